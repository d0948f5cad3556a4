"""Where the GPU tests save the measured series they check, for the record: the
directory named by the SC_TEST_OUTPUT environment variable, or nowhere when it
is unset."""
import json
import os


def save(name, record):
    d = os.environ.get("SC_TEST_OUTPUT")
    if not d:
        return
    try:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, name), "w") as fh:
            json.dump(record, fh, indent=1)
    except OSError:
        pass
