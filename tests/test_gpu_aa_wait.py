"""Failure detection of the persistent in-place step without a GPU fault: every
wait between neighbouring CTAs has a time limit. A test hook makes one CTA
withhold its progress reports, so its neighbours' waits run out after 50 ms; the
launch then ends early, the host reads SC_ETIMEOUT (sc_lbm_sync, and the status of
the diagnostics), and after a state is loaded again the same lattice steps to the
right bits: the device stayed usable."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03637_gb300 as mod
    mod.build()
    return mod


@pytest.mark.parametrize("bands", [1, 4])
@pytest.mark.parametrize("withhold", [0, "last"])
def test_withheld_progress_gives_etimeout_and_the_device_stays_usable(sc, withhold, bands):
    from paper_1701_03637_gb300.workloads import droplet
    params, init = droplet(48, 9.0, 7)
    lat = sc.Lattice(dict(params, layout="aa", staging="persistent"))
    assert lat.persist_bands(bands) == bands
    info = lat.launch_info()
    # one band: a 3 x 3 or larger tile grid; four bands of 12 sites: a few CTAs
    assert info["staging"] == "persistent" and info["ctas"] >= (9 if bands == 1 else 2)
    cta = info["ctas"] - 1 if withhold == "last" else withhold
    lat.init(init)
    lat.set_wait(50_000_000, cta)
    lat.step(3)
    with pytest.raises(sc.ScError) as e:
        lat.sync()
    assert e.value.code == -5  # SC_ETIMEOUT
    assert lat.diagnostics()["status"] == -5
    # restore: default limit, no withholding, a fresh state
    lat.set_wait(2_000_000_000, -1)
    lat.init(init)
    lat.step(5)
    lat.sync()
    ref = sc.Lattice(params)
    ref.init(init)
    ref.step(5)
    assert np.array_equal(lat.read_populations(), ref.read_populations())
    assert lat.diagnostics()["status"] == 0
    lat.close()
    ref.close()


def test_wait_policy_is_validated(sc):
    from paper_1701_03637_gb300.workloads import droplet
    params, _ = droplet(24, 5.0, 7)
    lat = sc.Lattice(dict(params, layout="aa", staging="persistent"))
    ctas = lat.launch_info()["ctas"]
    for args in ((0, -1), (1000, ctas), (1000, -2)):
        with pytest.raises(sc.ScError, match="-1"):
            lat.set_wait(*args)
    lat.close()
