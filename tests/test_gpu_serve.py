"""Served runs: a request served with continuous batching (admitted while others
run, stepped together with them) returns exactly the time series it returns when
run alone."""
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


def _alone(sc, req, storage, diag_every):
    from paper_1701_03637_gb300.serve import Result, _record
    lat = sc.Lattice(dict(req.params, storage=storage))
    lat.init(req.init)
    res = Result(req.rid, 0.0, 0.0, 0.0, req.steps, lat.n)
    assert _record(lat, res) == 0
    done = 0
    while done < req.steps:
        k = min(diag_every - done % diag_every, req.steps - done)
        lat.step(k)
        done += k
        assert _record(lat, res) == 0
    lat.close()
    return res


@pytest.mark.parametrize("storage", ["f16", "f32"])
def test_results_are_the_same_alone_and_in_the_mix(sc, storage):
    from paper_1701_03637_gb300.serve import Request, Server
    from paper_1701_03637_gb300.workloads import request_stream
    stream = request_stream(7, 400.0, seed=7, lo=20.0, hi=40.0, steps=(120, 420), storage=storage)
    reqs = [Request(k, t, p, i, n) for k, (t, p, i, n) in enumerate(stream)]
    need = max(sc.required_bytes(p) for _, p, _, _ in stream)
    srv = Server(3 * need + (1 << 20), storage, diag_every=50)
    res = srv.run(reqs)
    srv.close()
    waited = [r for r in res if r.admitted > r.arrival + 1e-3]
    assert waited, "the arena should have made some request wait"
    for r, q in zip(res, reqs):
        ref = _alone(sc, q, storage, 50)
        assert r.status == 0 and len(r.series) == len(ref.series)
        for a, b in zip(r.series, ref.series):
            step, iz, rad, flux, evap, mr = a
            assert (step, iz, rad, mr) == (b[0], b[1], b[2], b[5]), (q.rid, a, b)
            # cumulative sums over other partial sums: equal to FP64 rounding
            assert abs(flux - b[3]) <= 1e-12 * max(1.0, abs(b[3]))
            assert abs(evap - b[4]) <= 1e-12 * max(1.0, abs(b[4]))
