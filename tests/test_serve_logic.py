"""Host logic of the continuous-batching server, on a fake batch and a fake clock:
first-come admission by free arena, waiting while the arena is full, members
never stepped past their own step counts, a diagnostics record every diag_every
steps and at the end, and latencies measured from arrival."""
import pytest

from paper_1701_03637_gb300._native import ScError
from paper_1701_03637_gb300.serve import Request, Server, percentile


class FakeLattice:
    def __init__(self, n, fail=None):
        self.n = n
        self.step_count = 0
        self.fail = fail or {}  # seed -> first step whose diagnostics report SC_ENONFINITE

    def init(self, init):
        self.seed = init["seed"]

    def diagnostics(self):
        bad = self.seed in self.fail and self.step_count >= self.fail[self.seed]
        return dict(step=self.step_count, interface_z=float(self.seed), radius=0.0, flux_last=0.0,
                    evaporated_mass=0.0, mass_r=1.0, status=-4 if bad else 0)


class FakeBatch:
    """Arena of `capacity` units (a lattice of n sites takes n units); each step
    costs 1 ms on the fake clock per member."""

    def __init__(self, capacity, clock, fail=None):
        self.capacity = capacity
        self.clock = clock
        self.members = {}
        self.limits = {}
        self.log = []
        self.fail = fail

    def used(self):
        return sum(l.n for l in self.members.values())

    def add(self, params):
        n = params["nx"] * params["ny"] * params["nz"]
        if self.used() + n > self.capacity:
            raise ScError("arena full", -2)
        slot = 0
        while slot in self.members:
            slot += 1
        self.members[slot] = FakeLattice(n, self.fail)
        self.limits[slot] = None
        return slot, self.members[slot]

    def set_steps(self, slot, n):
        self.limits[slot] = n

    def step(self, k):
        for slot, lat in self.members.items():
            take = min(k, self.limits[slot] - lat.step_count)
            assert take == k, "a member would be stepped past its limit"
            lat.step_count += take
        self.clock.t += 1e-3 * k * len(self.members)
        self.log.append((k, sorted(self.members)))

    def remove(self, slot):
        del self.members[slot]
        del self.limits[slot]

    def configure(self, *a):
        pass


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 0.0)


def _req(rid, arrival, edge, steps):
    return Request(rid, arrival, dict(nx=edge, ny=edge, nz=edge), dict(seed=rid), steps)


def test_admission_waits_for_arena_and_series_are_complete():
    clock = Clock()
    fb = FakeBatch(capacity=2 * 10 ** 3, clock=clock)
    srv = Server(0, diag_every=100, batch=fb)
    reqs = [_req(0, 0.0, 10, 250), _req(1, 0.0, 10, 120), _req(2, 0.01, 10, 300), _req(3, 5.0, 5, 50)]
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    assert [r.rid for r in res] == [0, 1, 2, 3]
    for r, q in zip(res, reqs):
        steps = [s[0] for s in r.series]
        want = [0] + list(range(100, q.steps, 100)) + [q.steps]
        assert steps == want, (q.rid, steps)
        assert r.admitted >= q.arrival and r.finished > r.admitted
        assert r.latency == pytest.approx(r.finished - q.arrival)
        assert r.series[0][1] == float(q.rid)
    # request 2 arrived while 0 and 1 filled the arena: admitted only after 1 finished
    assert res[2].admitted >= res[1].finished
    # request 3 arrived after everything else was done: it waited for its arrival time
    assert res[3].admitted >= 5.0
    # never more than the arena holds
    assert all(len(m) <= 2 for _, m in fb.log)


def test_request_larger_than_an_empty_arena_is_an_error():
    clock = Clock()
    fb = FakeBatch(capacity=100, clock=clock)
    srv = Server(0, batch=fb)
    with pytest.raises(RuntimeError, match="does not fit"):
        srv.run([_req(0, 0.0, 10, 10)], clock=clock, sleep=clock.sleep)


def test_percentile():
    assert percentile([3, 1, 2], 50) == 2
    assert percentile([1, 2, 3, 4], 100) == 4
    assert percentile(list(range(101)), 99) == pytest.approx(99)


def test_site_cap_limits_the_active_set_but_always_admits_one():
    clock = Clock()
    fb = FakeBatch(capacity=10 ** 9, clock=clock)
    srv = Server(0, diag_every=100, batch=fb, max_active_sites=1500)
    reqs = [_req(0, 0.0, 10, 200), _req(1, 0.0, 10, 200), _req(2, 0.0, 20, 100)]
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    assert all(len(m) == 1 for _, m in fb.log)  # 1000 + 1000 > 1500; 8000 alone is admitted
    assert res[1].admitted >= res[0].finished and res[2].admitted >= res[1].finished


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_dispatch_serves_every_request_once_in_arrival_order(world):
    from paper_1701_03637_gb300.serve import Request, dispatch
    reqs = [Request(k, t, {}, {}, 100) for k, t in enumerate([0.5, 0.1, 0.3, 0.3, 0.9, 0.2, 0.7])]
    parts = [dispatch(reqs, r, world) for r in range(world)]
    assert sorted(q.rid for part in parts for q in part) == list(range(len(reqs)))
    order = sorted(reqs, key=lambda q: (q.arrival, q.rid))
    for r, part in enumerate(parts):
        assert [q.rid for q in part] == [q.rid for q in order[r::world]]
    with pytest.raises(ValueError):
        dispatch(reqs, world, world)


def test_a_failing_run_is_evicted_and_reported_while_the_others_finish():
    """Failure detection on the host: a run whose diagnostics report a non-finite
    density (status -4, injected by the fake lattice at step 200) leaves the batch at
    that record with its status; it is never stepped again and the others complete."""
    clock = Clock()
    batch = FakeBatch(10 ** 6, clock, fail={1: 200, 3: 0})
    srv = Server(0, batch=batch, diag_every=100)
    reqs = [_req(0, 0.0, 10, 500), _req(1, 0.0, 10, 500), _req(2, 0.0, 10, 300), _req(3, 0.0, 10, 400)]
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    by = {r.rid: r for r in res}
    assert [r.rid for r in res] == [0, 1, 2, 3]
    assert by[1].status == -4 and [s[0] for s in by[1].series] == [0, 100]
    assert by[3].status == -4 and by[3].series == []  # bad from the start: reported, never stepped
    for rid, steps in ((0, 500), (2, 300)):
        assert by[rid].status == 0 and by[rid].series[-1][0] == steps
    assert not batch.members
    assert by[1].finished < by[0].finished
