"""The benchmark reports the DRAM traffic of the step kernel from the committed ncu
summary only while that summary describes the kernel being timed: same source
digest, workload, storage and launch configuration; otherwise null."""
import pytest


def _summary(tmp_path, digest, tile="64x4", zchunk="32", workload="droplet_128", storage="f32"):
    p = tmp_path / "k_step.md"
    p.write_text(f"""# summary

- workload: `{workload}`
- storage: `{storage}`
- tile: `{tile}`
- zchunk: `{zchunk}`
- source_digest: `{digest}`
- dram_bytes_per_launch: `601070592`
""")
    return str(p)


@pytest.fixture()
def bench(monkeypatch):
    import bench as b
    return b


def test_traffic_when_everything_matches(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_FILE", _summary(tmp_path, bench.source_digest()))
    assert bench.profiled_traffic("droplet_128", "f32", "64x4", 32) == 601070592.0


@pytest.mark.parametrize("change", ["digest", "tile", "zchunk", "workload", "storage"])
def test_no_traffic_when_anything_differs(bench, tmp_path, monkeypatch, change):
    kw = dict(digest=bench.source_digest())
    if change == "digest":
        kw["digest"] = "0000000000000000"
    elif change == "tile":
        kw["tile"] = "32x4"
    elif change == "zchunk":
        kw["zchunk"] = "16"
    elif change == "workload":
        kw["workload"] = "droplet_512"
    else:
        kw["storage"] = "f16"
    monkeypatch.setattr(bench, "PROFILE_FILE", _summary(tmp_path, **kw))
    assert bench.profiled_traffic("droplet_128", "f32", "64x4", 32) is None


def test_missing_summary_gives_no_traffic(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_FILE", str(tmp_path / "absent.md"))
    assert bench.profiled_traffic("droplet_128", "f32", "64x4", 32) is None
