"""The benchmark reports the DRAM traffic of the step kernel from a committed ncu
summary only while that summary describes the kernel being timed: same source
digest, workload, storage, layout and launch configuration; otherwise null. Its
`config` is the same for both arms and says truthfully how the workload meets the
L2."""
import pytest


def _summary(tmp_path, digest, tile="64x4", zchunk="32", workload="droplet_128", storage="f32", layout=None):
    p = tmp_path / "k_step.md"
    lay = f"- layout: `{layout}`\n" if layout else ""
    p.write_text(f"""# summary

- workload: `{workload}`
- storage: `{storage}`
{lay}- tile: `{tile}`
- zchunk: `{zchunk}`
- source_digest: `{digest}`
- dram_bytes_per_launch: `601070592`
""")
    return str(tmp_path)


@pytest.fixture()
def bench(monkeypatch):
    import bench as b
    return b


def test_traffic_when_everything_matches(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_DIR", _summary(tmp_path, bench.source_digest()))
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
    monkeypatch.setattr(bench, "PROFILE_DIR", _summary(tmp_path, **kw))
    assert bench.profiled_traffic("droplet_128", "f32", "64x4", 32) is None


def test_missing_summary_gives_no_traffic(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_DIR", str(tmp_path / "absent"))
    assert bench.profiled_traffic("droplet_128", "f32", "64x4", 32) is None


def test_layout_must_match(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_DIR", _summary(tmp_path, bench.source_digest(), layout="aa"))
    assert bench.profiled_traffic("droplet_128", "f32", "64x4", 32) is None
    assert bench.profiled_traffic("droplet_128", "f32", "64x4", 32, layout="aa") == 601070592.0


def _args(bench, argv):
    import sys
    old = sys.argv
    sys.argv = ["bench.py"] + argv
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_default_line_is_the_512_droplet_in_place(bench):
    a = _args(bench, [])
    assert a.workload == "droplet_512" and a.layout == "aa" and a.storage == "f32"
    c = bench.arm_config(a, 1)
    assert c["sites"] == 512 ** 3 and c["layout"] == "aa"
    assert c["l2"].startswith("inputs larger than L2")


def test_l2_note_is_true_for_small_lattices(bench):
    a = _args(bench, ["--workload", "film_4x4x128"])
    assert a.layout == "two"
    assert bench.arm_config(a, 1)["l2"].startswith("populations fit in L2")


@pytest.mark.parametrize("argv", [[], ["--workload", "droplet_128"], ["--workload", "ensemble_64"],
                                  ["--workload", "serve"], ["--workload", "film_4x4x128", "--storage", "f16"],
                                  ["--workload", "ncomp3_128"], ["--workload", "droplet_1024"]])
def test_both_arms_print_the_same_config(bench, argv):
    """The oracle arm's config is computed by the same function from the same
    arguments: nothing in it depends on which arm runs."""
    a = _args(bench, argv)
    b = _args(bench, argv + ["--impl", "reference"])
    assert bench.arm_config(a, 1) == bench.arm_config(b, 1)


def test_slab_layout_config(bench):
    a = _args(bench, ["--workload", "droplet_128", "--layout", "slab"])
    b = _args(bench, ["--workload", "droplet_128", "--layout", "slab", "--impl", "reference"])
    c = bench.arm_config(a, 4)
    assert c == bench.arm_config(b, 4) and c["layout"] == "slab"
    assert "split along z over 4 ranks" in c["parallelism"] and str(2 * 19 * 2 * 128 * 128 * 4) in c["parallelism"]


def test_precision_record_prefers_the_longer_study(bench, tmp_path, monkeypatch):
    for study, case in (("precision_droplet_128", "1000 steps"), ("precision_droplet_128_5000", "5000 steps")):
        (tmp_path / f"{study}.md").write_text(f"- study: `{study}`\n- case: `{case}`\n- f32_linf: `1e-6`\n"
                                              f"- f32_l2: `1e-7`\n- f32_radius_error: `0.0`\n")
    monkeypatch.setattr(bench, "PROFILE_DIR", str(tmp_path))
    assert bench.precision_record()["case"] == "5000 steps"
    (tmp_path / "precision_droplet_128_5000.md").unlink()
    rec = bench.precision_record()
    assert rec["case"] == "1000 steps" and rec["f32"]["density_linf"] == 1e-6


def test_three_component_config(bench):
    a = _args(bench, ["--workload", "ncomp3_128"])
    c = bench.arm_config(a, 2)
    assert c["components"] == 3 and c["sites"] == 128 ** 3 and c["layout"] == "two"
    assert c["l2"].startswith("inputs larger than L2") and "replicas x2" in c["parallelism"]
