"""Host-side pieces of bench.py, without a GPU: the roofline arithmetic, the
launch-shape key of the traffic table, the workload description, the
--gpus / launcher consistency check, and the oracle sample of the CPU
baseline and the reference arm (two processes)."""
import math

import pytest


@pytest.fixture(scope="module")
def bench():
    import bench as mod     # the repository root is on sys.path (conftest)

    return mod


def test_roofline_fractions(bench):
    r = bench.roofline("k", 2e9, 1e-3, 1e9, 4000.0, "of measured", "x", "y")
    assert math.isclose(r["achieved"], 2000.0)
    assert math.isclose(r["frac"], 0.5)
    assert math.isclose(r["dram_frac"], 0.25)
    assert math.isclose(r["traffic_ratio"], 0.5)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    r = bench.roofline("k", 2e9, 1e-3, None, 4000.0, "of measured", "x", "y",
                       bound=bench.L2_BOUND)
    assert r["traffic"] is None and r["dram_frac"] is None and r["traffic_ratio"] is None
    assert r["bound"] == bench.L2_BOUND and r["denominator"] == "hbm"


def test_shape_key_tells_launch_shapes_apart(bench):
    base = {"batch": 2, "tile_rows": 0, "src_tile": 32, "groups": 1, "min_blocks": 5}
    keys = {bench.shape_key(dict(base)), bench.shape_key(dict(base, sweep=4)),
            bench.shape_key(dict(base, stream=1)), bench.shape_key(dict(base, tma=128)),
            bench.shape_key(dict(base, ring=4)), bench.shape_key(dict(base, groups=2))}
    assert len(keys) == 6
    assert bench.shape_key(dict(base)) == bench.shape_key(dict(base, sweep=0, stream=0, tma=0))


def test_traffic_is_reported_only_for_the_captured_sources(bench, monkeypatch):
    t = {"batch": 2, "tile_rows": 0, "src_tile": 32, "groups": 1, "min_blocks": 5}
    monkeypatch.setattr(bench, "TRAFFIC", {("w k", bench.shape_key(t), False):
                                           (1.5e9, bench.sources_sha1())})
    assert bench.traffic_for("w k", t) == 1.5e9
    assert bench.traffic_for("w k", dict(t, sweep=4)) is None
    monkeypatch.setattr(bench, "TRAFFIC", {("w k", bench.shape_key(t), False): (1.5e9, "0" * 40)})
    assert bench.traffic_for("w k", t) is None


def test_description_names_the_layout(bench):
    from workloads import configs

    w = configs.asteroid_2d(n_refine=1, S=4, nt=10)
    assert "kept in HBM" in bench.describe(w, "kept")
    assert "checkpoints every 256" in bench.describe(w, "checkpoints")


def test_gpus_must_match_the_launcher(bench, monkeypatch):
    class A:
        gpus = 2

    monkeypatch.setenv("WORLD_SIZE", "1")
    with pytest.raises(SystemExit):
        bench.relaunch_or_check(A())
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.relaunch_or_check(A()) is None
    A.gpus = 1
    monkeypatch.delenv("WORLD_SIZE")
    assert bench.relaunch_or_check(A()) is None      # one GPU: no relaunch


def test_oracle_sample_on_two_processes(bench, monkeypatch):
    monkeypatch.setattr(bench, "ORACLE_STEPS", 20)
    from workloads import configs
    from oracle import wave

    w = configs.asteroid_2d()
    m = w.mesh
    dt = w.cfl_fraction * wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc).cfl_dt()
    ora = bench.OracleSample(dt, cores=2)
    try:
        val, res = ora.run()
    finally:
        ora.close()
    assert len(res) == 2 and val > 0
    units = 3.0 * w.n_nodes * 20
    assert all(u == units for _, u in res)
    assert math.isclose(val, 2 * units / max(t for t, _ in res))
    assert "2 shots of 128" in ora.sample_text()


def test_lanes_per_row_and_entry_chunks(bench):
    """The bench's copy of the launch-shape rule (lanes per row) and the
    chunk each kind's launches use once the chunk-major entries are built."""
    assert bench.lanes_per_row(128, 2) == 16 and bench.lanes_per_row(64, 1) == 16
    assert bench.lanes_per_row(64, 2) == 8 and bench.lanes_per_row(256, 4) == 16
    assert bench.lanes_per_row(100, 2) == 25          # falls back to one float4 per lane
    t = {"forward": {"batch": 2, "tile_rows": 0, "groups": 1},
         "tangent": {"batch": 1, "tile_rows": 0, "groups": 2},
         "adjoint": {"batch": 2, "tile_rows": 64, "groups": 1}}
    bench.mark_chunk(t, 128, 16)
    assert [t[k]["ellc"] for k in ("forward", "tangent", "adjoint")] == [16, 16, 0]
    k = {"batch": 2, "tile_rows": 0, "groups": 1, "min_blocks": 5}
    assert bench.shape_key(dict(k, ellc=16)) != bench.shape_key(k)
