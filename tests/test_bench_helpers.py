"""Host-side helpers of bench.py: the kernel source hash that keys the
recorded DRAM traffic, the tiling parser, and the reference arm's sample."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_code_ignores_comments_and_blank_space():
    a = "int x = 1; // one\n/* block\n comment */ int y =  2;\n"
    b = "int x = 1;\n\n   int y = 2; // two"
    assert bench.kernel_code(a) == bench.kernel_code(b) == "int x = 1; int y = 2;"
    assert bench.kernel_code("int x = 1;") != bench.kernel_code("int x = 2;")


def test_kernel_source_hash_is_stable_and_sees_code(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() { int a = 1; }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ["k.cu"])
    h0 = bench.kernel_source_sha()
    src.write_text("// a comment\n__global__ void k() {\n  int a = 1;  /* same code */\n}\n")
    assert bench.kernel_source_sha() == h0
    src.write_text("__global__ void k() { int a = 2; }\n")
    assert bench.kernel_source_sha() != h0


def test_parse_tiling():
    from paper_2605_19926_gb300 import jx

    assert bench.parse_tiling(jx, "") is None
    t = bench.parse_tiling(jx, "4,1,64,8")
    assert t.as_tuple() == (4, 1, 64, 8, 1)  # staging buffers default to one
    assert bench.parse_tiling(jx, "2,2,128,16,2").as_tuple() == (2, 2, 128, 16, 2)
    with pytest.raises(ValueError):
        bench.parse_tiling(jx, "4,x,64,8")


def test_recorded_traffic_only_for_the_same_kernel_code(tmp_path, monkeypatch):
    """The recorded DRAM bytes apply only to the kernel code they were taken
    on and to the same env count; otherwise traffic is reported as null."""
    import json

    rec = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "kernel_source_sha", lambda sources=None: "abc")
    rec.write_text(json.dumps({"kernel_source_sha": "abc", "n_envs": 4096, "dram_bytes_per_env_step": 10000.0}))
    assert bench.recorded_traffic(4096, 128, str(rec)) == 10000.0 * 4096 * 128
    assert bench.recorded_traffic(2048, 128, str(rec)) is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda sources=None: "def")
    assert bench.recorded_traffic(4096, 128, str(rec)) is None
    assert bench.recorded_traffic(4096, 128, str(tmp_path / "missing.json")) is None


def test_recorded_traffic_scaling_and_tiling(tmp_path, monkeypatch):
    """A record taken on a smaller case applies to other env counts only when
    it says its traffic grows with the env-steps, and a batched-kernel record
    only to the tiling it was captured with."""
    import json

    rec = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "kernel_source_sha", lambda sources=None: "abc")
    rec.write_text(json.dumps({"kernel_source_sha": "abc", "n_envs": 4096, "dram_bytes_per_env_step": 100.0,
                               "scales_with_env_steps": True, "tiling": [4, 1, 64, 8, 1]}))
    assert bench.recorded_traffic(65536, 8, str(rec), tiling=(4, 1, 64, 8, 1)) == 100.0 * 65536 * 8
    assert bench.recorded_traffic(65536, 8, str(rec), tiling=(0, 0, 0, 0, 0)) == 100.0 * 65536 * 8  # no sides
    assert bench.recorded_traffic(65536, 8, str(rec)) is None
    rec.write_text(json.dumps({"kernel_source_sha": "abc", "n_envs": 4096, "dram_bytes_per_env_step": 100.0,
                               "scales_with_env_steps": True, "tiling": [4, 1, 64, 8, 1], "map_sides": [128]}))
    assert bench.recorded_traffic(65536, 8, str(rec), tiling=(2, 2, 8, 32, 1)) == 100.0 * 65536 * 8
    assert bench.recorded_traffic(65536, 8, str(rec), tiling=(4, 1, 0, 8, 1)) is None  # byte maps read less


def test_committed_records_are_well_formed():
    import json

    for path in (bench.TRAFFIC_FILE, bench.TRAFFIC_UNEVEN_FILE, bench.TRAFFIC_LARGE_FILE):
        rec = json.load(open(path))
        assert rec["dram_bytes_per_env_step"] == pytest.approx(
            (rec["dram_bytes_read"] + rec["dram_bytes_write"]) / (rec["n_envs"] * rec["capture_steps_per_launch"]),
            abs=0.1)


def test_tiling_key_sees_only_the_effective_map_kind():
    assert bench.tiling_key((4, 1, 8, 8, 1), [128]) == bench.tiling_key((4, 2, 64, 32, 2), [128])
    assert bench.tiling_key((4, 1, 8, 8, 1), [16, 128]) != bench.tiling_key((4, 1, 64, 8, 1), [16, 128])
    assert bench.tiling_key((4, 1, 0, 8, 1), [128]) != bench.tiling_key((4, 1, 128, 8, 1), [128])


@pytest.mark.parametrize("steps,warmup,ring_slots", [(20, 5, 128), (1, 3, 128), (129, 16, 128), (10000, 16, 128),
                                                     (3, 3, 2), (128, 3, 128), (500, 4, 7)])
def test_plan_indexes_stay_inside_the_action_stream(steps, warmup, ring_slots):
    """Every row the headline run reads lies inside the action stream it draws
    (warmup + steps rows), the timed launches cover exactly the timed steps in
    order, each fits the rollout buffer, and the graph replays read full rings."""
    p = bench.Plan(steps, warmup, ring_slots)
    assert p.stream_len == warmup + steps
    assert 1 <= p.ring <= ring_slots
    assert p.ring >= min(ring_slots, bench.MIN_RING)
    covered = []
    for start, n in p.launches:
        assert 1 <= n <= p.ring
        assert 0 <= start and start + n <= p.stream_len
        covered.extend(range(start, start + n))
    assert covered == list(range(warmup, warmup + steps))
    assert all(0 <= p.warmup_slot(s) < p.ring for s in range(warmup))
    assert 1 <= p.n_graph <= 16
    for c in range(p.n_graph):
        rows = p.graph_rows(c)
        assert len(rows) == p.ring and all(0 <= r < p.stream_len for r in rows)
    rows = p.wrapped(warmup, 300)
    assert len(rows) == 300 and all(0 <= r < p.stream_len for r in rows)


def test_plan_rejects_empty_runs():
    with pytest.raises(ValueError):
        bench.Plan(0, 3, 128)
    with pytest.raises(ValueError):
        bench.Plan(10, 3, 0)


@pytest.mark.parametrize("steps,warmup", [(20, 5), (1, 3), (129, 16), (10000, 16)])
def test_headline_roofline_is_bytes_per_step_times_steps_over_time(steps, warmup):
    """roofline.achieved = the timed launches' algorithmic bytes / the timed
    region: bytes per step x steps / seconds, whatever the launch split (a
    short last launch is not counted as a full one)."""
    from paper_2605_19926_gb300 import inputs

    cfg = inputs.batched_keydoor_mazes()
    p = bench.Plan(steps, warmup, 128)
    total = sum(bench.rollout_bytes(cfg, 4096, n) for _, n in p.launches)
    per_step = total / steps
    ms = 0.0096 * steps  # a made-up timed region
    r = bench.roofline(total, ms, 6785.5, "measured")
    assert r["achieved"] == pytest.approx(per_step * steps / (ms / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(per_step / (ms / steps / 1e3) / 1e9 / 6785.5)
    # frames dominate: per step a little over 4096 frames of 64 x 64 x 3 bytes
    assert 4096 * 12288 < per_step < 4096 * 12400


def test_clock_summary_uses_busy_samples():
    rows = ["0, 1000, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active, 0",
            "0, 1950, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Active, 100",
            "0, 1965, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active, 98"]
    s = bench.ClockSampler.summarise("\n".join(rows))
    assert s["sm_mhz"] == pytest.approx(1957.5) and s["samples"] == 3 and s["samples_under_load"] == 2
    assert s["reasons"] == ["sw_power_cap"] and s["sm_max_mhz"] == 2070
    assert bench.ClockSampler.summarise("") is None
