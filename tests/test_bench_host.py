"""Host logic of the benchmark (no GPU): the reference arm's JSON line on the
tiny workload, the clock record built from nvidia-smi samples, and the
roofline arithmetic."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_line_of_the_contract():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "tiny",
                        "--steps", "2", "--warmup", "1", "--ref-budget", "0.2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "updates/s"
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["name"] == "tiny" and d["config"]["workload"] == bench.WORKLOADS["tiny"]
    assert d["value"] > 0
    # one step is one whole layout: 30 iterations x 10 x S updates at the measured rate
    from synth import make_graph
    S = make_graph("tiny").n_steps
    assert d["ms_per_step"] == pytest.approx(30 * 10 * S / d["value"] * 1e3, rel=1e-9)
    # the same workload object as the GPU arm's line (sizes included)
    g = make_graph("tiny")
    assert d["config"] == bench.workload_config("tiny", g.n_nodes, g.n_paths, g.n_steps, 1)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_leaves_ranks_above_zero_idle():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "tiny",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT,
                       env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def _sample(sm, smax=2070, reasons=("Not Active",) * 4):
    return ", ".join([str(sm), str(smax), "900.0", "0x0"] + list(reasons))


def test_clock_record_takes_the_median_of_loaded_samples_and_every_reason_seen():
    lines = [_sample(900), _sample(2070), _sample(2055), _sample(2040, reasons=("Not Active",) * 3 + ("Active",)),
             "garbage", _sample("[N/A]"), _sample(2070)]
    c = bench.summarize_clocks(lines)
    # the idle 900 MHz sample is not under load; the malformed ones are skipped
    assert c["sm_mhz"] == 2062.5 and c["sm_max_mhz"] == 2070 and c["samples"] == 5
    assert c["reasons"] == ["sw_power_cap"]
    hot = bench.summarize_clocks([_sample(1500, reasons=("Active", "Not Active", "Active", "Not Active"))])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and hot["sm_mhz"] == 1500
    assert bench.summarize_clocks([])["reasons"] == ["no samples"]


def test_roofline_fraction_of_the_hbm_peak():
    r = bench.roofline_for("chrom", 4000.0, 6778.0, "measured", 6.58e11, 225.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6778.0
    assert r["frac"] == pytest.approx(4000.0 / 6778.0)
    assert r["bytes_per_update_model"] == bench.BYTES_PER_UPDATE == 192
    assert r["traffic"] == 6.58e11 and r["launch_ms"] == 225.0


def test_peaks_come_from_the_measured_file_when_present():
    peak, kind = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_traffic_record_belongs_to_the_current_update_kernel():
    """The benchmark reports the recorded ncu DRAM traffic only while the update
    kernel's source hash matches the one the record was taken on (the 2 M-node
    profiling graph: 1 GB resident, the chromosome graph's record sizes)."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "update_kernel_traffic_prof.json")))
    assert rec["kernel_rev"] == bench.kernel_revision()
    per_update = (rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]) / rec["updates_per_launch"]
    assert rec["dram_bytes_per_update"] == pytest.approx(per_update, abs=0.01)
    assert rec["updates_per_launch"] == 10 * 62_504_258  # 10 x S of the profiling graph


def test_phase_clocks_take_the_samples_inside_the_windows():
    from datetime import datetime
    t0 = datetime(2026, 12, 4, 6, 0, 0).timestamp()

    def line(sm, dt):
        ts = datetime.fromtimestamp(t0 + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return _sample(sm) + ", " + ts

    lines = [line(1500, 0.1), line(2000, 1.1), line(1990, 1.3), line(1700, 2.5), line(1980, 3.2)]
    c = bench.clocks_in_windows(lines, [(t0 + 1.0, t0 + 1.5), (t0 + 3.0, t0 + 3.5)])
    assert c["samples"] == 3 and c["sm_mhz_median"] == 1990 and c["sm_mhz_min"] == 1980
    assert bench.clocks_in_windows(lines, [(t0 + 5, t0 + 6)])["samples"] == 0
    # the summary over all samples still reads lines that carry the timestamp
    assert bench.summarize_clocks(lines)["samples"] == 5


def test_random_gather_fields_of_the_roofline():
    gather = {"reads_per_s": 48e9, "reads_per_s_with_node_reads": 37e9, "gbs_as_32B_sectors": 1536.0,
              "gbs_as_64B_accesses": 3072.0, "pattern": "p"}
    ref = {"kernel": "stress_kernel", "units_per_s": 22e9}
    r = bench.roofline_for("chrom", 4100.0, 6785.2, "measured", None, 218.6, gather, 42.9e9, ref, 21.4e9)
    assert r["random_gather_gbs"] == 1536.0
    assert r["frac_of_random_gather"] == pytest.approx(42.9 / 48)
    assert r["gather_reference"]["update_frac"] == pytest.approx(21.4 / 22)
    assert r["frac"] == pytest.approx(4100.0 / 6785.2)


def test_sampled_schedule_timing_scales_to_the_whole_layout():
    """The one-graph-at-a-time schedules are timed over the iterations of
    SAMPLED_ITERATIONS and scaled to ITERS; the rate is the timed updates over
    the timed milliseconds."""
    calls = []

    class FakeBatch:
        def __init__(self):
            self.pending = None

        def set_coords(self, xy):
            pass

        def set_option(self, k, v):
            pass

        def timing_read(self, reset=False):
            out, self.pending = self.pending, None
            return out if out else (0.0, 0, 0)

        def layout(self, iter_max, seeds=None, theta=None, iter_begin=0, iter_end=None):
            calls.append((iter_begin, iter_end))
            n = iter_end - iter_begin
            self.pending = (10.0 * n, 3 * n, 1_000_000 * n)  # ms, launches, updates per timed call

    out = bench._batch_sampled(FakeBatch(), None, None)
    its = sum(b - a for a, b in bench.SAMPLED_ITERATIONS)
    assert calls == [tuple(x) for x in bench.SAMPLED_ITERATIONS]
    assert out["timed_ms"] == 10.0 * its and out["ms"] == pytest.approx(10.0 * bench.ITERS)
    assert out["updates_per_s"] == pytest.approx(1e6 * its / (10.0 * its / 1e3))
    assert out["launches"] == 3 * bench.ITERS and out["ms_extrapolated"] is True
