"""The benchmark's host-side contract (CPU only): the reference arm's JSON
line (the oracle timed on a tiny sample of the 3-level channel), the clock
sampler's restriction to the timed region, and the roofline line's choice of
kernel class and arithmetic."""
import datetime
import importlib.util
import json
import os
import subprocess
import sys
import tempfile
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_contract_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-frac", "0.01", "--ref-iters", "1", "--config", "channel2d_l3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "unit", "scaling", "dtype", "data"):
        assert isinstance(line[k], str) and line[k]
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] >= 3
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["config"]["workload"] == "channel2d_l3"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def test_clock_sampler_keeps_the_samples_inside_the_timed_region():
    b = _bench()
    cs = b.ClockSampler(0)
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    t = time.time()
    rows = [(0.00, 1500, "Not Active"), (0.10, 2070, "Not Active"), (0.15, 1980, "Active"),
            (0.20, 2070, "Not Active"), (0.40, 900, "Not Active")]
    for dt, mhz, cap in rows:
        ts = datetime.datetime.fromtimestamp(t + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        f.write(f"{ts}, 0, {mhz}, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, {cap}\n")
    f.flush()
    cs.proc, cs.f, cs.t0, cs.t1 = _Proc(), f, t + 0.05, t + 0.25
    got = cs.stop()
    assert got["samples"] == 3 and got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"]
    # a region shorter than the polling interval takes the nearest sample
    f2 = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    for dt, mhz, cap in rows:
        ts = datetime.datetime.fromtimestamp(t + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        f2.write(f"{ts}, 0, {mhz}, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, {cap}\n")
    f2.flush()
    cs2 = b.ClockSampler(0)
    cs2.proc, cs2.f, cs2.t0, cs2.t1 = _Proc(), f2, t + 0.41, t + 0.42
    got = cs2.stop()
    assert got["samples"] == 1 and got["sm_mhz"] == 900.0


def _kst(ms, nbytes=0.0, flops=0.0, launches=10):
    return {"ms": ms, "bytes": nbytes, "flops": flops, "launches": launches}


@pytest.mark.parametrize("dominant", ["patch_apply", "patch_factor", "assemble"])
def test_roofline_picks_the_largest_class_and_divides_by_its_peak(dominant):
    b = _bench()
    kst = {"patch_apply": _kst(8.0, nbytes=8.0 * 4.0e6), "patch_factor": _kst(7.0, flops=7.0 * 1.0e10),
           "assemble": _kst(3.0, flops=3.0 * 5.0e8)}
    scale = 20.0 / kst[dominant]["ms"]   # make it the largest class at the same rate
    kst[dominant] = {k: (v * scale if k in ("ms", "bytes", "flops") else v) for k, v in kst[dominant].items()}
    key = "channel2d_l6 mixed"
    roof, classes = b._roofline(kst, steps=2, fp32_classes=("patch_factor",), traffic_key=key)
    assert roof["kernel"] == dominant
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["avg_launch_ms"] == pytest.approx(20.0 / 10)
    if dominant == "patch_apply":
        assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
        assert roof["achieved"] == pytest.approx(4.0e6 / 1e-3 / 1e9)     # bytes per ms -> GB/s
    elif dominant == "patch_factor":
        assert roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
        assert roof["achieved"] == pytest.approx(1.0e10 / 1e-3 / 1e12)
    else:
        assert roof["bound"] == "alu"
    assert roof["traffic"] == json.load(open(os.path.join(ROOT, "profiles", "traffic.json"))).get(key, {}).get(dominant)
    assert classes[dominant]["ms_per_step"] == pytest.approx(10.0)


def test_cpu_baseline_leg_serial_and_all_cores():
    """The cpu_baseline child process (one BLAS / OpenMP thread) times the
    oracle sample serially and spread over one process per core, and reports
    both with their core counts."""
    b = _bench()
    leg = b.CpuBaseline("channel2d_l3", 0.05, 1)
    out, why = leg.result(timeout=600)
    assert out is not None, why
    assert out["kind"] == "oracle" and out["cores"] == 1 and out["value"] > 0 and out["sample"]
    assert out["detail"]["frac"] == 0.05
    if b._cores() > 1:
        a = out["all_cores"]
        assert a["cores"] == b._cores() and a["value"] > 0
