"""Host logic of bench.py that needs no GPU: the clock-sample summary, the
measured-peak lookup, the traffic figures keyed by the kernel sources, and the
reference arm's JSON line.
"""
import hashlib
import json
import os
import re
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons(tmp_path):
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    cs.proc = object()  # as if nvidia-smi had run
    rows = [
        "0, 1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1010.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1950, 2070, 980.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    (tmp_path / "clocks.csv").write_text("\n".join(rows) + "\n")
    s = cs.summary()
    assert s["sm_mhz"] == 1965 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_slowdown(tmp_path):
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    cs.proc = object()
    (tmp_path / "clocks.csv").write_text("0, 1500, 2070, 1300, 0x20, Not Active, Active, Not Active, Not Active\n")
    assert cs.summary()["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_without_nvidia_smi():
    cs = bench.ClockSampler(0)
    assert cs.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6782.1, "bf16_tflops": 1900.0}))
    assert bench.measured_peaks() == (6782.1, "measured")


def _hash(csrc, files):
    """sha256 over each file's name and bytes, in the listed order, first 16 hex digits"""
    h = hashlib.sha256()
    for name in files:
        h.update(name.encode())
        h.update((csrc / name).read_bytes())
    return h.hexdigest()[:16]


def test_traffic_is_dropped_once_the_kernel_changes(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2407_10925_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cuh").write_text("// kernel\n")
    (csrc / "k.cu").write_text("#include \"k.cuh\"\n")
    files = ["k.cuh", "k.cu"]
    entry = {"source_files": files, "source_hash": _hash(csrc, files), "dram_bytes_per_launch": 1234}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"sweep": {"h16": entry}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("h16", "sweep") == 1234
    assert bench.profiled_traffic("h17", "sweep") is None  # no capture for that workload
    (csrc / "k.cuh").write_text("// kernel, changed\n")
    assert bench.profiled_traffic("h16", "sweep") is None


def _stored_states(cfg_name):
    c = bench.CONFIGS[cfg_name]
    n = c["sigma"] ** (c["d"] * c["h"])
    return n // 2 if c["sigma"] == 2 else n  # complement-half storage for sigma = 2


def test_committed_traffic_entries_are_consistent():
    """Each committed figure is its bytes per stored state times the stored
    states of its workload (the capture's bytes per state do not depend on h)."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        j = json.load(f)
    n = 0
    for kernel, per_cfg in j.items():
        if kernel.startswith("_"):
            continue
        for cfg_name, e in per_cfg.items():
            n += 1
            assert cfg_name in bench.CONFIGS and e["captured_config"] in bench.CONFIGS
            want = e["dram_bytes_per_stored_state"] * _stored_states(cfg_name)
            assert e["dram_bytes_per_launch"] == pytest.approx(want, rel=1e-4), (kernel, cfg_name)
            for name in e["source_files"]:
                assert os.path.exists(os.path.join(ROOT, "paper_2407_10925_gb300", "csrc", name))
            assert os.path.exists(os.path.join(ROOT, e["summary"]))
    assert n >= 1


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores, no GPU): one
    JSON line with the contract's keys, its value repeated in cpu_baseline and
    e2e, and ms_per_step the measured time of the sample each step ran."""
    import subprocess

    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in j, key
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC and j["unit"] == bench.METRIC
    assert j["higher_is_better"] is True and j["n_gpus"] == 1 and j["steps"] == 1 and j["warmup"] == 0
    assert j["value"] > 0 and j["cpu_baseline"]["value"] == j["value"] and j["e2e"]["value"] == j["value"]
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1 and j["cpu_baseline"]["sample"]
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0
    cfg = j["config"]
    assert cfg["states"] == 2 ** 32 and "workload" in cfg
    # the step is the sample it timed: ms_per_step is that time, not an extrapolation to the workload
    want_ms = cfg["states_per_step"] / j["value"] * 1e3
    assert j["ms_per_step"] == pytest.approx(want_ms, rel=1e-6)
    assert j["cpu_baseline"]["value_1core"] > 0 and j["cpu_baseline"]["value_all_cores"] == j["value"]


def test_readme_lists_every_bench_config():
    """The README's bench line names exactly the workloads bench.py defines."""
    text = open(os.path.join(ROOT, "README.md")).read()
    m = re.search(r"--config ((?:\w+\|)+\w+)", text)  # the list of all of them
    assert m, "README names no --config list"
    assert set(m.group(1).split("|")) == set(bench.CONFIGS)


def test_profile_summaries_name_runnable_commands():
    """Each ncu summary under profiles/ gives its command; every ncu there
    leaves the clocks alone (--clock-control none), and every script it runs
    is a committed file."""
    pdir = os.path.join(ROOT, "profiles")
    mds = [f for f in os.listdir(pdir) if f.endswith(".md")]
    assert mds
    for f in mds:
        text = open(os.path.join(pdir, f)).read()
        # join continued lines so each command reads as one
        text = re.sub(r"\\\n\s*", " ", text)
        ncu = [ln for ln in text.splitlines() if re.search(r"(^|\s)ncu\s+-", ln)]
        assert ncu, f
        for ln in ncu:
            assert "--clock-control none" in ln, (f, ln)
        for script in re.findall(r"python (\S+\.py)", text):
            assert os.path.exists(os.path.join(ROOT, script)), (f, script)


@pytest.mark.parametrize("s,d,h,m", [(2, 2, 5, 2), (2, 2, 4, 1), (3, 2, 3, 1), (2, 3, 3, 1), (4, 2, 2, 1)])
def test_cpu_baseline_window_reads_only_filled_blocks(s, d, h, m):
    """The CPU baseline times the oracle's F over a window whose arguments exist
    only in the blocks the window reads.  With every other value a sentinel far
    below, F over each aligned window must not see a sentinel: its values stay
    within the filled range (F of values near 200 units is within a unit of it)."""
    import numpy as np

    import oracle

    one = 1 << oracle.DEFAULT_FRAC_BITS
    n, W = s ** (d * h), s ** (d * m)
    for x0 in range(0, n, W * max(1, n // W // 5)):
        vs = [np.full(n, -(1 << 60), dtype=np.int64) for _ in range(d)]
        bench.window_arguments(s, d, h, x0, m, 7, vs)
        out = oracle.F(s, d, h, vs, arith="fx", x0=x0, x1=x0 + W)
        assert out.min() >= 190 * one and out.max() <= 210 * one, x0


def test_cpu_baseline_sample_runs():
    steps, rate_1core, cores, sample = bench.oracle_sample({"sigma": 2, "d": 2, "h": 16}, workers=2, steps=1, m=5)
    assert steps[0]["states"] == 2 * 4 ** 5 and steps[0]["seconds"] > 0
    assert rate_1core > 0 and cores == 2 and "orc_F_fx" in sample
