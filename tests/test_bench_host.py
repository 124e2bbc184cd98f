"""Host-side arithmetic and parsing of bench.py, on the CPU.

The roofline and e2e figures divide by per-row work; these tests recount that
work from the weight matrices a row actually multiplies and from the output
buffers' shapes, check the per-row totals of the scope table (14 / 35 /
100-input models), and exercise the clock-record parsing and the rule that
the ncu traffic is used only for the kernel source it was taken on.
"""
import numpy as np
import pytest

import bench
from paper_2510_19689_b300 import synth


def _params(name):
    return synth.make_params(synth.SPECS[name], synth.weight_seed(name))


def _macs_from_matrices(p):
    """Multiply-adds of one row: walk every FC matrix each step applies."""
    total = 0
    for s in range(p["n_steps"] + 1):
        for w in list(p["shared_fc"]) + list(p["ft"][s]["indep_fc"]):
            total += np.asarray(w).size                  # [2N, K]: 2N x K per row
        if s > 0:
            total += np.asarray(p["att"][s - 1]["fc"]).size   # [D_e, n_a]
    return total + np.asarray(p["final_w"]).size         # [C, n_d]


@pytest.mark.parametrize("name,macs", [("c1", 8_288), ("c2", 180_000), ("c3", 1_634_496)])
def test_mac_per_row(name, macs):
    p = _params(name)
    assert bench.mac_per_row(p) == _macs_from_matrices(p) == macs


@pytest.mark.parametrize("name,inp,out", [("c1", 56, 232), ("c2", 140, 848), ("c3", 400, 6812)])
def test_bytes_per_row(name, inp, out):
    p = _params(name)
    assert bench.bytes_per_row(p) == (inp, out)
    de = p["n_num"] + sum(p["cat_emb_dim"])
    d = p["n_num"] + len(p["cat_card"])
    # inputs: float32 numerics + int32 codes; outputs: logits, masks, aggregate
    assert inp == 4 * (p["n_num"] + len(p["cat_card"]))
    assert out == 4 * (p["n_classes"] + p["n_steps"] * de + d)


def test_clock_summary_median_and_reasons():
    c = bench.ClockSampler(0)
    # (sm MHz, max sm MHz, power W, clocks-event reason bits as NVML reports them)
    c.samples = [(2032.0, 2032.0, 800.1, 0x0), (1980.0, 2032.0, 1050.0, 0x4), (2010.0, 2032.0, 990.0, 0x1),
                 (1500.0, 2032.0, 700.0, 0x40 | 0x8)]
    c.how = "test"
    s = c.summary()
    assert s["sm_mhz"] == 1995.0 and s["sm_min_mhz"] == 1500.0 and s["sm_max_mhz"] == 2032.0
    assert s["power_w_max"] == 1050.0 and s["samples"] == 4
    # idle (0x1) is not a throttle reason; power cap, hardware slowdown and thermal are
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples():
    c = bench.ClockSampler(0)
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "how": None}


def _fake_root(tmp_path):
    csrc = tmp_path / "paper_2510_19689_b300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "tc_forward.cu").write_text("// kernel A\n")
    (csrc / "tc_ptx.cuh").write_text("// helpers\n")
    (csrc / "other.cu").write_text("// not a tensor-core source\n")
    (tmp_path / "profiles").mkdir()
    return csrc


def test_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = _fake_root(tmp_path)
    sha = bench.kernel_source_hash()
    (tmp_path / "profiles" / "tc_forward_c2_bf16x3.md").write_text(
        f"- kernel_source_sha = `{sha}`\n- dram_bytes_per_launch = 123456\n")
    assert bench.profiled_traffic("c2", "bf16x3") == 123456.0
    assert bench.profiled_traffic("c3", "bf16x3") is None          # no summary for that workload
    (csrc / "other.cu").write_text("// edits outside tc_* do not matter\n")
    assert bench.profiled_traffic("c2", "bf16x3") == 123456.0
    (csrc / "tc_forward.cu").write_text("// kernel B\n")           # the kernel changed
    assert bench.kernel_source_hash() != sha
    assert bench.profiled_traffic("c2", "bf16x3") is None


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == dict(hbm=6400.0, bf16=1800.0, bf16_sus=1400.0, src="fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(
        '{"hbm_gbs": 6489.3, "bf16_tflops": 1766.8, "bf16_tflops_sustained": 1387.8}')
    assert bench.peaks() == dict(hbm=6489.3, bf16=1766.8, bf16_sus=1387.8, src="measured")
