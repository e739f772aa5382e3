"""Host logic of bench.py's JSON line (CPU only): the roofline object and the
DRAM-traffic lookup keyed by the product sources' hash."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _res(prec="fp32", mirrored=True):
    stage_ms = {"XY": 1.0, "TU": 3.0, "Z": 2.0, "traces": 0.2, "Q": 0.3, "W": 1.5, "G": 0.1}
    flops = {k: 0.0 for k in bench.STAGES}
    flops.update({"XY": 6e9, "TU": 27e9, "Z": 36e9, "Q": 3e9, "W": 18e9})
    kernels = {"XY": "group-pipe-half", "TU": "group-pipe", "Z": "group-pipe-half", "Q": "group-pipe-half",
               "W": "group-pipe-half"}
    return {"prec": prec, "stage_ms": stage_ms, "flops_stage": flops, "kernels": kernels, "t_mirrored": mirrored}


def test_roofline_takes_the_slowest_product_stage():
    r = bench.roofline(_res())
    assert r["stage"] == "TU" and r["kernel_ms"] == 3.0
    assert abs(r["achieved"] - 27e9 / 3e-3 / 1e12) < 1e-3
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["algorithmic_flops_per_launch"] == 27e9
    assert "k_mirror_lower" in r["kernel"]


def test_roofline_labels_t_formed_whole():
    r = bench.roofline(_res(mirrored=False))
    assert "k_mirror_lower" not in r["kernel"] and r["kernel"].startswith("k_gw")


def test_roofline_peaks_per_precision():
    assert bench.roofline(_res("fp64"))["peak"] == round(bench.PEAK_TFLOPS["fp64"], 3)
    assert bench.roofline(_res("fp32"))["peak"] == round(bench.PEAK_TFLOPS["fp32"], 3)


def test_traffic_only_for_the_recorded_sources(monkeypatch):
    sha = bench.product_source_sha()
    got = bench.ncu_traffic("TU", "fp32")
    # the committed summary matches the committed kernels, or reports nothing
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    recorded = [ln.split() for ln in open(path) if not ln.startswith("#") and ln.strip()]
    if any(f[3] == sha for f in recorded):
        assert got is not None and got > 0
    else:
        assert got is None
    monkeypatch.setattr(bench, "product_source_sha", lambda: "000000000000")
    assert bench.ncu_traffic("TU", "fp32") is None


def test_roofline_of_a_tensor_core_stage():
    """A dominant stage on a tcgen05 kernel is reported against the dense
    TF32 peak (half the measured BF16 burst), with the FMA probe beside it."""
    res = _res()
    res["kernels"]["TU"] = "tensor-tile"
    r = bench.roofline(res, fma_tflops=76.0)
    tf32 = bench.measured_peaks()["bf16_tflops"] / 2.0
    assert r["bound"] == "tensor" and r["stage"] == "TU"
    assert abs(r["peak"] - round(tf32, 1)) < 1e-9
    assert abs(r["frac"] - r["achieved"] / tf32) < 1e-3
    assert abs(r["frac_of_fma_probe"] - r["achieved"] / 76.0) < 1e-3
    assert r["kernel"].startswith("k_umma_tile") and "k_mirror_lower" in r["kernel"]
    # the same stage on a SIMT kernel stays bound by the FMA pipe
    res["kernels"]["TU"] = "group-pipe"
    assert bench.roofline(res, fma_tflops=76.0)["bound"] == "alu"


def test_tensor_stage_list_and_single_pass_pins():
    """roofline_tensor lists exactly the tcgen05 stages; the single-pass
    measurement pins kernels 12 and 13 where 9 and 11 run, and names only
    kernels the binding knows."""
    from paper_0911_3584_gb300.lnv import Plan

    res = _res()
    res["kernels"].update({"TU": "tensor-tile", "Z": "tensor", "W": "tensor-1pass"})
    got = {t["stage"] for t in bench.roofline_tensor(res)}
    assert got == {"TU", "Z", "W"}
    pins = bench.SINGLE_PASS_KERNELS
    assert pins["mirror"] == "1"
    for st, k in pins.items():
        if st != "mirror":
            assert k in Plan.KERNELS and k in bench.KERNEL_NAME
    assert {pins[s] for s in ("Z", "W")} == {"tensor-1pass"}
    assert {pins[s] for s in ("TU", "Q")} == {"tensor-tile-1pass"}
