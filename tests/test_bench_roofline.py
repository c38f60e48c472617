"""bench.py's roofline bookkeeping on a synthetic kernel profile (CPU).

* the dominant class is the one with the largest total time, and its
  achieved rate is algorithmic work per launch over the average launch time;
* an FP64-pipe-bound class reports "alu" against the FP64 peak, a streaming
  class "hbm" against the measured copy bandwidth;
* the tensor-core projections are reported against the TF32 peak derived
  from the measured BF16 GEMM rate, with the executed 3xTF32 work beside it;
* the DRAM traffic ratio applies only while the listed sources hash to the
  recorded value.
"""
import json

import pytest


def _prof(**cls):
    base = {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0}
    return {"launches": 1, "classes": {k: dict(base, **v) for k, v in cls.items()}}


def test_dominant_class_alu():
    import bench
    prof = _prof(slab_f64={"launches": 10, "ms": 100.0, "flops": 10 * 6.0e9, "bytes": 10 * 4e8},
                 cg_f32={"launches": 100, "ms": 20.0, "flops": 1e9, "bytes": 1e11})
    r = bench.roofline(prof)
    assert r["kernel"] == "slab_f64" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(0.6, rel=1e-3)           # 6 GFLOP per 10 ms
    assert r["frac"] == pytest.approx(0.6 / bench.FP64_PEAK_TFLOPS, rel=1e-3)


def test_dominant_class_hbm():
    import bench
    hbm, _ = bench.measured_peaks()
    prof = _prof(cg_f32={"launches": 4, "ms": 4.0, "flops": 4 * 1e8, "bytes": 4 * 4e9})
    r = bench.roofline(prof)
    assert r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(4000.0, rel=1e-3)          # 4 GB per ms
    assert r["frac"] == pytest.approx(4000.0 / hbm, rel=1e-3)


def test_tensor_gemm_against_tf32_peak():
    import bench
    prof = _prof(gemm_tf32x3={"launches": 2, "ms": 2.0, "flops": 2e10, "bytes": 1e9})
    t = bench.tensor_gemm(prof)
    peak, _ = bench.tf32_peak()
    assert t["bound"] == "tensor"
    assert t["achieved"] == pytest.approx(10.0, rel=1e-3)            # 20 GFLOP in 2 ms
    assert t["executed_tf32"] == pytest.approx(30.0, rel=1e-3)
    assert t["frac"] == pytest.approx(10.0 / peak, abs=1e-4)        # rounded to 4 places
    assert bench.tensor_gemm(_prof(cg_f32={"launches": 1, "ms": 1.0})) is None


def test_traffic_needs_matching_sources(tmp_path, monkeypatch):
    import bench
    src = ["common.cuh", "fft.cuh"]
    good = {"classes": {"slab_f64": {"dram_over_algorithmic": 0.5, "sources": src,
                                     "sources_hash": bench.sources_hash(src)}}}
    f = tmp_path / "t.json"
    f.write_text(json.dumps(good))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.traffic_for("slab_f64", 100.0) == pytest.approx(50.0)
    assert bench.traffic_for("slab_f32", 100.0) is None
    good["classes"]["slab_f64"]["sources_hash"] = "0" * 16
    f.write_text(json.dumps(good))
    assert bench.traffic_for("slab_f64", 100.0) is None


def test_step_spread():
    import bench
    assert bench.step_spread([]) is None
    one = bench.step_spread([5.0])
    assert one == {"median": 5.0, "p10": 5.0, "p90": 5.0, "n": 1}
    sp = bench.step_spread([3.0, 1.0, 2.0, 5.0, 4.0])
    assert sp["median"] == 3.0 and sp["n"] == 5
    assert sp["p10"] == pytest.approx(1.4) and sp["p90"] == pytest.approx(4.6)
