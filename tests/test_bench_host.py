"""Host-side helpers of bench.py: the per-step arithmetic label, and the committed measurement
records (QP-gap error, DRAM traffic) that the bench line carries only while they were taken on the
current source of the tensor-core kernels."""
import importlib.util
import json
import os
import shutil
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_dtype_labels():
    b = _bench()
    assert b._dtype(types.SimpleNamespace(prec="fp64", screen="f32x2")) == "f64 (every step)"
    mixed = b._dtype(types.SimpleNamespace(prec="fp16x2", screen="f32x2"))
    assert "tensor cores" in mixed and "dielectric solve: f32x2" in mixed
    assert "dielectric solve: f32;" in b._dtype(types.SimpleNamespace(prec="fp16x2", screen="f32"))


def test_gap_record_follows_the_kernel_source(tmp_path):
    b = _bench()
    args = types.SimpleNamespace(screen="f32x2", omega=270.1, cont="cpe_mlp", gpus=1)
    rec = json.load(open(os.path.join(ROOT, "profiles", "gap_nk64_nb64.json")))
    got = b._gap_record("nk64_nb64", args, "fp16x2")
    if got:  # the committed record was taken on the current source
        assert got["gap_err_mev"]["cpe_ridge_1e-3"] == rec["gap_err_mev"]["mixed_f32x2/cpe_0.001"]
        assert got["gap_err_mev"]["pade"] == rec["gap_err_mev"]["mixed_f32x2/pade"]
        assert got["fp64_iteration_s"] == rec["fp64_iteration_s"]
    assert b._gap_record("nk64_nb64", args, "fp64") == {}
    # a copy of the tree whose kernel source differs from the one the record names: no record
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_1602_02313_gb300" / "csrc").mkdir(parents=True)
    for f in ("gap_nk64_nb64.json", "traffic.json"):
        shutil.copy(os.path.join(ROOT, "profiles", f), tmp_path / "profiles")
    src = open(os.path.join(ROOT, "paper_1602_02313_gb300", "csrc", "tc_mixed.cu")).read()
    (tmp_path / "paper_1602_02313_gb300" / "csrc" / "tc_mixed.cu").write_text(src + "\n// changed\n")
    b.ROOT = str(tmp_path)
    assert b._gap_record("nk64_nb64", args, "fp16x2") == {}
    assert b._traffic("k_pol_tc") is None
    # and the unchanged source: the traffic record is read
    (tmp_path / "paper_1602_02313_gb300" / "csrc" / "tc_mixed.cu").write_text(src)
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["k_pol_tc"]
    assert b._traffic("k_pol_tc") == (t["bytes_per_launch"] if t["src_sha"] == b.hashlib.sha256(
        src.encode()).hexdigest()[:16] else None)
