"""Host-side pieces of bench.py (no GPU): the accuracy helpers, the CPU
baseline leg and the argument contract."""
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_accuracy_helpers():
    rng = np.random.default_rng(11)
    xr, xi = rng.standard_normal((5, 32)), rng.standard_normal((5, 32))
    f = np.fft.fft(xr + 1j * xi)
    exact = bench._rel_l2(*bench._err_sums(f.real, f.imag, xr, xi))
    assert exact["rel_l2"] == 0.0 and exact["worst_transform"] == 0.0
    # a relative error of 1e-6 on one row's real part
    gr = f.real.copy()
    gr[2] *= 1 + 1e-6
    num, den = bench._err_sums(gr, f.imag, xr, xi)
    out = bench._rel_l2(num, den)
    want_row = 1e-6 * np.linalg.norm(f.real[2]) / np.linalg.norm(f[2])
    assert np.isclose(out["worst_transform"], want_row, rtol=1e-6)
    assert out["rel_l2"] < out["worst_transform"]
    # a single row (1-D) works too
    one = bench._rel_l2(*bench._err_sums(f.real[0], f.imag[0], xr[0], xi[0]))
    assert one["rel_l2"] == 0.0


def test_cpu_baseline_leg_reports_its_sample():
    r = bench.cpu_oracle_rate(target_s=0.2, max_batch=256)
    assert r["kind"] == "oracle" and r["unit"] == "Gpts/s" and r["value"] > 0
    assert r["cores"] >= 1 and "float64" in r["sample"]
    assert r["one_core"]["value"] > 0
    assert r["float32"]["value"] > 0 and "float32" in r["float32"]["sample"]


def test_warmup_contract():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True)
    assert p.returncode != 0 and "--warmup must be >= 3" in p.stderr


def test_source_hash_ignores_comments_only():
    a = "int f(int x) { return x + 1; }  // one\n/* two */"
    b = "/* another */ int f(int x)\n{ return x + 1; } // three"
    c = "int f(int x) { return x + 2; }"
    assert bench._code_only(a) == bench._code_only(b) != bench._code_only(c)
    # the stored traffic figure belongs to the kernel as it is
    assert bench._kernel_source_hash() == bench.NCU_TRAFFIC["fwd"]["hash"]
