"""Pins for the CPU oracle: checks against things other than the oracle itself.

Each ``pin_*`` function raises AssertionError when the oracle it is given
disagrees with what the paper or the mathematics fixes:

  * the paper's worked example N = 8 (Section III, Eqs. (7)-(8)), transcribed in
    ``golden/paper_n8.json`` -- the whole product and every intermediate stage;
  * ``numpy.fft.fft`` / ``ifft`` (a library routine that computes Eq. (1));
  * closed forms: delta -> ones, constant -> N delta, tone -> N delta_k0;
  * Parseval, linearity, F(F(x))[n] = N x[(-n) mod N];
  * the factors of Eq. (6) assembled with Kronecker products (as the paper
    writes them) and multiplied out, N <= 16;
  * exact integer sums at bins 0, N/4, N/2, 3N/4 for integer inputs;
  * adjoint identities: <F x, g> = <x, F^H g>, F^H F = N I, and
    F^H(x^r, x^i) = swap(F(x^i, x^r)).

They take the oracle's functions as arguments so the same pins can be run on
copies of the oracle with a planted mistake (tests/test_oracle_mutations.py).
"""
from __future__ import annotations

import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
R = 1.0 / np.sqrt(2.0)


def rel_l2(yr, yi, rr, ri) -> float:
    num = np.sum((np.asarray(yr, np.float64) - rr) ** 2 + (np.asarray(yi, np.float64) - ri) ** 2)
    den = np.sum(np.asarray(rr, np.float64) ** 2 + np.asarray(ri, np.float64) ** 2)
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))


def _rand(n, batch, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((batch, n)), rng.standard_normal((batch, n))


# ---------------------------------------------------------------- golden --
def _scalar(v):
    if isinstance(v, str):
        return {"r": R, "-r": -R}[v]
    return float(v)


def _named(name: str, g: dict) -> np.ndarray:
    if name.startswith("I") and name[1:].isdigit():
        return np.eye(int(name[1:]))
    if name == "H2":
        return np.array(g["H2"]["value"], dtype=float)
    if name == "S8":
        cols = g["S8_columns"]["value"]
        s = np.zeros((8, 8))
        for k, c in enumerate(cols):
            s[k, c] = 1.0
        return s
    if name.startswith("omega "):
        key = name.split()[1]
        return np.array([[_scalar(v) for v in row] for row in g["omega"][key]])
    return golden_matrix(name, g)


def _build(spec, g) -> np.ndarray:
    if isinstance(spec, str):
        return _named(spec, g)
    if "kron" in spec:
        out = np.eye(1)
        for part in spec["kron"]:
            out = np.kron(out, _build(part, g))
        return out
    if "dsum" in spec:
        blocks = [_build(part, g) for part in spec["dsum"]]
        n = sum(b.shape[0] for b in blocks)
        out = np.zeros((n, n))
        o = 0
        for b in blocks:
            out[o:o + b.shape[0], o:o + b.shape[0]] = b
            o += b.shape[0]
        return out
    raise ValueError(f"bad golden spec {spec}")


def load_golden() -> dict:
    with open(os.path.join(GOLDEN, "paper_n8.json")) as f:
        return json.load(f)


def golden_matrix(name: str, g: dict | None = None) -> np.ndarray:
    g = load_golden() if g is None else g
    return _build(g[name], g)


def interleave(xr, xi) -> np.ndarray:
    v = np.empty(2 * len(xr))
    v[0::2] = xr
    v[1::2] = xi
    return v


def operator_matrix(fn, n: int) -> np.ndarray:
    """The 2N x 2N real matrix of ``fn`` on the interleaved pair vector."""
    m = np.zeros((2 * n, 2 * n))
    for col in range(2 * n):
        e = np.zeros(2 * n)
        e[col] = 1.0
        yr, yi = fn(e[0::2].copy(), e[1::2].copy())
        m[:, col] = interleave(yr, yi)
    return m


def pin_golden_n8(fn):
    """fn on N = 8 equals the paper's product W3 D3 W2 D2 W1 D1 S16."""
    g = load_golden()
    prod = np.eye(16)
    for name in g["procedure"]["order"]:
        prod = golden_matrix(name, g) @ prod
    got = operator_matrix(fn, 8)
    assert np.max(np.abs(got - prod)) < 1e-13, "differs from the paper's N=8 example"


def pin_dit_stages_golden(dit_stages):
    """Every intermediate vector of Eq. (6) at N = 8 equals the paper's factors
    applied one at a time."""
    g = load_golden()
    rng = np.random.default_rng(11)
    x2 = rng.standard_normal(16)
    stages = dit_stages(x2)
    v = x2.copy()
    for k, name in enumerate(g["procedure"]["order"]):
        v = golden_matrix(name, g) @ v
        assert np.max(np.abs(stages[k] - v)) < 1e-13, f"stage {k} ({name}) differs"


# ------------------------------------------------------------- library --
def pin_numpy_fft(fn, sizes, batch=3, tol=1e-12):
    for n in sizes:
        xr, xi = _rand(n, batch, 100 + n)
        yr, yi = fn(xr, xi)
        ref = np.fft.fft(xr + 1j * xi, axis=-1)
        err = rel_l2(yr, yi, ref.real, ref.imag)
        assert err < tol, f"N={n}: rel err {err:.3e} vs numpy.fft.fft"


def pin_numpy_ifft_adjoint(adj, sizes, batch=3, tol=1e-12):
    """The adjoint is the unnormalised inverse: N * ifft."""
    for n in sizes:
        xr, xi = _rand(n, batch, 200 + n)
        yr, yi = adj(xr, xi)
        ref = n * np.fft.ifft(xr + 1j * xi, axis=-1)
        err = rel_l2(yr, yi, ref.real, ref.imag)
        assert err < tol, f"N={n}: rel err {err:.3e} vs N*numpy.fft.ifft"


# ----------------------------------------------------------- closed forms --
def pin_closed_forms(fn, sizes, tol=1e-12):
    for n in sizes:
        z = np.zeros(n)
        # delta -> all ones
        d = z.copy()
        d[0] = 1.0
        yr, yi = fn(d, z)
        assert np.max(np.abs(yr - 1.0)) < tol and np.max(np.abs(yi)) < tol, f"delta N={n}"
        # constant c -> N c delta
        c = 0.75 - 0.5j
        yr, yi = fn(np.full(n, c.real), np.full(n, c.imag))
        ref = np.zeros(n, complex)
        ref[0] = n * c
        assert np.max(np.abs(yr + 1j * yi - ref)) < tol * n, f"constant N={n}"
        # tone exp(+j 2 pi k0 t / N) -> N delta_{k0}
        for k0 in sorted({0, 1 % n, n // 3, n - 1}):
            t = np.arange(n)
            tone = np.exp(2j * np.pi * k0 * t / n)
            yr, yi = fn(tone.real.copy(), tone.imag.copy())
            ref = np.zeros(n, complex)
            ref[k0] = n
            assert np.max(np.abs(yr + 1j * yi - ref)) < 1e-10 * n, f"tone k0={k0} N={n}"


def pin_invariants(fn, sizes, tol=1e-12):
    for n in sizes:
        xr, xi = _rand(n, 2, 300 + n)
        yr, yi = fn(xr, xi)
        # Parseval: sum |y|^2 = N sum |x|^2
        lhs = np.sum(yr ** 2 + yi ** 2, axis=-1)
        rhs = n * np.sum(xr ** 2 + xi ** 2, axis=-1)
        assert np.max(np.abs(lhs - rhs) / rhs) < tol, f"Parseval N={n}"
        # linearity
        ur, ui = _rand(n, 2, 400 + n)
        a, b = 1.5, -0.25
        zr, zi = fn(a * xr + b * ur, a * xi + b * ui)
        vr, vi = fn(ur, ui)
        err = rel_l2(zr, zi, a * yr + b * vr, a * yi + b * vi)
        assert err < tol, f"linearity N={n}"
        # F(F(x))[t] = N x[(-t) mod N]
        wr, wi = fn(yr, yi)
        idx = (-np.arange(n)) % n
        err = rel_l2(wr, wi, n * xr[:, idx], n * xi[:, idx])
        assert err < tol, f"F(F(x)) N={n}"


def pin_integer_bins(fn, sizes):
    """Integer inputs: bins 0, N/4, N/2, 3N/4 are integer sums whose kernels
    are 1, (-j)^t, (-1)^t, (+j)^t; they must come out exactly."""
    rng = np.random.default_rng(5)
    for n in sizes:
        xr = rng.integers(-8, 9, size=n).astype(float)
        xi = rng.integers(-8, 9, size=n).astype(float)
        yr, yi = fn(xr, xi)
        x = xr.astype(np.int64) + 1j * xi.astype(np.int64)
        t = np.arange(n)
        kernels = {0: np.ones(n, complex), n // 2: (-1.0) ** t}
        if n % 4 == 0:
            kernels[n // 4] = (-1j) ** t
            kernels[3 * n // 4] = (1j) ** t
        for k, ker in kernels.items():
            exact = np.sum(x * np.round(ker.real) + x * 1j * np.round(ker.imag))
            # exactly: every term is an integer times 0 or +-1
            assert yr[k] == exact.real and yi[k] == exact.imag, f"integer bin k={k} N={n}"


# ------------------------------------------------------ Kronecker form --
def eq6_matrices(m: int):
    """Eq. (6) assembled from its printed definitions (with I_{2^{m-i}}):
    returns [S, D(1), W(1), ..., D(m), W(m)] as dense 2^{m+1} matrices."""
    n = 1 << m
    s = np.zeros((n, n))
    for k in range(n):
        rev = int(format(k, f"0{m}b")[::-1], 2) if m > 0 else 0
        s[k, rev] = 1.0
    mats = [np.kron(s, np.eye(2))]
    h2 = np.array([[1.0, 1.0], [1.0, -1.0]])
    for i in range(1, m + 1):
        rr = 1 << (i - 1)
        blocks = [np.eye(2 * rr)]
        for q in range(rr):
            th = 2 * np.pi * q / (1 << i)
            blocks.append(np.array([[np.cos(th), np.sin(th)], [-np.sin(th), np.cos(th)]]))
        size = sum(b.shape[0] for b in blocks)
        dsmall = np.zeros((size, size))
        o = 0
        for b in blocks:
            dsmall[o:o + b.shape[0], o:o + b.shape[0]] = b
            o += b.shape[0]
        mats.append(np.kron(np.eye(1 << (m - i)), dsmall))
        mats.append(np.kron(np.kron(np.eye(1 << (m - i)), h2), np.eye(1 << i)))
    return mats


def pin_kron_eq6(fn, max_m=4):
    for m in range(1, max_m + 1):
        prod = np.eye(2 << m)
        for mat in eq6_matrices(m):
            prod = mat @ prod
        got = operator_matrix(fn, 1 << m)
        assert np.max(np.abs(got - prod)) < 1e-12, f"Kronecker Eq. (6) m={m}"


def pin_eq9_kron(fn, max_m=4):
    """Eq. (9): S D(1) W(1) ... D(m) W(m), same factors as Eq. (6)."""
    for m in range(1, max_m + 1):
        mats = eq6_matrices(m)
        s, rest = mats[0], mats[1:]
        prod = np.eye(2 << m)
        for i in range(m, 0, -1):
            d, w = rest[2 * (i - 1)], rest[2 * (i - 1) + 1]
            prod = d @ (w @ prod)
        prod = s @ prod
        got = operator_matrix(fn, 1 << m)
        assert np.max(np.abs(got - prod)) < 1e-12, f"Kronecker Eq. (9) m={m}"


# --------------------------------------------------------------- adjoint --
def pin_adjoint(fwd, adj, sizes, tol=1e-12):
    for n in sizes:
        xr, xi = _rand(n, 2, 500 + n)
        gr, gi = _rand(n, 2, 600 + n)
        yr, yi = fwd(xr, xi)
        ar, ai = adj(gr, gi)
        lhs = np.sum(yr * gr + yi * gi, axis=-1)
        rhs = np.sum(xr * ar + xi * ai, axis=-1)
        scale = np.sqrt(np.sum(yr ** 2 + yi ** 2, axis=-1) * np.sum(gr ** 2 + gi ** 2, axis=-1))
        assert np.max(np.abs(lhs - rhs) / scale) < tol, f"<Fx,g> != <x,F^H g> N={n}"
        br, bi = adj(yr, yi)
        assert rel_l2(br, bi, n * xr, n * xi) < tol, f"F^H F != N I, N={n}"
        sr, si = fwd(xi, xr)
        assert rel_l2(si, sr, *adj(xr, xi)) < tol, f"swap identity N={n}"
