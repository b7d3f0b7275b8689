"""The CPU oracle against its pins (no GPU).

O1 = direct Eq. (1)/(3), O2 = Eq. (6), O3 = adjoint (transpose of Eq. (5)),
O3f = transpose of the Eq. (6) product, O4 = Eq. (9).
"""
import numpy as np
import pytest

import oracle_pins as P
from oracle import oracle as O

POW2 = [1 << m for m in range(0, 13)]          # 1 .. 4096
ANY_N = [1, 2, 3, 5, 6, 7, 12, 15, 100]        # O1 is defined for every N


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def test_golden_product_is_the_dft():
    """The paper's N = 8 factors (errata fixed) multiply out to E_16 of Eq. (1),
    and the example exactly as printed does not."""
    g = P.load_golden()
    prod = np.eye(16)
    for name in g["procedure"]["order"]:
        prod = P.golden_matrix(name, g) @ prod
    k = np.arange(8)
    e = np.exp(-2j * np.pi * np.outer(k, k) / 8)
    # real 16x16 form on the interleaved pair vector: (a + jb) -> [[Re, -Im], [Im, Re]]
    big = np.zeros((16, 16))
    big[0::2, 0::2] = e.real
    big[0::2, 1::2] = -e.imag
    big[1::2, 0::2] = e.imag
    big[1::2, 1::2] = e.real
    assert np.max(np.abs(prod - big)) < 1e-14
    printed = np.eye(16)
    for name in g["procedure"]["order"]:
        printed = P.golden_matrix("D3_as_printed" if name == "D3" else name, g) @ printed
    assert np.max(np.abs(printed - big)) > 0.1


def test_direct_golden():
    P.pin_golden_n8(O.dft_direct)


def test_dit_golden():
    P.pin_golden_n8(O.dft_factored_dit)


def test_dif_golden():
    P.pin_golden_n8(O.dft_factored_dif)


def test_dit_stages_golden():
    P.pin_dit_stages_golden(O.dit_stages)


def test_direct_numpy_pow2():
    P.pin_numpy_fft(O.dft_direct, POW2)


def test_direct_numpy_any_n():
    P.pin_numpy_fft(O.dft_direct, ANY_N)


def test_dit_numpy():
    P.pin_numpy_fft(O.dft_factored_dit, POW2 + [8192, 65536], batch=2)


def test_dif_numpy():
    P.pin_numpy_fft(O.dft_factored_dif, POW2 + [8192, 65536], batch=2)


def test_closed_forms():
    for fn in (O.dft_direct, O.dft_factored_dit, O.dft_factored_dif):
        P.pin_closed_forms(fn, [1, 2, 4, 8, 16, 64, 256, 1024])


def test_invariants():
    for fn in (O.dft_direct, O.dft_factored_dit, O.dft_factored_dif):
        P.pin_invariants(fn, [2, 4, 8, 32, 128, 512])
    P.pin_invariants(O.dft_factored_dit, [4096, 65536])


def test_integer_bins():
    for fn in (O.dft_direct, O.dft_factored_dit, O.dft_factored_dif):
        P.pin_integer_bins(fn, [2, 4, 8, 16, 32, 64, 1024])


def test_kronecker_eq6():
    for fn in (O.dft_direct, O.dft_factored_dit):
        P.pin_kron_eq6(fn, max_m=4)


def test_kronecker_eq9():
    P.pin_eq9_kron(O.dft_factored_dif, max_m=4)


def test_adjoint_direct():
    P.pin_adjoint(O.dft_direct, O.adjoint_direct, [1, 2, 4, 8, 16, 64, 256])
    P.pin_numpy_ifft_adjoint(O.adjoint_direct, [1, 2, 4, 8, 16, 64, 256, 1024])


def test_adjoint_factored():
    P.pin_adjoint(O.dft_factored_dit, O.adjoint_factored, [2, 4, 8, 64, 1024, 4096])
    P.pin_numpy_ifft_adjoint(O.adjoint_factored, [2, 4, 8, 64, 1024, 4096, 65536])


def test_adjoint_is_transpose_of_forward():
    for n in (2, 4, 8, 16):
        f = P.operator_matrix(O.dft_direct, n)
        a = P.operator_matrix(O.adjoint_direct, n)
        assert np.max(np.abs(a - f.T)) < 1e-12
        assert np.max(np.abs(P.operator_matrix(O.adjoint_factored, n) - f.T)) < 1e-12


def test_direct_bins_matches_direct():
    rng = np.random.default_rng(3)
    xr = rng.standard_normal((3, 64))
    xi = rng.standard_normal((3, 64))
    bins = np.array([0, 5, 16, 63, 32])
    br, bi = O.dft_direct_bins(xr, xi, bins)
    yr, yi = O.dft_direct(xr, xi)
    assert np.array_equal(br, yr[:, bins]) and np.array_equal(bi, yi[:, bins])


def test_factored_rejects_non_pow2():
    with pytest.raises(ValueError):
        O.dft_factored_dit(np.zeros((1, 6)), np.zeros((1, 6)))


def test_threading_does_not_change_results():
    rng = np.random.default_rng(9)
    xr = rng.standard_normal((16, 256))
    xi = rng.standard_normal((16, 256))
    a = O.dft_factored_dit(xr, xi, threads=1)
    b = O.dft_factored_dit(xr, xi, threads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
