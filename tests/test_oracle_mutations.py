"""Planted mistakes in the oracle are caught by its pins (no GPU).

Each case compiles a copy of the CPU oracle with one deliberate error (see the
SDFT_ORACLE_MUTATION hooks in oracle/sdft_oracle.c) and checks that the pins
reject it.  This shows the pins would catch a dropped term, a wrong sign, a
missing permutation or a misplaced twiddle.
"""
import functools

import pytest

import oracle_pins as P
from oracle import oracle as O

CASES = {
    1: ("sign of S in Eq. (3) flipped", "dft_direct"),
    2: ("omega^(i,q) conjugated", "dft_factored_dit"),
    3: ("bit-reversal S dropped", "dft_factored_dit"),
    4: ("D(i) applied to the top half of each block", "dft_factored_dit"),
    5: ("adjoint computed as the forward map", "adjoint_direct"),
}


def _pins_for(name, fn):
    if name.startswith("adjoint"):
        fwd = O.dft_direct
        return [lambda: P.pin_adjoint(fwd, fn, [4, 8, 16]),
                lambda: P.pin_numpy_ifft_adjoint(fn, [4, 8, 16])]
    return [lambda: P.pin_golden_n8(fn),
            lambda: P.pin_numpy_fft(fn, [4, 8, 16, 64]),
            lambda: P.pin_closed_forms(fn, [4, 8, 16])]


@pytest.mark.parametrize("mutation", sorted(CASES))
def test_pins_catch_planted_mistake(mutation):
    what, name = CASES[mutation]
    O.build(mutation)
    fn = functools.partial(getattr(O, name), mutation=mutation)
    failed = 0
    for pin in _pins_for(name, fn):
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed > 0, f"no pin caught the planted mistake: {what}"
    # the unmutated oracle passes the same pins
    for pin in _pins_for(name, getattr(O, name)):
        pin()
