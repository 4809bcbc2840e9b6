"""Acceptance checks of the parity tests (host only, no GPU needed).

The bound the method must meet is |C_gpu - C_oracle| <= TOL * sum|terms|,
where sum|terms| is the oracle's magnitude recursion (the same recursion run
on |G||S||S||S| blocks and |X||Y| products, summed over the sites of a slab):
TOL = 1e-13 for the FP64 path, 1e-6 for the FP32-product / compensated path.

That bound only means something where a wrong answer exceeds it. On random
Gaussian propagators the correlator cancels by many orders of magnitude
against sum|terms| (8Be: |C| / sum|terms| ~ 5e-14), so a zero output would
pass. Every comparison therefore also requires the reference itself to clear
the bound by MARGIN: max |C_ref| / sum|terms| >= MARGIN * TOL over the
compared entries. With MARGIN = 200 a zero or negated output fails, and so
does one perturbed by 1 % (its largest entry then misses by at least twice
the bound). A comparison that cannot fail raises NotDiscriminating, which
marks a test whose input has to change (near-identity propagators,
``synth.field(..., eps=...)``), not a kernel error.
"""
import numpy as np

TOL = {0: 1e-13, 1: 1e-6}
MARGIN = 200.0


class NotDiscriminating(AssertionError):
    pass


def margin(ref, scale) -> float:
    """max |ref| / scale over the compared entries."""
    ref = np.asarray(ref)
    sc = np.broadcast_to(np.asarray(scale, dtype=np.float64), ref.shape)
    return float(np.max(np.abs(ref) / sc))


def check(got, ref, scale, precision: int, what="") -> float:
    """Assert |got - ref| <= TOL * scale for every entry and that the
    comparison discriminates; returns max |got - ref| / scale."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    sc = np.broadcast_to(np.asarray(scale, dtype=np.float64), ref.shape)
    m = margin(ref, sc)
    if not m >= MARGIN * TOL[precision]:
        raise NotDiscriminating(f"{what}: max|ref|/scale = {m:.3e} < {MARGIN} x {TOL[precision]:.0e}")
    err = float(np.max(np.abs(got - ref) / sc))
    assert err <= TOL[precision], (what, precision, err)
    return err


def check_rel(got, ref, rtol: float, what="") -> float:
    """Assert |got - ref| <= rtol * sum |ref| (a closed form whose own scale
    is the sum of the magnitudes of its terms); returns the relative error.
    rtol must stay below 1 / MARGIN so that a 1 % error fails."""
    assert rtol * MARGIN <= 1.0, (what, rtol)
    got = np.asarray(got)
    ref = np.asarray(ref)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert err <= rtol, (what, err, rtol)
    return err
