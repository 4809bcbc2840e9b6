"""The parity checker rejects wrong answers (host only).

On the inputs the GPU parity tests use, a zero, negated or 1 %-perturbed
correlator fails ``parity.check``, and a comparison on inputs where the
bound cannot fail is refused. The references are the oracle's own values.
"""
import numpy as np
import pytest

import parity
import synth
from gpu_helpers import oracle_plan, oracle_slab


def _ref(n_p, n_n, D, spins, dims, eps, seed=31):
    field = synth.field(seed, 1, 1, dims, 0.4, eps=eps)
    comps = None if spins is None else spins
    from oracle import recursion
    plan = oracle_plan(n_p, n_n, D, comps if comps is not None else recursion.Plan(n_p, n_n, D).requests)
    return oracle_slab(plan, field[0, 0], dims, [(0, 0, 0), (1, 0, 0)])


CASES = [
    (1, 1, 2, None, (2, 2, 3)),
    (2, 1, 2, None, (2, 2, 3)),
    (2, 2, 2, None, (2, 2, 3)),
    (2, 2, 4, [((0, 1, 0, 1), (0, 1, 0, 1))], (1, 1, 2)),
]


@pytest.mark.parametrize("n_p,n_n,D,spins,dims", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_wrong_answers_fail(n_p, n_n, D, spins, dims, precision):
    ref, scale = _ref(n_p, n_n, D, spins, dims, eps=0.05)
    rng = np.random.default_rng(3)
    noise = parity.TOL[precision] * 0.1 * scale[None, :] * (rng.standard_normal(ref.shape) > 0)
    parity.check(ref + noise, ref, scale, precision)  # within the bound: passes
    for wrong in (np.zeros_like(ref), -ref, ref * 1.01):
        with pytest.raises(AssertionError) as ei:
            parity.check(wrong, ref, scale, precision)
        assert not isinstance(ei.value, parity.NotDiscriminating)


def test_gaussian_mixed_comparisons_are_refused():
    """On Gaussian propagators the mixed bound cannot fail for 4He: the
    checker says so instead of passing a zero output."""
    ref, scale = _ref(2, 2, 4, [((0, 1, 0, 1), (0, 1, 0, 1))], (1, 1, 2), eps=None)
    with pytest.raises(parity.NotDiscriminating):
        parity.check(np.zeros_like(ref), ref, scale, 1)
    # FP64 still discriminates on the same input
    with pytest.raises(AssertionError) as ei:
        parity.check(np.zeros_like(ref), ref, scale, 0)
    assert not isinstance(ei.value, parity.NotDiscriminating)


def test_relative_check():
    ref = np.array([3.0 + 1j, -2.0, 0.5j])
    parity.check_rel(ref * (1 + 1e-9), ref, 1e-8)
    for wrong in (np.zeros_like(ref), -ref, ref * 1.01):
        with pytest.raises(AssertionError):
            parity.check_rel(wrong, ref, 1e-5)
    with pytest.raises(AssertionError):
        parity.check_rel(ref, ref, 0.1)  # a tolerance that would pass a 1 % error
