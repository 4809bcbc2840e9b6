"""Closed-form counts of the paper (oracle, test infrastructure).

Test infrastructure only (see ``oracle/__init__.py``).

* multinomial C(n_1, ..., n_m) = (sum n)! / prod n_i! (Sec. 3 eq. gen_P);
* P(n_P, n_N) upper bound of stage components and Q_P / Q_N upper bounds of
  operations (Sec. 7), with D = 4 (relativistic) or 2 (nonrelativistic);
* maximal number of independent components of L (Sec. 3);
* naive operation count n_u! n_d! g^(2A) with g nonzero G entries per spin
  (Sec. 1, cost of the explicit Wick sum; the tables' naive column);
* UCA list sizes N_list = n_u! n_d! N_L, N_contr = N_list / 2^A (Sec. 8).
"""
from __future__ import annotations

from math import factorial


def multinomial(*parts) -> int:
    if any(p < 0 for p in parts):
        return 0
    n = factorial(sum(parts))
    for p in parts:
        n //= factorial(p)
    return n


def p_bound(n_p: int, n_n: int, D: int) -> int:
    """Upper bound of the components of F_-^(n_P, n_N) (Sec. 7)."""
    return (multinomial(n_p, D - n_p) * multinomial(n_n, D - n_n) *
            multinomial(2 * n_p + n_n, 3 * D - 2 * n_p - n_n) * multinomial(n_p + 2 * n_n, 3 * D - n_p - 2 * n_n))


def q_bound(n_p: int, n_n: int, D: int, add: str) -> int:
    """Upper bound of the operations adding a proton ('P') or neutron ('N')
    to F_-^(n_P, n_N) (Sec. 7)."""
    nu, nd = 2 * n_p + n_n, n_p + 2 * n_n
    if add == "P":
        return (multinomial(n_p, 1, D - 1 - n_p) * multinomial(n_n, D - n_n) *
                multinomial(nu, 2, 3 * D - 2 - nu) * multinomial(nd, 1, 3 * D - 1 - nd))
    return (multinomial(n_p, D - n_p) * multinomial(n_n, 1, D - 1 - n_n) *
            multinomial(nu, 1, 3 * D - 1 - nu) * multinomial(nd, 2, 3 * D - 2 - nd))


def q_sum_along(path, D: int) -> int:
    """Sum of the Q bounds along a recursion path ('P'/'N' letters)."""
    n_p = n_n = 0
    tot = 0
    for i, b in enumerate(path):
        if i > 0:
            tot += q_bound(n_p, n_n, D, b)
        if b == "P":
            n_p += 1
        else:
            n_n += 1
    return tot


def naive_ops(n_p: int, n_n: int, D: int) -> int:
    """n_u! n_d! g^(2A): g = 24 (rel) or 12 (nonrel) nonzero G entries per spin."""
    g = 24 if D == 4 else 12
    A = n_p + n_n
    return factorial(2 * n_p + n_n) * factorial(n_p + 2 * n_n) * g ** (2 * A)
