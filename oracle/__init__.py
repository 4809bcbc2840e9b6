"""CPU oracle for the recursive multibaryon contraction (test infrastructure).

This package is TEST INFRASTRUCTURE ONLY. Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import, call, link or execute anything in it. The
product path (the ``paper_1301_4895_gb300`` package and its CUDA library)
never does, and shares no code, table or helper with it.

Three independent forms of the same exact result (the method reorganises
Wick's theorem without approximation, Sec. 2 eqs. f_L_contr / tensor_L):

* O1 ``wick``      - the plain Wick definition: every sink and source
  spinor-colour assignment allowed by the G tensors (eq. def_g) times the
  signed sum over all same-flavour quark permutations (Sec. 1 eq.
  C_baryons, Sec. 2). Tiny inputs only (A <= 3).
* O2 ``minors``    - the same sum grouped by the sets of occupied indices:
  C = sum L(delta; U', D') L(alpha; U, D) det S_u[U'; U] det S_d[D'; D],
  with L written out from eq. tensor_L by brute-force enumeration.
* O3 ``recursion`` - the method in the paper's order (Sec. 3-4, 7): blocks
  (Sec. 2), antisymmetric components (Sec. 3), the bullet recursion for L
  (eq. recr_L) and F_- (eq. recr_F) with backward pruning (Sec. 3), the
  contraction eq. C_final. Plain C, compiled from ``recursion.c``.

Conventions the paper leaves open are fixed in ``gamma.py`` and listed there.
"""
