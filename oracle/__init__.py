"""CPU FP64 oracle for the IFFD-preconditioned PCG hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares
no code with the CUDA library (``paper_2512_20269_gb300``) and never imports it.

What it computes, plainly and slowly, in float64 (numpy / scipy):

* ``splines``   -- open knot vector, Cox-de Boor values and derivatives,
                   Gauss-Legendre quadrature, 1D mass ``M`` and stiffness ``K``
                   (Section 2), the symmetric cardinal B-spline recurrence
                   (Lemma 3, eq. "cardinal") and the coefficient-weighted 1D
                   matrices used by the variable-coefficient operator.
* ``splitting`` -- the splitting S = S^reg + S^out (Section 4, eqs.
                   "splitting", "reg_space", "reg_space_dim"), the special basis
                   of Section 6 (eqs. "Btilde", "special_basis"), the matrix
                   U_reg of Table 1, the numeric D~_reg / Lambda_reg (end of
                   Section 6), Q_out / Lambda_out (eq. "eigendecomposition_out"),
                   Q~ and Lambda~ (Section 4), and the closed forms of Lemma 3
                   and Theorem 3.
* ``operators`` -- the IFFD preconditioner (eq. "preconditioner"), the exact
                   Fast Diagonalization (eq. "exact_diagonalization"), the
                   Kronecker stiffness (eq. "system_matrix"), the separable
                   variable-coefficient stiffness, dense assembly for tiny
                   grids, textbook PCG (Section 3) and spectral estimates.
* ``general``   -- the stiffness of -div(C grad u) with a general symmetric
                   coefficient C(x) sampled at the tensor Gauss points (Section
                   2's Galerkin form; a geometry map of Section 7 pulled back to
                   the parameter domain has this form), by the plain
                   sum over derivative directions of G_k^T diag(w C_kl) G_l.

Pins (what fixes each function independently of itself) live in
``tests/test_oracle_*.py``. Every oracle function is pinned; the only values
the paper does not fix are the absolute scaling of D~_reg (Lemma 3's printed
normalisation is garbled; it is pinned here by a derivation from the periodic
symbols, and by the numeric route) and every time/throughput number.
"""

from . import splines, splitting, operators  # noqa: F401
