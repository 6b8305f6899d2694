"""FP64 CPU oracle for the Kronecker-product demagnetizing operator (arXiv 1212.3509).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables or constants with the CUDA library; both sides take their
inputs from ``synth.py`` only.

Plain numpy/scipy in float64.  Each function cites the part of the paper it
restates.  Modules:

* ``quadrature``  sinc nodes and weights of the Gaussian transform of
                  rho^{-3/2} (Sec. 3.3-3.4, Thm. 1, Eq. gauss_trans, Cor. 3).
* ``generators``  1D cell integrals h^(p)(tau) as Toeplitz generators
                  (Eq. sep_integrands, Eq. f_anal, Sec. 4.2).
* ``full``        the Kronecker operator on full tensors by mode products
                  (Eq. modemul, Eq. kron_operator), its adjoint, and the dense
                  quadrature matrix for tiny grids.
* ``exact``       the exact collocation matrix entries (Eq. matrix_op) by the
                  closed-form potential of a uniformly charged rectangle, and
                  the uniformly magnetized box.
* ``structured``  CP / Tucker / TT application (Eq. kron_eval_cp,
                  Eq. kron_eval_tuck, Eq. tt_3d_2) by direct Toeplitz matvecs.
* ``energy``      second-order stray field, demag energy and its gradient.

Readings of the paper used throughout (each is argued where it is used):

* sign: phi = +(1/4pi) int m . (x-y)/|x-y|^3 (the sign that satisfies
  Delta phi = div m with h_d = -grad phi, Eq. poisson / Eq. intop1);
* R = 2M+1 symmetric sinc nodes; the zero node drops out and +/-k fold into
  M terms with weights omega_k = 2 theta cosh t_k sinh^2 t_k (the trapezoid
  step theta and the fold factor 2 are part of the rule, Eq. sinc_int);
* theta = c0 ln(M)/M with the paper's "R" in that formula read as the number
  of non-zero terms M (Cor. 3: "R+1-term ... omitting the first");
* the domain is scaled so that its longest edge is 1 before the nodes are
  applied (Sec. 3.4), and phi is scaled back linearly.
"""

from . import quadrature, generators, full, exact, structured, energy  # noqa: F401
