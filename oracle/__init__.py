"""Independent CPU oracle for the half-range finite-difference lattice Boltzmann march.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or executes anything in this package; only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
do.  The oracle shares no code, header, table or constant with the CUDA path.

Contents (each function cites the passage of Ghiroldi & Gibelli,
"A finite-difference lattice Boltzmann approach for gas microflows",
arXiv:1308.0692, that it follows):

* ``quadrature``    -- half-range / full-range Gauss-Hermite rules in
                       extended precision (Table 1; Golub-Welsch on the
                       recurrence for the weight exp(-xi^2/2)).
* ``march``         -- plain FP64 C implementation of the fully discrete
                       scheme (Eqs. 1, 5-9 with first-order splitting,
                       first-order upwind transport, explicit Euler
                       relaxation), loaded through ctypes.
* ``couette_exact`` -- semi-discrete (exact in space and time) steady Couette
                       solution for any half-range set, and the paper's
                       closed form for D2Q^h_16 (Eqs. 10-11).
* ``fixed_point``   -- direct sparse solve of the fully discrete steady state
                       (the limit the march converges to), assembled as
                       matrices independently of the C loops.

Parity status: every function is pinned by tests under ``tests/`` that do not
use the oracle itself as the reference (Table 1, closed forms, exactness,
conservation, symmetry, grid convergence); see the module headers.
"""
