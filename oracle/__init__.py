"""CPU oracle for the explicit RKC / AMG-PCG EQS method (test infrastructure).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may
import it.  The CUDA library never calls it and shares no code with it; the
two meet only in the seeded input generators of ``eqs_inputs``.

Everything is plain FP64 numpy/scipy, written step by step from the paper's
statement of the method (Richter, Schoeps, Clemens, "GPU Accelerated Explicit
Time Integration Methods for Electro-Quasistatic Fields"):

* ``fem``      - P1 element operator K(x)x, assembled K(x) and M (Eq. 1-2,
                 Section III);
* ``system``   - Dirichlet elimination and the right-hand side F(t, y) of the
                 semi-discrete ODE (Eq. 2);
* ``rkc``      - Runge-Kutta-Chebyshev coefficients, stability polynomial and
                 step (Section II, the scheme of ref. [9]);
* ``amg``      - smoothed-aggregation AMG hierarchy and V-cycle used as the
                 constant preconditioner of the multiple right-hand-side
                 M-solve (Section II, Section IV; refs. [6-8]);
* ``pcg``      - preconditioned conjugate gradients (Section IV, ref. [3]);
* ``dtbound``  - a-priori bound of the spectral radius of M^-1 dK/dx and the
                 RKC step at the stability boundary;
* ``spe``      - subspace projection extrapolation start vector (Section IV,
                 Eq. 4-5);
* ``pod``      - POD-MOR start vectors, fixed (MOR) and rolling (MOR2)
                 snapshot sets (Section IV);
* ``mlp``      - the per-node initial-guess network (a project addition with
                 no counterpart in the paper): forward, backward, Adam.

Parity status per function is stated in each module header.
"""
