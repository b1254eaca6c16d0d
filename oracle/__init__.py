"""Plain FP64 CPU oracle for the explicit CG Euler right-hand side, DSS, inverse
mass and SSP-RK3 update of Kang, Giraldo & Camp (arXiv 2504.08157).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA path (no kernels,
tables, constants or helpers); the only thing both sides consume is the seeded
input generators in ``inputs/``, which hold none of the method's arithmetic.

The oracle is the method written out as the paper states it, step by step, in
numpy float64:

* ``lgl``    -- Legendre-Gauss-Lobatto nodes, weights and the nodal derivative
                matrix of the tensor-product Lagrange basis (Sec. 2.2, Eq. 5).
* ``mesh``   -- hexahedral elements of a (possibly affinely sheared) box, the
                local-to-global map ``intma`` (Alg. 1, Alg. 3) and per-node
                metric terms and Jacobians (Eq. 5, Eq. 8).
* ``euler``  -- the equation of state (Eq. 3), the conservative restatement of
                Eq. 1 and the CG right-hand side: gather (Alg. 1), reference
                derivatives (Alg. 2), pointwise S(q), quadrature weight times
                Jacobian (Eq. 8), DSS (Eqs. 9-11, Alg. 3 without atomics) and
                the inverse diagonal mass matrix (Eq. 12).
* ``ssprk3`` -- the three-stage strong-stability-preserving Runge-Kutta
                update (Shu-Osher form) that advances Eq. 12.
* ``closure`` -- the learned subgrid closure's pieces (not in the paper):
                per-node features (state, assembled gradients, heating),
                fine-to-coarse restriction by the elements' Lagrange
                interpolants, the 21-64-64-5 SiLU network with its
                back-propagated gradient, Adam, and the bfloat16 inference
                precision.
* ``dynamics`` -- the paper's remaining terms: the weak CG Laplacian with
                the tensor viscosity of Sec. 2.4, fourth-order
                hyper-diffusion (Eq. 14), the top sponge (Sec. 4.1) and the
                RI-velocity diagnostic (Sec. 5).
* ``imex``    -- the IMEX ARK2 time integrator of Sec. 2.3 with the linear
                fast-wave operator and Krylov stage solves.

Every function cites the passage it follows.  The pins that tie each function
to something other than itself live in ``tests/test_oracle_*.py``.

Parity status: every function here is pinned (closed forms, polynomial
exactness, brute-force assembly, a manufactured solution derived symbolically
from Eq. 1, conservation and rest-state invariants, the SSP-RK3 amplification
polynomial, inertial rotation; for the closure: finite-difference
gradients with planted mistakes, closed forms of the network and of Adam's
first step, bfloat16 ties, polynomial exactness of features and
restriction; for the dynamics: conservation, symmetry and definiteness of the
weak Laplacian, exact interior second derivatives of quadratics, spectral
convergence and the k^4 damping of a Fourier mode, the tensor's closed form,
the sponge profile, solid-body rotation for the RI velocity; for IMEX: the
tableau's order conditions, both stability functions, second-order
convergence with a planted wrong gamma losing it, the dense-solve step, and
the linear operator as the derivative of S at rest).  The synthetic config inputs themselves
(vortex, heating cells) are inputs, not oracle functions.
"""

from . import lgl, mesh, euler, ssprk3, closure, dynamics, imex  # noqa: F401
