"""CPU FP64 oracle for the assembly-free transient heat solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm call it. It shares no code with the CUDA path (the only common
module is ``workloads``, which draws seeded inputs and holds no FEM arithmetic).

What it computes is the plain definition of the method, not the GPU algorithm:

* ``fem``       -- Q1 element matrices by 2x2x2 Gauss quadrature, global CSR
                   assembly of M and K (§3.1, §3.2 Eq. 1), face flux loads,
                   Dirichlet node sets, and a row-by-row apply for sampled checks.
* ``pcg``       -- Jacobi-preconditioned CG following Algorithm 1 (§3.3), with
                   the readings listed below; dense Cholesky and sparse LU
                   solves of the same systems.
* ``transient`` -- the theta-scheme step system of §3.1,
                   [M/dt + theta K] U^n = [M/dt - (1-theta) K] U^{n-1} + F^n,
                   with symmetric elimination of Dirichlet nodes.

Readings of the paper used here (each also in the design notes):
  * Q1 hexahedra instead of the paper's linear tetrahedra (§4.1).
  * The step system is divided by dt (same solution, same relative tolerances).
  * Stopping rule: r^T P^-1 r <= rtol^2 * b^T P^-1 b (relative, preconditioned),
    checked before every iteration, including the first.
  * delta_old <- delta_new every iteration (standard PCG; Algorithm 1 omits it).
  * True residual r = b - A x when i > 0 and i % 50 == 0.
  * Initial guess x0 = 2 U^{n-1} - U^{n-2} (x0 = U^0 on the first step).
  * Flux F^n is on for steps n <= flux_steps (all steps if flux_steps < 0).
  * Dirichlet faces (not in the paper): rows and columns eliminated; values g.

Pins: every function here is checked in ``tests/test_oracle_pins.py`` against
closed forms (Q1 element matrices, exact discrete eigenmodes of the
theta-scheme, energy balance, patch tests) and against dense direct solves.
"""
