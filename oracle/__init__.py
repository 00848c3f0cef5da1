"""CPU FP64 oracle for the decoupled (interface-strain) Stokes operator and its multigrid.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plainly written reference that the
CUDA path is checked against.  Only the test-suite, the smoke check and the benchmark's CPU
baseline leg may import it; the library itself never does, and it shares no code with the
CUDA path (inputs come from ``paper_1604_07994_gb300.workloads``, which holds no method
arithmetic).

It follows the paper (Huber, Ruede, Waluga, Wohlmuth, arXiv:1604.07994) directly:

* ``mesh``     - Kuhn 6-tetrahedra split of a uniform hexahedral grid, generic P1 geometry
* ``forms``    - global sparse assembly of a_tr (eq. newbil), a_sym (eq. standard), the
                 gradient form, a_dev, b(v,q) = -(div v, q), the PSPG stabilisation C and
                 the right-hand side; boundary conditions (eq. boundary); interface rows
                 (Sec. 2.2, eq. equivalence-stencil)
* ``transfer`` - nested P1 prolongation / restriction between uniformly refined levels
* ``solvers``  - sparse direct solve, the Uzawa smoother (eq. Uzawa_smooth) and the
                 variable V-cycle of Sec. 5
* ``nn``       - the learned-initial-guess network (no counterpart in the paper): 3x3x3
                 convolutions, pooling, up-sampling, loss, backward pass and Adam

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms, the paper's
lemmas and identities, convergence to exact solutions, and the values the paper prints (the
relative differences of the layers and columns tables in Sec. 4.2.3-4.2.4, the V-cycle rates
of Sec. 5; ``tests/golden/``); see each docstring for the passage it follows.
"""
