"""FP64 CPU oracle for the Darcy-Boussinesq state solve, adjoint and sensitivities.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct restatement of
the method of Pollini, Sigmund, Andreasen & Alexandersen, "A 'poor man's' approach for
high-resolution three-dimensional topology optimization of natural convection problems"
(arXiv 1904.00182). Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it. The CUDA library never calls it
and shares no code with it: the only common module is ``synthetic`` (seeded input
generators, which hold none of the method's arithmetic).

Layout of the oracle (each function cites the passage it follows):

* ``mesh``       structured hex grid, connectivity, Dirichlet sets    (Sec. 4, Sec. 6.2, App. A)
* ``element``    Q1 tables, SUPG element residual / linearisation     (App. A, Eqs. weakstable,
                 / Jacobian / design derivatives                       govequation, finalsyseq)
* ``materials``  RAMP interpolation, kappa_f tuning formula           (Eqs. condRAMP, permRAMP,
                                                                       nusselt5)
* ``pde_filter`` Helmholtz (PDE) density filter and its transpose     (Sec. 5.1)
* ``solver``     assembly, damped Newton, adjoint, sensitivities,     (Sec. 5.1, 5.4, Eqs. objdiscr,
                 objective                                             optprob)

Equations are cited by the label they carry in the paper's LaTeX source (e.g. Eq. nusselt5);
sections by their number and title in the paper.

Every floating-point computation is FP64 (NumPy / SciPy sparse direct solves).

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against closed forms, invariants, finite differences or the
paper's Table 2, except the paper's printed objective values (Tables 5-10), which need
optimised designs that the paper does not ship: those are "parity unpinned" and are not
used by any test.
"""

from . import mesh, element, materials, pde_filter, solver  # noqa: F401
from .mesh import Mesh  # noqa: F401
from .solver import Problem, Params  # noqa: F401
