"""Plain FP64 CPU oracle for the fast spectral Boltzmann collision operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library and its
Python binding) imports, links or executes this package.  Only the test suite, the
``smoke()`` check of ``__graft_entry__`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may use it.

What it computes (Dimarco, Loubere, Narski, Rey, "An efficient numerical method for
solving the Boltzmann equation in multidimensions", arxiv 1608.08009):

* ``grid``      -- velocity grid, wave numbers, direction sets on the half sphere,
                   the separated kernel tables alpha, alpha', the loss multiplier D
                   (Sec. 3.3, Carleman representation and decoupling formula).
* ``operator``  -- forward/inverse spectral transforms (Eqs. FU/FC), the fast
                   collision operator Q = Q+ - f L (Sec. 3.3 / Sec. 4.2 algorithm),
                   the wrapped O(n^2) spectral sum (Eq. ode), the L2 conservation
                   projection (Sec. 3.2, Eq. minim1), moments (Eq. i5 / DM) and the
                   forward-Euler / Heun relaxation step (Eq. f_coll).
* ``plane``     -- the two-dimensional operator for Maxwell molecules (Sec. 3.3,
                   dimension two; Eq. dfor0) with its projection, relaxation and the 2D
                   BKW solution of Test 1.1 (Sec. 5).
* ``fks``       -- the Fast Kinetic Scheme in one space dimension (Sec. 3.1): exact
                   transport of the piecewise-constant distribution sampled at the cell
                   centres, coupled to the collision step, with Dirichlet boundary states.
* ``exact``     -- closed forms and independent quadratures used as pins: the exact
                   Carleman kernel at l=0, the classical kernel (Eq. KM) reduced to a
                   1D integral, the hard-sphere collision frequency of a Maxwellian,
                   a direct quadrature of the Boltzmann integral (Eq. bolt) and the
                   3D BKW solution for Maxwell molecules.

Everything is float64 numpy; library primitives (numpy FFT, scipy Bessel functions,
numpy Gauss-Legendre nodes, numpy linear solves) serve as steps.  Functions with no
independent pin say "parity unpinned" in their docstring; at present every exported
function has at least one pin in ``tests/test_oracle_pins.py``,
``tests/test_oracle_fks.py`` or ``tests/test_oracle_plane.py`` (the latter against the error magnitudes printed in the
paper's Table test1, stored in ``tests/golden/``).
"""

from .grid import (  # noqa: F401
    VelocityGrid,
    make_grid,
    directions,
    phi_hs,
    psi_hs,
    kernel_tables,
)
from .operator import (  # noqa: F401
    forward,
    inverse,
    collide,
    collide_brute_force,
    moments,
    project_Q,
    project_f,
    relax,
    constraint_matrix,
)
from . import exact  # noqa: F401
from . import fks  # noqa: F401
from . import plane  # noqa: F401
