"""FP64 CPU oracle of the decoupled ensemble Elsaesser scheme (Algorithm 1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (``paper_2108_05110_gb300``) never imports it, and this
package imports nothing from the product: the two share no code.  Inputs come
from ``workloads`` (seeded generators holding none of the method).

Plain, slow and obviously correct: numpy for element-wise arithmetic, scipy
sparse COO->CSR for assembly, SuperLU (``scipy.sparse.linalg.splu``) for the
linear systems, all in float64.

Discrete setting (the readings of the paper listed in the design doc):
* Taylor-Hood P2 velocity / P1 pressure on a conforming triangulation
  (Section 2, eq. infsup: any inf-sup stable pair);
* a 7-point degree-5 triangle quadrature derived in :mod:`oracle.quadrature`;
* skew-symmetric convection form by default (Section 2, trilinear form b);
* Dirichlet data by identity rows, pressure pinned at node 0 then shifted to
  mean zero (Q = L^2_0, Section 2);
* forcing as M times the P2 nodal interpolant.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
closed forms, exact integrals, brute force, the paper's convergence rates
(Tables 1-6), the stability inequality of Section 3.1 and the special cases of
Section 4.4 ("usual MHD").  Parity unpinned: the absolute error values of
Tables 1-6 (the paper uses Scott-Vogelius elements on barycenter-refined
meshes); only their rates are pinned.
"""
from .quadrature import triangle_rule_deg5  # noqa: F401
from .fe import P2Space  # noqa: F401
from .scheme import OracleRun, run_ensemble  # noqa: F401
