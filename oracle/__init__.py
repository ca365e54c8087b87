"""FP64 CPU oracle of the decoupled ensemble Elsaesser scheme (Algorithm 1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (``paper_2108_05110_gb300``) never imports it, and this
package imports nothing from the product: the two share no code.  Inputs come
from ``workloads`` (seeded generators holding none of the method).

Plain, slow and obviously correct: numpy for element-wise arithmetic, scipy
sparse COO->CSR for assembly, SuperLU (``scipy.sparse.linalg.splu``) for the
linear systems, all in float64.

Discrete setting (where the paper leaves a choice open, this is the reading
taken):
* Taylor-Hood P2 velocity / P1 pressure on a conforming triangulation
  (Section 2, eq. infsup: any inf-sup stable pair), or the paper's
  Scott-Vogelius pair P2 / P1disc on barycenter-refined meshes (Section 2,
  Section 4; ``OracleRun(..., element="SV")``);
* a 7-point degree-5 triangle quadrature derived in :mod:`oracle.quadrature`;
* skew-symmetric convection form by default (Section 2, trilinear form b);
* Dirichlet data by identity rows, pressure pinned at node 0 then shifted to
  mean zero (Q = L^2_0, Section 2);
* forcing as M times the P2 nodal interpolant.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
closed forms, exact integrals, brute force, the stability inequality of
Section 3.1, the special cases of Section 4.4 ("usual MHD") and the paper's
printed numbers: the spatial errors of Table 1 (Taylor-Hood with a
pressure-free velocity, where the element pair does not enter the velocity
error; Scott-Vogelius on barycenter-refined meshes with the printed pressure)
and of Table 3 (Scott-Vogelius), and the temporal errors of Table 4, values
and rates (``tests/golden/``).  The Scott-Vogelius space is further pinned by
pointwise zero divergence and pressure robustness (``tests/test_oracle_sv.py``).
Its adjoint (:mod:`oracle.adjoint`) is pinned by central differences of this
forward run.
"""
from .quadrature import triangle_rule_deg5  # noqa: F401
from .fe import P2Space  # noqa: F401
from .scheme import OracleRun, run_ensemble  # noqa: F401
