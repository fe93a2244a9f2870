"""FP64 CPU oracle of domain decomposition with flow updates (test infrastructure).

This package is the correctness reference for the CUDA library, and nothing
else: only the test suite, the smoke check in ``__graft_entry__`` and the
CPU-baseline leg of ``bench.py`` may import it. The library never calls it and
has no CPU fallback.

It follows the paper step by step, in float64, with plain numpy/scipy:

* ``geometry``  basic cells, the A/B composite partitions, the neighbourhood
  set (Def. 2.2, Fig. 3, Def. 3.1).
* ``cell``      the composite-cell entropic problem of Alg. 1, solved by
  log-domain Sinkhorn with DENSE (non-separable) log-sum-exp sums.
* ``domdec``    one domain-decomposition half-iteration on the basic-cell
  bounding-box state (Alg. 1 as restated for boxes in Alg. 4: BasicToComposite,
  cell solve, CompositeToBasic, balancing, truncation).
* ``flow``      the flow update with product gluing candidates (Def. 3.4,
  Def. 3.7, Remark 3.8), the min-cost flow Eq. (MinCostFlow) solved as a linear
  program by scipy's HiGHS, and the exchange Eq. (flow-update-cell-marginals).
* ``hybrid``    the hybrid schedule of Alg. 3 and the objective / marginal errors.
* ``dense``     a full-plan version for tiny grids (global Sinkhorn, Alg. 1 and
  Def. 3.4 on the explicit plan), used to pin the box version.
* ``warmstart`` (not in the paper) the inputs and training targets of the
  learned Sinkhorn initialisation of a composite cell.
* ``mlp``       (not in the paper) the warm-start network, its loss and its
  gradient by backpropagation.

Readings of the paper where it is silent or ambiguous are listed in the
module docstrings where they apply.
"""

from .geometry import Geometry  # noqa: F401
from .cell import cell_sinkhorn, sq_cost  # noqa: F401
from .domdec import Box, half_iteration, balance, truncate_box, basic_to_composite  # noqa: F401
from .flow import edge_costs, min_cost_flow, exchange  # noqa: F401
from .hybrid import OracleDD  # noqa: F401
