"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds no arithmetic of the domain-decomposition / flow-update
method. It only draws the problem data: the two grid measures mu and nu, and
initial couplings given as sparse (x, y, mass) lists or converted to the
basic-cell box format both sides read. The paper's test images (Gaussian
mixtures with random means, variances and magnitudes, Section A.2 "Test data")
are not available; these generators stand in for them with the same structure.
"""

from .measures import (  # noqa: F401
    gaussian_mixture,
    uniform_measure,
    four_bumps,
    workload,
    WORKLOADS,
)
from .couplings import (  # noqa: F401
    coarsen,
    prolongate,
    knothe_rosenblatt,
    product_coupling,
    boxes_from_coupling,
    rotation_coupling,
    rotation_contraction_coupling,
)
from .cellbench import cell_lse_sweep  # noqa: F401
