"""GB300-native (sm_103a) Swendsen-Wang cluster Monte Carlo and PCC feedback.

Lin & Zheng, "Two Parallel Swendsen-Wang Cluster Algorithms Using
Message-Passing Paradigm" (arXiv:0808.2109).  The compute path is the CUDA
library built from ``csrc/`` behind the C ABI of ``include/swgpu.h``;
``swgpu`` is its Python binding.
"""
from . import swgpu  # noqa: F401
from .swgpu import Lattice, SwError  # noqa: F401

__all__ = ["swgpu", "Lattice", "SwError"]
