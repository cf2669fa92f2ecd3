"""GB300-native recombination hot path of arXiv:2312.11448 (Ly-alpha packet
transport and the per-cell three-level-atom update with its adjoint).

The compute path is the CUDA library built from csrc/ and reached through the
C ABI in include/rec.h; `paper_2312_11448_gb300.rec` is the thin binding.
Importing the package does not load the library; `inputs` holds the seeded
synthetic workloads.
"""
__all__ = ["inputs", "rec"]
