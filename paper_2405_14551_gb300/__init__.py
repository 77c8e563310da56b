"""GB300-native two-component colour-gradient lattice Boltzmann step
(arXiv 2405.14551) with near-contact repulsion: CUDA kernels for sm_103a behind
the C ABI of include/lbcg.h, and a thin Python binding (``lbcg``)."""

__all__ = ["lbcg", "build"]
