"""GB300-native pressure projection (eigenexpansion solver with Method III
variable-density iteration) from Dalla Barba et al., arXiv:2005.11806.

``import paper_2005_11806_gb300`` is light: the CUDA library is loaded by
``paper_2005_11806_gb300.pressure`` on first use and raises if it is missing.
"""
__all__ = ["pressure", "workloads"]
