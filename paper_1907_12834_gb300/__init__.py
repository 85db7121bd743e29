"""GB300-native spin-2 BEC quantum lattice gas algorithm (arXiv:1907.12834).

``paper_1907_12834_gb300.qlga`` is the Python binding of the C-ABI library ``libqlga.so``
(hand-written CUDA for sm_103a); ``paper_1907_12834_gb300.inputs`` builds the paper's
analytic initial states.  Importing the package loads nothing; the CUDA library is loaded on
first use of the binding and its absence is an error, never a fallback.
"""
__all__ = ["qlga", "inputs"]
