"""GB300 (sm_103a) implementation of DuQuad's inexact (augmented) dual first-order
QP method (Necoara & Patrascu, arXiv 1504.05708).

The product is the C-ABI library ``libduquad.so`` (include/duquad.h); ``duquad``
is its thin Python binding.  There is no CPU fallback: importing the binding
fails if the library cannot be built or loaded.
"""
from . import duquad  # noqa: F401
from .duquad import Context, Problem, opts, solve_many  # noqa: F401
