"""FP64 CPU oracle of PDBO (arXiv 2509.21064) -- test infrastructure, not part of the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
"""
from .pdbo import *  # noqa: F401,F403
from . import pdbo  # noqa: F401
