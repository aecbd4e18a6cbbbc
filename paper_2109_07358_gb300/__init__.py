"""GB300 fast fermion sampling (arXiv 2109.07358): CUDA library + thin binding."""
from . import ffs  # noqa: F401
