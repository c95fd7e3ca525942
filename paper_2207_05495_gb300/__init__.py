"""Exact reset threshold and least shortest reset word on one GB300 GPU.

The search (Szykula and Zyzik, arXiv 2207.05495, Section 2.1) runs in the
CUDA library libsw.so behind the C-ABI of include/sw.h; `sw` is its Python
binding and `gen` makes seeded synthetic automata.  Importing the package
does not load the library; the first call through `sw` does, and fails
loudly if it has not been built.
"""

from . import gen  # noqa: F401
