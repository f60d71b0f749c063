"""GB300-native exact k-bisimulation refinement (arXiv 2111.12493, Algorithm 4).

The compute path lives in a C-ABI shared library built from ``csrc/``; the
Python layer in :mod:`paper_2111_12493_gb300.bisim` only marshals arguments.
Importing the package itself loads nothing: ``graphgen`` (seeded synthetic
inputs) stays usable on machines without a GPU.
"""

__all__ = ["graphgen"]
