"""GB300-native SPOCK: Chambolle-Pock + SuperMann/Anderson for multistage
risk-averse optimal control on a scenario tree (arXiv 2212.01110).

The compute path lives in the CUDA shared library built from ``csrc/``; the
Python module :mod:`paper_2212_01110_gb300.spock` marshals arguments to its
C-ABI.  Importing this package loads nothing: ``workloads`` (seeded input
generators) can be imported on machines without the library.
"""

__all__ = ["workloads", "spock"]
