"""Oracle for SPOCK (arXiv 2212.01110) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 CPU restatement of the method, written from the paper:
the scenario tree (Sec. "Scenario trees"), the splitting z, eta, S1, S2, S3
and the operator L (Sec. "Operator splitting"), prox of f and of g*
(Sec. "Proximal operator of f", Eq. (prox:g)), the Chambolle-Pock operator T
(Eq. (chambolle-pock-operator)), the residual/termination rule
(Sec. "The Chambolle-Pock method"), and SPOCK (Algorithm 3) with Anderson
directions (Sec. "Anderson's acceleration").  The projection onto the tree
dynamics S1 is a direct KKT solve, not the Riccati recursion of
Algorithms 1-2 used by the CUDA path.

It shares no code with the CUDA library and must never be imported by the
product path: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``
(its CPU-baseline and reference legs) may use it.

Parity status per function is stated in each module header.
"""
