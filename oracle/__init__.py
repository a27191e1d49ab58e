"""CPU oracle for the NCL KKT factor/solve path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library never calls it, and it imports nothing from the product.

Everything here is plain FP64: scipy.sparse for assembling the matrices
from their definitions, and the C file ``ldlt_oracle.c`` (a simplicial
up-looking LDL^T) for the factorisation.
"""
from .oracle import *  # noqa: F401,F403
