"""Sparse LDL^T factor + solve of the NCL KKT systems on one GB300 (sm_103a).

The compute path lives in the C-ABI library ``libncl_kkt.so`` (hand-written
CUDA, built from ``csrc/``); :mod:`.ncl_kkt` is the thin ctypes binding and
:mod:`.autograd` the ``torch.autograd.Function`` around it.  Importing this
package loads nothing: the library is opened on first use.
"""
