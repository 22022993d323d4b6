"""Time-fractional polymer-stress step on GB300 (sm_103a).

The compute path lives in the C-ABI library ``libtfs.so`` built from
``csrc/`` (declared in ``include/tfs.h``); ``tfs`` is its thin ctypes binding
and ``autograd`` the ``torch.autograd.Function`` around the forward step and
its hand-written adjoint.  Importing this package does not load CUDA; the
binding loads the library on first use and raises if it is missing.
"""

__all__ = ["tfs", "soe", "inputs", "autograd", "build"]
