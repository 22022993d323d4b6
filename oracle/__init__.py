"""Plain FP64 CPU oracle for the fractional polymer-stress step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product library never loads it and it never loads the product library: the two
share no code, header, constant or generator.  Inputs come from the neutral
seeded generators in ``paper_2411_17294_gb300.inputs`` (which hold none of the
method's arithmetic) and are passed to both sides.

Contents
--------
tfs_oracle.c   the per-step update and its reference adjoint, plain C, FP64
orc.py         ctypes wrapper: state, stepping, history, gradients
soe.py         sum-of-exponentials kernels: AAA with the division-by-s trick
               (Section 2.2) and a positive exponential quadrature
special.py     Mittag-Leffler function and convolution-quadrature weights
paper_form.py  the scheme in the paper's own variable Phi, Psi = D^{1-alpha} Phi
               (Section 3.4), pointwise, BDF2 with an optional SDIRK2 start
"""
