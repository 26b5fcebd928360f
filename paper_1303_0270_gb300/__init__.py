"""Computable compressed matrices on GB300 (sm_103a).

Integer matrices in the fixed-width "Supreme Minimum" bit-stream form of
Paixao and Coelho, *Computable Compressed Matrices* (Methods, Method 1), with
pack / unpack / element access / add / scale / matvec / matmul running as
hand-written CUDA kernels on the compressed form.  The C ABI is
``include/ccm.h`` (``libccm.so``); :mod:`paper_1303_0270_gb300.ccm` is its
Python binding (``from paper_1303_0270_gb300 import ccm``).
"""
