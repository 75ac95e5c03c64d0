"""Plain, slow, FP64 CPU oracle for the NFFT window-convolution path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this tree;
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code,
tables or constants with the CUDA path.

Modules
-------
window : Kaiser-Bessel window pair in the paper's scaled form (Sec. 2.2,
         window tensor product and the deconvolution vectors of Sec. 3.5),
         plus the LINEAR lookup-table size rule of Sec. 3.7.4.
ndft   : direct NDFT and adjoint NDFT, the exact definitions (Sec. 2.1,
         Eq. NDFT and Eq. NDFTH), and the exact node derivative.
nfft   : plain NFFT following Algorithm 1 (direct) and Algorithm 2 (adjoint),
         step by step, plus the derivative of the approximation with respect
         to the nodes.

Every oracle function is pinned by a ``-m "not gpu"`` test against something
other than itself (closed forms, brute force, invariants, printed values).
"""
from . import window, ndft, nfft  # noqa: F401
