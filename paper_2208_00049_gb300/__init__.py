"""GB300-native NFFT window-convolution path (arXiv 2208.00049, NFFT.jl).

The compute path is the CUDA library ``libnfft_gb300.so`` built from
``csrc/`` for sm_103a; ``binding`` marshals arguments to its C ABI and
``nfft`` wraps it in a plan object and ``torch.autograd.Function``s.
Importing this package does not load the library; the first call into
``binding`` does, and it raises if the library is missing.
"""
__all__ = ["binding", "nfft", "inputs"]
