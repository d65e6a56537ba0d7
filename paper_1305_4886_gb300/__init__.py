"""GB300-native Gaussian-process marginal log-likelihood (arXiv:1305.4886).

The compute path lives in the C-ABI library ``libgp.so`` (hand-written
sm_103a CUDA); ``paper_1305_4886_gb300.gp`` is its thin ctypes binding and
``paper_1305_4886_gb300.autograd`` wraps it for PyTorch.  Importing this
package does not load the library; the binding does, and fails loudly when
it is missing.
"""
__all__ = ["inputs"]
