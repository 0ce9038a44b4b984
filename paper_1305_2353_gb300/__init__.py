"""GB300-native compressed threshold pivoting for supernodal LDL^T (Hogg & Scott,
arXiv 1305.2353).  The compute path lives in ``libctp.so`` (hand-written CUDA for
sm_103a behind a C ABI); ``paper_1305_2353_gb300.ctp`` is its thin binding.
Importing the package does not load the library; ``ctp.load()`` does, and it
fails loudly when the library is missing."""
__all__ = ["ctp", "inputs"]
