"""B300 lifting engine: 2D segment embeddings onto 3D Gaussians (SLAG's Semantic Embedding stage).

The compute path is libslag.so (hand-written CUDA for sm_103a behind a C ABI,
declared in include/slag.h); `slag` is its ctypes binding.
"""
from .slag import Lifter, SlagError, load_library  # noqa: F401
