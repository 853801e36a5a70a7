"""GB300-native time-dependent four-body amplitude likelihood (arXiv:1702.06735).

The compute path lives in libtdmix.so (CUDA, sm_103a) behind the C ABI of
include/tdmix.h; ``tdmix`` is its Python binding and ``autograd`` exposes
the NLL to PyTorch.  Nothing here loads the library at import time.
"""
__all__ = ["tdmix", "samples"]
