"""GB300 (sm_103a) implementation of Multidimensional Contrast Limited Adaptive
Histogram Equalization (MCLAHE, arXiv:1906.11355).

The compute path is the C-ABI library ``libmclahe.so`` (hand-written CUDA
kernels); ``_native`` binds it with ctypes, ``api`` adds a PyTorch front end,
``synth`` draws seeded synthetic volumes.  Importing the package does not load
the library; the first call that needs it does, and fails loudly if it has not
been built.
"""

__version__ = "0.1.0"


def __getattr__(name):
    if name in ("MCLAHE", "mclahe"):
        from . import api

        return getattr(api, name)
    if name in ("MCLAHEFunction", "mclahe_autograd"):
        from . import autograd

        return getattr(autograd, name)
    raise AttributeError(name)
