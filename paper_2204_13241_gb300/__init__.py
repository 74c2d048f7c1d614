"""GB300-native direct-method XPCS / XSVS (arXiv 2204.13241).

The computation lives in the CUDA library libxs.so (include/xs_api.h);
``paper_2204_13241_gb300.api`` marshals torch tensors into its C ABI and
``workloads`` draws the seeded synthetic inputs.  Importing the package does
not load the library; the first call does, and fails loudly if it has not
been built.
"""
import importlib

from . import workloads  # noqa: F401

__all__ = ["workloads", "api"]


def __getattr__(name):
    if name == "api":
        return importlib.import_module(__name__ + ".api")
    raise AttributeError(name)
