"""mW water model on GB300: CUDA engine (libmw.so) behind a C ABI, thin Python binding.

``mw`` mirrors include/mw.h; ``inputs`` holds the seeded synthetic workloads.
The library is loaded on first use; nothing here falls back to the CPU.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "mw", "build"]


def __getattr__(name):
    if name in ("mw", "build", "torch_ops"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
