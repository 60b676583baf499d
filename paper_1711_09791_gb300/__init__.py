"""GB300-native separable width-5 convolution of planar 3-plane images
(arXiv 1711.09791, "2D Image Convolution using Three Parallel Programming
Models on the Xeon Phi").

The compute path is the CUDA library ``libsepconv5.so`` (C ABI declared in
``include/sepconv5.h``); :mod:`.sepconv5` is its thin ctypes binding.  The
binding is loaded lazily so that :mod:`.synth` (seeded inputs) can be imported
on a machine without the library.
"""
import importlib

__all__ = ["synth", "sepconv5"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
