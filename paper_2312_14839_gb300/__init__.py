"""GB300-native BHEM (bicubic Hermite element) thin-shell hot path.

``bhem`` is the ctypes binding of libbhem.so (C ABI in include/bhem.h); ``scenes`` generates
seeded synthetic inputs; ``build`` compiles the CUDA library for sm_103a.
"""
__all__ = ["bhem", "scenes", "build"]
