"""GB300-native time-step library for the 2DSW and UFLES programs of
arXiv:1711.04471 (Vanderbauwhede & Davidson).

The numerical work runs in libgbsw.so (CUDA, sm_103a); this package holds
the ctypes binding, the seeded input generators and the build script.
Importing it does not load the library; the first call does, and fails
loudly if the library is missing.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name == "SW":
        from .sw import SW
        return SW
    raise AttributeError(name)
