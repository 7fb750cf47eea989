"""Declarations of the later-added C-ABI entry points (see include/gbsw.h)."""


def declare(L, sig):
    pass
