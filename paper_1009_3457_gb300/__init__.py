"""GB300-native M2L / FGT Hermite-to-Taylor translation engine (Cruz, Layton & Barba, arXiv:1009.3457).

The compute path is the C-ABI library ``libfmmgb.so`` (hand-written sm_103a
CUDA).  ``paper_1009_3457_gb300.fmmgb`` is its thin ctypes binding, with the
same names as the C entry points.  Importing this package loads nothing; the
binding loads the library on first use and raises if it is missing.
"""
__all__ = ["fmmgb", "metrics"]
