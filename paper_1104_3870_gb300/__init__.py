"""GB300-native (sm_103a) stochastic-LapH quark-line library.

The compute lives in the CUDA library liblaph.so (csrc/, C ABI in
include/laph.h); `paper_1104_3870_gb300.laph` is its thin Python binding and
`paper_1104_3870_gb300.build` compiles it.  Importing the binding raises when
the library is not built: there is no CPU fallback.
"""
__all__ = ["build", "laph"]
