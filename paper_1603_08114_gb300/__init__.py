"""GB300-native HMC volatility update of the realized stochastic volatility model.

The compute path is ``librsv.so`` (hand-written CUDA for sm_103a behind a C ABI,
declared in ``include/rsv.h``); :mod:`.rsv` is its thin Python binding.  Nothing
here has a CPU fallback: calling into the library without the compiled
extension or without a GPU raises.
"""
