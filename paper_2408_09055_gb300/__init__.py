"""GB300 (sm_103a) execution of kernelized quantum circuits (arXiv 2408.09055).

The compute lives in ``libqsim.so`` (C ABI in include/qsim.h); ``qsim`` is
its ctypes binding.
"""
