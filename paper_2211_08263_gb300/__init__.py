"""GB300-native implicit FFT elastodynamics (arXiv 2211.08263): the matrix-free
spectral operator, the reference-medium preconditioner and the preconditioned
Krylov solve inside each beta-Newmark step, as hand-written sm_103a CUDA
behind a C ABI (``include/wfft.h``).

The CUDA library is loaded lazily by ``paper_2211_08263_gb300.wfft`` so that
the input generators (``paper_2211_08263_gb300.inputs``) import without it.
"""
__all__ = ["inputs", "wfft"]
