"""GB300-native discrete spherical Radon transform for cylindrical apertures.

The transform is computed as the composition of two circular Radon transforms
(Sec. 2 of the paper) applied as sparse matrices (Algorithm 1), with the
matched adjoint (Algorithm 2), by hand-written sm_103a CUDA kernels behind the
C ABI declared in ``include/srt.h``.  The CUDA library is loaded on first use;
there is no CPU fallback.
"""
__all__ = ["srt", "inputs"]
