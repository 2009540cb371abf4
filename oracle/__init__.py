"""FP64 CPU oracle for the P2S per-frame synthesis path (Mao, Chimitt & Chan, ICCV 2021).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, step-by-step
statement of what the simulator computes, written from the paper's equations
in double precision with NumPy.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the CUDA library never calls it,
and it shares no code, table or constant generator with the CUDA sources.

Modules, in the order the path runs:

  zernike   Noll-indexed Zernike polynomials (Sec. 2.2, Eq. 1)
  noll      Noll inter-mode covariance R_Z (Sec. 2.2, from Noll 1976)
  philox    Philox4x32-10 counter generator + Box-Muller normals
  fields    anchor-grid Zernike fields by Fourier filtering of white noise
            (Sec. 3.4), inter-mode colouring by chol(R_Z)
  warp      tilt modes -> sub-pixel backward bilinear warp (Sec. 2.2, 3.3)
  psf       pupil-FFT PSF (Eq. 2), PSF dictionary and SVD basis (Sec. 3.2)
  mlp       P2S network forward (Sec. 3.3)
  blur      basis blur, scatter and gather forms (Eq. 3-5), exact per-pixel blur
  frame     the whole frame, plus reduced-precision emulation
  precision round-to-nearest-even BF16 / FP8-E4M3 emulation

Parity status per function is stated in each module header.
"""
from . import zernike, noll, philox, fields, warp, psf, mlp, blur, precision, frame  # noqa: F401
