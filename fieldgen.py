"""Seeded synthetic density fields shaped like the paper's validation runs (Sec. 3).

This module is input synthesis only. It serves both sides of the parity tests, the
CUDA path (tests, bench) and the CPU oracle, and it holds none of the estimator's
arithmetic: no shells, no triple products, no normalisation of the bispectrum.

Recipe (Sec. 3, Eq. (3.1); power law as in Sec. 3 first paragraph):
  * w(x) ~ N(0, 1) i.i.d. on an Ng^3 grid, drawn with numpy's PCG64 from `seed`.
  * delta_G = IDFT[ DFT[w] * sqrt(P(|k|) / V_c) ], with the k = 0 mode set to zero and
    P(k) = k^-n_index, k in physical units 2*pi*|m|/L. With the unnormalised DFT this gives
    < |V_c DFT[delta_G](k)|^2 > = V P(k), the continuum convention of Eq. (2.1).
  * delta = delta_G + f_NG (delta_G^2 - mean(delta_G^2))   (Eq. (3.1); the sample mean
    stands in for the ensemble mean, which only touches k = 0).

Arrays are C-order [x][y][z]; z is the last axis, the axis halved by the real FFT and the
line of sight for redshift-space distortions.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

__all__ = ["gaussian_field", "quadratic_field", "gaussian_field_2d", "quadratic_field_2d", "spectrum",
           "half_spectrum_c64", "random_voxels", "random_weights"]


def _kmag_half(ng: int, box_len: float) -> np.ndarray:
    """|k| (physical units) on the half grid [ng][ng][ng//2+1]."""
    m = np.fft.fftfreq(ng, d=1.0 / ng)
    mz = np.arange(ng // 2 + 1, dtype=np.float64)
    q = m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2
    return (2.0 * np.pi / box_len) * np.sqrt(q)


def gaussian_field(ng: int, box_len: float, n_index: float, seed: int,
                   workers: int = -1) -> np.ndarray:
    """Gaussian random field delta_G(x) with power spectrum P(k) = k^-n_index (float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((ng, ng, ng))
    wk = sfft.rfftn(w, workers=workers)
    del w
    k = _kmag_half(ng, box_len)
    k[0, 0, 0] = 1.0
    vc = (box_len / ng) ** 3
    amp = np.sqrt(k ** (-n_index) / vc)
    amp[0, 0, 0] = 0.0
    wk *= amp
    del k, amp
    return sfft.irfftn(wk, s=(ng, ng, ng), workers=workers)


def quadratic_field(ng: int, box_len: float, n_index: float, f_ng: float, seed: int,
                    workers: int = -1) -> np.ndarray:
    """Local quadratic non-Gaussian field of Eq. (3.1) built on gaussian_field (float64)."""
    dg = gaussian_field(ng, box_len, n_index, seed, workers)
    sq = dg * dg
    return dg + f_ng * (sq - sq.mean())


def gaussian_field_2d(ng: int, box_len: float, n_index: float, seed: int) -> np.ndarray:
    """The 2D counterpart of gaussian_field on an Ng^2 grid of a square of side L (the 2D box of
    Sec. 2.1): < |A_c DFT[delta_G](k)|^2 > = A P(k), A = L^2, A_c = (L / Ng)^2 (float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    wk = sfft.rfftn(rng.standard_normal((ng, ng)))
    m = np.fft.fftfreq(ng, d=1.0 / ng)
    my = np.arange(ng // 2 + 1, dtype=np.float64)
    k = (2.0 * np.pi / box_len) * np.sqrt(m[:, None] ** 2 + my[None, :] ** 2)
    k[0, 0] = 1.0
    amp = np.sqrt(k ** (-n_index) / (box_len / ng) ** 2)
    amp[0, 0] = 0.0
    return sfft.irfftn(wk * amp, s=(ng, ng))


def quadratic_field_2d(ng: int, box_len: float, n_index: float, f_ng: float, seed: int) -> np.ndarray:
    """Eq. (3.1) on gaussian_field_2d (float64, [x][y], y the axis the real FFT halves)."""
    dg = gaussian_field_2d(ng, box_len, n_index, seed)
    sq = dg * dg
    return dg + f_ng * (sq - sq.mean())


def spectrum(delta: np.ndarray, workers: int = -1) -> np.ndarray:
    """Unnormalised forward real DFT sum_x delta(x) e^{-i k.x} on the half grid (complex128)."""
    return sfft.rfftn(delta, workers=workers)


def half_spectrum_c64(delta: np.ndarray, workers: int = -1) -> np.ndarray:
    """The half spectrum rounded to complex64, the input form of the FP32 paths."""
    return spectrum(delta, workers).astype(np.complex64)


def random_voxels(ng: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct flat voxel indices (for finite-difference checks), int64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(ng ** 3, size=count, replace=False)).astype(np.int64)


def random_weights(count: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) weights, e.g. an upstream gradient on the bispectrum bins."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(count)
