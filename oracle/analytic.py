"""Analytic expectations used to validate the estimator (test infrastructure).

  * b_ana: Eq. (3.2), B = 2 f_NG [P1 P2 + P2 P3 + P3 P1], first order in f_NG, for the
    local quadratic field of Eq. (3.1).
  * sigma_b: Eq. (3.3), sigma_B^2 = [V P1 P2 P3 + 3 B^2] / N_tri.
  * expected_binned: Eq. (2.5) with Eq. (3.2) inserted, summed over the actual grid
    triangles of each bin through the same plane-wave identity as Eq. (2.6):
       <B_abc> = 2 f_NG / T_abc * sum_x [(Pi)_a (Pi)_b i_c + (Pi)_b (Pi)_c i_a + (Pi)_c (Pi)_a i_b]
    with (Pi)_n(x) = sum_{k in n} P(|k|) e^{ik.x}, i_n the counting field of Eq. (2.11) and
    T_abc = sum_x i_a i_b i_c. With linear RSD (Eq. (3.4)) every mode carries the factor
    K(k) = 1 + beta mu_k^2, so P i -> K P i and i -> K i.
  * kaiser_monopole: orientation average of K(k1) K(k2) K(k3) over a closed triangle
    rotated uniformly, the ratio B^s / B of the RSD monopole to the real-space bispectrum
    (Sec. 3.1). The paper takes its formula from another work that is not reproduced in
    the paper; this is an own derivation from the isotropic moments of a unit vector n:
       <(n.u)^2> = 1/3, <(n.u)^2 (n.v)^2> = (1 + 2 c_uv^2)/15,
       <(n.u)^2 (n.v)^2 (n.w)^2> = (1 + 2 (c_uv^2 + c_vw^2 + c_wu^2) + 8 c_uv c_vw c_wu)/105.
    It is pinned by Monte Carlo in the tests and against the enhancement factors the paper
    prints in Sec. 3.1 (2.29 equilateral; 2.47 near squeezed; 2.32 and 2.68 at t = 0.73).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

from . import plan as P
from .fbe import kaiser_factor_half, triple_sums


def power_law(k, n_index: float):
    return np.asarray(k, dtype=np.float64) ** (-n_index)


def b_ana(p1, p2, p3, f_ng: float):
    """Eq. (3.2)."""
    return 2.0 * f_ng * (p1 * p2 + p2 * p3 + p3 * p1)


def sigma_b(p1, p2, p3, b, ntri, volume: float):
    """Eq. (3.3)."""
    return np.sqrt((volume * p1 * p2 * p3 + 3.0 * b * b) / ntri)


def _weighted_fields(plan: P.Plan, weight_half: np.ndarray, shells, workers=-1):
    ng = plan.ng
    sidx = P.shell_index_half(plan)
    out = {}
    for n in shells:
        masked = np.where(sidx == n, weight_half, 0.0).astype(np.complex128)
        out[n] = sfft.irfftn(masked, s=(ng, ng, ng), workers=workers) * float(ng) ** 3
    return out


def expected_binned(plan: P.Plan, triplets, n_index: float, f_ng: float,
                    beta: float | None = None, workers: int = -1) -> np.ndarray:
    """<B_abc> of the quadratic field at first order in f_NG, per bin (see module doc)."""
    ng = plan.ng
    m = np.fft.fftfreq(ng, d=1.0 / ng)
    mz = np.arange(ng // 2 + 1, dtype=np.float64)
    q = m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2
    q[0, 0, 0] = 1.0
    pk = (plan.kf * np.sqrt(q)) ** (-n_index)
    kz = np.ones_like(q) if beta is None else kaiser_factor_half(ng, beta)
    shells = sorted({s for t in triplets for s in t})
    pi_f = _weighted_fields(plan, kz * pk, shells, workers)
    i_f = _weighted_fields(plan, kz, shells, workers)
    i0 = _weighted_fields(plan, np.ones_like(q), shells, workers)
    t_abc = triple_sums(i0, triplets)
    s1 = triple_sums_mixed(pi_f, pi_f, i_f, triplets)
    s2 = triple_sums_mixed(i_f, pi_f, pi_f, triplets)
    s3 = triple_sums_mixed(pi_f, i_f, pi_f, triplets)
    return 2.0 * f_ng * (s1 + s2 + s3) / t_abc


def triple_sums_mixed(fa: dict, fb: dict, fc: dict, triplets) -> np.ndarray:
    """sum_x fa[a] fb[b] fc[c] per triplet."""
    return np.array([float(np.sum(fa[a] * fb[b] * fc[c])) for (a, b, c) in triplets])


def triangle_cosines(k1: float, k2: float, k3: float):
    """Cosines between the sides of a closed triangle k1 + k2 + k3 = 0 (law of cosines):
    khat_a . khat_b = (k_c^2 - k_a^2 - k_b^2) / (2 k_a k_b)."""
    c12 = (k3 * k3 - k1 * k1 - k2 * k2) / (2.0 * k1 * k2)
    c23 = (k1 * k1 - k2 * k2 - k3 * k3) / (2.0 * k2 * k3)
    c31 = (k2 * k2 - k3 * k3 - k1 * k1) / (2.0 * k3 * k1)
    return c12, c23, c31


def kaiser_monopole(k1: float, k2: float, k3: float, beta: float) -> float:
    """Orientation average of prod_a (1 + beta mu_a^2) over a rigidly rotated triangle."""
    c12, c23, c31 = triangle_cosines(k1, k2, k3)
    s2 = c12 * c12 + c23 * c23 + c31 * c31
    second = (3.0 + 2.0 * s2) / 15.0
    third = (1.0 + 2.0 * s2 + 8.0 * c12 * c23 * c31) / 105.0
    return 1.0 + beta + beta * beta * second + beta ** 3 * third


def kaiser_monopole_mu_t(mu: float, t: float, beta: float) -> float:
    """kaiser_monopole for the shape (mu, t) with k1 = 1 (Eq. (2.4) inverted):
    k2 = t, k3^2 = k1^2 + k2^2 - 2 k1 k2 mu."""
    k1, k2 = 1.0, t
    k3 = math.sqrt(max(k1 * k1 + k2 * k2 - 2.0 * k1 * k2 * mu, 0.0))
    return kaiser_monopole(k1, k2, k3, beta)
