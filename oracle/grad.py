"""Adjoint of the estimator with respect to the real-space field delta(x) (test infrastructure).

The estimator of Eq. (2.7) is B_t = c_t sum_x d_a d_b d_c with c_t = V_c^3 / (V T_t) and
d_n = Ng^3 H_n delta, where H_n = IDFT . S_n K . DFT (normalised inverse), S_n the shell
mask of Eq. (2.8) and K the optional Kaiser factor of Eq. (3.4). H_n is real and symmetric
(S_n K is even in k), so for an upstream gradient g_t = dL/dB_t

    dL/d delta = Ng^3 sum_n H_n G_n,   G_n = sum_t g_t c_t sum_{positions of n in t}
                                                    (product of the other two fields),

one term per position, so a bin with a repeated shell contributes once per repeat.
Pinned in the tests by central finite differences in float64.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from . import plan as P
from .fbe import kaiser_factor_half, shell_fields


def estimate_real(delta_x: np.ndarray, plan: P.Plan, trips, tsum, beta=None, workers=-1):
    """Per-bin B_t of a real field for a fixed list of bins (the forward of vjp)."""
    spec = sfft.rfftn(delta_x, workers=workers)
    if beta is not None:
        spec = spec * kaiser_factor_half(plan.ng, beta)
    shells = sorted({s for t in trips for s in t})
    d = shell_fields(spec, plan, shells, workers)
    norm = plan.vcell ** 3 / plan.volume
    return np.array([norm * float(np.sum(d[a] * d[b] * d[c])) / ts
                     for (a, b, c), ts in zip(trips, tsum)])


def vjp(delta_x: np.ndarray, plan: P.Plan, trips, tsum, g, beta=None, workers=-1):
    """dL/d delta(x) given g_t = dL/dB_t for the bins `trips` with counts `tsum`."""
    ng = plan.ng
    spec = sfft.rfftn(delta_x, workers=workers)
    weight = np.ones((ng, ng, ng // 2 + 1)) if beta is None else kaiser_factor_half(ng, beta)
    shells = sorted({s for t in trips for s in t})
    d = shell_fields(spec * weight, plan, shells, workers)
    norm = plan.vcell ** 3 / plan.volume
    gfield = {n: np.zeros((ng, ng, ng)) for n in shells}
    for (a, b, c), ts, gt in zip(trips, tsum, g):
        coef = float(gt) * norm / float(ts)
        gfield[a] += coef * d[b] * d[c]
        gfield[b] += coef * d[a] * d[c]
        gfield[c] += coef * d[a] * d[b]
    sidx = P.shell_index_half(plan)
    acc = np.zeros((ng, ng, ng // 2 + 1), dtype=np.complex128)
    for n in shells:
        gk = sfft.rfftn(gfield[n], workers=workers)
        acc += np.where(sidx == n, gk * weight, 0.0)
    return sfft.irfftn(acc, s=(ng, ng, ng), workers=workers) * float(ng) ** 3
