"""The FFT estimator carried from the bispectrum to the p-th order polyspectrum (test
infrastructure, float64). Sec. 4 notes that an FFT estimator of the p-th order polyspectrum must
keep every mode below 2 pi Ng / (p L), for the reason the bispectrum keeps them below
2 pi Ng / (3 L) (the cap after Eq. (2.12)): a sum of p modes must not wrap around the grid.

The estimator is the bin average of Eq. (2.3) with p shells instead of three, through the same
plane-wave identity as Eq. (2.6) - Eq. (2.11):
    P_{a_1 .. a_p} = V_c^p sum_x d_{a_1} ... d_{a_p} / (V sum_x i_{a_1} ... i_{a_p}),
    N_p = sum_x i_{a_1} ... i_{a_p} / Ng^3 = the number of ordered p-gons k_{a_1} + ... + k_{a_p} = 0
with one mode in each shell. p = 3 is the bispectrum estimator of fbe.py. The estimator is the
raw binned p-point sum: for p = 4 it keeps the disconnected part (pairs of modes that cancel),
which the paper does not discuss. Bins are the multisets a_1 >= ... >= a_p of shells that can
close: the smallest |k| of shell a_1 is at most the sum of the largest |k| of the others.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import dbe
from . import fbe
from . import plan as P


def cap_ok(ng: int, thresholds: np.ndarray, p: int) -> bool:
    """Every shell mode below 2 pi Ng / (p L): p^2 (Q_N - 1) < Ng^2."""
    return p * p * (int(thresholds[-1]) - 1) < ng * ng


def candidates(plan: P.Plan, p: int):
    """Multisets a_1 >= ... >= a_p (ascending lexicographic order) passing the closing test."""
    thr = plan.thresholds
    out = []
    for t in itertools.combinations_with_replacement(range(plan.ns), p):
        t = tuple(sorted(t, reverse=True))
        big = math.sqrt(float(thr[t[0]]))
        if big <= sum(math.sqrt(float(thr[s + 1] - 1)) for s in t[1:]):
            out.append(t)
    return sorted(out)


def multi_sums(fields: dict, bins) -> np.ndarray:
    """sum_x prod_j f[a_j] per bin."""
    out = np.empty(len(bins))
    for i, t in enumerate(bins):
        prod = fields[t[0]].copy()
        for s in t[1:]:
            prod *= fields[s]
        out[i] = float(np.sum(prod))
    return out


def kept_bins(plan: P.Plan, p: int):
    """Bins with at least one closed p-gon, their T = sum_x i...i and integer N_p."""
    if not cap_ok(plan.ng, plan.thresholds, p):
        raise ValueError("largest shell reaches k >= 2 pi Ng / (p L)")
    cand = candidates(plan, p)
    tsum = multi_sums(fbe.counting_fields(plan), cand)
    n = tsum / float(plan.ng) ** 3
    rnd = np.rint(n)
    if np.any(np.abs(n - rnd) > 1e-3):
        raise ArithmeticError("N_p not integral within 1e-3")
    keep = rnd > 0
    return [t for t, k in zip(cand, keep) if k], tsum[keep], rnd[keep].astype(np.int64)


def estimate(spec_half: np.ndarray, plan: P.Plan, p: int, with_abs: bool = False, counts=None):
    """Binned p-th order polyspectrum of one field: bins, T, N_p, sums and values."""
    bins, tsum, npoly = counts if counts is not None else kept_bins(plan, p)
    need = sorted({s for t in bins for s in t})
    d = fbe.shell_fields(np.asarray(spec_half, dtype=np.complex128), plan, need)
    msum = multi_sums(d, bins)
    norm = plan.vcell ** p / plan.volume
    res = dict(bins=bins, tsum=tsum, n=npoly, msum=msum, value=norm * msum / tsum)
    if with_abs:
        a = {k: np.abs(v) for k, v in d.items()}
        res["scale"] = norm * multi_sums(a, bins) / tsum
    return res


def direct_sums_4(spec_half, plan: P.Plan, count_only: bool = False):
    """({bin: sum F F F F}, {bin: N_4}) by enumeration: for every mode k_b of the ball and every
    ordered pair (k_c, k_e), the closing k_a = -(k_b + k_c + k_e) is looked up (non-periodic);
    the quadrilateral is added to bin (s_a, s_b, s_c, s_e) when s_a >= s_b >= s_c >= s_e."""
    modes, shell, r = dbe.ball_modes(plan)
    m = len(modes)
    vals = None if count_only else dbe.full_spectrum_values(spec_half, modes, plan.ng)
    span = 6 * r + 1
    off = 3 * r
    table = -np.ones((span, span, span), dtype=np.int64)
    table[modes[:, 0] + off, modes[:, 1] + off, modes[:, 2] + off] = np.arange(m)
    ns = plan.ns
    ic, ie = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    ic, ie = ic.ravel(), ie.ravel()
    pair = modes[ic] + modes[ie]
    nbin = ns ** 4
    cnt = np.zeros(nbin, dtype=np.int64)
    s_re = np.zeros(nbin)
    s_im = np.zeros(nbin)
    for ib in range(m):
        ka = -(modes[ib][None, :] + pair)
        ok = np.all(np.abs(ka) <= r, axis=1)
        ida = np.full(len(ka), -1, dtype=np.int64)
        ida[ok] = table[ka[ok, 0] + off, ka[ok, 1] + off, ka[ok, 2] + off]
        sel = ida >= 0
        ia, c, e = ida[sel], ic[sel], ie[sel]
        sa, sb, sc, se = shell[ia], shell[ib], shell[c], shell[e]
        keep = (sa >= sb) & (sb >= sc) & (sc >= se)
        ia, c, e, sa, sc, se = ia[keep], c[keep], e[keep], sa[keep], sc[keep], se[keep]
        key = ((sa * ns + sb) * ns + sc) * ns + se
        cnt += np.bincount(key, minlength=nbin)
        if vals is not None:
            w = vals[ia] * vals[ib] * vals[c] * vals[e]
            s_re += np.bincount(key, weights=w.real, minlength=nbin)
            s_im += np.bincount(key, weights=w.imag, minlength=nbin)
    out_s, out_n = {}, {}
    for key in np.nonzero(cnt)[0]:
        t = np.unravel_index(int(key), (ns,) * 4)
        t = tuple(int(v) for v in t)
        out_n[t] = int(cnt[key])
        out_s[t] = complex(s_re[key], s_im[key])
    return out_s, out_n
