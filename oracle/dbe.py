"""The direct bispectrum estimator (DBE), a literal evaluation of Eq. (2.3) and Eq. (2.9).

Test infrastructure. For every ordered pair of modes (k_b, k_c) of the ball covered by
the shells, the closing mode k_a = -(k_b + k_c) is formed as an ordinary (non-periodic)
vector sum; if it lies in a shell and the shells satisfy s(k_a) >= s(k_b) >= s(k_c),
the product Delta(k_a) Delta(k_b) Delta(k_c) and one triangle are added to bin
(s(k_a), s(k_b), s(k_c)). This is the loop over k_a2 x k_a3 with a membership test on
the third shell that the paper describes at the end of Sec. 2.1; here it serves all
bins at once. Cost O(M_ball^2): tiny grids only (Ng <= 64).

Values are in units of F (the unnormalised DFT): the returned sums are
  msum_abc = sum_{k_a in a, k_b in b, k_c in c, k_a+k_b+k_c = 0} F(k_a) F(k_b) F(k_c)
  ntri_abc = the number of such ordered triples.
"""
from __future__ import annotations

import numpy as np

from . import plan as P


def ball_modes(plan: P.Plan):
    """All integer modes with Q_0 <= |m|^2 < Q_Ns, their shell index, as (M, 3) int64."""
    r = int(np.ceil(np.sqrt(plan.thresholds[-1]))) + 1
    g = np.arange(-r, r + 1, dtype=np.int64)
    mx, my, mz = np.meshgrid(g, g, g, indexing="ij")
    m = np.stack([mx.ravel(), my.ravel(), mz.ravel()], axis=1)
    q = (m * m).sum(1)
    sel = (q >= plan.thresholds[0]) & (q < plan.thresholds[-1])
    m = m[sel]
    q = q[sel]
    s = np.searchsorted(plan.thresholds, q, side="right") - 1
    return m, s.astype(np.int64), r


def full_spectrum_values(spec_half: np.ndarray, modes: np.ndarray, ng: int) -> np.ndarray:
    """F(m) for integer modes m from the half grid, using F(-m) = conj F(m) (real delta)."""
    mx, my, mz = modes[:, 0], modes[:, 1], modes[:, 2]
    neg = mz < 0
    sx = np.where(neg, -mx, mx) % ng
    sy = np.where(neg, -my, my) % ng
    sz = np.where(neg, -mz, mz)
    v = spec_half[sx, sy, sz].astype(np.complex128)
    return np.where(neg, np.conj(v), v)


def direct_estimate(spec_half: np.ndarray, plan: P.Plan, count_only: bool = False):
    """Return ({(a,b,c): msum}, {(a,b,c): ntri}) over all bins with at least one triangle."""
    modes, shell, r = ball_modes(plan)
    nmode = len(modes)
    vals = None if count_only else full_spectrum_values(spec_half, modes, plan.ng)
    # lookup table: mode vector (offset by 2r, the largest |component| of a sum) -> mode id
    span = 4 * r + 1
    table = -np.ones((span, span, span), dtype=np.int64)
    table[modes[:, 0] + 2 * r, modes[:, 1] + 2 * r, modes[:, 2] + 2 * r] = np.arange(nmode)
    ns = plan.ns
    nbin = ns * ns * ns
    msum_re = np.zeros(nbin)
    msum_im = np.zeros(nbin)
    ntri = np.zeros(nbin, dtype=np.int64)
    for ib in range(nmode):
        kb = modes[ib]
        ka = -(kb[None, :] + modes)                  # closing mode for every k_c
        ida = table[ka[:, 0] + 2 * r, ka[:, 1] + 2 * r, ka[:, 2] + 2 * r]
        ok = ida >= 0
        ic = np.nonzero(ok)[0]
        ia = ida[ok]
        sa, sb, sc = shell[ia], shell[ib], shell[ic]
        order = (sa >= sb) & (sb >= sc)
        ia, ic, sa, sc = ia[order], ic[order], sa[order], sc[order]
        key = (sa * ns + sb) * ns + sc
        ntri += np.bincount(key, minlength=nbin)
        if vals is not None:
            w = vals[ia] * vals[ib] * vals[ic]
            msum_re += np.bincount(key, weights=w.real, minlength=nbin)
            msum_im += np.bincount(key, weights=w.imag, minlength=nbin)
    out_m, out_n = {}, {}
    for key in np.nonzero(ntri)[0]:
        a, rem = divmod(int(key), ns * ns)
        b, c = divmod(rem, ns)
        out_n[(a, b, c)] = int(ntri[key])
        out_m[(a, b, c)] = complex(msum_re[key], msum_im[key])
    return out_m, out_n


def direct_mean_k(plan: P.Plan):
    """{(a, b, c): (mean |k_a|, mean |k_b|, mean |k_c|)} over each bin's triangles (k_f units),
    by the same enumeration of ordered (k_b, k_c) pairs as direct_estimate."""
    modes, shell, r = ball_modes(plan)
    length = np.sqrt((modes * modes).sum(1).astype(np.float64))
    span = 4 * r + 1
    table = -np.ones((span, span, span), dtype=np.int64)
    table[modes[:, 0] + 2 * r, modes[:, 1] + 2 * r, modes[:, 2] + 2 * r] = np.arange(len(modes))
    ns = plan.ns
    nbin = ns * ns * ns
    ntri = np.zeros(nbin, dtype=np.int64)
    ksum = np.zeros((3, nbin))
    for ib in range(len(modes)):
        ka = -(modes[ib][None, :] + modes)
        ida = table[ka[:, 0] + 2 * r, ka[:, 1] + 2 * r, ka[:, 2] + 2 * r]
        ok = ida >= 0
        ic = np.nonzero(ok)[0]
        ia = ida[ok]
        sa, sb, sc = shell[ia], shell[ib], shell[ic]
        keep = (sa >= sb) & (sb >= sc)
        ia, ic, sa, sc = ia[keep], ic[keep], sa[keep], sc[keep]
        key = (sa * ns + sb) * ns + sc
        ntri += np.bincount(key, minlength=nbin)
        ksum[0] += np.bincount(key, weights=length[ia], minlength=nbin)
        ksum[1] += np.bincount(key, weights=np.full(len(key), length[ib]), minlength=nbin)
        ksum[2] += np.bincount(key, weights=length[ic], minlength=nbin)
    out = {}
    for key in np.nonzero(ntri)[0]:
        a, rem = divmod(int(key), ns * ns)
        b, c = divmod(rem, ns)
        out[(a, b, c)] = tuple(ksum[:, key] / ntri[key])
    return out
