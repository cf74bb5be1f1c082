"""The estimator on a 2D box: annular rings in place of spherical shells (test infrastructure,
float64). Sec. 2.1 introduces the binning on a 2D box (Figs. 1-2), Fig. 4 draws the aliasing of
the triangle counts for it, and the timing comparison of Sec. 2.2 (Fig. 5) is made in 2D.

The steps are those of plan.py / fbe.py / dbe.py with k = k_f (m_x, m_y), k_f = 2 pi / L:
  * ring n holds the modes with e_n^2 <= |m|^2 < e_{n+1}^2 (Q_n = ceil(e_n^2)); k = 0 is in no
    ring; k_n is the mean |m| over the ring's modes, summed over q = |m|^2 in ascending order.
  * every multiset a >= b >= c of rings passing the triangle inequality is a candidate bin; bins
    with N_tri > 0 are kept; labels by Eq. (2.4), cells and the allowed region as in 3D.
  * d_n(x) = sum_{k in n} F(k) e^{+i k.x} and i_n(x) = sum_{k in n} e^{+i k.x} on the Ng^2 grid
    (Eq. (2.8) and Eq. (2.11) in 2D), F the unnormalised 2D DFT and Delta = A_c F with the
    cell area A_c = (L / Ng)^2.
  * B_abc = A_c^3 sum_x d_a d_b d_c / (A sum_x i_a i_b i_c) with the box area A = L^2 (Eq. (2.7)
    with Eq. (2.10), area for volume), N_tri = sum_x i_a i_b i_c / Ng^2.
  * every ring mode needs |m| < Ng / 3 (the cap after Eq. (2.12), Fig. 4): 9 (Q_N - 1) < Ng^2.
  * direct_estimate: the loop of Sec. 2.1 over pairs (k_b, k_c) with k_a = -(k_b + k_c) looked
    up, for every bin at once (tiny grids only).
Arrays are C-order [x][y]; y is the axis the real FFT halves.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

from . import fbe
from . import plan as P


def q_counts_2d(qmax: int) -> np.ndarray:
    """count[q] = number of integer vectors m in Z^2 with |m|^2 = q, for q < qmax."""
    r = int(math.isqrt(max(qmax - 1, 0)))
    m = np.arange(-r, r + 1, dtype=np.int64)
    q = (m[:, None] ** 2 + m[None, :] ** 2).ravel()
    return np.bincount(q[q < qmax], minlength=qmax).astype(np.int64)


@dataclass
class Plan2D:
    ng: int
    box_len: float
    edges: np.ndarray
    thresholds: np.ndarray
    nmodes: np.ndarray
    kbar: np.ndarray               # units of k_f
    candidates: list
    n_mu: int = 10
    n_t: int = 10
    k1_merge: int = 1

    @property
    def ns(self) -> int:
        return len(self.thresholds) - 1

    @property
    def n_groups(self) -> int:
        return self.ns

    @property
    def kf(self) -> float:
        return 2.0 * math.pi / self.box_len

    @property
    def vcell(self) -> float:
        """Cell area A_c (the 2D counterpart of V_c)."""
        return (self.box_len / self.ng) ** 2

    @property
    def volume(self) -> float:
        """Box area A = L^2."""
        return self.box_len ** 2


def make_plan_2d(ng: int, box_len: float, edges_kf, n_mu: int = 10, n_t: int = 10,
                 allow_aliasing: bool = False) -> Plan2D:
    """Rings, their mode counts and mean lengths, and the candidate bins."""
    edges = np.asarray(edges_kf, dtype=np.float64)
    if edges.ndim != 1 or len(edges) < 2 or np.any(np.diff(edges) <= 0):
        raise ValueError("edges must increase")
    thr = P.shell_thresholds(edges)
    if not allow_aliasing and not P.aliasing_ok(ng, thr):
        raise ValueError("largest ring reaches k >= 2 pi Ng / (3 L)")
    cnt = q_counts_2d(int(thr[-1]))
    ns = len(thr) - 1
    nm = np.zeros(ns, dtype=np.int64)
    kb = np.zeros(ns)
    for n in range(ns):
        s, c = 0.0, 0
        for q in range(int(thr[n]), int(thr[n + 1])):
            if cnt[q]:
                s += float(cnt[q]) * math.sqrt(float(q))
                c += int(cnt[q])
        if c == 0:
            raise ValueError("a ring holds no modes")
        nm[n], kb[n] = c, s / c
    cand = [t for t in P.all_triplets(ns) if P.may_close(thr, *t)]
    return Plan2D(ng, float(box_len), edges, thr, nm, kb, cand, n_mu, n_t)


def ring_index_half(plan: Plan2D) -> np.ndarray:
    """Ring index (or -1) of every mode of the half grid [Ng][Ng/2+1]."""
    ng = plan.ng
    m = np.fft.fftfreq(ng, d=1.0 / ng).astype(np.int64)
    my = np.arange(ng // 2 + 1, dtype=np.int64)
    q = m[:, None] ** 2 + my[None, :] ** 2
    idx = np.searchsorted(plan.thresholds, q, side="right") - 1
    idx[(q < plan.thresholds[0]) | (q >= plan.thresholds[-1])] = -1
    return idx.astype(np.int32)


def ring_fields(spec_half: np.ndarray, plan: Plan2D, rings=None):
    """d_n(x): unnormalised inverse real 2D FFT of the spectrum masked to ring n."""
    ng = plan.ng
    ridx = ring_index_half(plan)
    rings = range(plan.ns) if rings is None else rings
    return {n: sfft.irfftn(np.where(ridx == n, spec_half, 0.0).astype(np.complex128), s=(ng, ng)) * float(ng) ** 2
            for n in rings}


def counting_fields(plan: Plan2D, rings=None):
    """i_n(x) = sum_{k in n} e^{+i k.x}."""
    ng = plan.ng
    return ring_fields(np.ones((ng, ng // 2 + 1), dtype=np.complex128), plan, rings)


def kept_triplets(plan: Plan2D):
    """Bins with at least one closed triangle, with T = sum_x i i i and integer N_tri."""
    tsum = fbe.triple_sums(counting_fields(plan), plan.candidates)
    ntri = tsum / float(plan.ng) ** 2
    rnd = np.rint(ntri)
    if np.any(np.abs(ntri - rnd) > 1e-3):
        raise ArithmeticError("N_tri not integral within 1e-3")
    keep = rnd > 0
    trips = [t for t, k in zip(plan.candidates, keep) if k]
    return trips, tsum[keep], rnd[keep].astype(np.int64)


def estimate(spec_half: np.ndarray, plan: Plan2D, with_abs: bool = False, counts=None):
    """The whole estimator on one 2D field; the same dict as fbe.estimate."""
    trips, tsum, ntri = counts if counts is not None else kept_triplets(plan)
    need = sorted({s for t in trips for s in t})
    d = ring_fields(np.asarray(spec_half, dtype=np.complex128), plan, need)
    msum = fbe.triple_sums(d, trips)
    norm = plan.vcell ** 3 / plan.volume
    labels = P.label_table(plan, trips)
    grid, gcount = fbe.merge_cells(plan, trips, labels, msum, tsum)
    res = dict(triplets=trips, tsum=tsum, ntri=ntri, msum=msum, b=norm * msum / tsum, labels=labels,
               grid=grid, grid_count=gcount)
    if with_abs:
        res["asum"] = fbe.triple_sums(d, trips, absolute=True)
        res["b_scale"] = norm * res["asum"] / tsum
    return res


def direct_estimate(spec_half, plan: Plan2D, count_only: bool = False):
    """({(a,b,c): sum F(k_a) F(k_b) F(k_c)}, {(a,b,c): N_tri}) over every bin with a triangle,
    enumerating ordered pairs (k_b, k_c) of the disc the rings cover."""
    r = int(math.ceil(math.sqrt(float(plan.thresholds[-1])))) + 1
    g = np.arange(-r, r + 1, dtype=np.int64)
    mx, my = np.meshgrid(g, g, indexing="ij")
    modes = np.stack([mx.ravel(), my.ravel()], axis=1)
    q = (modes * modes).sum(1)
    sel = (q >= plan.thresholds[0]) & (q < plan.thresholds[-1])
    modes, q = modes[sel], q[sel]
    ring = np.searchsorted(plan.thresholds, q, side="right") - 1
    vals = None
    if not count_only:
        ng = plan.ng
        neg = modes[:, 1] < 0
        sx = np.where(neg, -modes[:, 0], modes[:, 0]) % ng
        sy = np.where(neg, -modes[:, 1], modes[:, 1])
        v = np.asarray(spec_half, dtype=np.complex128)[sx, sy]
        vals = np.where(neg, np.conj(v), v)
    span = 4 * r + 1
    table = -np.ones((span, span), dtype=np.int64)
    table[modes[:, 0] + 2 * r, modes[:, 1] + 2 * r] = np.arange(len(modes))
    ns = plan.ns
    nbin = ns ** 3
    ntri = np.zeros(nbin, dtype=np.int64)
    m_re = np.zeros(nbin)
    m_im = np.zeros(nbin)
    for ib in range(len(modes)):
        ka = -(modes[ib][None, :] + modes)
        ida = table[ka[:, 0] + 2 * r, ka[:, 1] + 2 * r]
        ok = ida >= 0
        ic = np.nonzero(ok)[0]
        ia = ida[ok]
        sa, sb, sc = ring[ia], ring[ib], ring[ic]
        keep = (sa >= sb) & (sb >= sc)
        ia, ic, sa, sc = ia[keep], ic[keep], sa[keep], sc[keep]
        key = (sa * ns + sb) * ns + sc
        ntri += np.bincount(key, minlength=nbin)
        if vals is not None:
            w = vals[ia] * vals[ib] * vals[ic]
            m_re += np.bincount(key, weights=w.real, minlength=nbin)
            m_im += np.bincount(key, weights=w.imag, minlength=nbin)
    out_m, out_n = {}, {}
    for key in np.nonzero(ntri)[0]:
        a, rem = divmod(int(key), ns * ns)
        b, c = divmod(rem, ns)
        out_n[(a, b, c)] = int(ntri[key])
        out_m[(a, b, c)] = complex(m_re[key], m_im[key])
    return out_m, out_n


def expected_binned_2d(plan: Plan2D, triplets, n_index: float, f_ng: float) -> np.ndarray:
    """<B_abc> of the 2D quadratic field at first order in f_NG (Eq. (2.5) with Eq. (3.2)
    summed over the bin's grid triangles, as analytic.expected_binned does in 3D):
    2 f_NG / T_abc sum_x [(Pi)_a (Pi)_b i_c + (Pi)_b (Pi)_c i_a + (Pi)_c (Pi)_a i_b]."""
    ng = plan.ng
    m = np.fft.fftfreq(ng, d=1.0 / ng)
    my = np.arange(ng // 2 + 1, dtype=np.float64)
    q = m[:, None] ** 2 + my[None, :] ** 2
    q[0, 0] = 1.0
    pk = (plan.kf * np.sqrt(q)) ** (-n_index)
    rings = sorted({s for t in triplets for s in t})
    pi_f = ring_fields(pk.astype(np.complex128), plan, rings)
    i_f = counting_fields(plan, rings)
    t_abc = fbe.triple_sums(i_f, triplets)
    s = np.array([float(np.sum(pi_f[a] * pi_f[b] * i_f[c] + pi_f[b] * pi_f[c] * i_f[a]
                                + pi_f[c] * pi_f[a] * i_f[b])) for (a, b, c) in triplets])
    return 2.0 * f_ng * s / t_abc
