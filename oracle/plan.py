"""Binning plan of the estimator, float64 / integer arithmetic (test infrastructure).

Follows Sec. 2.1 of the paper:
  * k space is split into spherical shells of fixed radial width (Sec. 2.1, "annular rings
    ... replaced with spherical shells" in 3D). Shell edges are given in units of the
    fundamental mode k_f = 2 pi / L. A mode m (integer vector, k = k_f m) belongs to shell n
    iff e_n^2 <= |m|^2 < e_{n+1}^2; because |m|^2 is an integer this is the integer test
    Q_n <= |m|^2 < Q_{n+1} with Q_n = ceil(e_n^2). The k = 0 mode belongs to no shell.
  * every multiset a >= b >= c of shells is one bin of triangles (Sec. 2.1, the count
    C(N_r + 2, 3) of Fig. 2's discussion).
  * k_n is the average length of the modes in shell n (Sec. 2.1); the bin label is
    t = k2/k1 and mu = (k1/k2 + k2/k1 - (k3/k1)(k3/k2)) / 2 (Eq. (2.4)).
  * the allowed region is 0.5 <= mu, t <= 1 and 2 mu t >= 1 (Eq. (2.2)).
  * modes must satisfy k < 2 pi Ng / (3 L), i.e. 9 |m|^2 < Ng^2 (Eq. (2.12) and the text
    after it), otherwise the FFT sum also counts triangles that wind around the box.

Shell means are summed over the distinct values q = |m|^2 in ascending order,
sum_q count(q) sqrt(q) / sum_q count(q), so any implementation that takes the same
steps in float64 reaches the same bits; the (mu, t) cell of a bin is decided from them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def shell_thresholds(edges_kf) -> np.ndarray:
    """Integer thresholds Q_n = ceil(e_n^2) (Q_0 at least 1 so that k = 0 is excluded)."""
    q = [int(math.ceil(float(e) * float(e))) for e in edges_kf]
    q[0] = max(1, q[0])
    return np.asarray(q, dtype=np.int64)


def aliasing_ok(ng: int, thresholds: np.ndarray) -> bool:
    """True iff every shell mode has |m| < Ng/3 (Eq. (2.12) cap): 9 (Q_Ns - 1) < Ng^2."""
    return 9 * (int(thresholds[-1]) - 1) < ng * ng


def q_counts(qmax: int) -> np.ndarray:
    """count[q] = number of integer vectors m in Z^3 with |m|^2 = q, for q < qmax."""
    r = int(math.isqrt(max(qmax - 1, 0)))
    m = np.arange(-r, r + 1, dtype=np.int64)
    q = (m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2).ravel()
    q = q[q < qmax]
    return np.bincount(q, minlength=qmax).astype(np.int64)


def shell_means(thresholds: np.ndarray):
    """(mode count, mean |m|) per shell, the mean taken in ascending q order (Sec. 2.1)."""
    ns = len(thresholds) - 1
    cnt = q_counts(int(thresholds[-1]))
    nmodes = np.zeros(ns, dtype=np.int64)
    kbar = np.zeros(ns, dtype=np.float64)
    for n in range(ns):
        s = 0.0
        c = 0
        for q in range(int(thresholds[n]), int(thresholds[n + 1])):
            if cnt[q]:
                s += float(cnt[q]) * math.sqrt(float(q))
                c += int(cnt[q])
        nmodes[n] = c
        kbar[n] = s / c if c else float("nan")
    return nmodes, kbar


def all_triplets(ns: int):
    """Every multiset a >= b >= c of Ns shells, in ascending lexicographic (a, b, c) order."""
    return [(a, b, c) for a in range(ns) for b in range(a + 1) for c in range(b + 1)]


def may_close(thresholds: np.ndarray, a: int, b: int, c: int) -> bool:
    """Necessary condition for a closed triangle with one mode in each shell:
    smallest |k_a| <= largest |k_b| + largest |k_c| (triangle inequality)."""
    qa = float(thresholds[a])
    qb = float(thresholds[b + 1] - 1)
    qc = float(thresholds[c + 1] - 1)
    return math.sqrt(qa) <= math.sqrt(qb) + math.sqrt(qc)


def shape_label(k1: float, k2: float, k3: float):
    """(mu, t) of Eq. (2.4) from the mean lengths k1 >= k2 >= k3."""
    t = k2 / k1
    mu = 0.5 * (k1 / k2 + k2 / k1 - (k3 / k1) * (k3 / k2))
    return mu, t


def shape_cell(mu: float, t: float, n_mu: int, n_t: int):
    """Cell of a uniform n_mu x n_t grid over [0.5, 1]^2 (half-open, last cell closed at 1).
    mu is clamped to [0.5, 1] and t to [0.5, 1] first: mean lengths of shells that close only
    through the shell width can give mu > 1 or t < 0.5, outside the region of Eq. (2.2)."""
    mc = min(max(mu, 0.5), 1.0)
    tc = min(max(t, 0.5), 1.0)
    im = int(math.floor((mc - 0.5) * (2.0 * n_mu)))
    it = int(math.floor((tc - 0.5) * (2.0 * n_t)))
    return min(im, n_mu - 1), min(it, n_t - 1)


def in_region(mu: float, t: float) -> bool:
    """Eq. (2.2): 0.5 <= t, mu <= 1 and 2 mu t >= 1."""
    return 0.5 <= t <= 1.0 and 0.5 <= mu <= 1.0 and 2.0 * mu * t >= 1.0


@dataclass
class Plan:
    ng: int
    box_len: float
    edges: np.ndarray
    thresholds: np.ndarray
    nmodes: np.ndarray
    kbar: np.ndarray               # units of k_f
    candidates: list               # (a, b, c) passing may_close
    n_mu: int = 10
    n_t: int = 10
    extra: dict = field(default_factory=dict)
    k1_merge: int = 1              # k1 shells per (mu, t) cell group (Sec. 2.1, merging bins)
    label_k: str = "shell"         # "shell": k of Eq. (2.4) = shell means; "triangle": bin means

    @property
    def n_groups(self) -> int:
        return (self.ns + self.k1_merge - 1) // self.k1_merge

    @property
    def ns(self) -> int:
        return len(self.thresholds) - 1

    @property
    def kf(self) -> float:
        return 2.0 * math.pi / self.box_len

    @property
    def vcell(self) -> float:
        return (self.box_len / self.ng) ** 3

    @property
    def volume(self) -> float:
        return self.box_len ** 3


def make_plan(ng: int, box_len: float, edges_kf, n_mu: int = 10, n_t: int = 10,
              allow_aliasing: bool = False, k1_merge: int = 1, label_k: str = "shell") -> Plan:
    """Shells, their mode counts and means, and the candidate triplets (Sec. 2.1)."""
    edges = np.asarray(edges_kf, dtype=np.float64)
    if edges.ndim != 1 or len(edges) < 2 or np.any(np.diff(edges) <= 0):
        raise ValueError("edges must be strictly increasing, at least two")
    thr = shell_thresholds(edges)
    if np.any(np.diff(thr) <= 0):
        raise ValueError("an empty shell: two edges share the same integer threshold")
    if not allow_aliasing and not aliasing_ok(ng, thr):
        raise ValueError("largest shell edge reaches k >= 2 pi Ng / (3 L) (Eq. (2.12) cap)")
    nm, kb = shell_means(thr)
    if np.any(nm == 0):
        raise ValueError("a shell holds no modes")
    cand = [t for t in all_triplets(len(thr) - 1) if may_close(thr, *t)]
    if k1_merge < 1:
        raise ValueError("k1_merge must be >= 1")
    if label_k not in ("shell", "triangle"):
        raise ValueError("label_k must be 'shell' or 'triangle'")
    return Plan(ng, float(box_len), edges, thr, nm, kb, cand, n_mu, n_t, k1_merge=k1_merge,
                label_k=label_k)


def linear_edges(ns: int, lo: float, hi: float) -> np.ndarray:
    """Ns shells of equal width from lo to hi (units of k_f), the paper's preferred choice."""
    return np.linspace(lo, hi, ns + 1)


def label_table(plan: Plan, triplets, kvals=None):
    """Per triplet: (k1, k2, k3) in k_f units, mu, t, cell (i_mu, i_t), in-region flag. The
    lengths are the shells' mean |k| (kbar), or kvals[i] (one row of three per triplet) when
    given, e.g. the means over each bin's triangles."""
    out = []
    for i, (a, b, c) in enumerate(triplets):
        if kvals is None:
            k1, k2, k3 = plan.kbar[a], plan.kbar[b], plan.kbar[c]
        else:
            k1, k2, k3 = (float(v) for v in kvals[i])
        mu, t = shape_label(k1, k2, k3)
        im, it = shape_cell(mu, t, plan.n_mu, plan.n_t)
        out.append(dict(a=a, b=b, c=c, k1=k1, k2=k2, k3=k3, mu=mu, t=t,
                        i_mu=im, i_t=it, inside=in_region(mu, t)))
    return out


def shell_index_half(plan: Plan) -> np.ndarray:
    """Shell index (or -1) of every mode of the half grid [Ng][Ng][Ng/2+1]."""
    ng = plan.ng
    m = np.fft.fftfreq(ng, d=1.0 / ng).astype(np.int64)
    mz = np.arange(ng // 2 + 1, dtype=np.int64)
    q = m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2
    idx = np.searchsorted(plan.thresholds, q, side="right") - 1
    idx[(q < plan.thresholds[0]) | (q >= plan.thresholds[-1])] = -1
    return idx.astype(np.int32)
