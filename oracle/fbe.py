"""The FFT bispectrum estimator (FBE) written out plainly in float64 (test infrastructure).

Steps, in the paper's order (Sec. 2.2):
  1. Delta(k) = V_c F(k), F the unnormalised DFT sum_x delta(x) e^{-i k.x} (the input).
     Optional linear RSD, Eq. (3.4): Delta^s(k) = (1 + beta mu_k^2) Delta(k), mu_k = k_z/|k|.
  2. shell fields, Eq. (2.8): D(k_n, x) = sum_{k in shell n} Delta(k) e^{-i k.x}. With
     d_n(x) = sum_{k in n} F(k) e^{+i k.x} (an unnormalised inverse real FFT of the masked
     spectrum) one has D(k_n, x) = V_c d_n(-x); the sign of the exponent is immaterial
     because the sum over x in Eq. (2.7) runs over the whole periodic grid.
  3. counting fields, Eq. (2.11): i_n(x) = sum_{k in n} e^{+i k.x}.
  4. Eq. (2.7) with Eq. (2.10):
        B_abc = V_c^3 sum_x d_a d_b d_c / (V N_tri Ng^3),  N_tri = sum_x i_a i_b i_c / Ng^3,
     so B_abc = V_c^3 sum_x d_a d_b d_c / (V sum_x i_a i_b i_c); Ng^3 cancels.
  5. label every bin with (k1, mu, t) (Eq. (2.4)) and, for the (mu, t) grid, merge the bins
     of one k1 shell (or of plan.k1_merge neighbouring k1 shells) that fall in one cell as one
     bigger bin of Eq. (2.3):
        B_cell = V_c^3 sum_{bins} sum_x d d d / (V sum_{bins} sum_x i i i)
     (Sec. 2.1 last paragraph: merging adjacent bins).

A library routine (numpy/pocketfft irfftn, a matrix-vector product) serves as a step;
nothing is blocked, fused or reordered beyond that.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from . import plan as P


def kaiser_factor_half(ng: int, beta: float) -> np.ndarray:
    """1 + beta (m_z / |m|)^2 on the half grid (Eq. (3.4)); the k = 0 entry is 1."""
    m = np.fft.fftfreq(ng, d=1.0 / ng)
    mz = np.arange(ng // 2 + 1, dtype=np.float64)
    q = m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2
    q[0, 0, 0] = 1.0
    return 1.0 + beta * (mz[None, None, :] ** 2) / q


def shell_fields(spec_half: np.ndarray, plan: P.Plan, shells=None, workers: int = -1):
    """d_n(x) for the requested shells: unnormalised inverse real FFT of S_n F (Eq. (2.8))."""
    ng = plan.ng
    sidx = P.shell_index_half(plan)
    shells = range(plan.ns) if shells is None else shells
    out = {}
    for n in shells:
        masked = np.where(sidx == n, spec_half, 0.0).astype(np.complex128)
        out[n] = sfft.irfftn(masked, s=(ng, ng, ng), workers=workers) * float(ng) ** 3
    return out


def shell_fields_on_grid(spec_half: np.ndarray, plan: P.Plan, size: int, shells=None, workers: int = -1):
    """d_n of Eq. (2.8) sampled at x = (i, j, l) L / size on a size^3 grid, for a size that holds
    every shell mode (|m_i| < size / 2): each shell's modes are copied from the ng half spectrum
    into a size^3 half spectrum, which is inverse transformed (unnormalised)."""
    ng = plan.ng
    sidx = P.shell_index_half(plan)
    m = np.fft.fftfreq(size, d=1.0 / size).astype(np.int64) % ng
    mz = np.arange(size // 2 + 1)
    sub_spec = spec_half[np.ix_(m, m, mz)]
    sub_idx = sidx[np.ix_(m, m, mz)]
    shells = range(plan.ns) if shells is None else shells
    out = {}
    for n in shells:
        masked = np.where(sub_idx == n, sub_spec, 0.0).astype(np.complex128)
        out[n] = sfft.irfftn(masked, s=(size, size, size), workers=workers) * float(size) ** 3
    return out


def counting_fields(plan: P.Plan, shells=None, workers: int = -1):
    """i_n(x) = sum_{k in n} e^{+i k.x} (Eq. (2.11))."""
    ng = plan.ng
    ones = np.ones((ng, ng, ng // 2 + 1), dtype=np.complex128)
    return shell_fields(ones, plan, shells, workers)


def length_fields(plan: P.Plan, shells=None, workers: int = -1):
    """w_n(x) = sum_{k in n} |k| e^{+i k.x}, |k| in units of k_f: the counting field of
    Eq. (2.11) with every mode weighted by its length."""
    ng = plan.ng
    m = np.fft.fftfreq(ng, d=1.0 / ng)
    mz = np.arange(ng // 2 + 1, dtype=np.float64)
    q = m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2
    return shell_fields(np.sqrt(q).astype(np.complex128), plan, shells, workers)


def triangle_mean_k(plan: P.Plan, triplets, workers: int = -1) -> np.ndarray:
    """Per bin (a, b, c): the mean of |k_a|, |k_b| and |k_c| over its closed triangles (k_f
    units), the size and shape of the bin's average triangle (Sec. 2.1):
        kbar_1 = sum_x w_a i_b i_c / sum_x i_a i_b i_c   (likewise w_b for kbar_2, w_c for kbar_3),
    the sums of Eq. (2.10) with one counting field replaced by its length-weighted one."""
    need = sorted({s for t in triplets for s in t})
    f = dict(counting_fields(plan, need, workers))
    f.update({("w", n): v for n, v in length_fields(plan, need, workers).items()})
    tsum = triple_sums(f, triplets)
    out = np.empty((len(triplets), 3))
    for j in range(3):
        wt = [tuple(("w", s) if i == j else s for i, s in enumerate(t)) for t in triplets]
        out[:, j] = triple_sums(f, wt) / tsum
    return out


def triple_sums(fields: dict, triplets, absolute: bool = False) -> np.ndarray:
    """sum_x f_a f_b f_c for each (a, b, c) (Eq. (2.7) and Eq. (2.10) numerators).

    For each pair (a, b) the product f_a f_b is formed once and contracted with every f_c
    the pair needs (a matrix-vector product). `absolute` sums |f_a f_b f_c| instead,
    the scale against which rounding errors of a lower-precision path are measured."""
    out = np.zeros(len(triplets), dtype=np.float64)
    by_pair = {}
    for i, (a, b, c) in enumerate(triplets):
        by_pair.setdefault((a, b), []).append((i, c))
    for (a, b), lst in by_pair.items():
        prod = (fields[a] * fields[b]).ravel()
        cs = [c for _, c in lst]
        mat = np.stack([fields[c].ravel() for c in cs])
        if absolute:
            vals = np.abs(mat) @ np.abs(prod)
        else:
            vals = mat @ prod
        for (i, _), v in zip(lst, vals):
            out[i] = v
    return out


def triangle_counts(plan: P.Plan, workers: int = -1):
    """(T_abc = sum_x i_a i_b i_c, N_tri = T / Ng^3) over the plan's candidate triplets."""
    ifields = counting_fields(plan, workers=workers)
    tsum = triple_sums(ifields, plan.candidates)
    return tsum, tsum / float(plan.ng) ** 3


def kept_triplets(plan: P.Plan, workers: int = -1):
    """Bins with at least one closed triangle, with their T and integer N_tri."""
    tsum, ntri = triangle_counts(plan, workers)
    rnd = np.rint(ntri)
    if np.any(np.abs(ntri - rnd) > 1e-3):
        raise ArithmeticError("N_tri not integral within 1e-3")
    keep = rnd > 0
    trips = [t for t, k in zip(plan.candidates, keep) if k]
    return trips, tsum[keep], rnd[keep].astype(np.int64)


def estimate(spec_half: np.ndarray, plan: P.Plan, beta: float | None = None,
             workers: int = -1, with_abs: bool = False, counts=None):
    """The whole estimator on one field. Returns a dict with
    triplets, tsum, ntri, msum (sum_x d d d), b (per bin), labels, grid (Ns, Nmu, Nt)
    with NaN in empty cells, grid_count, and optionally asum (sum_x |d d d|)."""
    spec = np.asarray(spec_half, dtype=np.complex128)
    if beta is not None:
        spec = spec * kaiser_factor_half(plan.ng, beta)
    trips, tsum, ntri = counts if counts is not None else kept_triplets(plan, workers)
    needed = sorted({s for t in trips for s in t})
    dfields = shell_fields(spec, plan, needed, workers)
    msum = triple_sums(dfields, trips)
    norm = plan.vcell ** 3 / plan.volume
    b = norm * msum / tsum
    kvals = triangle_mean_k(plan, trips, workers) if plan.label_k == "triangle" else None
    labels = P.label_table(plan, trips, kvals)
    grid, gcount = merge_cells(plan, trips, labels, msum, tsum)
    res = dict(triplets=trips, tsum=tsum, ntri=ntri, msum=msum, b=b, labels=labels,
               grid=grid, grid_count=gcount)
    if with_abs:
        res["asum"] = triple_sums(dfields, trips, absolute=True)
        res["b_scale"] = norm * res["asum"] / tsum
    return res


def merge_cells(plan: P.Plan, trips, labels, msum, tsum):
    """Per (k1 group, mu cell, t cell): V_c^3 sum M / (V sum T), bins added in list order; a
    group holds plan.k1_merge consecutive k1 shells (the last one fewer)."""
    ns, nm, nt = plan.n_groups, plan.n_mu, plan.n_t
    num = np.zeros((ns, nm, nt))
    den = np.zeros((ns, nm, nt))
    cnt = np.zeros((ns, nm, nt), dtype=np.int64)
    for (a, _, _), lab, m, t in zip(trips, labels, msum, tsum):
        gi = a // plan.k1_merge
        num[gi, lab["i_mu"], lab["i_t"]] += m
        den[gi, lab["i_mu"], lab["i_t"]] += t
        cnt[gi, lab["i_mu"], lab["i_t"]] += 1
    norm = plan.vcell ** 3 / plan.volume
    with np.errstate(invalid="ignore", divide="ignore"):
        grid = np.where(cnt > 0, norm * num / den, np.nan)
    return grid, cnt
