"""Pins of the oracle's estimator (Sec. 2.2) to brute force, closed forms and invariants. CPU only."""
import numpy as np
import pytest

import fieldgen
from oracle import analytic as A
from oracle import dbe
from oracle import fbe
from oracle import plan as P


def _plan(ng, ns=8, top=None, **kw):
    return P.make_plan(ng, float(ng), P.linear_edges(ns, 1.0, top or ng / 4), **kw)


@pytest.mark.parametrize("ng,seed", [(16, 2), (32, 1)])
def test_fbe_equals_direct_summation(ng, seed):
    """Eq. (2.7)/(2.10) through FFTs equal Eq. (2.3)/(2.9) summed mode by mode."""
    pl = _plan(ng)
    spec = fieldgen.spectrum(fieldgen.quadratic_field(ng, float(ng), 2.0, 0.1, seed))
    res = fbe.estimate(spec, pl)
    msum_d, ntri_d = dbe.direct_estimate(spec, pl)
    assert set(ntri_d) == set(res["triplets"])
    ng3 = float(ng) ** 3
    for i, t in enumerate(res["triplets"]):
        assert ntri_d[t] == res["ntri"][i]
        m = msum_d[t]
        assert abs(m.imag) <= 1e-12 * abs(m.real) + 1e-9
        assert abs(res["msum"][i] / ng3 - m.real) <= 1e-12 * abs(m.real)


def test_triangle_counts_alias_above_cap():
    """Fig. 4: above k = 2 pi Ng/(3L) the FFT count exceeds the direct count; below it agrees."""
    ng = 16
    pl = _plan(ng, ns=6, top=7.0, allow_aliasing=True)
    tsum, ntri = fbe.triangle_counts(pl)
    _, ntri_d = dbe.direct_estimate(None, pl, count_only=True)
    over = 0
    for t, n in zip(pl.candidates, np.rint(ntri).astype(int)):
        nd = ntri_d.get(t, 0)
        kmax = np.sqrt(pl.thresholds[t[0] + 1] - 1)
        if 3 * kmax < ng:
            assert n == nd
        else:
            assert n >= nd
            over += n > nd
    assert over > 0


def test_closed_form_three_cosines():
    """delta = 2A [cos(k1.x) + cos(k2.x) + cos(k3.x)] with k1 + k2 + k3 = 0 in three shells:
    sum_x d_a d_b d_c = 8 A^3 Ng^9 sum_x cos cos cos = 2 A^3 Ng^12 (all other products vanish)."""
    ng, amp = 32, 0.7
    pl = _plan(ng)
    m1, m2 = np.array([6, 1, 2]), np.array([-2, -3, 1])
    m3 = -(m1 + m2)
    x = np.indices((ng, ng, ng)).reshape(3, -1).T
    delta = sum(2 * amp * np.cos(2 * np.pi * (x @ m) / ng) for m in (m1, m2, m3)).reshape(ng, ng, ng)
    sh = [int(np.searchsorted(pl.thresholds, (m * m).sum(), side="right") - 1) for m in (m1, m2, m3)]
    a, b, c = sorted(sh, reverse=True)
    assert a > b > c
    res = fbe.estimate(fieldgen.spectrum(delta), pl)
    i = res["triplets"].index((a, b, c))
    assert abs(res["msum"][i] - 2 * amp ** 3 * float(ng) ** 12) <= 1e-10 * 2 * amp ** 3 * float(ng) ** 12
    others = [abs(v) for j, v in enumerate(res["msum"]) if j != i]
    assert max(others) <= 1e-9 * float(ng) ** 12


def test_kaiser_factor_special_modes():
    """Eq. (3.4) at modes whose angle to the line of sight (z) is known by construction: along z
    the factor is 1 + beta, across it 1, at 45 degrees in the x-z plane 1 + beta/2, and on the
    3-4-5 direction (4, 0, 3) it is 1 + 9 beta/25; k = 0 keeps factor 1."""
    ng, beta = 16, 0.7
    f = fbe.kaiser_factor_half(ng, beta)
    assert f[0, 0, 0] == 1.0
    assert abs(f[0, 0, 5] - (1 + beta)) < 1e-15
    assert abs(f[5, 0, 0] - 1.0) < 1e-15 and abs(f[0, 5, 0] - 1.0) < 1e-15
    assert abs(f[3, 0, 3] - (1 + beta / 2)) < 1e-15 and abs(f[ng - 3, 0, 3] - (1 + beta / 2)) < 1e-15
    assert abs(f[4, 0, 3] - (1 + 9 * beta / 25)) < 1e-15 and abs(f[0, ng - 4, 3] - (1 + 9 * beta / 25)) < 1e-15


def test_closed_form_three_cosines_with_rsd():
    """Three plane waves of amplitude 2A on a 3-4-5 triangle, m1 = (0, 0, 3) along the line of
    sight, m2 = (4, 0, -3), m3 = (-4, 0, 0) across it: linear RSD (Eq. (3.4)) multiplies each wave
    by 1 + beta mu^2 with mu^2 = 1, 9/25 and 0 (the cosines of the triangle's angles with z), so
    the bin's triple sum is the real-space closed form 2 A^3 Ng^12 times (1 + beta)(1 + 9 beta/25).
    Using mu for mu^2, the x axis for z, or |m| for |m|^2 changes the product."""
    ng, amp, beta = 32, 0.7, 0.6
    pl = _plan(ng)
    m1, m2 = np.array([0, 0, 3]), np.array([4, 0, -3])
    m3 = -(m1 + m2)
    x = np.indices((ng, ng, ng)).reshape(3, -1).T
    delta = sum(2 * amp * np.cos(2 * np.pi * (x @ m) / ng) for m in (m1, m2, m3)).reshape(ng, ng, ng)
    sh = [int(np.searchsorted(pl.thresholds, (m * m).sum(), side="right") - 1) for m in (m1, m2, m3)]
    a, b, c = sorted(sh, reverse=True)
    assert a > b > c
    res = fbe.estimate(fieldgen.spectrum(delta), pl, beta=beta)
    i = res["triplets"].index((a, b, c))
    want = 2 * amp ** 3 * float(ng) ** 12 * (1 + beta) * (1 + 9 * beta / 25)
    assert abs(res["msum"][i] - want) <= 1e-10 * want
    others = [abs(v) for j, v in enumerate(res["msum"]) if j != i]
    assert max(others) <= 1e-9 * float(ng) ** 12


def test_invariants():
    """Translation, the cube symmetries, delta -> alpha delta (alpha^3) and delta -> -delta."""
    ng = 16
    pl = _plan(ng)
    d = fieldgen.quadratic_field(ng, float(ng), 2.0, 0.3, 5)
    counts = fbe.kept_triplets(pl)
    b0 = fbe.estimate(fieldgen.spectrum(d), pl, counts=counts)["b"]
    scale = np.abs(b0).max()

    def b(x):
        return fbe.estimate(fieldgen.spectrum(x), pl, counts=counts)["b"]

    assert np.abs(b(np.roll(d, (3, -5, 7), axis=(0, 1, 2))) - b0).max() <= 1e-12 * scale
    assert np.abs(b(np.transpose(d, (2, 0, 1))) - b0).max() <= 1e-12 * scale
    assert np.abs(b(d[::-1, :, ::-1]) - b0).max() <= 1e-12 * scale
    assert np.abs(b(2.5 * d) - 2.5 ** 3 * b0).max() <= 1e-12 * 2.5 ** 3 * scale
    assert np.abs(b(-d) + b0).max() <= 1e-12 * scale


def test_parseval_shell_power():
    """sum_x d_n^2 = Ng^3 sum_{k in n} |F(k)|^2 over the full grid (Parseval)."""
    ng = 32
    pl = _plan(ng)
    d = fieldgen.quadratic_field(ng, float(ng), 1.5, 0.1, 9)
    spec = fieldgen.spectrum(d)
    fields = fbe.shell_fields(spec, pl)
    full = np.fft.fftn(d)
    m = np.fft.fftfreq(ng, 1.0 / ng)
    q = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    for n in range(pl.ns):
        sel = (q >= pl.thresholds[n]) & (q < pl.thresholds[n + 1])
        lhs = float(np.sum(fields[n] ** 2))
        rhs = float(ng) ** 3 * float(np.sum(np.abs(full[sel]) ** 2))
        assert abs(lhs - rhs) <= 1e-12 * rhs


@pytest.mark.parametrize("beta", [None, 0.5])
def test_ensemble_mean_matches_expected_bispectrum(beta):
    """Mean over 100 realisations of the quadratic field (Eq. (3.1), f_NG = 0.5 as in Sec. 3)
    against Eq. (2.5) with Eq. (3.2) summed over the grid triangles (with Eq. (3.4) factors for
    RSD); chi^2 per bin about 1. A 30 percent error gives chi^2/dof ~ 10, a sign error ~ 500."""
    ng, f = 32, 0.5
    pl = _plan(ng)
    counts = fbe.kept_triplets(pl)
    exp = A.expected_binned(pl, counts[0], 2.0, f, beta=beta)
    bs = np.array([fbe.estimate(fieldgen.spectrum(fieldgen.quadratic_field(ng, float(ng), 2.0, f, 1000 + s)),
                                pl, beta=beta, counts=counts)["b"] for s in range(100)])
    z = (bs.mean(0) - exp) / (bs.std(0, ddof=1) / np.sqrt(len(bs)))
    assert np.mean(z ** 2) < 2.0
    assert np.mean(np.abs(z) > 4) < 0.02


def test_gaussian_field_has_zero_mean_bispectrum():
    ng = 32
    pl = _plan(ng)
    counts = fbe.kept_triplets(pl)
    bs = np.array([fbe.estimate(fieldgen.spectrum(fieldgen.gaussian_field(ng, float(ng), 2.0, 50 + s)),
                                pl, counts=counts)["b"] for s in range(60)])
    z = bs.mean(0) / (bs.std(0, ddof=1) / np.sqrt(len(bs)))
    assert np.mean(z ** 2) < 2.0


def test_expected_binned_tends_to_eq_3_2_at_shell_means():
    """For bins far from the squeezed and linear limits, the grid-summed expectation is close
    to Eq. (3.2) evaluated at the shell means (finite-width effects of a few percent)."""
    ng, f = 64, 0.5
    pl = _plan(ng, ns=8)
    trips = [(7, 7, 7), (7, 6, 5), (6, 6, 6), (7, 7, 6)]
    exp = A.expected_binned(pl, trips, 2.0, f)
    for (a, b, c), e in zip(trips, exp):
        p = A.power_law(pl.kf * pl.kbar[[a, b, c]], 2.0)
        ana = A.b_ana(p[0], p[1], p[2], f)
        assert abs(e - ana) <= 0.05 * ana


def test_condition_scale_bounds_the_sum():
    ng = 16
    pl = _plan(ng)
    spec = fieldgen.spectrum(fieldgen.quadratic_field(ng, float(ng), 2.0, 0.1, 3))
    res = fbe.estimate(spec, pl, with_abs=True)
    assert np.all(np.abs(res["msum"]) <= res["asum"] * (1 + 1e-12))


def test_fields_on_a_coarser_grid():
    """Shell fields sampled on a coarser S^3 grid: (i) S = Ng reproduces shell_fields; (ii) values
    equal the plane-wave sum of Eq. (2.8) at the sample points; (iii) triple sums times (Ng/S)^3
    equal the Ng^3 sums whenever S exceeds 3 (r_max - 1), the largest wavevector component a
    triple product holds (the exactness the GPU plan's evaluation grid relies on)."""
    ng = 32
    pl = _plan(ng)                               # shells up to |m| < 8: r_max - 1 = 7
    spec = fieldgen.spectrum(fieldgen.quadratic_field(ng, float(ng), 2.0, 0.3, 17))
    full = fbe.shell_fields(spec, pl)
    same = fbe.shell_fields_on_grid(spec, pl, ng)
    for n in range(pl.ns):
        assert np.allclose(same[n], full[n], rtol=0, atol=1e-9 * np.abs(full[n]).max())
    size = 24                                    # > 3 * 7 = 21
    coarse = fbe.shell_fields_on_grid(spec, pl, size)
    modes, shell, _ = dbe.ball_modes(pl)
    vals = dbe.full_spectrum_values(spec, modes, ng)
    rng = np.random.default_rng(4)
    for n in (0, 3, 7):
        sel = shell == n
        for _ in range(3):
            j = rng.integers(0, size, 3)
            x = j * (ng / size)                  # grid units of the Ng grid
            direct = np.sum(vals[sel] * np.exp(2j * np.pi * (modes[sel] @ x) / ng))
            assert abs(direct.imag) < 1e-6 * abs(direct) + 1e-6
            assert abs(coarse[n][tuple(j)] - direct.real) <= 1e-9 * np.abs(coarse[n]).max()
    trips = fbe.kept_triplets(pl)[0]
    want = fbe.triple_sums(full, trips)
    got = fbe.triple_sums(coarse, trips) * (ng / size) ** 3
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-10
    # below the bound the coarse grid aliases: S = 16 < 21 no longer reproduces every bin
    small = fbe.shell_fields_on_grid(spec, pl, 16)
    bad = fbe.triple_sums(small, trips) * (ng / 16) ** 3
    assert np.max(np.abs(bad - want) / np.abs(want)) > 1e-3


@pytest.mark.parametrize("k1_merge,n_mu,n_t", [(1, 4, 4), (3, 4, 4), (8, 1, 1)])
def test_merged_cells_are_bigger_bins_summed_mode_by_mode(k1_merge, n_mu, n_t):
    """The (mu, t) grid (Sec. 2.1, merging adjacent bins): every cell is one bigger bin of
    Eq. (2.3), here built from the direct mode sums of Eq. (2.9) over the triangles of its member
    bins (k1 shell a with a // k1_merge = group, labels in the cell), divided by their direct
    triangle count. k1_merge = Ns with one (mu, t) cell merges every bin into one number."""
    ng = 16
    pl = _plan(ng, k1_merge=k1_merge, n_mu=n_mu, n_t=n_t)
    spec = fieldgen.spectrum(fieldgen.quadratic_field(ng, float(ng), 2.0, 0.2, 31))
    res = fbe.estimate(spec, pl)
    msum_d, ntri_d = dbe.direct_estimate(spec, pl)
    num = np.zeros((pl.n_groups, n_mu, n_t))
    den = np.zeros((pl.n_groups, n_mu, n_t))
    for t in res["triplets"]:
        k = [pl.kbar[s] for s in t]
        mu, tt = P.shape_label(*k)
        im, it = P.shape_cell(mu, tt, n_mu, n_t)
        num[t[0] // k1_merge, im, it] += msum_d[t].real
        den[t[0] // k1_merge, im, it] += ntri_d[t]
    want = np.full(num.shape, np.nan)
    ok = den > 0
    want[ok] = pl.vcell ** 3 / pl.volume * num[ok] / den[ok]
    got = res["grid"]
    assert got.shape == (-(-pl.ns // k1_merge), n_mu, n_t)
    assert np.array_equal(np.isnan(got), ~ok)
    assert np.max(np.abs(got[ok] - want[ok]) / np.abs(want[ok])) < 1e-10
    if k1_merge == pl.ns:
        assert got.shape == (1, 1, 1)


@pytest.mark.parametrize("ng", [16, 32])
def test_triangle_mean_lengths_equal_mode_by_mode_means(ng):
    """Labels from each bin's average triangle (Sec. 2.1): the FFT sums with length-weighted
    counting fields equal the means of |k_a|, |k_b|, |k_c| over the triangles enumerated one by
    one; each mean lies inside its shell, and two equal shells give equal means (symmetry)."""
    pl = _plan(ng, label_k="triangle")
    trips, _, _ = fbe.kept_triplets(pl)
    got = fbe.triangle_mean_k(pl, trips)
    want = dbe.direct_mean_k(pl)
    assert set(want) == set(trips)
    for i, t in enumerate(trips):
        assert np.all(np.abs(got[i] - want[t]) <= 1e-12 * np.asarray(want[t]))
        for j, s in enumerate(t):
            assert np.sqrt(pl.thresholds[s]) - 1e-12 <= got[i, j] < np.sqrt(pl.thresholds[s + 1])
        if t[0] == t[1]:
            assert abs(got[i, 0] - got[i, 1]) <= 1e-12 * got[i, 0]
        if t[1] == t[2]:
            assert abs(got[i, 1] - got[i, 2]) <= 1e-12 * got[i, 1]


def test_triangle_labels_in_the_estimate():
    """With label_k = 'triangle' the estimate's labels come from the bins' mean triangles, the
    values B are unchanged, and on one-radius shells (every mode of a shell has the same |k|)
    both label choices coincide."""
    ng = 16
    spec = fieldgen.spectrum(fieldgen.quadratic_field(ng, float(ng), 2.0, 0.2, 33))
    shell = fbe.estimate(spec, _plan(ng))
    tri = fbe.estimate(spec, _plan(ng, label_k="triangle"))
    assert np.array_equal(shell["b"], tri["b"])
    km = fbe.triangle_mean_k(_plan(ng), tri["triplets"])
    assert [l["k1"] for l in tri["labels"]] == list(km[:, 0])
    assert any(abs(l1["mu"] - l2["mu"]) > 1e-3 for l1, l2 in zip(shell["labels"], tri["labels"]))
    # shells of one radius each: |m|^2 = 9 .. 26 (15 and 23 are no sums of three squares and
    # join the shell below); every triangle of a bin then has the shells' lengths
    qs = [q for q in range(9, 28) if q not in (15, 23)]
    pl1 = P.make_plan(ng, float(ng), np.sqrt(np.array(qs, dtype=float)) - 1e-9, label_k="triangle")
    assert list(pl1.thresholds) == qs
    one = fbe.estimate(spec, pl1)
    for (a, b, c), lab in zip(one["triplets"], one["labels"]):
        want = np.sqrt([pl1.thresholds[a], pl1.thresholds[b], pl1.thresholds[c]])
        assert np.all(np.abs(np.array([lab["k1"], lab["k2"], lab["k3"]]) - want) <= 1e-12 * want)
        assert np.allclose(want, pl1.kbar[[a, b, c]], rtol=1e-15, atol=0)
