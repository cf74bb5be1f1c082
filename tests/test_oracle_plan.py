"""Pins of the oracle's binning plan (Sec. 2.1, Eqs. (2.2), (2.4), (2.12)) to values the paper
prints and to closed forms. CPU only."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import plan as P
from oracle import fbe


def test_sum_of_three_squares_counts():
    # r_3(n), the number of integer vectors with |m|^2 = n (number theory; OEIS A005875)
    known = [1, 6, 12, 8, 6, 24, 24, 0, 12, 30, 24, 24, 8, 24, 48, 0, 6]
    assert P.q_counts(len(known)).tolist() == known


def test_paper_triplet_counting():
    g = {k: int(float(v)) for k, v in read_golden("paper_binning.txt")}
    nr = g["n_r"]
    trips = P.all_triplets(nr)
    assert len(trips) == g["triplets_total"] == math.comb(nr + 2, 3)
    assert sum(1 for t in trips if t[0] == nr - 1) == g["triplets_largest_k1"]
    assert sum(1 for t in trips if t[0] == nr - 2) == g["triplets_second_k1"]
    assert all(a >= b >= c for a, b, c in trips)
    assert trips == sorted(trips)


def _paper_plan(nr, step):
    return P.make_plan(384, 215.0, 1.0 + step * np.arange(nr + 1))


def test_paper_shell_centre_and_width():
    # Sec. 2.1: delta k = 0.0584 Mpc^-1 (2 grid spacings), largest ring at k = 0.88 Mpc^-1
    pl = _paper_plan(15, 2)
    assert abs(2 * pl.kf - 0.0584) < 5e-5
    assert abs(pl.kbar[-1] * pl.kf - 0.88) < 5e-3


def test_paper_labels_reproduced():
    for nr, step, mu, t, digits, *_ in read_golden("paper_labels.txt"):
        nr, step, mu, t, digits = int(nr), int(step), float(mu), float(t), int(digits)
        pl = _paper_plan(nr, step)
        labs = P.label_table(pl, [x for x in P.all_triplets(nr) if x[0] == nr - 1])
        best = min(labs, key=lambda l: abs(l["mu"] - mu) + abs(l["t"] - t))
        tol = 10.0 ** (-digits)
        assert abs(best["mu"] - mu) <= tol and abs(best["t"] - t) <= tol, (nr, mu, t, best)


def test_shape_label_closed_forms():
    # equilateral -> (0.5, 1); k2 = k3 = k1/2 (stretched) -> (1, 0.5); k3 -> 0 -> (1, 1)
    assert P.shape_label(3.0, 3.0, 3.0) == (0.5, 1.0)
    mu, t = P.shape_label(2.0, 1.0, 1.0)
    assert abs(mu - 1.0) < 1e-15 and t == 0.5
    mu, t = P.shape_label(5.0, 5.0, 1e-6)
    assert abs(mu - 1.0) < 1e-12 and t == 1.0
    # right angle (3, 4, 5): mu = cos of the angle between k1 and -k2 = 4/5, t = 4/5
    mu, t = P.shape_label(5.0, 4.0, 3.0)
    assert abs(mu - 0.8) < 1e-15 and abs(t - 0.8) < 1e-15


def test_ordered_means_stay_on_region_edges():
    # for k1 >= k2 >= k3 > 0: mu >= 1/2 and 2 mu t - 1 = (k2^2 - k3^2)/k1^2 >= 0 (Eq. (2.2))
    rng = np.random.default_rng(0)
    for _ in range(2000):
        k = np.sort(rng.uniform(0.1, 10.0, 3))[::-1]
        mu, t = P.shape_label(*k)
        assert mu >= 0.5 - 1e-12
        assert abs((2 * mu * t - 1) - (k[1] ** 2 - k[2] ** 2) / k[0] ** 2) < 1e-10


def test_shape_cells():
    assert P.shape_cell(0.5, 0.5, 10, 10) == (0, 0)
    assert P.shape_cell(1.0, 1.0, 10, 10) == (9, 9)          # last cell closed at 1
    assert P.shape_cell(1.2, 0.3, 10, 10) == (9, 0)          # clamped
    assert P.shape_cell(0.55, 0.75, 10, 10) == (1, 5)        # half-open lower edges
    assert P.shape_cell(0.5499999, 0.7499999, 10, 10) == (0, 4)
    assert P.in_region(0.5, 1.0) and P.in_region(1.0, 0.5)
    assert not P.in_region(0.6, 0.6)                         # 2 mu t < 1
    assert not P.in_region(1.0001, 0.9)


def test_aliasing_cap():
    # Eq. (2.12): modes must have k < 2 pi Ng / (3 L), i.e. 9 |m|^2 < Ng^2
    assert P.aliasing_ok(48, P.shell_thresholds([1.0, 15.9]))
    assert P.aliasing_ok(48, P.shell_thresholds([1.0, 16.0]))      # |m|^2 < 256 -> max 255
    assert not P.aliasing_ok(48, P.shell_thresholds([1.0, 16.1]))
    with pytest.raises(ValueError):
        P.make_plan(16, 16.0, [1.0, 3.0, 6.0])
    P.make_plan(16, 16.0, [1.0, 3.0, 6.0], allow_aliasing=True)


def test_shell_means_brute_force():
    pl = P.make_plan(32, 32.0, P.linear_edges(8, 1, 8))
    g = np.arange(-9, 10)
    m = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    k = np.sqrt((m * m).sum(1))
    for n in range(pl.ns):
        sel = (k * k >= pl.edges[n] ** 2) & (k * k < pl.edges[n + 1] ** 2) & (k > 0)
        assert pl.nmodes[n] == sel.sum()
        assert abs(pl.kbar[n] - k[sel].mean()) < 1e-12
    # Ng=32 mode counts per shell, edges 1..8 in 8 equal steps
    assert pl.nmodes.tolist() == [26, 54, 122, 186, 230, 402, 482, 600]


@pytest.mark.slow
def test_paper_triangle_counts_magnitude():
    g = {k: float(v) for k, v in read_golden("paper_ntri.txt")}
    pl = _paper_plan(15, 2)
    f = fbe.counting_fields(pl, shells=[14, 10, 9, 3])
    ng3 = 384.0 ** 3
    equi = fbe.triple_sums(f, [(14, 14, 14)])[0] / ng3
    right = fbe.triple_sums(f, [(14, 10, 9)])[0] / ng3    # mu ~ t: right-angled
    linear = fbe.triple_sums(f, [(14, 10, 3)])[0] / ng3   # mu ~ 1: linear
    assert abs(equi - round(equi)) < 1e-3
    assert 0.5 * g["equilateral_order"] < equi < 5 * g["equilateral_order"]
    assert 0.5 * g["right_angle_drop"] < equi / right < 2 * g["right_angle_drop"]
    assert 0.5 * g["linear_drop"] < equi / linear < 2 * g["linear_drop"]
