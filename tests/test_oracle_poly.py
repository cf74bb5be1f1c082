"""Pins of the oracle's p-th order polyspectrum estimator (the extension Sec. 4 notes, with its
cap 2 pi Ng / (p L)) to the bispectrum estimator, brute-force enumeration, the aliasing onset,
a closed form and the Gaussian (disconnected) expectation. CPU only."""
import math

import numpy as np
import pytest

import fieldgen
from oracle import fbe
from oracle import plan as P
from oracle import poly


def _plan(ng, ns, top, **kw):
    return P.make_plan(ng, float(ng), P.linear_edges(ns, 1.0, top), **kw)


def test_order_three_is_the_bispectrum():
    ng = 32
    pl = _plan(ng, 8, 8.0)
    spec = fieldgen.spectrum(fieldgen.quadratic_field(ng, float(ng), 2.0, 0.1, 1))
    b = fbe.estimate(spec, pl)
    p3 = poly.estimate(spec, pl, 3)
    assert p3["bins"] == b["triplets"]
    assert np.array_equal(p3["n"], b["ntri"])
    assert np.max(np.abs(p3["value"] - b["b"]) / np.abs(b["b"])) < 1e-12


@pytest.mark.parametrize("ng,ns,top", [(16, 4, 3.9), (20, 3, 4.9)])
def test_order_four_equals_direct_enumeration(ng, ns, top):
    pl = _plan(ng, ns, top)
    spec = fieldgen.spectrum(fieldgen.quadratic_field(ng, float(ng), 2.0, 0.2, 4))
    res = poly.estimate(spec, pl, 4)
    s_d, n_d = poly.direct_sums_4(spec, pl)
    assert set(n_d) == set(res["bins"])
    for i, t in enumerate(res["bins"]):
        assert n_d[t] == res["n"][i]
        s = s_d[t]
        assert abs(s.imag) <= 1e-12 * abs(s.real) + 1e-9
        assert abs(res["msum"][i] / float(ng) ** 3 - s.real) <= 1e-11 * abs(s.real)


def test_order_four_aliases_above_its_cap():
    """Shells below Ng/3 (the bispectrum's cap) but reaching Ng/4: the FFT count of some
    quadrilaterals exceeds the direct count, and agrees where 4 |m|_max < Ng."""
    ng = 16
    pl = _plan(ng, 5, 5.0)
    assert P.aliasing_ok(ng, pl.thresholds) and not poly.cap_ok(ng, pl.thresholds, 4)
    cand = poly.candidates(pl, 4)
    n_fft = np.rint(poly.multi_sums(fbe.counting_fields(pl), cand) / ng ** 3).astype(int)
    _, n_d = poly.direct_sums_4(None, pl, count_only=True)
    over = 0
    for t, n in zip(cand, n_fft):
        if 4 * math.sqrt(pl.thresholds[t[0] + 1] - 1) < ng:
            assert n == n_d.get(t, 0)
        else:
            assert n >= n_d.get(t, 0)
            over += n > n_d.get(t, 0)
    assert over > 0
    with pytest.raises(ValueError):
        poly.kept_bins(pl, 4)


def test_closed_form_four_cosines():
    """delta = 2A sum_i cos(k_i.x), k1 + k2 + k3 + k4 = 0 in four shells, no other signed sum
    zero: sum_x d d d d = 16 A^4 Ng^12 sum_x prod cos = 2 A^4 Ng^15."""
    ng, amp = 32, 0.5
    pl = _plan(ng, 8, 7.9)
    ms = [np.array([5, 2, 1]), np.array([-3, 1, 3]), np.array([1, -2, 0])]
    ms.append(-(ms[0] + ms[1] + ms[2]))
    x = np.indices((ng, ng, ng)).reshape(3, -1).T
    delta = sum(2 * amp * np.cos(2 * np.pi * (x @ m) / ng) for m in ms).reshape(ng, ng, ng)
    sh = sorted((int(np.searchsorted(pl.thresholds, (m * m).sum(), side="right") - 1) for m in ms), reverse=True)
    assert len(set(sh)) == 4
    res = poly.estimate(fieldgen.spectrum(delta), pl, 4)
    i = res["bins"].index(tuple(sh))
    want = 2 * amp ** 4 * float(ng) ** 15
    assert abs(res["msum"][i] - want) <= 1e-9 * want


def test_gaussian_disconnected_part():
    """For a Gaussian field the bins (a, a, b, b), a != b, hold the pairs k_a' = -k_a, k_b' = -k_b:
    <sum over quadrilaterals of Delta^4> = V^2 sum_{k in a} P(k) sum_{k in b} P(k), so the mean
    estimate is V sum_a P sum_b P / N_4; bins of four distinct shells have mean zero."""
    ng, n_index = 16, 2.0
    pl = _plan(ng, 4, 3.9)
    bins, tsum, n4 = poly.kept_bins(pl, 4)
    counts = (bins, tsum, n4)
    vals = np.array([poly.estimate(fieldgen.spectrum(fieldgen.gaussian_field(ng, float(ng), n_index, 500 + s)),
                                   pl, 4, counts=counts)["value"] for s in range(400)])
    m = np.fft.fftfreq(ng, 1.0 / ng)
    q = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    pk = np.where(q > 0, (pl.kf * np.sqrt(np.where(q > 0, q, 1.0))) ** (-n_index), 0.0)
    psum = [float(np.sum(pk[(q >= pl.thresholds[n]) & (q < pl.thresholds[n + 1])])) for n in range(pl.ns)]
    mean, err = vals.mean(0), vals.std(0, ddof=1) / np.sqrt(len(vals))
    tested = 0
    for i, (a, b, c, e) in enumerate(bins):
        if a == b and c == e and a != c:
            want = pl.volume * psum[a] * psum[c] / n4[i]
            assert abs(mean[i] - want) < 4 * err[i] + 0.05 * want
            assert abs(mean[i] - want) < 0.2 * want
            tested += 1
        elif len({a, b, c, e}) == 4:
            assert abs(mean[i]) < 4 * err[i]
    assert tested >= 3
