"""Pins of the Kaiser monopole factor and of the oracle adjoint. CPU only."""
import numpy as np
import pytest

import fieldgen
from conftest import read_golden
from oracle import analytic as A
from oracle import fbe
from oracle import grad as G
from oracle import plan as P


def _random_rotations(n, rng):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1)], 1)


@pytest.mark.parametrize("mu,t", [(0.5, 1.0), (0.8, 0.8), (0.95, 0.6), (0.7, 0.9)])
def test_kaiser_monopole_monte_carlo(mu, t):
    """Closed form against a direct average of prod (1 + beta mu_a^2) over random rotations."""
    beta = 0.8
    k1 = np.array([1.0, 0.0, 0.0])
    ang = np.arccos(-mu)                      # mu = -k1.k2 / (k1 k2) (Sec. 2.1)
    k2 = t * np.array([np.cos(ang), np.sin(ang), 0.0])
    k3 = -(k1 + k2)
    rng = np.random.default_rng(7)
    rot = _random_rotations(400000, rng)
    prod = np.ones(len(rot))
    for k in (k1, k2, k3):
        kz = (rot @ k)[:, 2] / np.linalg.norm(k)
        prod *= 1.0 + beta * kz * kz
    mc = prod.mean()
    err = prod.std() / np.sqrt(len(prod))
    assert abs(mc - A.kaiser_monopole_mu_t(mu, t, beta)) < 5 * err


def test_kaiser_monopole_limits():
    # beta -> 0: 1; linear triangles: <(1 + beta mu^2)^3> = 1 + beta + 3 beta^2/5 + beta^3/7
    assert A.kaiser_monopole_mu_t(0.6, 0.9, 0.0) == 1.0
    b = 0.7
    assert abs(A.kaiser_monopole_mu_t(1.0, 0.7, b) - (1 + b + 3 * b * b / 5 + b ** 3 / 7)) < 1e-12


def test_kaiser_monopole_vs_paper_factors():
    """Sec. 3.1 prints B^s/B (beta = 1) and states +-7 percent agreement with theory."""
    for mu, t, fac in read_golden("paper_rsd_factors.txt"):
        r = A.kaiser_monopole_mu_t(float(mu), float(t), 1.0)
        assert abs(r / float(fac) - 1.0) < 0.07, (mu, t, r, fac)


@pytest.mark.parametrize("beta", [None, 0.5])
def test_adjoint_matches_finite_differences(beta):
    ng = 16
    pl = P.make_plan(ng, float(ng), P.linear_edges(6, 1.0, 4.0))
    trips, tsum, _ = fbe.kept_triplets(pl)
    delta = fieldgen.quadratic_field(ng, float(ng), 2.0, 0.3, 11)
    g = fieldgen.random_weights(len(trips), 12)
    grad = G.vjp(delta, pl, trips, tsum, g, beta=beta)

    def loss(x):
        return float(np.dot(g, G.estimate_real(x, pl, trips, tsum, beta=beta)))

    h = 1e-3 * delta.std()
    vox = fieldgen.random_voxels(ng, 12, 13)
    flat = delta.ravel()
    for v in vox:
        e = np.zeros_like(flat)
        e[v] = h
        fd = (loss((flat + e).reshape(delta.shape)) - loss((flat - e).reshape(delta.shape))) / (2 * h)
        assert abs(fd - grad.ravel()[v]) <= 1e-6 * np.abs(grad).max()
    # one random direction
    u = np.random.default_rng(3).standard_normal(delta.shape)
    fd = (loss(delta + h * u) - loss(delta - h * u)) / (2 * h)
    assert abs(fd - float(np.sum(grad * u))) <= 1e-6 * abs(fd)


def test_forward_of_adjoint_matches_estimator():
    ng = 16
    pl = P.make_plan(ng, float(ng), P.linear_edges(6, 1.0, 4.0))
    trips, tsum, ntri = fbe.kept_triplets(pl)
    delta = fieldgen.quadratic_field(ng, float(ng), 2.0, 0.3, 4)
    b1 = G.estimate_real(delta, pl, trips, tsum)
    b2 = fbe.estimate(fieldgen.spectrum(delta), pl, counts=(trips, tsum, ntri))["b"]
    assert np.allclose(b1, b2, rtol=1e-12, atol=0)


def test_gaussian_scatter_follows_eq_3_3():
    """For a Gaussian field (B = 0) and three distinct shells every closed triangle is its own
    term (Wick pairings match only identical triangles), so Var(B_hat) = V sum_T P_a P_b P_c /
    N_tri^2; Eq. (3.3) at the shells' mean powers gives the same to the spread of P over a
    shell. Both against the scatter of 400 seeded realisations."""
    ng, n_index = 32, 2.0
    pl = P.make_plan(ng, float(ng), P.linear_edges(8, 1.0, 8.0))
    trips, tsum, ntri = fbe.kept_triplets(pl)
    sel = [i for i, (a, b, c) in enumerate(trips) if a > b > c]
    m = np.fft.fftfreq(ng, 1.0 / ng)
    mz = np.arange(ng // 2 + 1, dtype=np.float64)
    q = m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2
    pk = np.where(q > 0, (pl.kf * np.sqrt(np.where(q > 0, q, 1.0))) ** (-n_index), 0.0)
    pf = fbe.shell_fields(pk, pl)
    sum_ppp = fbe.triple_sums(pf, [trips[i] for i in sel]) / float(ng) ** 3
    n = ntri[sel].astype(float)
    var_exact = pl.volume * sum_ppp / n ** 2
    counts = (trips, tsum, ntri)
    bs = np.array([fbe.estimate(fieldgen.spectrum(fieldgen.gaussian_field(ng, float(ng), n_index, 700 + s)),
                                pl, counts=counts)["b"][sel] for s in range(400)])
    ratio = bs.var(0, ddof=1) / var_exact
    assert 0.85 < np.median(ratio) < 1.15
    assert np.all((ratio > 0.6) & (ratio < 1.6))
    # Eq. (3.3) with B = 0 at the mean power of each shell's modes
    sidx = P.shell_index_half(pl)
    full = np.ones_like(q)
    full[..., 1:ng // 2] = 2.0                       # half-grid modes stand for two of the full grid
    pbar = np.array([np.sum((pk * full)[sidx == s]) / np.sum(full[sidx == s]) for s in range(pl.ns)])
    a, b, c = (np.array([trips[i][j] for i in sel]) for j in range(3))
    sig = A.sigma_b(pbar[a], pbar[b], pbar[c], 0.0, n, pl.volume)
    # the shell-mean form is an approximation where P changes fast across a shell (k^-2 on the
    # innermost shells, whose width is comparable to their radius)
    dev = np.abs(sig ** 2 / var_exact - 1.0)
    assert np.median(dev) < 0.05 and np.max(dev) < 0.5
