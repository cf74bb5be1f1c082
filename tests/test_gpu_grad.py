"""The forward spectrum, the adjoint (bsp_grad) and the autograd Function against the FP64
oracle's adjoint (itself pinned by finite differences). Needs a GB300."""
import numpy as np
import pytest

import fieldgen
from oracle import fbe
from oracle import grad as G
from oracle import plan as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14564_gb300 import binding
    return binding


def _setup(lib, ng, ns, top, seed, beta=None, prec="fp32"):
    edges = P.linear_edges(ns, 1.0, top)
    delta = fieldgen.quadratic_field(ng, float(ng), 1.5, 0.2, seed).astype(np.float32)
    gp = lib.Plan(ng, float(ng), edges, rsd=beta is not None, beta=beta or 0.0, precision=prec)
    pl = P.make_plan(ng, float(ng), edges)
    return edges, delta, gp, pl


def test_spectrum_on_shell_modes(lib):
    ng = 128
    _, delta, gp, pl = _setup(lib, ng, 8, 32.0, 3)
    spec = gp.spectrum(torch.from_numpy(delta).cuda()).cpu().numpy()
    want = np.fft.rfftn(delta.astype(np.float64))
    sidx = P.shell_index_half(pl)
    sel = sidx >= 0
    err = np.abs(spec[sel] - want[sel]).max() / np.abs(want[sel]).max()
    assert err < 1e-5
    assert np.all(spec[~sel] == 0)


@pytest.mark.parametrize("beta,prec", [(None, "fp32"), (0.5, "fp32"), (None, "mixed_bf16x3")])
def test_adjoint_matches_oracle(lib, beta, prec):
    ng = 128
    _, delta, gp, pl = _setup(lib, ng, 8, 32.0, 5, beta, prec)
    trips = [tuple(int(v) for v in t) for t in zip(gp.triplets["a"], gp.triplets["b"], gp.triplets["c"])]
    tsum = gp.triplets["tsum"]
    g = fieldgen.random_weights(len(trips), 9)
    want = G.vjp(delta.astype(np.float64), pl, trips, tsum, g, beta=beta)
    d = torch.from_numpy(delta).cuda()
    spec = gp.spectrum(d)
    got = gp.grad(spec, torch.from_numpy(g).cuda()).cpu().numpy()
    gp.check()
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 1e-4, err


def test_autograd_function_loss(lib):
    """loss = sum (B - B_ana)^2 / B_ana^2 over the bins; d loss / d delta via backward() against the
    oracle adjoint driven by the same dL/dB."""
    from oracle import analytic as A
    from paper_2107_14564_gb300.autograd import bispectrum
    ng = 128
    _, delta, gp, pl = _setup(lib, ng, 8, 32.0, 7)
    tr = gp.triplets
    kf = pl.kf
    p = [A.power_law(kf * tr[k], 1.5) for k in ("k1", "k2", "k3")]
    bana = torch.from_numpy(A.b_ana(p[0], p[1], p[2], 0.2)).cuda()
    d = torch.from_numpy(delta).cuda().requires_grad_(True)
    b = bispectrum(d, gp)
    loss = (((b - bana) / bana) ** 2).sum()
    loss.backward()
    g = (2.0 * (b.detach() - bana) / bana ** 2).cpu().numpy()
    trips = [tuple(int(v) for v in t) for t in zip(tr["a"], tr["b"], tr["c"])]
    want = G.vjp(delta.astype(np.float64), pl, trips, tr["tsum"], g)
    got = d.grad.cpu().numpy()
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-4
    # and the forward equals the oracle estimate of the same field
    res = fbe.estimate(np.fft.rfftn(delta.astype(np.float64)), pl, with_abs=True)
    assert np.max(np.abs(b.detach().cpu().numpy() - res["b"]) / res["b_scale"]) < 1e-4


@pytest.mark.slow
def test_adjoint_ng256_24_shells_sampled_voxels(lib):
    """Ng=256, 24 shells up to k_Nyq/2, FP32: the adjoint at 64 seeded voxels against the oracle."""
    ng = 256
    _, delta, gp, pl = _setup(lib, ng, 24, 64.0, 5)
    tr = gp.triplets
    trips = [tuple(int(v) for v in t) for t in zip(tr["a"], tr["b"], tr["c"])]
    g = fieldgen.random_weights(len(trips), 6)
    want = G.vjp(delta.astype(np.float64), pl, trips, tr["tsum"], g)
    spec = gp.spectrum(torch.from_numpy(delta).cuda())
    got = gp.grad(spec, torch.from_numpy(g).cuda()).cpu().numpy()
    vox = fieldgen.random_voxels(ng, 64, 6)
    scale = np.abs(want).max()
    assert np.abs(got.ravel()[vox] - want.ravel()[vox]).max() / scale < 1e-4
    assert np.abs(got - want).max() / scale < 1e-4


@pytest.mark.slow
def test_adjoint_on_a_384_evaluation_grid(lib):
    """The adjoint's forward transforms at length 384 (16 lanes per line, radices 8, 8, 6): Ng = 384
    with shells up to 96 k_f puts the evaluation grid at 384. The upstream gradient is non-zero
    on 12 bins only, so the oracle's adjoint needs only those."""
    ng = 384
    _, delta, gp, pl = _setup(lib, ng, 16, 96.0, 8)
    assert gp.ng_eval == 384
    trips = [tuple(int(v) for v in t) for t in zip(gp.triplets["a"], gp.triplets["b"], gp.triplets["c"])]
    g = np.zeros(len(trips))
    pick = np.linspace(0, len(trips) - 1, 12).astype(int)
    g[pick] = fieldgen.random_weights(len(pick), 10)
    want = G.vjp(delta.astype(np.float64), pl, [trips[i] for i in pick], gp.triplets["tsum"][pick], g[pick])
    spec = gp.spectrum(torch.from_numpy(delta).cuda())
    got = gp.grad(spec, torch.from_numpy(g).cuda()).cpu().numpy()
    gp.check()
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 1e-4, err


def test_adjoint_under_a_memory_budget(lib):
    """Shell fields, adjoint products and their transforms along z one x-slab at a time (slabs of
    20 planes of the 128^3 evaluation grid, the last one 8), with RSD: the gradient and the
    estimate against the oracle."""
    ng, beta = 128, 0.5
    edges = P.linear_edges(8, 1.0, 32.0)
    delta = fieldgen.quadratic_field(ng, float(ng), 1.5, 0.2, 5).astype(np.float32)
    gp = lib.Plan(ng, float(ng), edges, rsd=True, beta=beta, precision="fp32",
                  mem_budget_bytes=20 * 8 * 128 * 128 * 4)
    assert gp.ng_eval == 128 and gp.slabs == (20, 7)
    pl = P.make_plan(ng, float(ng), edges)
    trips = [tuple(int(v) for v in t) for t in zip(gp.triplets["a"], gp.triplets["b"], gp.triplets["c"])]
    g = fieldgen.random_weights(len(trips), 9)
    want = G.vjp(delta.astype(np.float64), pl, trips, gp.triplets["tsum"], g, beta=beta)
    spec = gp.spectrum(torch.from_numpy(delta).cuda())
    got = gp.grad(spec, torch.from_numpy(g).cuda()).cpu().numpy()
    b, _ = gp.estimate(spec)
    gp.check()
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-4
    res = fbe.estimate(spec.cpu().numpy().astype(np.complex128), pl, beta=beta, with_abs=True)
    assert np.max(np.abs(b.cpu().numpy() - res["b"]) / res["b_scale"]) < 1e-4


@pytest.mark.slow
def test_config5_loss_gradient_finite_differences(lib):
    """The differentiable workload at its size: Ng=256, 24 shells k_f..64 k_f, the quadratic field
    with P = k^-1.5 and f = 0.05, loss L = sum_t (B_t - B_ana,t)^2 / B_ana,t^2 (B_ana of Eq. (3.2)
    at the bins' shell means). dL/d delta from autograd (forward bsp_estimate of the FP32 plan,
    backward the hand-written adjoint bsp_grad) against central differences of L at 64 seeded
    voxels and along one seeded random direction, the differences taken with the FP64 GPU plan's
    forward on delta +- h e (spectra shifted on the device by +- h e^{-i k.x_v}). L is a polynomial
    of degree 6 in delta and h = 1e-3 of the field's r.m.s., so the differences' truncation error is
    ~1e-6 relative; the FP32 gradient's own rounding dominates."""
    from oracle import analytic as A
    from paper_2107_14564_gb300.autograd import bispectrum
    ng, ns = 256, 24
    edges = P.linear_edges(ns, 1.0, 64.0)
    delta64 = fieldgen.quadratic_field(ng, float(ng), 1.5, 0.05, 5)
    delta = delta64.astype(np.float32)
    gp = lib.Plan(ng, float(ng), edges, 20, 20, precision="fp32")
    g64 = lib.Plan(ng, float(ng), edges, 20, 20, precision="fp64")
    pl = P.make_plan(ng, float(ng), edges)
    tr = gp.triplets
    p = [A.power_law(pl.kf * tr[k], 1.5) for k in ("k1", "k2", "k3")]
    bana = torch.from_numpy(A.b_ana(p[0], p[1], p[2], 0.05)).cuda()

    d = torch.from_numpy(delta).cuda().requires_grad_(True)
    b = bispectrum(d, gp)
    loss = (((b - bana) / bana) ** 2).sum()
    loss.backward()
    grad = d.grad.double()
    gp.check()

    # FP64 forward on spectra of delta +- h e
    spec0 = torch.from_numpy(np.fft.rfftn(delta.astype(np.float64))).cuda()
    m = torch.fft.fftfreq(ng, d=1.0 / ng, dtype=torch.float64, device="cuda")
    mz = torch.arange(ng // 2 + 1, dtype=torch.float64, device="cuda")

    def loss64(spec):
        bb, _ = g64.estimate(spec.contiguous(), with_grid=False)
        return float((((bb - bana) / bana) ** 2).sum())

    h = 1e-3 * float(delta.astype(np.float64).std())
    vox = fieldgen.random_voxels(ng, 64, 6)
    fd = np.empty(len(vox))
    for i, v in enumerate(vox):
        x, y, z = np.unravel_index(int(v), (ng, ng, ng))
        ph = torch.exp(-2j * np.pi * (m[:, None, None] * x + m[None, :, None] * y + mz[None, None, :] * z) / ng)
        fd[i] = (loss64(spec0 + h * ph) - loss64(spec0 - h * ph)) / (2 * h)
    got = grad.reshape(-1)[torch.from_numpy(vox).cuda()].cpu().numpy()
    gmax = float(grad.abs().max())
    err = np.abs(got - fd)
    print(f"\n[grad FD] 64 voxels: max |err| / |fd| {np.max(err / np.abs(fd)):.2e}, median {np.median(err / np.abs(fd)):.2e}; "
          f"max |err| / max|grad| {err.max() / gmax:.2e}")
    assert np.all(err <= 1e-3 * np.abs(fd) + 1e-4 * gmax), (err, fd)
    # one random direction u: (L(delta + h u) - L(delta - h u)) / 2h = grad . u
    u = fieldgen.random_weights(ng ** 3, 7).reshape(ng, ng, ng)
    u /= np.sqrt((u * u).sum())
    su = torch.from_numpy(np.fft.rfftn(u)).cuda()
    hu = 1e-3 * float(np.sqrt((delta.astype(np.float64) ** 2).sum()))
    fdu = (loss64(spec0 + hu * su) - loss64(spec0 - hu * su)) / (2 * hu)
    gu = float((grad.cpu().numpy() * u).sum())
    print(f"[grad FD] direction: fd {fdu:.6e} grad.u {gu:.6e} rel {abs(gu - fdu) / abs(fdu):.2e}")
    assert abs(gu - fdu) <= 1e-3 * abs(fdu)
    g64.check()
