"""The 2D ring estimator (dim = 2 plans: the 2D box of Sec. 2.1 and Sec. 2.2) through the C ABI
against the 2D oracle. Needs a GB300."""
import numpy as np
import pytest

import fieldgen
from oracle import plan as P
from oracle import ring2d as R

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14564_gb300 import binding
    return binding


def _check_tables(gp, res):
    tr = gp.triplets
    assert [(int(a), int(b), int(c)) for a, b, c in zip(tr["a"], tr["b"], tr["c"])] == res["triplets"]
    assert np.array_equal(tr["ntri"].astype(np.int64), res["ntri"])
    labs = res["labels"]
    assert np.array_equal(tr["i_mu"], [l["i_mu"] for l in labs])
    assert np.array_equal(tr["i_t"], [l["i_t"] for l in labs])
    assert np.array_equal(tr["mu"], [l["mu"] for l in labs])


@pytest.mark.parametrize("ng,nr", [(64, 12), (96, 10)])
def test_fp64_2d_parity(lib, ng, nr):
    """FP64 2D plans: bins, N_tri and cells exactly, B within 1e-10, merged cells, host entry."""
    edges = P.linear_edges(nr, 1.0, ng / 4)
    spec = fieldgen.spectrum(fieldgen.quadratic_field_2d(ng, float(ng), 2.0, 0.2, 51))
    pl = R.make_plan_2d(ng, float(ng), edges)
    res = R.estimate(spec, pl)
    gp = lib.Plan(ng, float(ng), edges, precision="fp64", dim=2)
    assert gp.spec_shape() == (ng, ng // 2 + 1)
    _check_tables(gp, res)
    b, g = gp.estimate(torch.from_numpy(spec).cuda())
    gp.check()
    b, g = b.cpu().numpy(), g.cpu().numpy()
    assert np.max(np.abs(b - res["b"]) / np.abs(res["b"])) < 1e-10
    assert np.array_equal(np.isnan(g), np.isnan(res["grid"]))
    ok = ~np.isnan(g)
    assert np.max(np.abs(g[ok] - res["grid"][ok]) / np.abs(res["grid"][ok])) < 1e-10
    bh, _ = gp.estimate_host(spec)
    assert np.array_equal(bh, b)


def test_fp32_paper_2d_box(lib):
    """The 2D box of Sec. 2.1: L = 215, Ng = 384, N_r = 15 rings of width 2 k_f; FP32 plan within
    1e-4 of each bin's condition scale; the shell-fields / contraction entry points agree."""
    ng, box = 384, 215.0
    edges = 1.0 + 2.0 * np.arange(16)
    spec = fieldgen.spectrum(fieldgen.quadratic_field_2d(ng, box, 2.0, 0.5, 52))
    pl = R.make_plan_2d(ng, box, edges)
    res = R.estimate(spec, pl, with_abs=True)
    gp = lib.Plan(ng, box, edges, precision="fp32", dim=2)
    _check_tables(gp, res)
    s32 = torch.from_numpy(spec.astype(np.complex64)).cuda()
    b, _ = gp.estimate(s32)
    gp.check()
    b = b.cpu().numpy()
    assert np.max(np.abs(b - res["b"]) / res["b_scale"]) < 1e-4
    fields = gp.shell_fields(s32)
    assert tuple(fields.shape) == (15, gp.ng_eval, gp.ng_eval)
    msum = gp.contract(fields).cpu().numpy()
    assert np.max(np.abs(msum - res["msum"]) / res["asum"]) < 1e-4


def test_2d_batched_and_unsupported_calls(lib):
    """Several 2D plans in one captured graph equal their single estimates; the 3D-only entry
    points refuse a 2D plan."""
    plans, specs, single = [], [], []
    for i, ng in enumerate((64, 128, 192)):
        gp = lib.Plan(ng, float(ng), P.linear_edges(10, 1.0, ng / 4), precision="fp32", dim=2)
        sp = torch.from_numpy(fieldgen.half_spectrum_c64(fieldgen.quadratic_field_2d(ng, float(ng), 1.5, 0.1, 60 + i))).cuda()
        plans.append(gp)
        specs.append(sp)
        single.append(gp.estimate(sp)[0].cpu().numpy())
    batch = lib.Batch(plans, specs)
    out = batch.run()
    torch.cuda.synchronize()
    for got, want in zip(out, single):
        assert np.array_equal(got.cpu().numpy(), want)
    batch.close()
    with pytest.raises(lib.BispecError) as e:
        plans[1].grad(specs[1], torch.zeros(plans[1].n_triplets, dtype=torch.float64, device="cuda"))
    assert e.value.status == 6
