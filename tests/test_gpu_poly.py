"""Order-4 plans (the binned 4-point sum the FFT estimator extends to, Sec. 4) through the C ABI
against the oracle's polyspectrum estimator. Needs a GB300."""
import numpy as np
import pytest

import fieldgen
from oracle import plan as P
from oracle import poly
from oracle import ring2d as R

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14564_gb300 import binding
    return binding


def _bins(gp):
    tr = gp.triplets
    return [(int(a), int(b), int(c), int(e)) for a, b, c, e in zip(tr["a"], tr["b"], tr["c"], tr["e"])]


def test_order4_fp64_parity(lib):
    """Ng = 32, 6 shells below Ng/4: bins and quadrilateral counts exactly, values within 1e-10."""
    ng = 32
    edges = P.linear_edges(6, 1.0, 7.9)
    spec = fieldgen.spectrum(fieldgen.quadratic_field(ng, float(ng), 2.0, 0.2, 81))
    pl = P.make_plan(ng, float(ng), edges, 1, 1)
    res = poly.estimate(spec, pl, 4)
    gp = lib.Plan(ng, float(ng), edges, 1, 1, precision="fp64", order=4)
    assert _bins(gp) == res["bins"]
    assert np.array_equal(gp.triplets["ntri"].astype(np.int64), res["n"])
    assert np.all(np.isnan(gp.triplets["mu"]))
    b, g = gp.estimate(torch.from_numpy(spec).cuda())
    gp.check()
    b = b.cpu().numpy()
    assert np.max(np.abs(b - res["value"]) / np.abs(res["value"])) < 1e-10
    # one cell per k1 shell: the merged bin sum V_c^4 sum M / (V sum T)
    g = g.cpu().numpy()[:, 0, 0]
    a = np.array([t[0] for t in res["bins"]])
    norm = pl.vcell ** 4 / pl.volume
    for k in range(pl.ns):
        sel = a == k
        if sel.any():
            want = norm * res["msum"][sel].sum() / res["tsum"][sel].sum()
            assert abs(g[k] - want) <= 1e-10 * abs(want)
    with pytest.raises(lib.BispecError):
        gp.contract(gp.shell_fields(torch.from_numpy(spec).cuda()))


def test_order4_fp32_parity(lib):
    """Ng = 64, 10 shells below Ng/4, FP32 plan: every bin within 1e-4 of its condition scale."""
    ng = 64
    edges = P.linear_edges(10, 1.0, 15.9)
    spec = fieldgen.spectrum(fieldgen.quadratic_field(ng, float(ng), 1.5, 0.1, 82))
    pl = P.make_plan(ng, float(ng), edges, 1, 1)
    res = poly.estimate(spec, pl, 4, with_abs=True)
    gp = lib.Plan(ng, float(ng), edges, 1, 1, precision="fp32", order=4)
    assert _bins(gp) == res["bins"]
    assert np.array_equal(gp.triplets["ntri"].astype(np.int64), res["n"])
    b, _ = gp.estimate(torch.from_numpy(spec.astype(np.complex64)).cuda())
    gp.check()
    assert np.max(np.abs(b.cpu().numpy() - res["value"]) / res["scale"]) < 1e-4


def test_order4_on_a_2d_box(lib):
    """dim = 2, order 4: rings below Ng/4; the oracle's ring fields and multi-sums."""
    ng = 64
    edges = P.linear_edges(8, 1.0, 15.9)
    spec = fieldgen.spectrum(fieldgen.quadratic_field_2d(ng, float(ng), 2.0, 0.2, 83))
    pl = R.make_plan_2d(ng, float(ng), edges, 1, 1)
    cand = poly.candidates(pl, 4)
    tsum = poly.multi_sums(R.counting_fields(pl), cand)
    n = np.rint(tsum / ng ** 2)
    keep = n > 0
    bins = [t for t, k in zip(cand, keep) if k]
    msum = poly.multi_sums(R.ring_fields(spec, pl), bins)
    want = pl.vcell ** 4 / pl.volume * msum / tsum[keep]
    gp = lib.Plan(ng, float(ng), edges, 1, 1, precision="fp64", dim=2, order=4)
    assert _bins(gp) == bins
    assert np.array_equal(gp.triplets["ntri"], n[keep])
    b, _ = gp.estimate(torch.from_numpy(spec).cuda())
    assert np.max(np.abs(b.cpu().numpy() - want) / np.abs(want)) < 1e-10
