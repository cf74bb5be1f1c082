"""Full-size parity in the bench's launch configuration: the Ng=512 redshift-space workload
(32 shells k_f..k_Nyq/2, Kaiser beta=0.5, 20x20 cells, split-BF16 contraction) and the Ng=256 FP32
workload, on bins the FP64 oracle can compute one by one (their shell fields and counting
fields at the full grid). Needs a GB300 and about a minute of host FFTs."""
import numpy as np
import pytest

import fieldgen
from oracle import fbe
from oracle import plan as P

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14564_gb300 import binding
    return binding


def _sampled(lib, ng, ns, top, n_index, f, seed, beta, prec, picks, budgets=(0,)):
    """Condition-scaled and plain relative errors of the picked bins, one row per memory budget."""
    edges = np.linspace(1.0, top, ns + 1)
    delta = fieldgen.quadratic_field(ng, float(ng), n_index, f, seed)
    spec = fieldgen.half_spectrum_c64(delta)
    del delta
    bs = []
    for budget in budgets:
        gp = lib.Plan(ng, float(ng), edges, 20, 20, rsd=beta is not None, beta=beta or 0.0, precision=prec,
                      mem_budget_bytes=budget)
        if budget:  # fields produced and reduced x-slab by x-slab; the plan holds less than all fields
            assert gp.slabs[1] > 1 and gp.device_bytes < gp.field_bytes
        bs.append(gp.estimate(torch.from_numpy(spec).cuda(), with_grid=False)[0].cpu().numpy())
        gp.check()
        tr = gp.triplets
        gp.close()
        torch.cuda.empty_cache()
    keys = [(int(a), int(bb), int(c)) for a, bb, c in zip(tr["a"], tr["b"], tr["c"])]
    pl = P.make_plan(ng, float(ng), edges, 20, 20)
    assert len(keys) <= len(pl.candidates)
    trips = [keys[i] for i in picks]
    shells = sorted({s for t in trips for s in t})
    spec64 = spec.astype(np.complex128)
    if beta is not None:
        spec64 = spec64 * fbe.kaiser_factor_half(ng, beta)
    d = fbe.shell_fields(spec64, pl, shells)
    msum = fbe.triple_sums(d, trips)
    asum = fbe.triple_sums(d, trips, absolute=True)
    del d
    i = fbe.counting_fields(pl, shells)
    tsum = fbe.triple_sums(i, trips)
    del i
    norm = pl.vcell ** 3 / pl.volume
    want = norm * msum / tsum
    scale = norm * asum / tsum
    got = np.stack([b[picks] for b in bs])
    assert np.array_equal(np.rint(tsum / float(ng) ** 3), tr["ntri"][picks])
    cond = np.abs(got - want) / scale
    rel = np.abs(got - want) / np.abs(want)
    return cond, rel


def test_ng512_rsd_mixed_sampled_bins(lib):
    # bins of the largest k1 shell (equilateral, squeezed, linear), a mid shell and the lowest
    picks = [-1, -2, -17, 1500, 0, 7]
    cond, rel = _sampled(lib, 512, 32, 128.0, 1.5, 0.05, 4, 0.5, "mixed_bf16x3", picks)
    assert np.max(cond) < 1e-4, (cond, rel)


def test_ng256_fp32_sampled_bins(lib):
    picks = [-1, -3, -40, 600, 0, 11]
    cond, rel = _sampled(lib, 256, 24, 64.0, 1.5, 0.05, 3, None, "fp32", picks)
    assert np.max(cond) < 1e-4, (cond, rel)


def test_ng768_fp32_forward_sampled_bins(lib):
    """The forward-only Ng=768 FP32 workload (24 shells k_f..192 k_f), with every field resident
    (24 x 768^3 FP32 = 43.5 GB) and under an 8 GiB budget for shell fields (x-slabs of 151
    planes, plan-time FP64 counts in slabs too); bins of the largest, a middle and the smallest
    k1 shell against the oracle."""
    picks = [-1, -2, 300, 0]
    cond, rel = _sampled(lib, 768, 24, 192.0, 1.5, 0.05, 7, None, "fp32", picks, budgets=(0, 8 << 30))
    assert np.max(cond) < 1e-4, (cond, rel)
