"""Full-size parity in the bench's launch configuration: the Ng=512 redshift-space workload
(32 shells k_f..k_Nyq/2, Kaiser beta=0.5, 20x20 cells, split-BF16 contraction) and the Ng=256 FP32
workload, on bins the FP64 oracle computes one by one (their shell fields and counting fields on
the full grid). The bins are chosen from the plan's own layout (bsp_plan_bin_levels) so that every
contraction level, and every tensor-core tile of the top level, sums at least one of them. Each
test prints its measured errors. Needs a GB300 and a few minutes of host FFTs."""
from collections import OrderedDict

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


def _oracle_bins(spec64, pl, trips, cache_size=8):
    """FP64 oracle sums of the given bins: sum_x d d d, sum_x |d d d| and sum_x i i i (Eqs. (2.7),
    (2.10)), holding at most `cache_size` full-grid fields at a time."""
    cache = OrderedDict()
    ones = None

    def field(kind, n):
        nonlocal ones
        key = (kind, n)
        if key in cache:
            cache.move_to_end(key)
            return cache[key]
        if kind == "d":
            f = fbe.shell_fields(spec64, pl, [n])[n]
        else:
            if ones is None:
                ones = np.ones_like(spec64)
            f = fbe.shell_fields(ones, pl, [n])[n]
        cache[key] = f
        while len(cache) > cache_size:
            cache.popitem(last=False)
        return f

    msum = np.zeros(len(trips))
    asum = np.zeros(len(trips))
    tsum = np.zeros(len(trips))
    for kind in ("d", "i"):
        cache.clear()
        for j in sorted(range(len(trips)), key=lambda j: trips[j]):
            a, b, c = trips[j]
            fa, fb, fc = field(kind, a), field(kind, b), field(kind, c)
            p = fa * fb
            if kind == "d":
                msum[j] = float(np.vdot(p.ravel(), fc.ravel()))
                asum[j] = float(np.vdot(np.abs(p).ravel(), np.abs(fc).ravel()))
            else:
                tsum[j] = float(np.vdot(p.ravel(), fc.ravel()))
    return msum, asum, tsum


def _layout_picks(plan, extra):
    """Bins covering the plan's launch structure: the first and last bin of every contraction
    level and, for split-BF16 plans, the bins of the lowest and highest slot of every tile of each
    level; plus the `extra` indices."""
    lev, slot = plan.bin_level, plan.bin_slot
    picks = set(int(i) % plan.n_triplets for i in extra)
    for lv in np.unique(lev):
        idx = np.flatnonzero(lev == lv)
        picks.update([int(idx[0]), int(idx[-1])])
        if slot[idx[0]] >= 0:
            tiles = slot[idx] // 64
            for t in np.unique(tiles):
                sel = idx[tiles == t]
                s = slot[sel]
                picks.update([int(sel[np.argmin(s)]), int(sel[np.argmax(s)])])
    return sorted(picks)


def _sampled(lib, ng, ns, top, n_index, f, seed, beta, prec, extra, budgets=(0,), layout=True, variants=None):
    """Condition-scaled and plain relative errors of the picked bins, one row per memory budget
    (or per (precision, budget) in `variants`); with `layout`, every level and tile is covered."""
    edges = np.linspace(1.0, top, ns + 1)
    delta = fieldgen.quadratic_field(ng, float(ng), n_index, f, seed)
    spec = fieldgen.half_spectrum_c64(delta)
    del delta
    bs = []
    picks = None
    for prec_v, budget in (variants or [(prec, b) for b in budgets]):
        gp = lib.Plan(ng, float(ng), edges, 20, 20, rsd=beta is not None, beta=beta or 0.0, precision=prec_v,
                      mem_budget_bytes=budget)
        if budget:  # fields produced and reduced x-slab by x-slab; the plan holds less than all fields
            assert gp.slabs[1] > 1 and gp.device_bytes < gp.field_bytes
        if picks is None:
            picks = _layout_picks(gp, extra) if layout else sorted(int(i) % gp.n_triplets for i in extra)
            lev, slot = gp.bin_level[picks], gp.bin_slot[picks]
            if layout:  # every level, and every tensor-core tile of every level, has a picked bin
                assert set(lev) == set(gp.bin_level)
                assert set(zip(gp.bin_level, gp.bin_slot // 64)) == set(zip(lev, slot // 64))
        bs.append(gp.estimate(torch.from_numpy(spec).cuda(), with_grid=False)[0].cpu().numpy())
        gp.check()
        tr = gp.triplets
        gp.close()
        torch.cuda.empty_cache()
    keys = [(int(a), int(bb), int(c)) for a, bb, c in zip(tr["a"], tr["b"], tr["c"])]
    pl = P.make_plan(ng, float(ng), edges, 20, 20)
    trips = [keys[i] for i in picks]
    spec64 = spec.astype(np.complex128)
    if beta is not None:
        spec64 = spec64 * fbe.kaiser_factor_half(ng, beta)
    msum, asum, tsum = _oracle_bins(spec64, pl, trips)
    norm = pl.vcell ** 3 / pl.volume
    want = norm * msum / tsum
    scale = norm * asum / tsum
    got = np.stack([b[picks] for b in bs])
    assert np.array_equal(np.rint(tsum / float(ng) ** 3), tr["ntri"][picks])
    cond = np.abs(got - want) / scale
    rel = np.abs(got - want) / np.abs(want)
    cancel = scale / np.abs(want)  # how far each bin's sum cancels below its terms
    print(f"\n[{prec} Ng={ng}] condition-scaled max per plan: {', '.join(f'{c:.2e}' for c in cond.max(axis=1))}")
    print(f"[{prec} Ng={ng}] {len(picks)} bins: condition-scaled max {cond.max():.2e} median {np.median(cond):.2e}; "
          f"relative max {rel.max():.2e} median {np.median(rel):.2e}; relative max over bins cancelling < 1e3: "
          f"{rel[:, cancel < 1e3].max() if np.any(cancel < 1e3) else float('nan'):.2e}")
    return cond, rel


def test_ng512_rsd_mixed_sampled_bins(lib):
    # the layout picks plus bins of the largest k1 shell (equilateral, squeezed, linear), a mid
    # shell and the lowest
    cond, rel = _sampled(lib, 512, 32, 128.0, 1.5, 0.05, 4, 0.5, "mixed_bf16x3", [-1, -2, -17, 1500, 0, 7])
    assert np.max(cond) < 2e-6, (cond, rel)  # the stated split-BF16 bound


def test_ng256_fp32_sampled_bins(lib):
    cond, rel = _sampled(lib, 256, 24, 64.0, 1.5, 0.05, 3, None, "fp32", [-1, -3, -40, 600, 0, 11])
    assert np.max(cond) < 1e-7, (cond, rel)  # the stated FP32 bound


def test_ng768_fp32_forward_sampled_bins(lib):
    """The forward-only Ng=768 workload (24 shells k_f..192 k_f): the FP32 plan with every field
    resident (24 x 768^3 FP32 = 43.5 GB) and under an 8 GiB budget for shell fields (x-slabs of 151
    planes, plan-time FP64 counts in slabs too), and the split-BF16 plan under the same budget
    (split fields of one slab, one tensor-core level); bins of the largest, a middle and the
    smallest k1 shell against the oracle."""
    cond, rel = _sampled(lib, 768, 24, 192.0, 1.5, 0.05, 7, None, "fp32/mixed", [-1, -2, 300, 0], layout=False,
                         variants=[("fp32", 0), ("fp32", 8 << 30), ("mixed_bf16x3", 8 << 30)])
    assert np.max(cond) < 1e-6, (cond, rel)


def test_ng256_all_bins_fp32_and_mixed(lib):
    """Every bin of the Ng=256 workload (24 shells, 20x20 cells) against the full FP64 oracle
    estimate, for the FP32 and the split-BF16 plans: the condition-scaled error of every bin (the
    stated bounds, 1e-7 and 2e-6), and
    the plain relative error of the bins whose sums cancel to no less than 1e-3 (FP32) or 1e-2
    (split BF16) of their terms. Plain relative error = condition-scaled error x cancellation ratio,
    so each bin class inherits its bound from the condition-scaled one."""
    ng, ns = 256, 24
    edges = np.linspace(1.0, 64.0, ns + 1)
    spec = fieldgen.half_spectrum_c64(fieldgen.quadratic_field(ng, float(ng), 1.5, 0.05, 3))
    pl = P.make_plan(ng, float(ng), edges, 20, 20)
    res = fbe.estimate(spec.astype(np.complex128), pl, with_abs=True)
    want, scale = res["b"], res["b_scale"]
    cancel = scale / np.abs(want)
    for prec, bound, cmax in (("fp32", 1e-7, 1e3), ("mixed_bf16x3", 2e-6, 1e2)):
        gp = lib.Plan(ng, float(ng), edges, 20, 20, precision=prec)
        got = gp.estimate(torch.from_numpy(spec).cuda(), with_grid=False)[0].cpu().numpy()
        gp.check()
        gp.close()
        cond = np.abs(got - want) / scale
        rel = np.abs(got - want) / np.abs(want)
        ok = cancel < cmax
        print(f"\n[{prec} Ng={ng}] all {len(want)} bins: condition-scaled max {cond.max():.2e} median "
              f"{np.median(cond):.2e}; relative max {rel.max():.2e} median {np.median(rel):.2e}; relative max over "
              f"{ok.sum()} bins cancelling < {cmax:.0e}: {rel[ok].max():.2e}")
        assert cond.max() < bound, (prec, cond.max())
        assert rel[ok].max() < 1e-4, (prec, rel[ok].max())
