"""Parity of the CUDA path (through the C ABI) with the FP64 oracle. Needs a GB300."""
import numpy as np
import pytest

import fieldgen
from oracle import dbe
from oracle import fbe
from oracle import plan as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14564_gb300 import binding
    return binding


def _edges(ng, ns, top=None):
    return P.linear_edges(ns, 1.0, top or ng / 4)


def _spec(ng, n_index, f, seed, c64):
    d = fieldgen.quadratic_field(ng, float(ng), n_index, f, seed)
    s = fieldgen.spectrum(d)
    if c64:
        s = s.astype(np.complex64)
    return s


def _oracle(spec, ng, edges, n_mu=10, n_t=10, beta=None, with_abs=False, counts=None):
    pl = P.make_plan(ng, float(ng), edges, n_mu, n_t)
    return pl, fbe.estimate(spec.astype(np.complex128), pl, beta=beta, with_abs=with_abs, counts=counts)


def _check_plan_tables(gp, res, pl):
    """Bins, triangle counts and (mu, t) cells are integers and flags: they must agree exactly;
    labels are computed in FP64 by the same steps on both sides and must agree to the bit."""
    tr = gp.triplets
    assert [(int(a), int(b), int(c)) for a, b, c in zip(tr["a"], tr["b"], tr["c"])] == res["triplets"]
    assert np.array_equal(tr["ntri"].astype(np.int64), res["ntri"])
    labs = res["labels"]
    assert np.array_equal(tr["i_mu"], [l["i_mu"] for l in labs])
    assert np.array_equal(tr["i_t"], [l["i_t"] for l in labs])
    assert np.array_equal(tr["inside"].astype(bool), [l["inside"] for l in labs])
    assert np.array_equal(tr["mu"], [l["mu"] for l in labs])
    assert np.array_equal(tr["t"], [l["t"] for l in labs])
    assert np.array_equal(tr["k1"], pl.kbar[tr["a"]])


def test_fp64_ng32_8_shells_parity(lib):
    """Ng=32, L=32, 8 linear shells k_f..k_Nyq/2, P=k^-2, f=0.1, 10x10 cells, FP64: 1e-10."""
    ng = 32
    edges = _edges(ng, 8)
    spec = _spec(ng, 2.0, 0.1, 1, c64=False)
    pl, res = _oracle(spec, ng, edges)
    gp = lib.Plan(ng, float(ng), edges, 10, 10, precision="fp64")
    _check_plan_tables(gp, res, pl)
    b, g = gp.estimate(torch.from_numpy(spec).cuda())
    b = b.cpu().numpy()
    g = g.cpu().numpy()
    assert np.max(np.abs(b - res["b"]) / np.abs(res["b"])) < 1e-10
    assert np.array_equal(np.isnan(g), np.isnan(res["grid"]))
    ok = ~np.isnan(g)
    assert np.max(np.abs(g[ok] - res["grid"][ok]) / np.abs(res["grid"][ok])) < 1e-10


def test_fp64_matches_direct_summation(lib):
    """GPU FP64 against the literal Eq. (2.3) loop on Ng=16 (independent of the FFT oracle)."""
    ng = 16
    edges = _edges(ng, 8)
    spec = _spec(ng, 2.0, 0.1, 2, c64=False)
    pl = P.make_plan(ng, float(ng), edges)
    msum_d, ntri_d = dbe.direct_estimate(spec, pl)
    gp = lib.Plan(ng, float(ng), edges, precision="fp64")
    b, _ = gp.estimate(torch.from_numpy(spec).cuda())
    b = b.cpu().numpy()
    vc = 1.0
    for i, (a, bb, c) in enumerate(zip(gp.triplets["a"], gp.triplets["b"], gp.triplets["c"])):
        key = (int(a), int(bb), int(c))
        assert ntri_d[key] == gp.triplets["ntri"][i]
        want = vc ** 3 * msum_d[key].real / (float(ng) ** 3 * ntri_d[key])
        assert abs(b[i] - want) <= 1e-10 * abs(want)


@pytest.mark.parametrize("ng", [48, 64, 96])
def test_fp64_other_grids(lib, ng):
    """Radix-3 lengths (48, 96) and several FFT blocks per pass, FP64 at 1e-10."""
    edges = _edges(ng, 6)
    spec = _spec(ng, 1.5, 0.2, 7 + ng, c64=False)
    pl, res = _oracle(spec, ng, edges)
    gp = lib.Plan(ng, float(ng), edges, precision="fp64")
    _check_plan_tables(gp, res, pl)
    b, _ = gp.estimate(torch.from_numpy(spec).cuda())
    assert np.max(np.abs(b.cpu().numpy() - res["b"]) / np.abs(res["b"])) < 1e-10


def test_fp64_rsd_parity(lib):
    ng = 32
    edges = _edges(ng, 8)
    spec = _spec(ng, 2.0, 0.1, 3, c64=False)
    pl, res = _oracle(spec, ng, edges, beta=0.5)
    gp = lib.Plan(ng, float(ng), edges, rsd=True, beta=0.5, precision="fp64")
    b, _ = gp.estimate(torch.from_numpy(spec).cuda())
    assert np.max(np.abs(b.cpu().numpy() - res["b"]) / np.abs(res["b"])) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shell_fields_parity(lib, prec):
    ng = 64
    edges = _edges(ng, 8)
    c64 = prec != "fp64"
    spec = _spec(ng, 1.5, 0.1, 4, c64=c64)
    pl = P.make_plan(ng, float(ng), edges)
    gp = lib.Plan(ng, float(ng), edges, precision=prec)
    want = fbe.shell_fields_on_grid(spec.astype(np.complex128), pl, gp.ng_eval)
    got = gp.shell_fields(torch.from_numpy(spec).cuda()).cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 2e-6
    for n in range(pl.ns):
        scale = np.abs(want[n]).max()
        assert np.abs(got[n] - want[n]).max() <= tol * scale, n


def _cond_err(b, res):
    """Error against the condition scale V_c^3 sum|d d d| / (V T) of each bin."""
    return np.abs(b - res["b"]) / res["b_scale"]


@pytest.mark.parametrize("prec", ["fp32", "mixed_bf16x3"])
def test_fp32_parity_ragged(lib, prec):
    """Ng=64 with 12 shells: several contraction tiles and voxel chunks; FP32 within 1e-4 of the
    condition scale (the relative error itself is reported by the bench)."""
    ng = 64
    edges = _edges(ng, 12)
    spec = _spec(ng, 1.5, 0.05, 5, c64=True)
    pl, res = _oracle(spec, ng, edges, 20, 20, with_abs=True)
    gp = lib.Plan(ng, float(ng), edges, 20, 20, precision=prec)
    _check_plan_tables(gp, res, pl)
    b, g = gp.estimate(torch.from_numpy(spec).cuda())
    assert np.max(_cond_err(b.cpu().numpy(), res)) < 1e-4
    assert np.array_equal(np.isnan(g.cpu().numpy()), np.isnan(res["grid"]))


@pytest.mark.parametrize("prec", ["fp32", "mixed_bf16x3"])
def test_rsd_parity_on_the_warp_passes(lib, prec):
    """Kaiser RSD (Eq. (3.4), beta = 0.5) through the warp FFT passes, whose X pass applies the
    factor in FP32 as it reads each tile: Ng = 192 with 12 shells up to 48 k_f (a 192^3
    evaluation grid), shell fields and the estimate against the oracle."""
    ng = 192
    edges = P.linear_edges(12, 1.0, 48.0)
    spec = _spec(ng, 1.5, 0.05, 24, c64=True)
    pl, res = _oracle(spec, ng, edges, beta=0.5, with_abs=True)
    gp = lib.Plan(ng, float(ng), edges, rsd=True, beta=0.5, precision=prec)
    assert gp.ng_eval >= 128  # the warp passes
    d = torch.from_numpy(spec).cuda()
    b = gp.estimate(d)[0].cpu().numpy()
    gp.check()
    assert np.max(_cond_err(b, res)) < (1e-6 if prec == "fp32" else 1e-4)
    if prec == "fp32":
        spec64 = spec.astype(np.complex128) * fbe.kaiser_factor_half(ng, 0.5)
        want = fbe.shell_fields_on_grid(spec64, pl, gp.ng_eval)
        got = gp.shell_fields(d).cpu().numpy()
        for n in range(pl.ns):
            assert np.abs(got[n] - want[n]).max() <= 2e-6 * np.abs(want[n]).max(), n
    gp.close()


def test_contract_on_oracle_fields(lib):
    """The contraction alone, fed the oracle's FP64 fields sampled on the plan's evaluation grid;
    its sums must equal the oracle's sums over the full Ng^3 grid (the coarser grid is exact)."""
    ng = 32
    edges = _edges(ng, 8)
    spec = _spec(ng, 2.0, 0.1, 6, c64=False)
    pl, res = _oracle(spec, ng, edges)
    gp = lib.Plan(ng, float(ng), edges, precision="fp64")
    assert gp.ng_eval < ng
    fields = fbe.shell_fields_on_grid(spec, pl, gp.ng_eval)
    stack = np.stack([fields[n] for n in range(pl.ns)])
    msum = gp.contract(torch.from_numpy(stack).cuda()).cpu().numpy()
    assert np.max(np.abs(msum - res["msum"]) / np.abs(res["msum"])) < 1e-10


def test_host_entry_point(lib):
    ng = 32
    edges = _edges(ng, 8)
    spec = _spec(ng, 2.0, 0.1, 1, c64=True)
    gp = lib.Plan(ng, float(ng), edges, precision="fp32")
    b_dev, g_dev = gp.estimate(torch.from_numpy(spec).cuda())
    # pinned and pageable host memory
    for host in (torch.from_numpy(spec).pin_memory(), np.ascontiguousarray(spec)):
        b_h, g_h = gp.estimate_host(host)
        assert np.array_equal(b_h, b_dev.cpu().numpy())
        assert np.array_equal(np.nan_to_num(g_h, nan=-1.0), np.nan_to_num(g_dev.cpu().numpy(), nan=-1.0))


def test_errors_are_reported(lib):
    with pytest.raises(lib.BispecError) as e:
        lib.Plan(32, 32.0, [1.0, 5.0, 11.0])
    assert e.value.status == 2                       # BSP_ERR_ALIASING
    with pytest.raises(lib.BispecError) as e:
        lib.Plan(30, 30.0, [1.0, 3.0, 5.0])         # 30 = 2*3*5 is not supported
    assert e.value.status == 6
    with pytest.raises(lib.BispecError):
        lib.Plan(32, 32.0, [1.5, 1.6])               # empty shell


@pytest.mark.parametrize("ng,ns,top", [(32, 6, 8.0), (64, 12, 16.0), (128, 40, 32.0)])
def test_mixed_contraction_shapes(lib, ng, ns, top):
    """Tensor-core contraction with 6 (padded to 32), 12 and 40 (padded to 64) shells; bins
    spread over one to several M tiles of 128 pairs. Within 1e-4 of the condition scale."""
    edges = P.linear_edges(ns, 1.0, top)
    spec = _spec(ng, 1.5, 0.1, 30 + ns, c64=True)
    pl, res = _oracle(spec, ng, edges, with_abs=True)
    gp = lib.Plan(ng, float(ng), edges, precision="mixed_bf16x3")
    b, _ = gp.estimate(torch.from_numpy(spec).cuda())
    gp.check()
    err = _cond_err(b.cpu().numpy(), res)
    assert np.max(err) < 1e-4, np.max(err)


def test_mixed_contract_on_oracle_fields(lib):
    """The tensor-core contraction alone, fed FP32 copies of the oracle's fields."""
    ng = 64
    edges = _edges(ng, 10)
    spec = _spec(ng, 2.0, 0.1, 8, c64=False)
    pl, res = _oracle(spec, ng, edges, with_abs=True)
    gp = lib.Plan(ng, float(ng), edges, precision="mixed_bf16x3")
    size = gp.ng_eval
    fields = fbe.shell_fields_on_grid(spec, pl, size)
    stack = np.stack([fields[n] for n in range(pl.ns)]).astype(np.float32)
    exact = fbe.triple_sums({n: stack[n].astype(np.float64) for n in range(pl.ns)}, res["triplets"])
    exact *= (ng / size) ** 3
    msum = gp.contract(torch.from_numpy(stack).cuda()).cpu().numpy()
    gp.check()
    assert np.max(np.abs(msum - exact) / res["asum"]) < 1e-4


def test_autotuned_plan_matches(lib):
    """The autotuner only changes how each level's voxels are split over blocks: the estimate
    agrees with the untuned plan to the FP32 partial-sum rounding (condition-scaled)."""
    ng = 128
    edges = _edges(ng, 20, 32.0)
    spec = _spec(ng, 1.5, 0.05, 21, c64=True)
    pl, res = _oracle(spec, ng, edges, with_abs=True)
    d = torch.from_numpy(spec).cuda()
    a = lib.Plan(ng, float(ng), edges, precision="mixed_bf16x3")
    b = lib.Plan(ng, float(ng), edges, precision="mixed_bf16x3", autotune=True)
    assert [g for g, _ in a.tuning] == [g for g, _ in b.tuning]
    assert all(m in (1, 2, 4) for _, m in b.tuning)
    ba = a.estimate(d)[0].cpu().numpy()
    bb = b.estimate(d)[0].cpu().numpy()
    a.check()
    b.check()
    assert np.max(np.abs(ba - bb) / res["b_scale"]) < 1e-5
    assert np.max(_cond_err(bb, res)) < 1e-4
    # the FFT pass grids change no value: the shell fields are the same bits
    assert a.pass_tuning == (0, 0) and all(v % torch.cuda.get_device_properties(0).multi_processor_count == 0
                                           for v in b.pass_tuning)
    assert torch.equal(a.shell_fields(d), b.shell_fields(d))


def test_mixed_levels_merge_only_upwards(lib):
    """Split-BF16 plans merge a contraction level into the next one up where the level's pairs
    cost less in that level's tile groups. Every bin must then sit on a grid at least as fine as
    the smallest exact one (the FP32 plan's level of the same bin), no level may be empty, and the
    estimate stays within the bound."""
    ng = 128
    edges = _edges(ng, 20, 32.0)
    spec = _spec(ng, 1.5, 0.05, 22, c64=True)
    pl, res = _oracle(spec, ng, edges, with_abs=True)
    m = lib.Plan(ng, float(ng), edges, precision="mixed_bf16x3")
    f = lib.Plan(ng, float(ng), edges, precision="fp32")
    side_m = np.array([g for g, _ in m.tuning])[m.bin_level]
    side_f = np.array([g for g, _ in f.tuning])[f.bin_level]
    assert np.all(side_m >= side_f)
    assert np.all(m.ng_eval % side_m == 0)
    assert set(m.bin_level) == set(range(len(m.tuning)))
    assert len(m.tuning) <= len(f.tuning)
    b = m.estimate(torch.from_numpy(spec).cuda())[0].cpu().numpy()
    m.check()
    assert np.max(_cond_err(b, res)) < 1e-4
    print(f"\nlevels FP32 {[g for g, _ in f.tuning]} split BF16 {[g for g, _ in m.tuning]}")
    m.close()
    f.close()


def test_bounded_wait_running_out_is_reported(lib):
    """The device-side failure path: a bounded mbarrier wait that runs out (the self-test kernel
    waits on a barrier nothing arrives at) raises the plan's flag; bsp_plan_check reports
    BSP_ERR_TIMEOUT once and clears it, and the plan's next estimate is still correct."""
    ng = 64
    edges = _edges(ng, 8)
    spec = _spec(ng, 1.5, 0.05, 23, c64=True)
    pl, res = _oracle(spec, ng, edges, with_abs=True)
    gp = lib.Plan(ng, float(ng), edges, precision="mixed_bf16x3")
    gp.check()
    lib.bsp_selftest_wait_timeout(gp.handle)
    with pytest.raises(RuntimeError, match="BSP_ERR_TIMEOUT"):
        gp.check()
    gp.check()  # reported once
    b = gp.estimate(torch.from_numpy(spec).cuda())[0].cpu().numpy()
    gp.check()
    assert np.max(_cond_err(b, res)) < 1e-4
    gp.close()


def test_host_entry_reads_only_the_shell_box(lib):
    """bsp_estimate_host copies only |m_x|, |m_y|, m_z < r of the outermost shell: NaN written
    everywhere else in the host spectrum changes nothing."""
    ng = 64
    edges = _edges(ng, 10)
    spec = _spec(ng, 1.5, 0.05, 23, c64=True)
    gp = lib.Plan(ng, float(ng), edges, precision="mixed_bf16x3")
    b_dev, g_dev = gp.estimate(torch.from_numpy(spec).cuda())
    pl = P.make_plan(ng, float(ng), edges)
    r = int(np.sqrt(pl.thresholds[-1] - 1)) + 1
    m = np.fft.fftfreq(ng, 1.0 / ng).astype(int)
    inside = (np.abs(m)[:, None, None] < r) & (np.abs(m)[None, :, None] < r) & (np.arange(ng // 2 + 1)[None, None, :] < r)
    dirty = spec.copy()
    dirty[~inside] = np.nan
    assert gp.host_input_bytes == int(inside.sum()) * 8
    b_h, g_h = gp.estimate_host(torch.from_numpy(dirty).pin_memory())
    assert np.array_equal(b_h, b_dev.cpu().numpy())
    assert np.array_equal(np.nan_to_num(g_h, nan=-1.0), np.nan_to_num(g_dev.cpu().numpy(), nan=-1.0))


@pytest.mark.parametrize("prec", ["fp32", "mixed_bf16x3"])
def test_log_spaced_shells(lib, prec):
    """Shells of growing width (log-spaced edges, Sec. 2.1 allows any ring widths): plan tables
    and values against the oracle."""
    ng = 64
    edges = np.geomspace(1.0, 16.0, 11)
    spec = _spec(ng, 1.5, 0.05, 24, c64=True)
    pl, res = _oracle(spec, ng, edges, with_abs=True)
    gp = lib.Plan(ng, float(ng), edges, precision=prec)
    _check_plan_tables(gp, res, pl)
    b, _ = gp.estimate(torch.from_numpy(spec).cuda())
    gp.check()
    assert np.max(_cond_err(b.cpu().numpy(), res)) < 1e-4


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed_bf16x3"])
def test_degenerate_inputs(lib, prec):
    """One shell (bins (0, 0, 0) only) and a zero field (every sum exactly zero)."""
    ng = 32
    dtype = np.complex128 if prec == "fp64" else np.complex64
    one = lib.Plan(ng, float(ng), [2.0, 6.0], precision=prec)
    tr = one.triplets
    assert len(tr) == 1 and (tr["a"][0], tr["b"][0], tr["c"][0]) == (0, 0, 0)
    spec = _spec(ng, 2.0, 0.1, 25, c64=prec != "fp64")
    pl, res = _oracle(spec, ng, [2.0, 6.0], with_abs=True)
    b, _ = one.estimate(torch.from_numpy(spec).cuda())
    assert abs(b.cpu().numpy()[0] - res["b"][0]) <= (1e-10 if prec == "fp64" else 1e-4) * res["b_scale"][0]
    many = lib.Plan(ng, float(ng), _edges(ng, 8), precision=prec)
    zero = torch.zeros((ng, ng, ng // 2 + 1), dtype=torch.from_numpy(np.zeros(1, dtype)).dtype, device="cuda")
    bz, gz = many.estimate(zero)
    many.check()
    assert np.all(bz.cpu().numpy() == 0.0)
    g = gz.cpu().numpy()
    assert np.all((g == 0.0) | np.isnan(g))


def test_shell_count_limits(lib):
    """The tensor-core contraction takes at most 64 shells (N <= 64 per MMA); FP32 plans more."""
    ng = 256
    edges = np.linspace(1.0, 66.0, 66)                  # 65 shells of width 1
    with pytest.raises(lib.BispecError) as e:
        lib.Plan(ng, float(ng), edges, precision="mixed_bf16x3")
    assert e.value.status == 6                          # BSP_ERR_NOT_SUPPORTED
    gp = lib.Plan(ng, float(ng), np.linspace(1.0, 64.0, 65), precision="mixed_bf16x3")
    assert gp.n_shells == 64
    gp.close()


@pytest.mark.parametrize("k1_merge", [2, 3])
def test_merged_k1_groups(lib, k1_merge):
    """(mu, t) cells spanning k1_merge neighbouring k1 shells (Sec. 2.1, merging adjacent bins),
    FP64 plan, device and host entries: grid shape, empty cells and values against the oracle."""
    ng = 32
    edges = _edges(ng, 8)
    spec = _spec(ng, 2.0, 0.1, 41, c64=False)
    pl = P.make_plan(ng, float(ng), edges, 6, 6, k1_merge=k1_merge)
    res = fbe.estimate(spec, pl)
    gp = lib.Plan(ng, float(ng), edges, 6, 6, precision="fp64", k1_merge=k1_merge)
    assert gp.n_groups == pl.n_groups == -(-8 // k1_merge)
    b, g = gp.estimate(torch.from_numpy(spec).cuda())
    _, gh = gp.estimate_host(spec)
    for grid in (g.cpu().numpy(), gh):
        assert grid.shape == res["grid"].shape
        assert np.array_equal(np.isnan(grid), np.isnan(res["grid"]))
        ok = ~np.isnan(grid)
        assert np.max(np.abs(grid[ok] - res["grid"][ok]) / np.abs(res["grid"][ok])) < 1e-10
    assert np.max(np.abs(b.cpu().numpy() - res["b"]) / np.abs(res["b"])) < 1e-10


def test_triangle_mean_labels(lib):
    """label_k = 'triangle' (the bin's average triangle, Sec. 2.1): the plan's side lengths are
    FP64 sums of Eq. (2.10) with one |k|-weighted counting field; against the oracle's to 1e-12,
    (mu, t) and cells from them, and the bin values unchanged by the choice of labels."""
    ng = 32
    edges = _edges(ng, 8)
    spec = _spec(ng, 2.0, 0.1, 43, c64=False)
    pl = P.make_plan(ng, float(ng), edges, 10, 10, label_k="triangle")
    res = fbe.estimate(spec, pl)
    gp = lib.Plan(ng, float(ng), edges, 10, 10, precision="fp64", label_k="triangle")
    tr = gp.triplets
    assert [(int(a), int(b), int(c)) for a, b, c in zip(tr["a"], tr["b"], tr["c"])] == res["triplets"]
    labs = res["labels"]
    for k in ("k1", "k2", "k3", "mu", "t"):
        want = np.array([l[k] for l in labs])
        assert np.max(np.abs(tr[k] - want) / np.abs(want)) < 1e-12, k
    # cells agree wherever the label is not within rounding of a cell edge
    for k, n, cell in (("mu", 10, "i_mu"), ("t", 10, "i_t")):
        want = np.array([l[k] for l in labs])
        frac = (np.clip(want, 0.5, 1.0) - 0.5) * 2 * n
        clear = np.abs(frac - np.rint(frac)) > 1e-9
        assert np.array_equal(tr[cell][clear], np.array([l[cell] for l in labs])[clear])
    shell = lib.Plan(ng, float(ng), edges, 10, 10, precision="fp64")
    assert np.any(np.abs(shell.triplets["mu"] - tr["mu"]) > 1e-3)
    b, _ = gp.estimate(torch.from_numpy(spec).cuda())
    b0, _ = shell.estimate(torch.from_numpy(spec).cuda())
    assert np.array_equal(b.cpu().numpy(), b0.cpu().numpy())
    assert np.max(np.abs(b.cpu().numpy() - res["b"]) / np.abs(res["b"])) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_memory_budget_slabs(lib, prec):
    """Under a budget of 7 x-planes of shell fields the plan produces and reduces the fields one
    x-slab of the evaluation grid at a time (the last slab thinner), and counts the triangles at
    plan time in slabs too: plan tables exact, values against the oracle and against the plan
    that holds every field."""
    ng = 64
    edges = _edges(ng, 12)
    spec = _spec(ng, 1.5, 0.05, 27, c64=prec != "fp64")
    pl, res = _oracle(spec, ng, edges, with_abs=True)
    full = lib.Plan(ng, float(ng), edges, precision=prec)
    size = full.ng_eval
    elem = 8 if prec == "fp64" else 4
    gp = lib.Plan(ng, float(ng), edges, precision=prec, mem_budget_bytes=7 * 12 * size * size * elem)
    assert gp.slabs == (7, -(-size // 7)) and size % 7 != 0
    assert full.slabs == (0, 1)
    assert gp.device_bytes < full.device_bytes
    _check_plan_tables(gp, res, pl)
    b, g = gp.estimate(torch.from_numpy(spec).cuda())
    b0, _ = full.estimate(torch.from_numpy(spec).cuda())
    gp.check()
    b, b0, g = b.cpu().numpy(), b0.cpu().numpy(), g.cpu().numpy()
    if prec == "fp64":
        assert np.max(np.abs(b - res["b"]) / np.abs(res["b"])) < 1e-10
        assert np.max(np.abs(b - b0) / res["b_scale"]) < 1e-13
    else:
        assert np.max(_cond_err(b, res)) < 1e-4
        assert np.max(np.abs(b - b0) / res["b_scale"]) < 1e-5
    assert np.array_equal(np.isnan(g), np.isnan(res["grid"]))


def test_mixed_memory_budget_slabs(lib):
    """A split-BF16 plan under a budget of 40 x-planes of shell fields (Ng = 128, evaluation grid
    128^3, 12 shells: slabs of 40 planes, the last 8): the Z pass writes each slab's split fields,
    the tensor-core contraction reads them through a full-slab or a last-slab tensor map and adds
    the slabs' sums. Against the oracle and the plan that holds every field, with and without the
    autotuner (whose Z-pass timing then runs on the first slab only)."""
    ng = 128
    edges = _edges(ng, 12)
    spec = _spec(ng, 1.5, 0.05, 29, c64=True)
    pl, res = _oracle(spec, ng, edges, with_abs=True)
    full = lib.Plan(ng, float(ng), edges, precision="mixed_bf16x3")
    size = full.ng_eval
    assert size == 128
    b0, _ = full.estimate(torch.from_numpy(spec).cuda())
    b0 = b0.cpu().numpy()
    for tune in (False, True):
        gp = lib.Plan(ng, float(ng), edges, precision="mixed_bf16x3", autotune=tune,
                      mem_budget_bytes=40 * 12 * size * size * 4)
        assert gp.slabs == (40, 4)
        assert gp.device_bytes < full.device_bytes
        b, g = gp.estimate(torch.from_numpy(spec).cuda())
        gp.check()
        b, g = b.cpu().numpy(), g.cpu().numpy()
        assert np.max(_cond_err(b, res)) < 1e-4
        assert np.max(np.abs(b - b0) / res["b_scale"]) < 1e-5
        assert np.array_equal(np.isnan(g), np.isnan(res["grid"]))
        gp.close()
