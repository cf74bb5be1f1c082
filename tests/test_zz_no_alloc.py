"""bsp_triple_sums_noalloc: the allocation-free contraction for callers that cannot call
cudaMalloc (for example code whose device memory is owned by a framework allocator). Fed FP32
copies of the oracle's shell fields, it must give the oracle's triple sums of those fields and
agree with the plan-based contraction (bsp_contract) on them, call after call, and it must turn
shell indices outside the fields into NaN without reading outside its inputs.

This file is named so that pytest collects it last. Needs a GB300."""
import ctypes as C

import numpy as np
import pytest

import fieldgen
from oracle import fbe
from oracle import plan as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14564_gb300 import _lib, binding
    ng = 64
    edges = P.linear_edges(12, 1.0, ng / 4)
    spec = fieldgen.half_spectrum_c64(fieldgen.quadratic_field(ng, float(ng), 1.5, 0.05, 21))
    plan = binding.Plan(ng, float(ng), edges, 20, 20, precision="fp32")
    size = plan.ng_eval
    pl = P.make_plan(ng, float(ng), edges, 20, 20)
    res = fbe.estimate(spec.astype(np.complex128), pl, with_abs=True)
    # the oracle's fields on the plan's evaluation grid, rounded to FP32: the input of both calls
    of = fbe.shell_fields_on_grid(spec.astype(np.complex128), pl, size)
    stack = np.stack([of[n] for n in range(pl.ns)]).astype(np.float32)
    scale = (ng / size) ** 3  # sums over the size^3 grid -> sums over the Ng^3 grid
    exact = fbe.triple_sums({n: stack[n].astype(np.float64) for n in range(pl.ns)}, res["triplets"]) * scale
    fields = torch.from_numpy(stack).cuda()
    tr = plan.triplets
    assert [tuple(t) for t in zip(tr["a"], tr["b"], tr["c"])] == [tuple(t) for t in res["triplets"]]
    trip = torch.from_numpy(np.stack([tr["a"], tr["b"], tr["c"]], 1).astype(np.int32).ravel()).cuda()
    ref = plan.contract(fields).cpu().numpy()  # the plan-based entry point on the same fields
    return _lib, plan, fields, trip, exact, ref, res["asum"], scale


def _call(lib_mod, fields, ns, nvox, trip, n, out):
    lib = lib_mod.load()
    st = lib.bsp_triple_sums_noalloc(C.c_void_p(fields.data_ptr()), ns, nvox, C.c_void_p(trip.data_ptr()),
                                     n, C.c_void_p(out.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_matches_oracle_and_plan_contraction_twice(setup):
    lib_mod, plan, fields, trip, exact, ref, asum, scale = setup
    n = plan.n_triplets
    nvox = plan.ng_eval ** 3
    outs = []
    free_after = []
    for _ in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib_mod, fields, plan.n_shells, nvox, trip, n, out) == 0
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
        outs.append(out.cpu().numpy() * scale)
    for got in outs:
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - exact) / asum) < 1e-4  # the oracle's sums of the same fields
        assert np.max(np.abs(got - ref) / asum) < 1e-4    # the plan-based contraction
    # the second call allocated nothing on the device
    assert free_after[0] == free_after[1]


def test_noalloc_rejects_sizes_beyond_its_scratch(setup):
    lib_mod, plan, fields, trip, *_ = setup
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    assert _call(lib_mod, fields, plan.n_shells, plan.ng_eval ** 3, trip, 4097, out) == 1
    assert b"4096" in lib_mod.load().bsp_last_error()
    assert _call(lib_mod, fields, 65, plan.ng_eval ** 3, trip, 8, out) == 1


def test_noalloc_out_of_range_shells_give_nan(setup):
    """Bins naming shell n_shells, 63, 64 or -1 (outside the fields) come back NaN; the others are
    unchanged. The kernel checks each index before it reads shared or global memory."""
    lib_mod, plan, fields, trip, exact, _, asum, scale = setup
    n = plan.n_triplets
    t = trip.clone().view(n, 3)
    bad = [0, 3, n // 2, n - 1]
    t[bad[0], 0] = plan.n_shells
    t[bad[1], 1] = 63
    t[bad[2], 2] = 64
    t[bad[3], 0] = -1
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert _call(lib_mod, fields, plan.n_shells, plan.ng_eval ** 3, t.reshape(-1).contiguous(), n, out) == 0
    got = out.cpu().numpy() * scale
    assert np.all(np.isnan(got[bad]))
    keep = np.setdiff1d(np.arange(n), bad)
    assert np.all(np.isfinite(got[keep]))
    assert np.max(np.abs(got[keep] - exact[keep]) / asum[keep]) < 1e-4
