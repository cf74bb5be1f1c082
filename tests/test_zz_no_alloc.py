"""bsp_triple_sums_noalloc: the allocation-free contraction for callers that cannot call
cudaMalloc (for example code whose device memory is owned by a framework allocator). It must
agree with the plan-based contraction (bsp_contract) on the same fields, call after call.

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
    fields = plan.shell_fields(torch.from_numpy(spec).cuda())
    ref = plan.contract(fields).cpu().numpy()
    tr = plan.triplets
    trip = torch.from_numpy(np.stack([tr["a"], tr["b"], tr["c"]], 1).astype(np.int32).ravel()).cuda()
    # condition scale sum_x |d_a d_b d_c| of each bin, from the oracle on the same input
    pl = P.make_plan(ng, float(ng), edges, 20, 20)
    res = fbe.estimate(spec.astype(np.complex128), pl, with_abs=True)
    return _lib, plan, fields, trip, ref, res["asum"]


def _call(lib_mod, fields, ns, nvox, trip, n, out):
    lib = lib_mod.load()
    st = lib.bsp_triple_sums_noalloc(C.c_void_p(fields.data_ptr()), ns, nvox, C.c_void_p(trip.data_ptr()),
                                     n, C.c_void_p(out.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_matches_plan_contraction_twice(setup):
    lib_mod, plan, fields, trip, ref, asum = setup
    n = plan.n_triplets
    nvox = plan.ng_eval ** 3
    scale = (plan.ng / plan.ng_eval) ** 3  # plan sums refer to the Ng^3 grid
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
        assert np.max(np.abs(got - ref) / asum) < 1e-4
    # the second call allocated nothing on the device
    assert free_after[0] == free_after[1]


def test_noalloc_rejects_sizes_beyond_its_scratch(setup):
    lib_mod, plan, fields, trip, _, _ = setup
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    assert _call(lib_mod, fields, plan.n_shells, plan.ng_eval ** 3, trip, 4097, out) == 1
    assert b"4096" in lib_mod.load().bsp_last_error()
    assert _call(lib_mod, fields, 65, plan.ng_eval ** 3, trip, 8, out) == 1
