"""Batched estimates over uneven grids (the 64-realisation workload's shape at reduced counts):
bsp_estimate_batched and a captured CUDA-graph batch reproduce single estimates exactly, and a
realisation of each grid agrees with the FP64 oracle. Needs a GB300."""
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
    from paper_2107_14564_gb300 import binding
    plans, specs, np_specs = [], [], []
    for ng, prec, count in ((128, "fp32", 2), (192, "fp32", 2), (256, "mixed_bf16x3", 2)):
        edges = P.linear_edges(16, 1.0, ng / 4)
        plan = binding.Plan(ng, float(ng), edges, 10, 10, precision=prec)
        for i in range(count):
            sp = fieldgen.half_spectrum_c64(fieldgen.quadratic_field(ng, float(ng), 1.5, 0.05, 100 + ng + i))
            plans.append(plan)
            np_specs.append(sp)
            specs.append(torch.from_numpy(sp).cuda())
    return binding, plans, specs, np_specs


def test_batched_equals_single(setup):
    lib, plans, specs, _ = setup
    ref = [p.estimate(s, with_grid=False)[0].clone() for p, s in zip(plans, specs)]
    outs = [torch.empty_like(r) for r in ref]
    lib.bsp_estimate_batched(plans, specs, outs)
    torch.cuda.synchronize()
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)


def test_graph_batch_replays(setup):
    lib, plans, specs, _ = setup
    ref = [p.estimate(s, with_grid=False)[0].clone() for p, s in zip(plans, specs)]
    batch = lib.Batch(plans, specs)
    for _ in range(2):
        outs = batch.run()
        torch.cuda.synchronize()
        for r, o in zip(ref, outs):
            assert torch.equal(r, o)
    batch.close()


def test_batch_against_oracle(setup):
    _, plans, specs, np_specs = setup
    seen = set()
    for p, s, sp in zip(plans, specs, np_specs):
        if p.ng in seen:
            continue
        seen.add(p.ng)
        pl = P.make_plan(p.ng, float(p.ng), P.linear_edges(16, 1.0, p.ng / 4), 10, 10)
        res = fbe.estimate(sp.astype(np.complex128), pl, with_abs=True)
        b = p.estimate(s, with_grid=False)[0].cpu().numpy()
        assert np.max(np.abs(b - res["b"]) / res["b_scale"]) < 1e-4


@pytest.mark.slow
def test_batch64_graph_equals_single_estimates(setup):
    """The 64-field workload at its full size (16 fields at Ng = 128, 24 at 192, 24 at 256, 16
    shells each, split-BF16 plans): one captured-graph replay of all 64 estimates gives, field by
    field, exactly the bins of the single estimates, twice."""
    lib = setup[0]
    plans, specs = [], []
    by_ng = {}
    for ng, count in ((128, 16), (192, 24), (256, 24)):
        by_ng[ng] = lib.Plan(ng, float(ng), P.linear_edges(16, 1.0, ng / 4), 10, 10, precision="mixed_bf16x3")
        for i in range(count):
            sp = fieldgen.half_spectrum_c64(fieldgen.quadratic_field(ng, float(ng), 1.5, 0.05, 1000 + len(specs)))
            plans.append(by_ng[ng])
            specs.append(torch.from_numpy(sp).cuda())
    ref = [p.estimate(s, with_grid=False)[0].clone() for p, s in zip(plans, specs)]
    batch = lib.Batch(plans, specs)
    for _ in range(2):
        outs = batch.run()
        torch.cuda.synchronize()
        assert len(outs) == 64
        for r, o in zip(ref, outs):
            assert torch.equal(r, o)
    batch.close()
    for p in by_ng.values():
        p.check()
        p.close()
