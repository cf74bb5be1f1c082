#!/usr/bin/env python
"""Throughput of the FFT bispectrum estimator on GB300 (one JSON line on stdout).

A step is one full estimate (all shell FFT passes, the triple-product contraction and the
(k1, mu, t) map) of one synthetic field already resident in device memory. The default
workload is the Ng=512 redshift-space case: L=512, linear RSD (Kaiser, beta=0.5, line of sight
z) on the quadratic non-Gaussian field (P(k)=k^-1.5, f_NG=0.05), 32 linear shells from k_f to
k_Nyq/2, 20x20 (mu, t) cells per k1 shell, monopole.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl ours|reference]

Under torchrun every rank estimates its own independently seeded field (replicas of one
problem: weak scaling, no collective on the data path); value = bins of all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "ng512_rsd": dict(ng=512, box=512.0, n_index=1.5, f_ng=0.05, beta=0.5, ns=32, top=128.0,
                      n_mu=20, n_t=20, seed=4,
                      text="Ng=512 L=512 quadratic NG field P=k^-1.5 f=0.05, Kaiser RSD beta=0.5 "
                           "(LoS z), 32 linear shells k_f..k_Nyq/2, 20x20 (mu,t) cells, monopole"),
    "ng256": dict(ng=256, box=256.0, n_index=1.5, f_ng=0.05, beta=None, ns=24, top=64.0,
                  n_mu=20, n_t=20, seed=3,
                  text="Ng=256 L=256 quadratic NG field P=k^-1.5 f=0.05, 24 linear shells "
                       "k_f..k_Nyq/2, 20x20 (mu,t) cells"),
}
WORKLOADS["prof384"] = dict(ng=384, box=384.0, n_index=1.5, f_ng=0.05, beta=None, ns=8, top=96.0,
                            n_mu=10, n_t=10, seed=11,
                            text="profiling case: Ng=384 L=384, 8 linear shells k_f..k_Nyq/2, 10x10 cells")
WORKLOADS["prof256"] = dict(ng=256, box=256.0, n_index=1.5, f_ng=0.05, beta=None, ns=32, top=64.0,
                            n_mu=10, n_t=10, seed=12,
                            text="profiling case: Ng=256 L=256, 32 linear shells k_f..k_Nyq/2, 10x10 cells "
                                 "(full 128-row tensor-core tiles on a 256^3 grid, 2 GB of fields)")
WORKLOADS["ng768"] = dict(ng=768, box=768.0, n_index=1.5, f_ng=0.05, beta=None, ns=24, top=192.0,
                          n_mu=20, n_t=20, seed=7,
                          text="forward-only Ng=768 L=768 quadratic NG field P=k^-1.5 f=0.05, 24 linear shells "
                               "k_f..k_Nyq/2, 20x20 (mu,t) cells (run FP32, optionally under --mem-budget-gb)")
WORKLOADS["fig_time"] = dict(text="timing against Ng (Sec. 2.2, Fig. 5): the equilateral bin of one ring (2D) or "
                                  "shell (3D) with edges 29 and 31 k_f at Ng=384, L=215, both scaled with Ng at "
                                  "fixed grid resolution (L = 215 Ng / 384); quadratic NG field P=k^-2 f=0.5",
                             ng2d=(96, 192, 384, 768, 1536, 3072), ng3d=(96, 192, 288, 384, 512),
                             dbe2d=(96, 192, 384, 768, 1536, 3072), seed=70)
WORKLOADS["batch64"] = dict(text="64 seeded quadratic NG fields (P=k^-1.5, f=0.05) on uneven grids: 16 x 128^3, "
                                 "24 x 192^3, 24 x 256^3 (L=Ng), 16 linear shells k_f..k_Nyq/2 each, 10x10 "
                                 "(mu,t) cells, one captured CUDA graph",
                            grids=((128, 16), (192, 24), (256, 24)), ns=16, n_mu=10, n_t=10)
DTYPES = {"fp64": "f64", "fp32": "f32", "mixed_bf16x3": "bf16x3/f32"}
STAGES = ["xpass", "ypass", "zpass", "contract", "finalize"]
STAGE_KERNEL_SRC = {"xpass": "bispec_fft_warp.cu", "ypass": "bispec_fft_warp.cu", "zpass": "bispec_fft_warp.cu",
                    "contract": "bispec_contract_tc.cu", "finalize": "bispec_contract.cu"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def src_hash(name):
    path = os.path.join(ROOT, "paper_2107_14564_gb300", "csrc", name)
    with open(path, "rb") as fh:
        return hashlib.sha1(fh.read()).hexdigest()[:12]


def ncu_traffic(stage, workload, precision):
    """DRAM bytes per launch of the stage's kernel from the committed ncu summary, or None when
    the kernel source changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            tab = json.load(fh)
    except OSError:
        return None
    e = tab.get(f"{workload}/{precision}/{stage}")
    if not e or e.get("src_sha1") != src_hash(STAGE_KERNEL_SRC[stage]):
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows if len(r) >= 9 for n, v in zip(names, r[5:9])
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(sm)}


def make_input(w, seed):
    import fieldgen
    delta = fieldgen.quadratic_field(w["ng"], w["box"], w["n_index"], w["f_ng"], seed)
    return fieldgen.half_spectrum_c64(delta)


def edges_of(w):
    import numpy as np
    return np.linspace(1.0, w["top"], w["ns"] + 1)


# ------------------------------------------------------------------ CPU oracle baseline
def oracle_sample(w, spec_c64, n_triplets, n_pairs):
    """Time the FP64 oracle on a bounded sample of the workload and extrapolate to one full
    estimate: ns shell FFTs (with the RSD factor), n_pairs pair products, n_triplets dot
    products. Returns (bins/s, seconds of the sample, description)."""
    import numpy as np
    from oracle import fbe
    from oracle import plan as P
    pl = P.make_plan(w["ng"], w["box"], edges_of(w), w["n_mu"], w["n_t"])
    spec = spec_c64.astype(np.complex128)
    t0 = time.perf_counter()
    if w["beta"] is not None:
        spec = spec * fbe.kaiser_factor_half(w["ng"], w["beta"])
    f = fbe.shell_fields(spec, pl, shells=[w["ns"] - 1, w["ns"] - 2])
    t1 = time.perf_counter()
    t_fft = (t1 - t0) / 2
    a, b = w["ns"] - 1, w["ns"] - 2
    # the oracle's per-pair steps (fbe.triple_sums): the pair product, a stacked copy of the third
    # fields the pair needs, one matrix-vector product; timed here with two third fields
    # as many third fields as an average pair has (the stacked copy's size drives its cost)
    m = max(1, round(n_triplets / n_pairs))
    t1 = time.perf_counter()
    prod = (f[a] * f[b]).ravel()
    t2 = time.perf_counter()
    mat = np.stack([f[a].ravel() if i % 2 == 0 else f[b].ravel() for i in range(m)])
    t3 = time.perf_counter()
    mat @ prod
    t4 = time.perf_counter()
    del mat
    t_pair = t2 - t1
    t_third = (t3 - t2 + t4 - t3) / m  # per third field: its copy and its dot product
    total = w["ns"] * t_fft + n_pairs * t_pair + n_triplets * t_third
    desc = (f"oracle timed on 2 of {w['ns']} shell FFTs and one pair's product, copied {m} third fields and "
            f"dot products ({n_pairs} pairs, {n_triplets} bins) at full Ng={w['ng']}, extrapolated to one "
            f"estimate ({total:.1f} s); a lower bound: checked against full timed estimates at Ng=256 "
            f"(bench.py --validate-oracle-model) it came out 40-50% short")
    return n_triplets / total, t4 - t0, desc


def run_reference(args, w):
    """Reference arm: the FP64 CPU oracle on the same workload, metric and unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import fbe
    from oracle import plan as P
    spec = make_input(w, w["seed"])
    pl = P.make_plan(w["ng"], w["box"], edges_of(w), w["n_mu"], w["n_t"])
    # bin list from the data-independent counts (plan time, excluded as in the GPU arm)
    n_trip, n_pairs = oracle_bin_counts(pl)
    for _ in range(args.warmup):
        oracle_sample(w, spec, n_trip, n_pairs)
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        v, _, desc = oracle_sample(w, spec, n_trip, n_pairs)
        vals.append(v)
    elapsed = time.perf_counter() - t_all
    value = statistics.mean(vals)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": metric_name(w), "value": value, "unit": "bins/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            # one step is one (extrapolated) oracle estimate; the timed samples took sample_ms each
            "ms_per_step": 1000.0 * n_trip / value, "sample_ms": 1000.0 * elapsed / max(args.steps, 1),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, "fp64"),
            "cpu_baseline": {"value": value, "unit": "bins/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "bins/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def validate_oracle_model(args):
    """Check the cpu_baseline extrapolation against a full timed oracle estimate (workload
    --workload, Ng=256 by default; the counting fields, plan time in both arms, are computed first
    and not timed). Prints one JSON line with the predicted and the measured seconds."""
    import numpy as np
    from oracle import fbe
    from oracle import plan as P
    w = WORKLOADS["ng256" if args.workload == "ng512_rsd" and not args.full_size_oracle else args.workload]
    spec = make_input(w, w["seed"])
    pl = P.make_plan(w["ng"], w["box"], edges_of(w), w["n_mu"], w["n_t"])
    n_trip, n_pairs = oracle_bin_counts(pl)
    oracle_sample(w, spec, n_trip, n_pairs)  # warm-up
    preds = [n_trip / oracle_sample(w, spec, n_trip, n_pairs)[0] for _ in range(3)]
    if args.full_size_oracle:  # the bins' counts only divide: skip the (untimed) counting pass
        counts = (list(pl.candidates), np.ones(n_trip), np.ones(n_trip))
    else:
        counts = fbe.kept_triplets(pl)
    assert len(counts[0]) == n_trip
    t0 = time.perf_counter()
    fbe.estimate(spec.astype(np.complex128), pl, beta=w["beta"], counts=counts)
    full = time.perf_counter() - t0
    pred = statistics.median(preds)
    print(json.dumps({"oracle_model_check": f"ng{w['ng']}", "bins": n_trip, "bins_per_s": round(n_trip / full, 3), "predicted_s": round(pred, 2), "measured_s": round(full, 2),
                      "model_error": round(pred / full - 1.0, 3), "cores": os.cpu_count()}), flush=True)


def oracle_bin_counts(pl):
    """(bins, distinct pairs (a, b)) of the oracle's candidate list: the bins whose shell edges
    allow a closed triangle. Counting the closed triangles themselves (N_tri > 0) takes the
    oracle's counting-field FFTs, too slow for a bench step; for the bench workloads the candidate
    list equals the kept bins (3624 at Ng=512 and 1654 at Ng=256, the CUDA plans' counts)."""
    trips = pl.candidates
    pairs = {(a, b) for a, b, _ in trips}
    return len(trips), len(pairs)


def metric_name(w):
    return f"triangle bins/sec at Ng={w['ng']} (all (k1,mu,t) bins)"


def config_of(w, precision):
    return {"workload": w["text"], "ng": w["ng"], "box_len": w["box"], "n_shells": w["ns"],
            "n_mu": w["n_mu"], "n_t": w["n_t"], "rsd_beta": w["beta"], "precision": precision,
            "l2": "no flush: every step streams its spectrum, FFT intermediates and shell fields, all larger "
                  "than the 129 MB L2"}


# ------------------------------------------------------------------ replicas over ranks
def rank_seed(seed, rank):
    """Each rank estimates its own independently seeded field (replicas, no data exchange)."""
    return seed + 1000 * rank


def max_over_ranks(x, dist):
    """The largest x over all ranks (x itself without a process group): the job's time is the
    slowest rank's."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_max):
    """Whole-job throughput: the units all ranks processed per second of the slowest rank."""
    return units_per_rank * world / (ms_max / 1000.0)


# ------------------------------------------------------------------ GPU arm
def run_ours(args, w):
    import numpy as np
    import torch
    from paper_2107_14564_gb300 import _lib, binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    spec_np = make_input(w, rank_seed(w["seed"], rank))
    spec = torch.from_numpy(spec_np).cuda()
    t0 = time.perf_counter()
    plan = binding.Plan(w["ng"], w["box"], edges_of(w), w["n_mu"], w["n_t"],
                        rsd=w["beta"] is not None, beta=w["beta"] or 0.0, precision=args.precision,
                        autotune=not args.no_autotune, mem_budget_bytes=int(args.mem_budget_gb * 2 ** 30))
    plan_s = time.perf_counter() - t0
    log(f"[bench] plan: {plan.n_triplets} bins, {plan.device_bytes / 1e9:.1f} GB on device, "
        f"{plan_s:.1f} s, x-slabs {plan.slabs}")
    for _ in range(args.warmup):
        plan.estimate(spec)
    torch.cuda.synchronize()
    lib = _lib.load()
    _lib.check(lib.bsp_timing_enable(plan.handle, 1, args.steps))
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.estimate(spec)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    import ctypes as C
    st_ms = (C.c_double * 5)()
    ncalls = C.c_int()
    nlaunch = C.c_longlong()
    _lib.check(lib.bsp_timing_read(plan.handle, st_ms, C.byref(ncalls), C.byref(nlaunch)))
    _lib.check(lib.bsp_timing_enable(plan.handle, 0, 0))
    wb = (C.c_double * 5)()
    wf = (C.c_double * 5)()
    _lib.check(lib.bsp_plan_stage_work(plan.handle, wb, wf))
    ms_max = max_over_ranks(ms, dist)
    bins = plan.n_triplets * world
    value = job_rate(plan.n_triplets, world, ms_max)
    fields_per_s = job_rate(plan.n_shells, world, ms_max)

    # end to end through the host-buffer entry point
    pinned = torch.from_numpy(spec_np).pin_memory()
    plan.estimate_host(pinned)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.estimate_host(pinned)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dist)
    e2e = {"value": bins / e2e_s, "unit": "bins/s",
           "h2d_bytes_per_step": int(plan.host_input_bytes),  # the spectrum box the shells reach
           "d2h_bytes_per_step": int(8 * (plan.n_triplets + plan.n_groups * w["n_mu"] * w["n_t"]))}

    plain = None
    if args.precision != "fp32" and not args.no_plain and world == 1:
        pplan = binding.Plan(w["ng"], w["box"], edges_of(w), w["n_mu"], w["n_t"],
                             rsd=w["beta"] is not None, beta=w["beta"] or 0.0, precision="fp32")
        for _ in range(args.warmup):
            pplan.estimate(spec)
        torch.cuda.synchronize()
        k = max(3, args.steps // 2)
        e0.record(stream)
        for _ in range(k):
            pplan.estimate(spec)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / k
        plain = {"precision": "fp32", "value": pplan.n_triplets / (pms / 1000.0), "unit": "bins/s",
                 "ms_per_step": pms, "steps": k,
                 "speedup_of_main": round(pms / ms_max, 3)}
        pplan.close()

    pk, pk_kind = peaks()
    stages = {}
    for i, name in enumerate(STAGES):
        t = st_ms[i] / 1000.0
        d = {"ms": round(st_ms[i], 4), "algo_bytes": wb[i], "algo_flops": wf[i]}
        if t > 0:
            d["gbs"] = round(wb[i] / t / 1e9, 1)
            d["hbm_frac"] = round(wb[i] / t / 1e9 / pk["hbm_gbs"], 3)
            if wf[i] > 0:
                d["tflops"] = round(wf[i] / t / 1e12, 2)
        stages[name] = d
    dom = max(range(5), key=lambda i: st_ms[i])
    dname = STAGES[dom]
    tdom = st_ms[dom] / 1000.0
    slabbed = plan.slabs[1] > 1
    if slabbed:
        # under a memory budget the Z pass and the contraction alternate slab by slab: the library
        # times them as one stage (its Z-pass stage; the contraction stage is empty)
        t = (st_ms[2] + st_ms[3]) / 1000.0
        zc = {"ms": round(st_ms[2] + st_ms[3], 4), "algo_bytes": wb[2] + wb[3], "algo_flops": wf[3]}
        if t > 0:
            zc["gbs"] = round((wb[2] + wb[3]) / t / 1e9, 1)
            zc["hbm_frac"] = round((wb[2] + wb[3]) / t / 1e9 / pk["hbm_gbs"], 3)
        stages = {"xpass": stages["xpass"], "ypass": stages["ypass"], "zpass+contract": zc,
                  "finalize": stages["finalize"]}
    tr = plan.triplets
    npairs = len({(int(a), int(b)) for a, b in zip(tr["a"], tr["b"])})
    nvox = float(plan.ng_eval) ** 3
    if slabbed and dom in (2, 3):
        t = (st_ms[2] + st_ms[3]) / 1000.0
        ach = (wb[2] + wb[3]) / t / 1e9
        roof = {"bound": "hbm", "kernel": "zpass+contract (x-slabs, timed as one stage)", "achieved": round(ach, 1),
                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(ach / pk["hbm_gbs"], 4),
                "peak_kind": f"{pk_kind} hbm_gbs", "traffic": None}
    elif dname == "contract" and args.precision == "mixed_bf16x3":
        # split-BF16 GEMM work from the library: 3 MMAs x 2 flops per (pair, padded shell column,
        # voxel), each pair on its smallest exact contraction level
        tflop = wf[dom] / 1e12
        ach = tflop / tdom
        roof = {"bound": "tensor", "kernel": "contract_tc_kernel (tcgen05 kind::f16, bf16x3)",
                "achieved": round(ach, 2), "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                "frac": round(ach / pk["bf16_tflops"], 4),
                "peak_kind": f"{pk_kind} bf16_tflops (burst, cuBLAS)",
                "work": f"3 x 2 x pairs x 32 shell columns x g^3 voxels, each pair on its smallest exact level "
                        f"({tflop:.3f} TFLOP per estimate)",
                "traffic": ncu_traffic(dname, args.workload, args.precision)}
    elif dname == "contract" and args.precision == "fp32":
        sm_mhz = pk.get("sm_max_mhz", 2070.0)
        alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        ach = wf[dom] / tdom / 1e12
        roof = {"bound": "alu", "kernel": "contract_simt_kernel<float>", "achieved": round(ach, 2),
                "peak": round(alu_peak, 1), "unit": "TFLOP/s", "frac": round(ach / alu_peak, 4),
                "peak_kind": f"FP32 CUDA-core FMA, 152 SM x 128 lanes x 2 x {sm_mhz:.0f} MHz",
                "traffic": ncu_traffic(dname, args.workload, args.precision)}
    else:
        ach = wb[dom] / tdom / 1e9
        roof = {"bound": "hbm", "kernel": dname, "achieved": round(ach, 1), "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": round(ach / pk["hbm_gbs"], 4),
                "peak_kind": f"{pk_kind} hbm_gbs",
                "traffic": ncu_traffic(dname, args.workload, args.precision)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, secs, desc = oracle_sample(w, spec_np, plan.n_triplets, npairs)
        cpu = {"value": v, "unit": "bins/s", "cores": os.cpu_count(), "kind": "oracle", "sample": desc}

    line = {"metric": metric_name(w), "value": value, "unit": "bins/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic", "config": config_of(w, args.precision),
            "fields_per_sec": fields_per_s, "n_bins": plan.n_triplets, "roofline": roof,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(nlaunch.value), "clocks": clk,
            "stages": stages, "plan_seconds": round(plan_s, 2), "plain_fp32": plain,
            "eval_grid": plan.ng_eval, "contraction_levels": plan.tuning,
            "device_bytes": plan.device_bytes, "x_slabs": list(plan.slabs),
            "fft_grid_blocks": {"ypass": plan.pass_tuning[0], "zpass": plan.pass_tuning[1]}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


def run_batch(args, w):
    """The batched workload: every field's estimate in one CUDA-graph replay per step."""
    import numpy as np
    import torch
    import fieldgen
    from paper_2107_14564_gb300 import _lib, binding
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    plans, specs, nbytes = [], [], 0
    for ng, count in w["grids"]:
        plan = binding.Plan(ng, float(ng), np.linspace(1.0, ng / 4, w["ns"] + 1), w["n_mu"], w["n_t"],
                            precision=args.precision, autotune=not args.no_autotune)
        for i in range(count):
            sp = fieldgen.half_spectrum_c64(fieldgen.quadratic_field(ng, float(ng), 1.5, 0.05, 100 + len(specs)))
            nbytes += sp.nbytes
            plans.append(plan)
            specs.append(torch.from_numpy(sp).cuda())
    bins = sum(p.n_triplets for p in plans)
    # kernels per estimate of each plan, counted by the library on one timed estimate
    import ctypes as C
    lib = _lib.load()
    per_plan = {}
    for p, sp in zip(plans, specs):
        if id(p) in per_plan:
            continue
        _lib.check(lib.bsp_timing_enable(p.handle, 1, 1))
        p.estimate(sp, with_grid=False)
        st_ms = (C.c_double * 5)()
        ncalls, nl = C.c_int(), C.c_longlong()
        _lib.check(lib.bsp_timing_read(p.handle, st_ms, C.byref(ncalls), C.byref(nl)))
        _lib.check(lib.bsp_timing_enable(p.handle, 0, 0))
        per_plan[id(p)] = int(nl.value) // max(1, int(ncalls.value))
    launches = sum(per_plan[id(p)] for p in plans)
    batch = binding.Batch(plans, specs)
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        batch.run()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # the same estimates launched one by one (no graph) for comparison
    e0.record(stream)
    for p, sp in zip(plans, specs):
        p.estimate(sp, with_grid=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1)
    line = {"metric": "triangle bins/sec over the 64-field batch", "value": bins / (ms / 1000.0),
            "unit": "bins/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": w["text"], "precision": args.precision, "fields": len(specs),
                       "l2": "inputs larger than L2 (%.1f GB of spectra)" % (nbytes / 1e9)},
            "n_bins": bins, "fields_per_sec": sum(p.n_shells for p in plans) / (ms / 1000.0),
            "ms_without_graph": ms_loop, "gpu_launches": launches * args.steps, "clocks": clk,
            "roofline": None, "cpu_baseline": None, "e2e": None}
    print(json.dumps(line), flush=True)
    batch.close()


def run_fig_time(args, w):
    """Fig. 5: FBE time of the equilateral bin against Ng in 2D and 3D (GPU, FP32 plans, CUDA
    events), with the triangle count of the bin, and the direct summation (DBE) and the FBE of
    the FP64 oracle on the host for 2D (the paper's single-core comparison)."""
    import numpy as np
    import torch
    import fieldgen
    from paper_2107_14564_gb300 import binding
    rows = []
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    clocks.start()
    for dim, ngs in ((2, w["ng2d"]), (3, w["ng3d"])):
        for ng in ngs:
            sc = ng / 384.0
            box, edges = 215.0 * sc, [29.0 * sc, 31.0 * sc]
            if dim == 2:
                spec = fieldgen.half_spectrum_c64(fieldgen.quadratic_field_2d(ng, box, 2.0, 0.5, w["seed"]))
            else:
                spec = fieldgen.half_spectrum_c64(fieldgen.quadratic_field(ng, box, 2.0, 0.5, w["seed"]))
            plan = binding.Plan(ng, box, edges, 1, 1, precision="fp32", dim=dim)
            if plan.n_triplets == 0:  # a ring this thin on this grid closes no triangle
                log(f"[fig_time] {dim}D Ng={ng}: no closed triangle")
                plan.close()
                continue
            sp = torch.from_numpy(spec).cuda()
            for _ in range(args.warmup):
                plan.estimate(sp, with_grid=False)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                plan.estimate(sp, with_grid=False)
            e1.record(stream)
            torch.cuda.synchronize()
            rows.append({"dim": dim, "ng": ng, "eval_grid": plan.ng_eval, "ntri": float(plan.triplets["ntri"][0]),
                         "fbe_gpu_ms": e0.elapsed_time(e1) / args.steps})
            log(f"[fig_time] {dim}D Ng={ng}: {rows[-1]}")
            plan.close()
            del sp
    clk = clocks.stop()
    # host side: the oracle's direct summation and FFT estimator of the same 2D bin (FP64)
    from oracle import ring2d as R
    cpu = []
    for ng in w["dbe2d"]:
        sc = ng / 384.0
        box, edges = 215.0 * sc, [29.0 * sc, 31.0 * sc]
        spec = fieldgen.spectrum(fieldgen.quadratic_field_2d(ng, box, 2.0, 0.5, w["seed"]))
        pl = R.make_plan_2d(ng, box, edges, 1, 1)
        t0 = time.perf_counter()
        _, ntri = R.direct_estimate(spec, pl)
        t1 = time.perf_counter()
        if (0, 0, 0) in ntri:
            R.estimate(spec, pl)
        t2 = time.perf_counter()
        cpu.append({"ng": ng, "ntri": ntri.get((0, 0, 0), 0), "dbe_s": t1 - t0, "fbe_s": t2 - t1})
        log(f"[fig_time] oracle 2D Ng={ng}: {cpu[-1]}")

    def slope(xs, ys):
        return float(np.polyfit(np.log(xs), np.log(ys), 1)[0])

    r2 = [r for r in rows if r["dim"] == 2]
    r3 = [r for r in rows if r["dim"] == 3]
    ref = next(r for r in r2 if r["ng"] == 384)
    line = {"metric": "seconds for the equilateral bin of the largest ring against Ng (Fig. 5)",
            "value": ref["fbe_gpu_ms"], "unit": "ms (2D FBE, Ng=384, GPU)", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ref["fbe_gpu_ms"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["text"], "l2": "small grids fit L2: launch- and latency-bound"},
            "rows": rows, "clocks": clk,
            "slopes": {"ntri_2d": slope([r["ng"] for r in r2], [r["ntri"] for r in r2]),
                       "ntri_3d": slope([r["ng"] for r in r3], [r["ntri"] for r in r3]),
                       "dbe_2d_host": slope([c["ng"] for c in cpu if c["dbe_s"] > 0.05],
                                            [c["dbe_s"] for c in cpu if c["dbe_s"] > 0.05]),
                       "fbe_2d_gpu": slope([r["ng"] for r in r2], [r["fbe_gpu_ms"] for r in r2]),
                       "fbe_3d_gpu": slope([r["ng"] for r in r3], [r["fbe_gpu_ms"] for r in r3])},
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "rows": cpu,
                             "sample": "direct summation and FP64 FFT estimator of the 2D bin, one run each"},
            "roofline": None, "e2e": None}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "mixed_bf16x3", "fp64"], default="mixed_bf16x3")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip timing the plain FP32 (CUDA-core contraction) form beside the main one")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="ng512_rsd")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mem-budget-gb", type=float, default=0.0,
                    help="GiB of shell fields a plan may hold (0: all); FP32/FP64 plans then stream x-slabs")
    ap.add_argument("--no-autotune", action="store_true",
                    help="plans skip the contraction autotuner (fixed split: one voxel block per SM)")
    ap.add_argument("--validate-oracle-model", action="store_true",
                    help="compare the cpu_baseline extrapolation with a full timed oracle estimate (Ng=256 unless "
                         "--full-size-oracle)")
    ap.add_argument("--full-size-oracle", action="store_true",
                    help="with --validate-oracle-model: time the full oracle estimate of the bench workload itself")
    args = ap.parse_args()
    if args.validate_oracle_model:
        validate_oracle_model(args)
        return
    if args.warmup < 3:
        log("[bench] warmup raised to 3")
        args.warmup = 3
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
    elif args.workload == "batch64":
        run_batch(args, w)
    elif args.workload == "fig_time":
        run_fig_time(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
