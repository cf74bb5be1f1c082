"""Thin Python binding of the C ABI (include/bispec.h) for torch device memory and streams.

Every function with a `bsp_` name marshals its arguments and calls the C entry point of the
same name; all arithmetic of the estimator runs in the library's CUDA kernels. `Plan` bundles
a plan handle with torch tensors for its outputs.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import PRECISIONS, BispecError, PlanDesc, Triplet, check

TRIPLET_DTYPE = np.dtype([("a", "i4"), ("b", "i4"), ("c", "i4"), ("i_mu", "i4"), ("i_t", "i4"),
                          ("inside", "i4"), ("ntri", "f8"), ("tsum", "f8"), ("k1", "f8"),
                          ("k2", "f8"), ("k3", "f8"), ("mu", "f8"), ("t", "f8"), ("e", "i4"),
                          ("reserved", "i4")])


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int:
    return int(t.data_ptr())


# ------------------------------------------------------------------ C names
def bsp_plan_create(desc: PlanDesc, stream=None) -> C.c_void_p:
    out = C.c_void_p()
    check(_lib.load().bsp_plan_create(C.byref(desc), C.c_void_p(_stream_ptr(stream)), C.byref(out)))
    return out


def bsp_plan_destroy(handle) -> None:
    check(_lib.load().bsp_plan_destroy(handle))


def bsp_plan_info(handle):
    nt, ns, fb, db = C.c_int(), C.c_int(), C.c_size_t(), C.c_size_t()
    check(_lib.load().bsp_plan_info(handle, C.byref(nt), C.byref(ns), C.byref(fb), C.byref(db)))
    return nt.value, ns.value, fb.value, db.value


def bsp_plan_grid(handle) -> int:
    n = C.c_int()
    check(_lib.load().bsp_plan_grid(handle, C.byref(n)))
    return n.value


def bsp_plan_pass_tuning(handle):
    """(Y-pass blocks, Z-pass blocks) the autotuner picked; 0 = as many as fit."""
    y, z = C.c_int(), C.c_int()
    check(_lib.load().bsp_plan_pass_tuning(handle, C.byref(y), C.byref(z)))
    return y.value, z.value


def bsp_plan_slabs(handle):
    """(x-planes per slab, number of slabs) an estimate streams; (0, 1) without a memory budget."""
    planes, n = C.c_int(), C.c_int()
    check(_lib.load().bsp_plan_slabs(handle, C.byref(planes), C.byref(n)))
    return planes.value, n.value


def bsp_plan_host_input_bytes(handle) -> int:
    n = C.c_size_t(0)
    check(_lib.load().bsp_plan_host_input_bytes(handle, C.byref(n)))
    return int(n.value)


def bsp_plan_tuning(handle):
    """[(level side g, voxel blocks per tile group / SM count)] in ascending g."""
    n = C.c_int(0)
    check(_lib.load().bsp_plan_tuning(handle, C.byref(n), None, None, 0))
    side = (C.c_int * max(n.value, 1))()
    mult = (C.c_int * max(n.value, 1))()
    check(_lib.load().bsp_plan_tuning(handle, C.byref(n), side, mult, n.value))
    return [(int(side[i]), int(mult[i])) for i in range(n.value)]


def bsp_plan_bin_levels(handle, n: int):
    """(level index, tensor-core tile x 64 + slot or -1) of each kept bin."""
    lev = (C.c_int * max(n, 1))()
    slot = (C.c_int * max(n, 1))()
    check(_lib.load().bsp_plan_bin_levels(handle, n, lev, slot))
    return np.array(lev[:n], dtype=np.int64), np.array(slot[:n], dtype=np.int64)


def bsp_plan_triplets(handle) -> np.ndarray:
    tab = C.POINTER(Triplet)()
    n = C.c_int()
    check(_lib.load().bsp_plan_triplets(handle, C.byref(tab), C.byref(n)))
    if n.value == 0:
        return np.zeros(0, dtype=TRIPLET_DTYPE)
    raw = C.string_at(C.cast(tab, C.c_void_p), n.value * C.sizeof(Triplet))
    return np.frombuffer(raw, dtype=TRIPLET_DTYPE).copy()


def bsp_shell_fields(handle, spec: torch.Tensor, fields_out: torch.Tensor, stream=None) -> None:
    check(_lib.load().bsp_shell_fields(handle, C.c_void_p(_ptr(spec)), C.c_void_p(_ptr(fields_out)),
                                       C.c_void_p(_stream_ptr(stream))))


def bsp_contract(handle, fields: torch.Tensor, msum: torch.Tensor, stream=None) -> None:
    check(_lib.load().bsp_contract(handle, C.c_void_p(_ptr(fields)), C.c_void_p(_ptr(msum)),
                                   C.c_void_p(_stream_ptr(stream))))


def bsp_estimate(handle, spec: torch.Tensor, b_triplet: torch.Tensor, b_grid, stream=None) -> None:
    grid = C.c_void_p(_ptr(b_grid)) if b_grid is not None else C.c_void_p(0)
    check(_lib.load().bsp_estimate(handle, C.c_void_p(_ptr(spec)), C.c_void_p(_ptr(b_triplet)), grid,
                                   C.c_void_p(_stream_ptr(stream))))


def bsp_estimate_host(handle, spec_host, b_triplet_host, b_grid_host, stream=None) -> None:
    def hp(x):
        if x is None:
            return C.c_void_p(0)
        return C.c_void_p(x.data_ptr() if isinstance(x, torch.Tensor) else x.ctypes.data)
    check(_lib.load().bsp_estimate_host(handle, hp(spec_host), hp(b_triplet_host), hp(b_grid_host),
                                        C.c_void_p(_stream_ptr(stream))))


def bsp_spectrum(handle, delta_x: torch.Tensor, spec_out: torch.Tensor, stream=None) -> None:
    check(_lib.load().bsp_spectrum(handle, C.c_void_p(_ptr(delta_x)), C.c_void_p(_ptr(spec_out)),
                                   C.c_void_p(_stream_ptr(stream))))


def bsp_grad(handle, spec: torch.Tensor, dl_db: torch.Tensor, dl_ddelta: torch.Tensor, stream=None) -> None:
    check(_lib.load().bsp_grad(handle, C.c_void_p(_ptr(spec)), C.c_void_p(_ptr(dl_db)),
                               C.c_void_p(_ptr(dl_ddelta)), C.c_void_p(_stream_ptr(stream))))


def bsp_last_sums(handle) -> int:
    p = C.c_void_p()
    check(_lib.load().bsp_last_sums(handle, C.byref(p)))
    return p.value


def bsp_plan_check(handle, stream=None) -> None:
    check(_lib.load().bsp_plan_check(handle, C.c_void_p(_stream_ptr(stream))))


def bsp_selftest_wait_timeout(handle, stream=None) -> None:
    check(_lib.load().bsp_selftest_wait_timeout(handle, C.c_void_p(_stream_ptr(stream))))


def bsp_version() -> str:
    return _lib.load().bsp_version().decode()


def _ptr_array(items):
    arr = (C.c_void_p * len(items))()
    for i, x in enumerate(items):
        arr[i] = None if x is None else (x.handle.value if isinstance(x, Plan) else _ptr(x))
    return arr


def bsp_estimate_batched(plans, specs, b_triplets, b_grids=None, stream=None) -> None:
    n = len(plans)
    grids = _ptr_array(b_grids) if b_grids is not None else None
    check(_lib.load().bsp_estimate_batched(_ptr_array(plans), _ptr_array(specs), n, _ptr_array(b_triplets),
                                           grids, C.c_void_p(_stream_ptr(stream))))


class Batch:
    """A captured CUDA graph of estimates over (plan, spectrum) pairs with preallocated outputs.
    The spectra tensors must stay alive (and unchanged in place) while the batch is used."""

    def __init__(self, plans, specs, stream=None, with_grid=False):
        self.plans = list(plans)
        self.specs = list(specs)
        for p, sp in zip(self.plans, self.specs):
            p._check_spec(sp)
        dev = self.specs[0].device
        self.b = [torch.empty(p.n_triplets, dtype=torch.float64, device=dev) for p in self.plans]
        self.grid = [torch.empty((p.n_groups, p.n_mu, p.n_t), dtype=torch.float64, device=dev)
                     for p in self.plans] if with_grid else None
        out = C.c_void_p()
        grids = _ptr_array(self.grid) if self.grid is not None else None
        check(_lib.load().bsp_batch_create(_ptr_array(self.plans), _ptr_array(self.specs), len(self.plans),
                                           _ptr_array(self.b), grids, C.c_void_p(_stream_ptr(stream)),
                                           C.byref(out)))
        self.handle = out

    def run(self, stream=None):
        check(_lib.load().bsp_batch_run(self.handle, C.c_void_p(_stream_ptr(stream))))
        return self.b

    def close(self):
        if self.handle is not None:
            check(_lib.load().bsp_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ convenience object
class Plan:
    """A binning plan plus its output tensors on the current CUDA device.

    ng, box_len, edges_kf: grid, box side and shell edges in units of k_f = 2 pi / L;
    n_mu, n_t: (mu, t) cells; rsd/beta: linear RSD along z (Eq. (3.4));
    precision: 'fp64', 'fp32' or 'mixed_bf16x3'; autotune: time the contraction's voxel split
    per level at creation and keep the fastest (tensor-core plans); k1_merge: (mu, t) cells span
    this many neighbouring k1 shells (b_grid has ceil(Ns / k1_merge) groups); label_k: 'shell'
    forms (mu, t) from the shells' mean |k|, 'triangle' from the mean sides of each bin's
    triangles; mem_budget_bytes: the most bytes of shell fields to hold at once (0: all; else
    fields are produced and reduced x-slab by x-slab, see .slabs); dim: 3 for an Ng^3 cube in
    spherical shells, 2 for an Ng^2 square in annular rings (spectrum [Ng, Ng/2+1]); order: 3 for
    the bispectrum, 4 for the binned 4-point sum over bins a >= b >= c >= e (triplets["e"])."""

    def __init__(self, ng, box_len, edges_kf, n_mu=10, n_t=10, rsd=False, beta=0.0,
                 precision="fp32", stream=None, autotune=False, k1_merge=1,
                 label_k="shell", mem_budget_bytes=0, dim=3, order=3):
        self._edges = np.ascontiguousarray(np.asarray(edges_kf, dtype=np.float64))
        desc = PlanDesc()
        desc.ng = int(ng)
        desc.box_len = float(box_len)
        desc.n_shells = len(self._edges) - 1
        desc.edges_kf = self._edges.ctypes.data_as(C.POINTER(C.c_double))
        desc.n_mu = int(n_mu)
        desc.n_t = int(n_t)
        desc.rsd = 1 if rsd else 0
        desc.beta = float(beta)
        desc.precision = PRECISIONS[precision]
        desc.mem_budget_bytes = int(mem_budget_bytes)
        desc.autotune = 1 if autotune else 0
        desc.k1_merge = int(k1_merge)
        if label_k not in ("shell", "triangle"):
            raise ValueError("label_k must be 'shell' or 'triangle'")
        desc.label_k = 0 if label_k == "shell" else 1
        desc.dim = int(dim)
        desc.order = int(order)
        self.handle = None
        self.handle = bsp_plan_create(desc, stream)
        self.ng, self.box_len, self.n_mu, self.n_t = int(ng), float(box_len), int(n_mu), int(n_t)
        self.dim = 2 if dim == 2 else 3
        self.precision = precision
        self.real_dtype = torch.float64 if precision == "fp64" else torch.float32
        self.complex_dtype = torch.complex128 if precision == "fp64" else torch.complex64
        self.n_triplets, self.n_shells, self.field_bytes, self.device_bytes = bsp_plan_info(self.handle)
        self.k1_merge = max(int(k1_merge), 1)
        self.n_groups = (self.n_shells + self.k1_merge - 1) // self.k1_merge
        self.triplets = bsp_plan_triplets(self.handle)
        self.ng_eval = bsp_plan_grid(self.handle)
        self.tuning = bsp_plan_tuning(self.handle)
        self.bin_level, self.bin_slot = bsp_plan_bin_levels(self.handle, self.n_triplets)
        self.host_input_bytes = bsp_plan_host_input_bytes(self.handle)
        self.slabs = bsp_plan_slabs(self.handle)
        self.pass_tuning = bsp_plan_pass_tuning(self.handle)

    def close(self):
        if self.handle is not None:
            bsp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spec_shape(self):
        return (self.ng,) * (self.dim - 1) + (self.ng // 2 + 1,)

    def _check_spec(self, spec: torch.Tensor):
        if not spec.is_cuda or spec.dtype != self.complex_dtype or tuple(spec.shape) != self.spec_shape() \
                or not spec.is_contiguous():
            raise ValueError(f"spec must be a contiguous CUDA {self.complex_dtype} tensor of shape "
                             f"{self.spec_shape()}")

    def estimate(self, spec: torch.Tensor, stream=None, with_grid=True):
        """(b_triplet [n_triplets], b_grid [n_groups, n_mu, n_t]) as float64 CUDA tensors."""
        self._check_spec(spec)
        dev = spec.device
        b = torch.empty(self.n_triplets, dtype=torch.float64, device=dev)
        g = torch.empty((self.n_groups, self.n_mu, self.n_t), dtype=torch.float64, device=dev) \
            if with_grid else None
        bsp_estimate(self.handle, spec, b, g, stream)
        return b, g

    def estimate_host(self, spec_host, stream=None):
        """Host-in, host-out estimate (copies inside the call). spec_host: pinned torch or numpy."""
        b = np.empty(self.n_triplets, dtype=np.float64)
        g = np.empty((self.n_groups, self.n_mu, self.n_t), dtype=np.float64)
        bsp_estimate_host(self.handle, spec_host, b, g, stream)
        return b, g

    def spectrum(self, delta_x: torch.Tensor, stream=None) -> torch.Tensor:
        """Half spectrum of a real FP32 field on the modes the plan uses (other entries zero)."""
        if not delta_x.is_cuda or delta_x.dtype != torch.float32 or not delta_x.is_contiguous() \
                or tuple(delta_x.shape) != (self.ng,) * 3:
            raise ValueError(f"delta_x must be a contiguous CUDA float32 tensor of shape {(self.ng,) * 3}")
        spec = torch.zeros(self.spec_shape(), dtype=torch.complex64, device=delta_x.device)
        bsp_spectrum(self.handle, delta_x, spec, stream)
        return spec

    def grad(self, spec: torch.Tensor, dl_db: torch.Tensor, stream=None) -> torch.Tensor:
        """dL/d delta(x) on the Ng^3 grid for dl_db = dL/dB per kept bin (float32 CUDA tensor)."""
        self._check_spec(spec)
        g = dl_db.to(device=spec.device, dtype=torch.float64).contiguous()
        if g.numel() != self.n_triplets:
            raise ValueError("dl_db must have one entry per kept bin")
        out = torch.empty((self.ng,) * 3, dtype=torch.float32, device=spec.device)
        bsp_grad(self.handle, spec, g, out, stream)
        return out

    def check(self, stream=None):
        """Raise if a bounded device-side wait gave up in an earlier call (synchronises)."""
        bsp_plan_check(self.handle, stream)

    def shell_fields(self, spec: torch.Tensor, stream=None) -> torch.Tensor:
        self._check_spec(spec)
        s = self.ng_eval
        out = torch.empty((self.n_shells,) + (s,) * self.dim, dtype=self.real_dtype, device=spec.device)
        bsp_shell_fields(self.handle, spec, out, stream)
        return out

    def contract(self, fields: torch.Tensor, stream=None) -> torch.Tensor:
        if not fields.is_cuda or fields.dtype != self.real_dtype or not fields.is_contiguous() \
                or fields.numel() != self.n_shells * self.ng_eval ** self.dim:
            raise ValueError("fields must be the contiguous [Ns, S, S, S] output of shell_fields")
        msum = torch.empty(self.n_triplets, dtype=torch.float64, device=fields.device)
        bsp_contract(self.handle, fields, msum, stream)
        return msum


__all__ = ["Plan", "BispecError", "bsp_plan_create", "bsp_plan_destroy", "bsp_plan_info",
           "bsp_plan_triplets", "bsp_plan_grid", "bsp_plan_tuning", "bsp_plan_bin_levels", "bsp_plan_host_input_bytes", "bsp_plan_slabs", "bsp_plan_pass_tuning", "bsp_shell_fields", "bsp_contract", "bsp_estimate",
           "bsp_estimate_host", "bsp_estimate_batched", "Batch", "bsp_spectrum", "bsp_grad", "bsp_last_sums", "bsp_plan_check", "bsp_selftest_wait_timeout", "bsp_version", "TRIPLET_DTYPE"]
