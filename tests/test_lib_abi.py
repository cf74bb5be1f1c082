"""The C ABI library builds, loads and exports every entry point include/bispec.h declares;
argument checks that precede any CUDA call work without a GPU. CPU only."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2107_14564_gb300 import _lib, build
    build.build_library()
    return _lib.load()


def declared_entry_points():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^BSP_API\s+[\w\s\*]+?\b(bsp_\w+)\s*\(", txt, flags=re.M)
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (bsp_\w+)", out))
    assert set(names) <= exported, set(names) - exported
    from paper_2107_14564_gb300 import _lib
    assert set(names) == set(_lib.SIGNATURES)


P_EDGES = list(np.linspace(1.0, 8.0, 9))   # 8 shells up to Ng/4 at Ng = 32


def _desc(lib_mod, edges, ng=32, prec=1, n_mu=10, n_t=10, rsd=0, beta=0.0, k1_merge=1, label_k=0, budget=0, dim=0, order=0):
    e = np.ascontiguousarray(edges, dtype=np.float64)
    d = lib_mod.PlanDesc()
    d.ng, d.box_len, d.n_shells = ng, float(ng), len(e) - 1
    d.edges_kf = e.ctypes.data_as(C.POINTER(C.c_double))
    d.n_mu, d.n_t, d.rsd, d.beta, d.precision, d.mem_budget_bytes = n_mu, n_t, rsd, beta, prec, budget
    d.k1_merge, d.label_k, d.dim, d.order = k1_merge, label_k, dim, order
    return d, e


@pytest.mark.parametrize("kw,status", [
    (dict(edges=[1.0, 5.0, 11.0]), 2),              # beyond the cap of Eq. (2.12): 9*120 >= 32^2
    (dict(edges=[1.0, 3.0, 5.0], ng=30), 6),        # 30 = 2*3*5
    (dict(edges=[1.0, 3.0, 5.0], ng=2048), 6),
    (dict(edges=[1.0, 3.0, 2.0]), 1),               # not increasing
    (dict(edges=[1.5, 1.6]), 1),                    # empty shell: ceil(2.25) == ceil(2.56)
    (dict(edges=[1.0, 3.0], prec=9), 1),
    (dict(edges=[1.0, 3.0], n_mu=0), 1),
    (dict(edges=[1.0, 3.0], k1_merge=-1), 1),
    (dict(edges=[1.0, 3.0], label_k=2), 1),
    (dict(edges=P_EDGES, budget=1000), 1),           # below one x-plane of the 8 shells (S = 24)
    (dict(edges=P_EDGES, prec=2, budget=100000), 6),  # split-BF16 fields do not stream in slabs
    (dict(edges=P_EDGES, dim=5), 1),
    (dict(edges=P_EDGES, dim=2, prec=2), 6),         # 2D plans: FP64 or FP32
    (dict(edges=P_EDGES, dim=2, rsd=1), 6),
    (dict(edges=[1.0, 3.0], dim=2, ng=8192), 6),
    (dict(edges=[1.0, 5.0, 11.0], dim=2), 2),         # the cap after Eq. (2.12) holds in 2D too
    (dict(edges=P_EDGES, order=5), 1),
    (dict(edges=[1.0, 4.0, 7.0], order=4, n_mu=1, n_t=1, prec=2), 6),
    (dict(edges=[1.0, 4.0, 7.0], order=4), 1),              # order 4: one (mu, t) cell
    (dict(edges=[1.0, 4.0, 10.0], order=4, n_mu=1, n_t=1), 2),  # below Ng/3 but not below Ng/4
])
def test_argument_errors_without_gpu(lib, kw, status):
    from paper_2107_14564_gb300 import _lib
    d, keep = _desc(_lib, **kw)
    out = C.c_void_p(123)
    assert lib.bsp_plan_create(C.byref(d), None, C.byref(out)) == status
    assert out.value is None
    assert len(lib.bsp_last_error()) > 0


def test_null_arguments(lib):
    assert lib.bsp_plan_create(None, None, None) == 1
    assert lib.bsp_estimate(None, None, None, None, None) == 1
    assert lib.bsp_plan_destroy(None) == 0


def test_version(lib):
    assert b"sm_103a" in lib.bsp_version()


def test_plan_desc_layout_matches_the_header():
    """The binding's PlanDesc lists the fields of bsp_plan_desc in the header's order."""
    from paper_2107_14564_gb300 import _lib
    txt = open(os.path.join(ROOT, "include", "bispec.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} bsp_plan_desc;", txt, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            names += [re.sub(r"[\s\*]", "", n.split()[-1] if i == 0 else n)
                      for i, n in enumerate(decl.split(","))]
    assert names == [f[0] for f in _lib.PlanDesc._fields_]


def _struct_fields(name):
    txt = open(os.path.join(ROOT, "include", "bispec.h")).read()
    body = re.search(r"typedef struct \{([^{}]*)\} " + name + ";", txt).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            names += [re.sub(r"[\s\*]", "", n.split()[-1] if i == 0 else n) for i, n in enumerate(decl.split(","))]
    return names


def test_triplet_layout_matches_the_header():
    """The binding's Triplet and its numpy dtype list bsp_triplet's fields in the header's order."""
    from paper_2107_14564_gb300 import _lib, binding
    names = _struct_fields("bsp_triplet")
    assert names == [f[0] for f in _lib.Triplet._fields_] == list(binding.TRIPLET_DTYPE.names)
    assert C.sizeof(_lib.Triplet) == binding.TRIPLET_DTYPE.itemsize
