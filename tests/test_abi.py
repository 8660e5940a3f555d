"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (CPU only: no compute calls), plus one GPU-marked test
of the handles' lifetimes."""
import ctypes as C
import glob
import os
import re

import pytest

import paper_2001_01158_gb300 as lcg
from paper_2001_01158_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"LC_EXPORT[^;(]*?\b(lc_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["lc_mark_residual", "lc_mark_gradient", "lc_extract", "lc_pcg_solve",
                     "lc_solve_local_then_global", "lc_ctx_create", "lc_op_create_stencil", "lc_op_create_csr"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    path = build_library()
    L = C.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_error_strings_and_no_device_path():
    L = lcg.lib()
    assert L.lc_error_string(0) == b"ok"
    assert L.lc_error_string(5).startswith(b"Krylov breakdown")
    assert L.lc_error_string(999) == b"unknown error"
    h = C.c_void_p()
    # an out-of-range device is rejected without touching a GPU
    assert L.lc_ctx_create(C.byref(h), 1 << 20) == 1 and not h.value
    assert L.lc_ctx_create(None, 0) == 1


def test_struct_layouts_match_header():
    # sizes of the parameter structs as the C compiler lays them out
    assert C.sizeof(lcg.MarkParams) == 24
    assert C.sizeof(lcg.SolveParams) == 32
    assert C.sizeof(lcg.Params) == 120
    assert C.sizeof(lcg.Stats) == 88
    assert lcg.Params.global_.offset == 48 and lcg.Params.local.offset == 80


LAYOUT_PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "lc_api.h"
int main(void) {
    printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(lc_mark_params), sizeof(lc_solve_params),
           sizeof(lc_params), sizeof(lc_stats), sizeof(lc_heat2d_params), sizeof(lc_heat2d_stats),
           offsetof(lc_params, global), offsetof(lc_heat2d_params, params), offsetof(lc_heat2d_params, max_picard),
           offsetof(lc_heat2d_stats, t_total_ms));
    return 0;
}
"""


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """ctypes layouts of the binding equal what a C compiler makes of lc_api.h."""
    import subprocess
    src = tmp_path / "probe.c"
    src.write_text(LAYOUT_PROBE)
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(lcg.MarkParams), C.sizeof(lcg.SolveParams), C.sizeof(lcg.Params), C.sizeof(lcg.Stats),
            C.sizeof(lcg.HeatParams), C.sizeof(lcg.HeatStats), lcg.Params.global_.offset,
            lcg.HeatParams.params.offset, lcg.HeatParams.max_picard.offset, lcg.HeatStats.t_total_ms.offset]
    assert got == want


def test_noalloc_binding_rejects_a_3d_shape_without_z_faces():
    """A grid with nz > 1 given without Tz is refused on the host before the
    C call: run as 2D, it would mark only the first nx*ny cells."""
    import torch
    t = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(ValueError, match="Tz is None"):
        lcg.mark_residual_stencil_noalloc((4, 3, 2), t, t, t, None, t, t,
                                          lcg.MarkParams(lcg.THR_REL_MAX, 1e-3, lcg.EXP_NONE, 0),
                                          torch.zeros(1, dtype=torch.uint8), t, torch.zeros(1, dtype=torch.int32))


@pytest.mark.gpu
def test_context_may_be_destroyed_before_its_operators():
    """Handles are released in any order: an operator destroyed after its
    context (as a garbage collector may order them) still finds the context
    it was created on; no CUDA error is left behind for a later call."""
    import torch
    lcg.build()
    L = lcg.lib()
    ctx = C.c_void_p()
    assert L.lc_ctx_create(C.byref(ctx), 0) == 0
    n = 16
    D = torch.full((n,), 4.0, dtype=torch.float64, device="cuda")
    T = torch.ones(n, dtype=torch.float64, device="cuda")
    sh = (C.c_int32 * 3)(4, 4, 1)
    op = C.c_void_p()
    assert L.lc_op_create_stencil(ctx, C.byref(op), 2, sh, C.c_void_p(D.data_ptr()), C.c_void_p(T.data_ptr()),
                                  C.c_void_p(T.data_ptr()), None) == 0
    assert L.lc_ctx_destroy(ctx) == 0
    assert L.lc_op_destroy(op) == 0
    # a new context and operator are created without inheriting an error
    ctx2 = lcg.Context(0)
    lcg.StencilOperator(ctx2, (4, 4, 1), D, T, T)


def test_checked_entry_points_in_an_ordinary_build():
    """The bounds-checked diagnostics exist in every build; the ordinary one
    answers LC_ERR_UNSUPPORTED, reports no failures and launches nothing
    (callable without a GPU)."""
    L = C.CDLL(build_library())
    L.lc_checked_status.argtypes = [C.POINTER(C.c_int32), C.c_char_p, C.c_int32]
    L.lc_checked_selftest.argtypes = [C.c_void_p]
    n = C.c_int32(7)
    buf = C.create_string_buffer(64)
    assert L.lc_checked_status(C.byref(n), buf, len(buf)) == 8
    assert n.value == 0 and buf.value == b"not a bounds-checked build"
    assert L.lc_checked_status(None, None, 0) == 8
    assert L.lc_checked_selftest(None) == 8


def test_checked_library_is_selected_by_the_environment(monkeypatch):
    from paper_2001_01158_gb300.build import CHECKED_LIB, LIB
    monkeypatch.delenv("LC_CHECKED", raising=False)
    assert lcg.library_path() == LIB
    monkeypatch.setenv("LC_CHECKED", "1")
    assert lcg.library_path() == CHECKED_LIB and CHECKED_LIB != LIB


def test_binding_refuses_host_tensors():
    """There is no CPU path: every array the binding hands to the library
    must be a CUDA tensor of the declared type, and a host tensor is refused
    before any call."""
    import numpy as np
    import torch
    with pytest.raises(TypeError, match="CUDA tensor"):
        lcg._ptr(torch.zeros(4, dtype=torch.float64), torch.float64, "b")
    with pytest.raises(TypeError, match="CUDA tensor"):
        lcg._ptr(np.zeros(4), torch.float64, "b")
    assert lcg._ptr(None) is None
