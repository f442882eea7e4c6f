"""The C-ABI library builds for sm_103a, loads, exports every function that
include/lbmd.h declares, and rejects bad arguments before touching the GPU.
No kernel runs here."""
import ctypes

import numpy as np
import pytest

from paper_0711_2665_gb300 import workloads


def test_library_exports_every_declared_symbol(lbmd_lib):
    L = lbmd_lib.lib()
    names = lbmd_lib.declared_symbols()
    assert "lbmd_init" in names and "lbmd_step" in names and "lbmd_observables" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_structs_match_header_layout(lbmd_lib, tmp_path):
    """The ctypes mirrors have the sizes and field offsets a C compiler gives
    the structs of include/lbmd.h."""
    import subprocess
    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "lbmd.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(lbmd_config),"
        " sizeof(lbmd_obs), sizeof(lbmd_diag), sizeof(lbmd_kernel_time), offsetof(lbmd_config, seed),"
        " offsetof(lbmd_obs, step), offsetof(lbmd_config, precision), sizeof(lbmd_transloc),"
        " offsetof(lbmd_transloc, rg_u_origin), offsetof(lbmd_diag, rg_translocated)); return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", lbmd_lib.HEADER.rsplit("/", 1)[0], "-o", str(exe), str(src)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(lbmd_lib.Config), ctypes.sizeof(lbmd_lib.Obs),
                   ctypes.sizeof(lbmd_lib.Diag), ctypes.sizeof(lbmd_lib.KernelTime),
                   lbmd_lib.Config.seed.offset, lbmd_lib.Obs.step.offset,
                   lbmd_lib.Config.precision.offset, ctypes.sizeof(lbmd_lib.Transloc),
                   lbmd_lib.Transloc.rg_u_origin.offset, lbmd_lib.Diag.rg_translocated.offset]


def _cfg(lbmd_lib, **kw):
    w = workloads.get("plain_fp64_small", **kw)
    return lbmd_lib.make_config(w)


def test_required_bytes_and_validation(lbmd_lib):
    L = lbmd_lib.lib()
    off = np.array([0, 20], dtype=np.int32)
    n = ctypes.c_size_t(0)
    c = _cfg(lbmd_lib)
    assert L.lbmd_required_bytes(ctypes.byref(c), off.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)) == 0
    ns = 32 * 16 * 16
    assert n.value >= 3 * 19 * ns * 4 + 24 * ns  # two population buffers + staging + G
    for bad in (dict(tau=0.5), dict(tau=0.3), dict(nx=0), dict(md_outer=0), dict(wall_x=40),
                dict(pore_h=-1), dict(nx=5000)):
        c = _cfg(lbmd_lib, **bad)
        assert L.lbmd_required_bytes(ctypes.byref(c), off.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(n)) == 1, bad
    c = _cfg(lbmd_lib)
    too_many = np.array([0, 1025], dtype=np.int32)
    assert L.lbmd_required_bytes(ctypes.byref(c), too_many.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.byref(n)) == 1
    decreasing = np.array([0, 5, 3], dtype=np.int32)
    c.n_real = 2
    assert L.lbmd_required_bytes(ctypes.byref(c), decreasing.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.byref(n)) == 1


def test_init_rejects_bad_buffer_without_gpu(lbmd_lib):
    """Argument checks happen before any CUDA call: a null or misaligned
    buffer returns LBMD_ERR_BUFFER and no handle."""
    L = lbmd_lib.lib()
    c = _cfg(lbmd_lib)
    off = np.array([0, 0], dtype=np.int32)
    solid = np.zeros(32 * 16 * 16, dtype=np.uint8)
    h = ctypes.c_void_p()
    st = L.lbmd_init(ctypes.byref(c), solid.ctypes.data_as(ctypes.c_void_p),
                     off.ctypes.data_as(ctypes.c_void_p), None, None, 0, None, ctypes.byref(h))
    assert st == 6 and not h.value
    st = L.lbmd_init(ctypes.byref(c), solid.ctypes.data_as(ctypes.c_void_p),
                     off.ctypes.data_as(ctypes.c_void_p), None, ctypes.c_void_p(0x1001), 1 << 30, None,
                     ctypes.byref(h))
    assert st == 6 and not h.value
    assert L.lbmd_status_string(5) == b"fixed-capacity list overflowed"


def test_binding_fails_loudly_without_gpu(lbmd_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    inp = workloads.build_inputs(workloads.get("plain_fp64_small"))
    with pytest.raises(RuntimeError):
        lbmd_lib.Simulation(workloads.get("plain_fp64_small"), inp["solid"], inp["offsets"], inp["r0"])
