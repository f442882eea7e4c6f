"""The allocation-free fluid sums, called through the C ABI, against the
regular observables.

lbmd_population_sums_static is for callers that cannot allocate device
memory where they call it (a monitoring loop on a GPU whose memory another
framework already holds, or code that cannot take cudaMalloc's device-wide
synchronisation).  It keeps its scratch in a device array of the library.
This file is named so that pytest collects it last; it also passes on its own
in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import small_workload

pytestmark = pytest.mark.gpu


def _sums_static(lib, f_dev, solid_dev, w, out_dev, stream):
    st = lib.lbmd_population_sums_static(ctypes.c_void_p(f_dev.data_ptr()),
                                         ctypes.c_void_p(solid_dev.data_ptr()),
                                         w["nx"], w["ny"], w["nz"],
                                         ctypes.c_void_p(out_dev.data_ptr()),
                                         ctypes.c_void_p(stream.cuda_stream))
    assert st == 0
    stream.synchronize()
    return out_dev.cpu().numpy().copy()


def test_static_sums_match_observables_on_two_calls():
    import torch
    from paper_0711_2665_gb300 import lbmd, workloads

    w = small_workload()
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    lib = lbmd.lib()
    stream = sim.stream
    solid_dev = torch.from_numpy(np.ascontiguousarray(inp["solid"], dtype=np.uint8).reshape(-1)).cuda()
    out_dev = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        sim.step(6)
        obs = sim.observables()[0]
        f_dev = torch.from_numpy(sim.get_deviations()[0].reshape(-1).copy()).cuda()
        torch.cuda.synchronize()
        got = _sums_static(lib, f_dev, solid_dev, w, out_dev, stream)
        # same tolerances as the observables-vs-oracle parity test
        assert got[0] == pytest.approx(obs["mass"], rel=1e-9), call
        for a, k in enumerate("xyz"):
            assert got[1 + a] == pytest.approx(obs[f"p_fluid_{k}"], rel=1e-5, abs=1e-8), (call, k)


def test_static_sums_under_lazy_module_loading():
    """The same two-call check in a fresh process with lazy module loading
    asked for explicitly: the first call loads the array's module on the
    device, the second reuses it."""
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); "
            "import test_zz_no_alloc as t; t.test_static_sums_match_observables_on_two_calls(); print('ok')"
            % (here, os.path.dirname(here)))
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0 and p.stdout.strip().endswith("ok"), p.stderr[-2000:]


def test_static_sums_reject_oversized_lattice():
    from paper_0711_2665_gb300 import lbmd
    lib = lbmd.lib()
    # 2048^2 x 4 sites exceeds the stated maximum; rejected before any launch
    st = lib.lbmd_population_sums_static(ctypes.c_void_p(16), None, 2048, 2048, 4, ctypes.c_void_p(16), None)
    assert st == 5
