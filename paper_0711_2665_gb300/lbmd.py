"""Python binding of the C ABI in ``include/lbmd.h`` (argument marshalling only).

Every step of the coupled LB-MD path runs in the CUDA kernels of
``liblbmd.so``; this module only converts arrays, allocates the one device
buffer the library works in (through PyTorch's caching allocator) and passes
the current PyTorch CUDA stream.  There is no fallback: if the library or a
GPU is missing, constructing a :class:`Simulation` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbmd.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lbmd.h")

LBMD_Q = 19
MAX_BEADS_PER_REALIZATION = 1024
DIAG_RING = 1024
FP32, FP16DEV = 0, 1

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "non-finite value",
          4: "timeout", 5: "capacity exceeded", 6: "device buffer too small or misaligned"}


class LbmdError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_real", ctypes.c_int32), ("tau", ctypes.c_double),
                ("body_force", ctypes.c_double * 3), ("wall_x", ctypes.c_int32),
                ("pore_h", ctypes.c_int32), ("k_bond", ctypes.c_double), ("r0", ctypes.c_double),
                ("kappa_bend", ctypes.c_double), ("lj_sigma", ctypes.c_double),
                ("lj_eps", ctypes.c_double), ("wall_sigma", ctypes.c_double),
                ("wall_eps", ctypes.c_double), ("E", ctypes.c_double), ("gamma", ctypes.c_double),
                ("kT", ctypes.c_double), ("md_outer", ctypes.c_int32), ("md_inner", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("real_base", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("interp", ctypes.c_int32), ("integrator", ctypes.c_int32), ("lb_kT", ctypes.c_double),
                ("slab_x0", ctypes.c_int32), ("slab_nx", ctypes.c_int32)]


class SlabIO(ctypes.Structure):
    _fields_ = [("up", ctypes.c_void_p), ("send_lo", ctypes.c_void_p), ("send_hi", ctypes.c_void_p),
                ("recv_lo", ctypes.c_void_p), ("recv_hi", ctypes.c_void_p), ("plane_bytes", ctypes.c_size_t)]


class Obs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("p_fluid", ctypes.c_double * 3),
                ("p_beads", ctypes.c_double * 3), ("com", ctypes.c_double * 3),
                ("n_translocated", ctypes.c_double), ("dWH_dt", ctypes.c_double),
                ("dWE_dt", ctypes.c_double), ("rg_untranslocated", ctypes.c_double),
                ("rg_translocated", ctypes.c_double), ("step", ctypes.c_int64),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


class Diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("mass", ctypes.c_double), ("p_fluid", ctypes.c_double * 3),
                ("p_beads", ctypes.c_double * 3), ("com", ctypes.c_double * 3),
                ("n_translocated", ctypes.c_double), ("dWH_dt", ctypes.c_double),
                ("dWE_dt", ctypes.c_double), ("rg_untranslocated", ctypes.c_double),
                ("rg_translocated", ctypes.c_double)]


class Transloc(ctypes.Structure):
    _fields_ = [("t_origin", ctypes.c_int64), ("t_first", ctypes.c_int64), ("t_x", ctypes.c_int64),
                ("rg_u_origin", ctypes.c_double), ("rg_t_x", ctypes.c_double),
                ("max_translocated", ctypes.c_double)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_lib = None


def declared_symbols() -> list[str]:
    """Names of every function ``include/lbmd.h`` declares."""
    import re
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(lbmd_[a-z_0-9]+)\s*\(", text)))


def lib():
    """Load liblbmd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_0711_2665_gb300.build.build_library()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "lbmd_required_bytes": [P(Config), vp, P(sz)],
        "lbmd_init": [P(Config), vp, vp, vp, vp, sz, vp, P(vp)],
        "lbmd_step": [vp, i64],
        "lbmd_observables": [vp, P(Obs)],
        "lbmd_check": [vp],
        "lbmd_diagnostics": [vp, P(Diag), i32, P(i32)],
        "lbmd_translocation": [vp, P(Transloc)],
        "lbmd_reset_translocation": [vp],
        "lbmd_init_fluid": [vp, vp, vp],
        "lbmd_get_populations": [vp, vp],
        "lbmd_get_deviations": [vp, vp],
        "lbmd_set_populations": [vp, vp],
        "lbmd_set_deviations": [vp, vp],
        "lbmd_get_beads": [vp, vp, vp],
        "lbmd_set_beads": [vp, vp, vp],
        "lbmd_get_coupling": [vp, vp, vp],
        "lbmd_get_step": [vp, P(i64)],
        "lbmd_set_step": [vp, i64],
        "lbmd_set_graph": [vp, i32],
        "lbmd_set_tiles": [vp, i32, i32],
        "lbmd_get_tiles": [vp, P(i32), P(i32)],
        "lbmd_autotune": [vp, i32, P(i32), P(i32)],
        "lbmd_profile": [vp, i32],
        "lbmd_kernel_times": [vp, P(KernelTime), i32, P(i32)],
        "lbmd_launch_count": [vp, P(i64)],
        "lbmd_population_sums_static": [vp, vp, i32, i32, i32, vp, vp],
        "lbmd_set_md_shape": [vp, i32, i32],
        "lbmd_set_overlap": [vp, i32],
        "lbmd_get_overlap": [vp, P(i32)],
        "lbmd_get_md_shape": [vp, P(i32), P(i32)],
        "lbmd_set_md_exchange": [vp, i32],
        "lbmd_get_md_exchange": [vp, P(i32)],
        "lbmd_set_md_bonded": [vp, i32],
        "lbmd_get_md_bonded": [vp, P(i32)],
        "lbmd_get_md_reserve": [vp, P(i32)],
        "lbmd_set_md_reserve": [vp, i32],
        "lbmd_set_wait_probe": [vp, i32],
        "lbmd_set_drive": [vp, ctypes.c_double, ctypes.c_double],
        "lbmd_step_loop": [vp, i64],
        "lbmd_adjoint_required_bytes": [vp, i32, i32, P(sz)],
        "lbmd_adjoint": [vp, i32, i32, vp, sz, vp, vp, vp, vp],
        "lbmd_philox4x32_10": [vp, vp, i64, vp],
        "lbmd_slab_buffers": [vp, P(SlabIO)],
        "lbmd_slab_gather": [vp],
        "lbmd_slab_advance": [vp],
        "lbmd_slab_import": [vp],
        "lbmd_noise_gauss3": [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, i64, i64, ctypes.c_uint32, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.lbmd_status_string.argtypes = [ctypes.c_int]
    L.lbmd_status_string.restype = ctypes.c_char_p
    L.lbmd_last_error.argtypes = [vp]
    L.lbmd_last_error.restype = ctypes.c_char_p
    L.lbmd_destroy.argtypes = [vp]
    L.lbmd_destroy.restype = None
    _lib = L
    return L


def philox4x32_10(ctr_key, device: str = "cuda:0") -> np.ndarray:
    """Philox4x32-10 on the GPU (the generator of the noise): ctr_key is an
    (n, 6) array of uint32 (ctr0..ctr3, key0, key1); returns (n, 4) uint32."""
    import torch
    a = np.ascontiguousarray(ctr_key, dtype=np.uint32).reshape(-1, 6)
    src = torch.from_numpy(a.view(np.int32).copy()).to(device)
    out = torch.empty((a.shape[0], 4), dtype=torch.int32, device=device)
    st = torch.cuda.current_stream(device)
    s = lib().lbmd_philox4x32_10(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(out.data_ptr()), a.shape[0],
                                 ctypes.c_void_p(st.cuda_stream))
    if s != 0:
        raise LbmdError(s, "lbmd_philox4x32_10")
    st.synchronize()
    return out.cpu().numpy().view(np.uint32)


def noise_gauss3(seed: int, realization: int, bead0: int, n: int, step: int, substep: int,
                 device: str = "cuda:0") -> np.ndarray:
    """The bead-noise normals the particle kernel draws, (n, 3) float32."""
    import torch
    out = torch.empty((n, 3), dtype=torch.float32, device=device)
    st = torch.cuda.current_stream(device)
    s = lib().lbmd_noise_gauss3(seed, realization, bead0, n, step, substep, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(st.cuda_stream))
    if s != 0:
        raise LbmdError(s, "lbmd_noise_gauss3")
    st.synchronize()
    return out.cpu().numpy()


def make_config(w: dict) -> Config:
    """lbmd_config from a parameter dict (see workloads.py for the keys)."""
    c = Config()
    c.nx, c.ny, c.nz = int(w["nx"]), int(w["ny"]), int(w["nz"])
    c.n_real = int(w.get("n_real", 1))
    c.tau = float(w["tau"])
    c.body_force = (ctypes.c_double * 3)(*[float(v) for v in w.get("body_force", (0, 0, 0))])
    c.wall_x = int(w.get("wall_x", -1))
    c.pore_h = int(w.get("pore_h", 0))
    for k in ("k_bond", "r0", "kappa_bend", "lj_sigma", "lj_eps", "wall_sigma", "wall_eps", "E",
              "gamma", "kT"):
        setattr(c, k, float(w[k]))
    c.md_outer = int(w.get("md_outer", 5))
    c.md_inner = int(w.get("md_inner", 20))
    prec = w.get("precision", "fp32")
    c.precision = FP16DEV if prec in ("fp16dev", FP16DEV) else FP32
    c.real_base = int(w.get("real_base", 0))
    c.interp = int(w.get("interp", 0))
    c.integrator = int(w.get("integrator", 0))
    c.lb_kT = float(w.get("lb_kT", 0.0))
    c.seed = int(w.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    slab = w.get("slab")
    c.slab_x0, c.slab_nx = (int(slab[0]), int(slab[1])) if slab else (0, 0)
    return c


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class Simulation:
    """One handle of the library: n_real realizations on one GPU."""

    def __init__(self, params: dict, solid: np.ndarray, offsets, r_init, device: str = "cuda:0"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Simulation needs a CUDA GPU; there is no CPU path")
        self._lib = lib()
        self.cfg = make_config(params)
        self.device = torch.device(device)
        self.n_real = self.cfg.n_real
        # x planes of this handle's populations: the lattice's, or a slab's
        # own planes with one ghost plane on the left and two on the right
        self.nx_local = self.cfg.slab_nx + 3 if self.cfg.slab_nx > 0 else self.cfg.nx
        self.ns = self.nx_local * self.cfg.ny * self.cfg.nz
        ns_all = self.cfg.nx * self.cfg.ny * self.cfg.nz
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int32)
        self.total_beads = int(self.offsets[-1])
        solid = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        if solid.size != ns_all:
            raise ValueError("solid mask must have nx*ny*nz entries")
        r = np.ascontiguousarray(r_init, dtype=np.float64).reshape(-1)
        if r.size != 3 * self.total_beads:
            raise ValueError("r_init must have 3 * total_beads entries")
        nbytes = ctypes.c_size_t(0)
        self._check(self._lib.lbmd_required_bytes(ctypes.byref(self.cfg), _ptr(self.offsets),
                                                  ctypes.byref(nbytes)), "lbmd_required_bytes")
        self.nbytes = nbytes.value
        with torch.cuda.device(self.device):
            self.buffer = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.buffer.data_ptr()
            aligned = (base + 255) & ~255
            # the library orders its work on the caller's current stream; the
            # legacy default stream cannot be captured into a CUDA graph, so a
            # simulation created there gets a stream of its own
            self.stream = torch.cuda.current_stream(self.device)
            if self.stream.cuda_stream == 0:
                self.stream = torch.cuda.Stream(device=self.device)
                self.stream.wait_stream(torch.cuda.current_stream(self.device))
            h = ctypes.c_void_p()
            st = self._lib.lbmd_init(ctypes.byref(self.cfg), _ptr(solid), _ptr(self.offsets), _ptr(r),
                                     ctypes.c_void_p(aligned), self.nbytes,
                                     ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise LbmdError(st, "lbmd_init")
        self._h = h

    # -- plumbing --------------------------------------------------------
    def _check(self, st: int, where: str):
        if st != 0:
            detail = ""
            h = getattr(self, "_h", None)
            if h:
                detail = self._lib.lbmd_last_error(h).decode()
            raise LbmdError(st, where, detail)

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.lbmd_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stepping --------------------------------------------------------
    def step(self, n: int = 1):
        self._check(self._lib.lbmd_step(self._h, int(n)), "lbmd_step")

    def step_loop(self, n: int):
        """n steps in one launch of the device-side step loop (lbmd_step_loop)."""
        self._check(self._lib.lbmd_step_loop(self._h, int(n)), "lbmd_step_loop")

    def check(self):
        self._check(self._lib.lbmd_check(self._h), "lbmd_check")

    def set_graph(self, steps_per_graph: int):
        self._check(self._lib.lbmd_set_graph(self._h, int(steps_per_graph)), "lbmd_set_graph")

    def set_tiles(self, by: int, zc: int):
        self._check(self._lib.lbmd_set_tiles(self._h, int(by), int(zc)), "lbmd_set_tiles")

    def tiles(self):
        by, zc = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.lbmd_get_tiles(self._h, ctypes.byref(by), ctypes.byref(zc)), "lbmd_get_tiles")
        return by.value, zc.value

    def set_md_shape(self, threads_per_bead: int = 0, blocks_per_chain: int = 0):
        self._check(self._lib.lbmd_set_md_shape(self._h, int(threads_per_bead), int(blocks_per_chain)),
                    "lbmd_set_md_shape")

    def set_md_exchange(self, mode: str = "auto"):
        """Chain exchange between the blocks of a cluster: "push", "pull" or
        "auto" (lbmd_autotune chooses)."""
        code = {"auto": 0, "push": 1, "pull": 2}[mode]
        self._check(self._lib.lbmd_set_md_exchange(self._h, code), "lbmd_set_md_exchange")

    def md_exchange(self) -> str:
        m = ctypes.c_int32()
        self._check(self._lib.lbmd_get_md_exchange(self._h, ctypes.byref(m)), "lbmd_get_md_exchange")
        return "pull" if m.value == 2 else "push"

    def set_md_bonded(self, mode: str = "auto"):
        """Bonded terms of the particle kernel: "lanes" (every bead's lanes),
        "warp" (one extra warp per block) or "auto"."""
        code = {"auto": 0, "lanes": 1, "warp": 2}[mode]
        self._check(self._lib.lbmd_set_md_bonded(self._h, code), "lbmd_set_md_bonded")

    def md_bonded(self) -> str:
        m = ctypes.c_int32()
        self._check(self._lib.lbmd_get_md_bonded(self._h, ctypes.byref(m)), "lbmd_get_md_bonded")
        return "warp" if m.value == 2 else "lanes"

    def set_md_reserve(self, mode: str = "auto"):
        """SMs of the particle kernel: "reserve" (its blocks claim their SMs'
        shared memory), "share" or "auto" (lbmd_autotune chooses)."""
        code = {"auto": 0, "share": 1, "reserve": 2}[mode]
        self._check(self._lib.lbmd_set_md_reserve(self._h, code), "lbmd_set_md_reserve")

    def set_wait_probe(self, on: bool):
        """Test hook: the tensor-copy lattice pass waits on a barrier nothing
        completes and reports a timeout (lbmd_set_wait_probe)."""
        self._check(self._lib.lbmd_set_wait_probe(self._h, int(bool(on))), "lbmd_set_wait_probe")

    def md_reserve(self) -> bool:
        m = ctypes.c_int32()
        self._check(self._lib.lbmd_get_md_reserve(self._h, ctypes.byref(m)), "lbmd_get_md_reserve")
        return bool(m.value)

    def set_overlap(self, overlap: bool):
        self._check(self._lib.lbmd_set_overlap(self._h, int(bool(overlap))), "lbmd_set_overlap")

    def md_shape(self):
        t, c = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.lbmd_get_md_shape(self._h, ctypes.byref(t), ctypes.byref(c)), "lbmd_get_md_shape")
        return t.value, c.value

    def autotune(self, reps: int = 5):
        by, zc = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.lbmd_autotune(self._h, int(reps), ctypes.byref(by), ctypes.byref(zc)),
                    "lbmd_autotune")
        return by.value, zc.value

    @property
    def step_count(self) -> int:
        s = ctypes.c_int64()
        self._check(self._lib.lbmd_get_step(self._h, ctypes.byref(s)), "lbmd_get_step")
        return s.value

    def set_step(self, n: int):
        self._check(self._lib.lbmd_set_step(self._h, int(n)), "lbmd_set_step")

    # -- state -----------------------------------------------------------
    def init_fluid(self, rho=None, u=None):
        """Equilibrium populations of rho (n_real, nz, ny, nx) and u (n_real,
        3, nz, ny, nx) over this handle's planes (None: rho = 1, u = 0)."""
        r = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1) if rho is not None else None
        uu = np.ascontiguousarray(u, dtype=np.float64).reshape(-1) if u is not None else None
        if r is not None and r.size != self.n_real * self.ns:
            raise ValueError("rho must have n_real * sites entries")
        if uu is not None and uu.size != 3 * self.n_real * self.ns:
            raise ValueError("u must have 3 * n_real * sites entries")
        self._check(self._lib.lbmd_init_fluid(self._h, _ptr(r), _ptr(uu)), "lbmd_init_fluid")

    def get_populations(self) -> np.ndarray:
        f = np.empty(self.n_real * LBMD_Q * self.ns, dtype=np.float32)
        self._check(self._lib.lbmd_get_populations(self._h, _ptr(f)), "lbmd_get_populations")
        return f.reshape(self.n_real, LBMD_Q, self.cfg.nz, self.cfg.ny, self.nx_local)

    def get_deviations(self) -> np.ndarray:
        """f - w_i as stored (FP32), shape (n_real, 19, nz, ny, nx)."""
        f = np.empty(self.n_real * LBMD_Q * self.ns, dtype=np.float32)
        self._check(self._lib.lbmd_get_deviations(self._h, _ptr(f)), "lbmd_get_deviations")
        return f.reshape(self.n_real, LBMD_Q, self.cfg.nz, self.cfg.ny, self.nx_local)

    # slab mode ------------------------------------------------------------
    def slab_views(self) -> dict:
        """Torch views into this handle's buffer of its slab exchange areas:
        up (total_beads, 4) float32; send_lo, recv_hi (19, 2, nz, ny) and
        send_hi, recv_lo (19, 1, nz, ny) in the population storage type."""
        import torch
        io = SlabIO()
        self._check(self._lib.lbmd_slab_buffers(self._h, ctypes.byref(io)), "lbmd_slab_buffers")
        base = self.buffer.data_ptr()
        dt = torch.float16 if self.cfg.precision == FP16DEV else torch.float32
        esz = 2 if dt == torch.float16 else 4
        nz, ny = self.cfg.nz, self.cfg.ny

        def view(ptr, nbytes, dtype, shape):
            off = ptr - base
            return self.buffer[off:off + nbytes].view(dtype).view(shape)
        pb = io.plane_bytes
        assert pb == LBMD_Q * ny * nz * esz
        return {"up": view(io.up, 16 * max(self.total_beads, 1), torch.float32, (max(self.total_beads, 1), 4)),
                "send_lo": view(io.send_lo, 2 * pb, dt, (LBMD_Q, 2, nz, ny)),
                "send_hi": view(io.send_hi, pb, dt, (LBMD_Q, 1, nz, ny)),
                "recv_lo": view(io.recv_lo, pb, dt, (LBMD_Q, 1, nz, ny)),
                "recv_hi": view(io.recv_hi, 2 * pb, dt, (LBMD_Q, 2, nz, ny))}

    def slab_gather(self):
        self._check(self._lib.lbmd_slab_gather(self._h), "lbmd_slab_gather")

    def slab_advance(self):
        self._check(self._lib.lbmd_slab_advance(self._h), "lbmd_slab_advance")

    def slab_import(self):
        self._check(self._lib.lbmd_slab_import(self._h), "lbmd_slab_import")

    def set_deviations(self, h):
        """Load f - w_i (FP32), shape (n_real, 19, nz, ny, nx)."""
        a = np.ascontiguousarray(h, dtype=np.float32).reshape(-1)
        if a.size != self.n_real * LBMD_Q * self.ns:
            raise ValueError("deviations must have n_real*19*nsites entries")
        self._check(self._lib.lbmd_set_deviations(self._h, _ptr(a)), "lbmd_set_deviations")

    def set_populations(self, f):
        a = np.ascontiguousarray(f, dtype=np.float32).reshape(-1)
        if a.size != self.n_real * LBMD_Q * self.ns:
            raise ValueError("populations must have n_real*19*nsites entries")
        self._check(self._lib.lbmd_set_populations(self._h, _ptr(a)), "lbmd_set_populations")

    def get_beads(self):
        r = np.zeros(3 * max(self.total_beads, 1))
        v = np.zeros(3 * max(self.total_beads, 1))
        self._check(self._lib.lbmd_get_beads(self._h, _ptr(r), _ptr(v)), "lbmd_get_beads")
        n = self.total_beads
        return r[:3 * n].reshape(n, 3), v[:3 * n].reshape(n, 3)

    def set_beads(self, r, v=None):
        rr = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
        vv = np.ascontiguousarray(v, dtype=np.float64).reshape(-1) if v is not None else None
        self._check(self._lib.lbmd_set_beads(self._h, _ptr(rr), _ptr(vv)), "lbmd_set_beads")

    def get_coupling(self):
        n = self.total_beads
        up = np.zeros(3 * max(n, 1), dtype=np.float32)
        J = np.zeros(3 * max(n, 1), dtype=np.float32)
        self._check(self._lib.lbmd_get_coupling(self._h, _ptr(up), _ptr(J)), "lbmd_get_coupling")
        return up[:3 * n].reshape(n, 3), J[:3 * n].reshape(n, 3)

    # -- measurements ----------------------------------------------------
    def observables(self) -> list[dict]:
        arr = (Obs * self.n_real)()
        self._check(self._lib.lbmd_observables(self._h, arr), "lbmd_observables")
        out = []
        for o in arr:
            out.append(dict(mass=o.mass, p_fluid_x=o.p_fluid[0], p_fluid_y=o.p_fluid[1],
                            p_fluid_z=o.p_fluid[2], p_beads_x=o.p_beads[0], p_beads_y=o.p_beads[1],
                            p_beads_z=o.p_beads[2], com_x=o.com[0], com_y=o.com[1], com_z=o.com[2],
                            n_translocated=o.n_translocated, dWH_dt=o.dWH_dt, dWE_dt=o.dWE_dt,
                            rg_untranslocated=o.rg_untranslocated, rg_translocated=o.rg_translocated,
                            step=o.step, status=o.status))
        return out

    def diagnostics(self, max_rows: int = DIAG_RING) -> np.ndarray:
        """Per-step rows [n_real, rows] as a structured numpy array."""
        buf = (Diag * (self.n_real * max_rows))()
        rows = ctypes.c_int32()
        self._check(self._lib.lbmd_diagnostics(self._h, buf, int(max_rows), ctypes.byref(rows)),
                    "lbmd_diagnostics")
        dt = np.dtype([("step", np.int64), ("mass", np.float64), ("p_fluid", np.float64, 3),
                       ("p_beads", np.float64, 3), ("com", np.float64, 3),
                       ("n_translocated", np.float64), ("dWH_dt", np.float64), ("dWE_dt", np.float64),
                       ("rg_untranslocated", np.float64), ("rg_translocated", np.float64)])
        a = np.frombuffer(buf, dtype=dt).reshape(self.n_real, max_rows)
        return a[:, :rows.value].copy()

    def translocation(self) -> np.ndarray:
        """Translocation record of every realization (Sec. IV.A) as a structured
        array: t_origin, t_first, t_x (-1 = not yet), rg_u_origin, rg_t_x,
        max_translocated."""
        arr = (Transloc * self.n_real)()
        self._check(self._lib.lbmd_translocation(self._h, arr), "lbmd_translocation")
        dt = np.dtype([("t_origin", np.int64), ("t_first", np.int64), ("t_x", np.int64),
                       ("rg_u_origin", np.float64), ("rg_t_x", np.float64), ("max_translocated", np.float64)])
        return np.frombuffer(arr, dtype=dt).copy()

    def reset_translocation(self):
        """Restart every translocation record at the current step."""
        self._check(self._lib.lbmd_reset_translocation(self._h), "lbmd_reset_translocation")

    def profile(self, enable: bool):
        self._check(self._lib.lbmd_profile(self._h, int(bool(enable))), "lbmd_profile")

    def kernel_times(self) -> dict:
        arr = (KernelTime * 16)()
        n = ctypes.c_int32()
        self._check(self._lib.lbmd_kernel_times(self._h, arr, 16, ctypes.byref(n)), "lbmd_kernel_times")
        return {arr[k].name.decode(): (arr[k].launches, arr[k].total_ms) for k in range(n.value)}

    def launch_count(self) -> int:
        n = ctypes.c_int64()
        self._check(self._lib.lbmd_launch_count(self._h, ctypes.byref(n)), "lbmd_launch_count")
        return n.value

    # -- reverse mode ----------------------------------------------------
    def set_drive(self, gamma: float, E: float):
        self._check(self._lib.lbmd_set_drive(self._h, float(gamma), float(E)), "lbmd_set_drive")

    def adjoint_bytes(self, K: int, checkpoint_every: int) -> int:
        n = ctypes.c_size_t(0)
        self._check(self._lib.lbmd_adjoint_required_bytes(self._h, int(K), int(checkpoint_every), ctypes.byref(n)),
                    "lbmd_adjoint_required_bytes")
        return n.value

    def adjoint(self, K: int, checkpoint_every: int) -> dict:
        """Loss L_r = mean x(K) - mean x(0) of every chain over the next K steps
        and its gradient w.r.t. gamma, E and the initial bead positions
        (lbmd_adjoint); the simulation ends K steps later."""
        import torch
        nbytes = self.adjoint_bytes(K, checkpoint_every)
        with torch.cuda.device(self.device):
            scratch = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (scratch.data_ptr() + 255) & ~255
        loss = np.zeros(self.n_real)
        dg = np.zeros(self.n_real)
        dE = np.zeros(self.n_real)
        dr0 = np.zeros(3 * max(self.total_beads, 1))
        self._check(self._lib.lbmd_adjoint(self._h, int(K), int(checkpoint_every), ctypes.c_void_p(aligned), nbytes,
                                           _ptr(loss), _ptr(dg), _ptr(dE), _ptr(dr0)), "lbmd_adjoint")
        del scratch
        return dict(loss=loss, dgamma=dg, dE=dE, dr0=dr0[:3 * self.total_beads].reshape(self.total_beads, 3))


def com_displacement(sim: Simulation, r0, gamma, E, K: int, checkpoint_every: int = 20, fluid=None):
    """Differentiable centre-of-mass displacement of every chain along the
    field over K coupled steps, as a function of the initial bead positions
    r0 [total_beads, 3], the friction gamma and the pore field E (0-d
    tensors).  The forward and the reverse sweep both run in the library
    (lbmd_adjoint): the forward call computes the gradient too and keeps it
    for backward.  The simulation restarts from fluid (populations as
    get_populations returns them; None = fluid at rest) at step 0 and ends K
    steps later."""
    import torch

    class _ComDisplacement(torch.autograd.Function):
        @staticmethod
        def forward(ctx, r0_t, gamma_t, E_t):
            sim.set_drive(float(gamma_t), float(E_t))
            if fluid is None:
                sim.init_fluid()
            else:
                sim.set_populations(fluid)
            sim.set_step(0)
            sim.set_beads(r0_t.detach().cpu().double().numpy())
            out = sim.adjoint(K, checkpoint_every)
            dev = r0_t.device
            ctx.save_for_backward(torch.as_tensor(out["dr0"], dtype=r0_t.dtype, device=dev),
                                  torch.as_tensor(out["dgamma"], dtype=r0_t.dtype, device=dev),
                                  torch.as_tensor(out["dE"], dtype=r0_t.dtype, device=dev))
            ctx.offsets = sim.offsets
            return torch.as_tensor(out["loss"], dtype=r0_t.dtype, device=dev)

        @staticmethod
        def backward(ctx, gl):
            dr0, dg, dE = ctx.saved_tensors
            counts = torch.as_tensor(np.diff(ctx.offsets), device=gl.device)
            per_bead = torch.repeat_interleave(gl, counts)
            return dr0 * per_bead[:, None], (dg * gl).sum(), (dE * gl).sum()

    return _ComDisplacement.apply(r0, gamma, E)


def from_workload(w: dict, device: str = "cuda:0", inputs: dict | None = None) -> tuple[Simulation, dict]:
    """Build a Simulation for a named workload dict (paper_0711_2665_gb300.workloads)."""
    from . import workloads
    inp = inputs if inputs is not None else workloads.build_inputs(w)
    sim = Simulation(w, inp["solid"], inp["offsets"], inp["r0"], device=device)
    return sim, inp
