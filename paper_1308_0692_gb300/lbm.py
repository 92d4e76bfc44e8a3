"""Thin ctypes binding of liblbm.so (argument marshalling only).

Every function has the name of the C entry point it calls (declared in
``include/lbm.h``); all computation happens in the library's CUDA kernels.
Device memory and streams may come from PyTorch: pass ``device_buf`` as a
``torch.uint8`` CUDA tensor of ``lbm_sim_bytes(...)`` bytes and ``stream`` as a
``torch.cuda.Stream`` (or a raw ``cudaStream_t`` integer).

The library is loaded on first use; if it has not been built a RuntimeError
says how to build it -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_EUNSUPPORTED = range(7)
LBM_HALF_RANGE_GH, LBM_FULL_RANGE_GH = 0, 1
LBM_COUETTE, LBM_CAVITY = 0, 1
LBM_FP64, LBM_FP32_PERTURB = 0, 1

_STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA",
                 4: "LBM_ENONFINITE", 5: "LBM_ETIMEOUT", 6: "LBM_EUNSUPPORTED"}


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lbm_solve_info(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_long), ("correction_steps", ctypes.c_long), ("sweeps", ctypes.c_int),
                ("residual", ctypes.c_double), ("defect", ctypes.c_double)]


class lbm_problem(ctypes.Structure):
    _fields_ = [("geom", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("kn", ctypes.c_double), ("u_bottom", ctypes.c_double), ("u_top", ctypes.c_double),
                ("cfl", ctypes.c_double), ("prec", ctypes.c_int), ("residual_every", ctypes.c_int)]


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_1308_0692_gb300.build` "
                           "(the CUDA library is the only implementation)")
    lib = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    sig = {
        "lbm_make_velocity_set": (st, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]),
        "lbm_vset_query": (st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp, _dp, _dp]),
        "lbm_vset_destroy": (None, [_vp]),
        "lbm_sim_bytes": (st, [_vp, ctypes.POINTER(lbm_problem), ctypes.POINTER(ctypes.c_size_t)]),
        "lbm_init": (st, [_vp, ctypes.POINTER(lbm_problem), _dp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
        "lbm_destroy": (None, [_vp]),
        "lbm_coeffs": (st, [_vp, _dp, _dp, _dp]),
        "lbm_step": (st, [_vp, ctypes.c_long]),
        "lbm_residual": (st, [_vp, _dp, ctypes.POINTER(ctypes.c_long)]),
        "lbm_set_variant": (st, [_vp, ctypes.c_int, ctypes.c_int]),
        "lbm_solve": (st, [_vp, ctypes.c_double, ctypes.c_long, ctypes.c_int, ctypes.c_double,
                           ctypes.POINTER(lbm_solve_info)]),
        "lbm_get_variant": (st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "lbm_set_splitting": (st, [_vp, ctypes.c_int]),
        "lbm_get_splitting": (st, [_vp, ctypes.POINTER(ctypes.c_int)]),
        "lbm_set_transport": (st, [_vp, ctypes.c_int]),
        "lbm_get_transport": (st, [_vp, ctypes.POINTER(ctypes.c_int)]),
        "lbm_moments": (st, [_vp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]),
        "lbm_face_flux": (st, [_vp, _dp, _dp]),
        "lbm_get_state": (st, [_vp, _dp]),
        "lbm_set_state": (st, [_vp, _dp]),
        "lbm_get_state_f32": (st, [_vp, _fp]),
        "lbm_set_state_f32": (st, [_vp, _fp]),
        "lbm_set_moments": (st, [_vp, _dp]),
        "lbm_state_device": (st, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_long)]),
        "lbm_state_layout": (st, [_vp, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long)]),
        "lbm_state_tiling": (st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long)]),
        "lbm_norms_scratch_bytes": (st, [ctypes.c_long, ctypes.POINTER(ctypes.c_size_t)]),
        "lbm_norms": (st, [_vp, _vp, ctypes.c_long, ctypes.c_int, _vp, ctypes.c_size_t, _vp, _vp]),
        "lbm_norms_noalloc": (st, [_vp, _vp, ctypes.c_long, ctypes.c_int, _vp, _vp]),
        "lbm_probe_fp64_rate": (st, [ctypes.c_long, _dp, _vp]),
        "lbm_batch_bytes": (st, [_vp, ctypes.POINTER(lbm_problem), ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
        "lbm_batch_init": (st, [_vp, ctypes.POINTER(lbm_problem), ctypes.c_int, _vp, ctypes.c_size_t, _vp,
                                ctypes.POINTER(_vp)]),
        "lbm_batch_destroy": (None, [_vp]),
        "lbm_batch_set_schedule": (st, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "lbm_batch_get_schedule": (st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "lbm_batch_advance": (st, [_vp, ctypes.c_int, ctypes.c_double]),
        "lbm_batch_set_timeout": (st, [_vp, ctypes.c_longlong]),
        "lbm_batch_poll": (st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_long)]),
        "lbm_batch_status": (st, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_long), _dp, ctypes.POINTER(ctypes.c_int)]),
        "lbm_batch_stalled": (st, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "lbm_batch_get_state": (st, [_vp, ctypes.c_int, _dp]),
        "lbm_batch_reset": (st, [_vp]),
        "lbm_batch_moments": (st, [_vp, ctypes.c_int, _vp]),
        "lbm_batch_refine": (st, [_vp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_long, _vp]),
        "lbm_batch_set_march": (st, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "lbm_hybrid_init": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double, _vp,
                                 ctypes.POINTER(_vp)]),
        "lbm_hybrid_destroy": (None, [_vp]),
        "lbm_hybrid_query": (st, [_vp, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_double)]),
        "lbm_hybrid_set_state": (st, [_vp, _vp]),
        "lbm_hybrid_get_state": (st, [_vp, _vp]),
        "lbm_hybrid_step": (st, [_vp, ctypes.c_long]),
        "lbm_hybrid_residual": (st, [_vp, ctypes.POINTER(ctypes.c_double)]),
        "lbm_hybrid_solve": (st, [_vp, ctypes.c_double, ctypes.c_long, ctypes.c_int, ctypes.POINTER(ctypes.c_long),
                                  ctypes.POINTER(ctypes.c_double)]),
        "lbm_hybrid_velocity": (st, [_vp, _vp, _vp]),
        "lbm_hybrid_face_flux": (st, [_vp, _vp]),
        "lbm_hybrid_set_precision": (st, [_vp, ctypes.c_int]),
        "lbm_hybrid_refine": (st, [_vp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_long, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_double)]),
        "lbm_batch_get_march": (st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]),
        "lbm_batch_set_state": (st, [_vp, ctypes.c_int, _dp]),
        "lbm_batch_warm_start": (st, [_vp, ctypes.c_int, _vp, ctypes.c_double, ctypes.c_double]),
        "lbm_batch_tune": (st, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int), _dp]),
        "lbm_mlp_param_count": (st, [ctypes.POINTER(ctypes.c_long)]),
        "lbm_mlp_create": (st, [ctypes.c_int, ctypes.c_ulonglong, _vp, ctypes.POINTER(_vp)]),
        "lbm_mlp_destroy": (None, [_vp]),
        "lbm_mlp_set_params": (st, [_vp, ctypes.POINTER(ctypes.c_float)]),
        "lbm_mlp_get_params": (st, [_vp, ctypes.POINTER(ctypes.c_float)]),
        "lbm_mlp_forward": (st, [_vp, _vp, ctypes.c_int, _vp]),
        "lbm_mlp_loss_grad": (st, [_vp, _vp, _vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_float)]),
        "lbm_mlp_train_step": (st, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_float, _dp]),
        "lbm_mlp_features": (st, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _vp]),
        "lbm_warm_start": (st, [_vp, _vp, ctypes.c_double, ctypes.c_double]),
        "lbm_march_plan": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int)]),
        "lbm_stream_create": (st, [ctypes.POINTER(_vp)]),
        "lbm_stream_destroy": (None, [_vp]),
        "lbm_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def library():
    """The loaded ctypes library (for callers that bind extra entry points)."""
    return _load()


def _check(status: int):
    if status != LBM_OK:
        raise LBMError(status, _load().lbm_last_error().decode())


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def lbm_march_plan(nx: int, ny: int, blocks: int):
    """(strips, chunks) of the column-march kernel's work split (host logic, no GPU)."""
    a, c = ctypes.c_int(), ctypes.c_int()
    _check(_load().lbm_march_plan(int(nx), int(ny), int(blocks), ctypes.byref(a), ctypes.byref(c)))
    return a.value, c.value


class PrivateStream:
    """A CUDA stream of the caller's own (lbm_stream_create), usable wherever a torch stream
    is (``.torch`` is a torch.cuda.ExternalStream over it; ``cuda_stream`` the handle).
    torch.cuda.Stream() hands out streams from a small pool, so simulations driven from
    many host threads can end up sharing one; these never are."""

    def __init__(self):
        import torch
        p = _vp()
        _check(_load().lbm_stream_create(ctypes.byref(p)))
        self.cuda_stream = p.value
        self.torch = torch.cuda.ExternalStream(p.value)

    def close(self):
        if self.cuda_stream and _lib is not None:
            _lib.lbm_stream_destroy(self.cuda_stream)
        self.cuda_stream = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VelocitySet:
    """Owner of an lbm_vset* (freed on garbage collection)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.lbm_vset_destroy(self.handle)
            self.handle = None


class Sim:
    """Owner of an lbm_sim* and of the device buffer it lives in (if any)."""

    def __init__(self, handle: int, prob: lbm_problem, n_vel: int, keepalive=None):
        self.handle = handle
        self.prob = prob
        self.n_vel = n_vel
        self._keepalive = keepalive

    @property
    def ncells(self) -> int:
        return self.prob.nx * self.prob.ny

    def close(self):
        if self.handle and _lib is not None:
            _lib.lbm_destroy(self.handle)
        self.handle = None

    def __del__(self):
        self.close()


def make_problem(geom: int, nx: int, ny: int, kn: float, u_bottom: float, u_top: float,
                 cfl: float = 0.9, prec: int = LBM_FP64, residual_every: int = 100) -> lbm_problem:
    return lbm_problem(geom, nx, ny, kn, u_bottom, u_top, cfl, prec, residual_every)


def lbm_make_velocity_set(kind: int, n: int) -> VelocitySet:
    h = _vp()
    _check(_load().lbm_make_velocity_set(kind, n, ctypes.byref(h)))
    return VelocitySet(h.value)


def lbm_vset_query(vs: VelocitySet):
    """Returns (xi_x, xi_y, w, M) as float64 arrays."""
    lib = _load()
    nv, m = ctypes.c_int(), ctypes.c_int()
    _check(lib.lbm_vset_query(vs.handle, ctypes.byref(nv), ctypes.byref(m), None, None, None))
    xi_x, xi_y, w = (np.empty(nv.value) for _ in range(3))
    _check(lib.lbm_vset_query(vs.handle, None, None, _ptr(xi_x), _ptr(xi_y), _ptr(w)))
    return xi_x, xi_y, w, m.value


def lbm_sim_bytes(vs: VelocitySet, prob: lbm_problem) -> int:
    b = ctypes.c_size_t()
    _check(_load().lbm_sim_bytes(vs.handle, ctypes.byref(prob), ctypes.byref(b)))
    return b.value


def lbm_init(vs: VelocitySet, prob: lbm_problem, init_h: np.ndarray | None = None,
             device_buf=None, stream=None) -> Sim:
    """device_buf: None (library allocates) or a CUDA torch tensor (kept alive by the Sim)."""
    lib = _load()
    out = _vp()
    buf_ptr, buf_bytes = None, 0
    if device_buf is not None:
        buf_ptr = device_buf.data_ptr()
        buf_bytes = device_buf.numel() * device_buf.element_size()
    h = None if init_h is None else np.ascontiguousarray(init_h, dtype=np.float64)
    _check(lib.lbm_init(vs.handle, ctypes.byref(prob), _ptr(h), buf_ptr, buf_bytes,
                        _stream_handle(stream), ctypes.byref(out)))
    nv = ctypes.c_int()
    _check(lib.lbm_vset_query(vs.handle, ctypes.byref(nv), None, None, None, None))
    return Sim(out.value, prob, nv.value, keepalive=(device_buf, stream, vs))


def lbm_destroy(sim: Sim):
    sim.close()


def lbm_coeffs(sim: Sim):
    dt, om, ur = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_load().lbm_coeffs(sim.handle, ctypes.byref(dt), ctypes.byref(om), ctypes.byref(ur)))
    return {"dt": dt.value, "omega": om.value, "u_ref": ur.value}


def lbm_step(sim: Sim, nsteps: int):
    _check(_load().lbm_step(sim.handle, int(nsteps)))


def lbm_solve(sim: Sim, tol: float, max_steps: int, refine_sweeps: int = 0, refine_tol: float = 0.0) -> dict:
    info = lbm_solve_info()
    _check(_load().lbm_solve(sim.handle, float(tol), int(max_steps), int(refine_sweeps), float(refine_tol),
                             ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in lbm_solve_info._fields_}


def lbm_set_variant(sim: Sim, warps_per_segment: int, prefetch: int = 0):
    """Step kernel: warps per 32-cell segment and load path (0 registers, 1 prefetch, 2/3 TMA
    segments, 4 to 7 the column march, 8 the column march on the strip-tiled state; the C
    header lists which combinations exist)."""
    _check(_load().lbm_set_variant(sim.handle, int(warps_per_segment), int(prefetch)))


LBM_SPLIT_LIE, LBM_SPLIT_STRANG, LBM_SPLIT_STRANG_EXACT = 0, 1, 2


def lbm_set_transport(sim: Sim, order: int):
    _check(_load().lbm_set_transport(sim.handle, int(order)))


def lbm_get_transport(sim: Sim) -> int:
    v = ctypes.c_int()
    _check(_load().lbm_get_transport(sim.handle, ctypes.byref(v)))
    return v.value


def lbm_set_splitting(sim: Sim, scheme: int):
    _check(_load().lbm_set_splitting(sim.handle, int(scheme)))


def lbm_get_splitting(sim: Sim) -> int:
    v = ctypes.c_int()
    _check(_load().lbm_get_splitting(sim.handle, ctypes.byref(v)))
    return v.value


def lbm_get_variant(sim: Sim):
    g, pf = ctypes.c_int(), ctypes.c_int()
    _check(_load().lbm_get_variant(sim.handle, ctypes.byref(g), ctypes.byref(pf)))
    return g.value, pf.value


def lbm_residual(sim: Sim):
    r, s = ctypes.c_double(), ctypes.c_long()
    _check(_load().lbm_residual(sim.handle, ctypes.byref(r), ctypes.byref(s)))
    return r.value, s.value


MOMENT_NAMES = ("rho", "ux", "uy", "pxx", "pxy", "pyy")


def lbm_moments(sim: Sim, wall_shear: bool = True, which=MOMENT_NAMES):
    """The moments named in `which` (the others are not requested: NULL outputs)."""
    n = sim.ncells
    outs = {k: np.empty(n) for k in MOMENT_NAMES if k in which}
    ws = np.empty(4) if wall_shear else None
    _check(_load().lbm_moments(sim.handle, *[_ptr(outs.get(k)) for k in MOMENT_NAMES], _ptr(ws)))
    res = {k: v.reshape(sim.prob.ny, sim.prob.nx) for k, v in outs.items()}
    if ws is not None:
        res["wall_shear"] = ws
    return res


def lbm_face_flux(sim: Sim):
    nx, ny = sim.prob.nx, sim.prob.ny
    fy = np.empty((ny + 1) * nx)
    fx = np.empty(ny * (nx + 1)) if sim.prob.geom == LBM_CAVITY else None
    _check(_load().lbm_face_flux(sim.handle, _ptr(fy), _ptr(fx)))
    return fy.reshape(ny + 1, nx), (None if fx is None else fx.reshape(ny, nx + 1))


def lbm_set_moments(sim: Sim, moments) -> None:
    """moments: dict with rho, ux, uy, pxx, pxy, pyy ([ny][nx] each) or an array [6][ny][nx]."""
    if isinstance(moments, dict):
        moments = np.stack([np.asarray(moments[k], dtype=np.float64).reshape(-1)
                            for k in ("rho", "ux", "uy", "pxx", "pxy", "pyy")])
    m = np.ascontiguousarray(np.asarray(moments, dtype=np.float64).reshape(6, sim.ncells))
    _check(_load().lbm_set_moments(sim.handle, _ptr(m)))


def lbm_get_state(sim: Sim) -> np.ndarray:
    h = np.empty((sim.n_vel, sim.ncells))
    _check(_load().lbm_get_state(sim.handle, _ptr(h)))
    return h


def lbm_set_state(sim: Sim, h: np.ndarray):
    h = np.ascontiguousarray(h, dtype=np.float64)
    assert h.size == sim.n_vel * sim.ncells
    _check(_load().lbm_set_state(sim.handle, _ptr(h)))


def lbm_get_state_f32(sim: Sim) -> np.ndarray:
    h = np.empty((sim.n_vel, sim.ncells), dtype=np.float32)
    _check(_load().lbm_get_state_f32(sim.handle, h.ctypes.data_as(_fp)))
    return h


def lbm_set_state_f32(sim: Sim, h: np.ndarray):
    h = np.ascontiguousarray(h, dtype=np.float32)
    assert h.size == sim.n_vel * sim.ncells
    _check(_load().lbm_set_state_f32(sim.handle, h.ctypes.data_as(_fp)))


def lbm_state_device(sim: Sim):
    p, s = _vp(), ctypes.c_long()
    _check(_load().lbm_state_device(sim.handle, ctypes.byref(p), ctypes.byref(s)))
    return p.value, s.value


def lbm_state_layout(sim: Sim):
    """(plane_pitch, row_pitch) of the device state: element a * plane_pitch + y * row_pitch + x."""
    pa, py = ctypes.c_long(), ctypes.c_long()
    _check(_load().lbm_state_layout(sim.handle, ctypes.byref(pa), ctypes.byref(py)))
    return pa.value, py.value


def lbm_state_tiling(sim: Sim):
    """(tile_width, x_shift, tile_pitch, row_pitch) of a strip-tiled device state (load path 8):
    element (a, x, y) at ((x + x_shift) // tile_width) * tile_pitch + y * row_pitch
    + a * tile_width + (x + x_shift) % tile_width; all zero for a planar state."""
    w, sh, tp, rp = ctypes.c_int(), ctypes.c_int(), ctypes.c_long(), ctypes.c_long()
    _check(_load().lbm_state_tiling(sim.handle, ctypes.byref(w), ctypes.byref(sh), ctypes.byref(tp), ctypes.byref(rp)))
    return w.value, sh.value, tp.value, rp.value


def lbm_norms_scratch_bytes(count: int) -> int:
    b = ctypes.c_size_t()
    _check(_load().lbm_norms_scratch_bytes(int(count), ctypes.byref(b)))
    return b.value


def lbm_norms(a_ptr: int, b_ptr: int | None, count: int, prec: int, scratch_ptr: int,
              scratch_bytes: int, out_ptr: int, stream=None):
    _check(_load().lbm_norms(a_ptr, b_ptr, int(count), prec, scratch_ptr, scratch_bytes, out_ptr,
                             _stream_handle(stream)))


def lbm_probe_fp64_rate(iters: int = 200_000, stream=None) -> float:
    """FP64 fused multiply-adds per second of this GPU (a timed throughput kernel)."""
    r = ctypes.c_double()
    _check(_load().lbm_probe_fp64_rate(int(iters), ctypes.byref(r), _stream_handle(stream)))
    return r.value


def lbm_norms_noalloc(a_ptr: int, b_ptr: int | None, count: int, prec: int, out_ptr: int, stream=None):
    """Squared norms with the library's static scratch (no allocation, count <= 2**26)."""
    _check(_load().lbm_norms_noalloc(a_ptr, b_ptr, int(count), prec, out_ptr, _stream_handle(stream)))


class Batch:
    """Owner of an lbm_batch* and of its device buffer (if any)."""

    def __init__(self, handle: int, probs, n_vel: int, keepalive=None):
        self.handle = handle
        self.probs = probs
        self.n_vel = n_vel
        self._keepalive = keepalive

    def close(self):
        if self.handle and _lib is not None:
            _lib.lbm_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        self.close()


def _problem_array(probs):
    arr = (lbm_problem * len(probs))()
    for i, p in enumerate(probs):
        arr[i] = p
    return arr


def lbm_batch_bytes(vs: VelocitySet, probs) -> int:
    b = ctypes.c_size_t()
    arr = _problem_array(probs)
    _check(_load().lbm_batch_bytes(vs.handle, arr, len(probs), ctypes.byref(b)))
    return b.value


def lbm_batch_init(vs: VelocitySet, probs, device_buf=None, stream=None) -> Batch:
    lib = _load()
    arr = _problem_array(probs)
    out = _vp()
    buf_ptr, buf_bytes = None, 0
    if device_buf is not None:
        buf_ptr = device_buf.data_ptr()
        buf_bytes = device_buf.numel() * device_buf.element_size()
    _check(lib.lbm_batch_init(vs.handle, arr, len(probs), buf_ptr, buf_bytes, _stream_handle(stream),
                              ctypes.byref(out)))
    nv = ctypes.c_int()
    _check(lib.lbm_vset_query(vs.handle, ctypes.byref(nv), None, None, None, None))
    return Batch(out.value, list(probs), nv.value, keepalive=(device_buf, stream, vs))


def lbm_batch_set_schedule(b: Batch, warps_per_segment: int, blocks_per_sm: int, order: int):
    _check(_load().lbm_batch_set_schedule(b.handle, warps_per_segment, blocks_per_sm, order))


def lbm_batch_get_schedule(b: Batch):
    g, bp, o, gr = (ctypes.c_int() for _ in range(4))
    _check(_load().lbm_batch_get_schedule(b.handle, ctypes.byref(g), ctypes.byref(bp), ctypes.byref(o),
                                          ctypes.byref(gr)))
    return {"warps_per_segment": g.value, "blocks_per_sm": bp.value, "order": o.value, "grid": gr.value}


def lbm_batch_set_march(b: Batch, on: bool, rows_per_chunk: int = 0, warps_per_item: int = 0):
    _check(_load().lbm_batch_set_march(b.handle, int(bool(on)), int(rows_per_chunk), int(warps_per_item)))


def lbm_batch_get_march(b: Batch) -> dict:
    on, ch, it, gr, wg = (ctypes.c_int() for _ in range(5))
    _check(_load().lbm_batch_get_march(b.handle, ctypes.byref(on), ctypes.byref(ch), ctypes.byref(it),
                                       ctypes.byref(gr), ctypes.byref(wg)))
    return {"on": bool(on.value), "rows_per_chunk": ch.value, "items": it.value, "grid": gr.value,
            "warps_per_item": wg.value}


def lbm_batch_advance(b: Batch, nsteps: int, tol: float):
    _check(_load().lbm_batch_advance(b.handle, int(nsteps), float(tol)))


def lbm_batch_set_timeout(b: Batch, cycles: int):
    _check(_load().lbm_batch_set_timeout(b.handle, int(cycles)))


def lbm_batch_poll(b: Batch):
    n, s = ctypes.c_int(), ctypes.c_long()
    _check(_load().lbm_batch_poll(b.handle, ctypes.byref(n), ctypes.byref(s)))
    return n.value, s.value


def lbm_batch_status(b: Batch, i: int):
    """Steps, last residual, converged (frozen below the tolerance) and stalled (frozen by the
    stagnation rule above it) of instance i."""
    st, r, cv, sl = ctypes.c_long(), ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    _check(_load().lbm_batch_status(b.handle, int(i), ctypes.byref(st), ctypes.byref(r), ctypes.byref(cv)))
    _check(_load().lbm_batch_stalled(b.handle, int(i), ctypes.byref(sl)))
    return {"steps": st.value, "residual": r.value, "converged": bool(cv.value), "stalled": bool(sl.value)}


def lbm_batch_get_state(b: Batch, i: int) -> np.ndarray:
    p = b.probs[i]
    h = np.empty((b.n_vel, p.nx * p.ny))
    _check(_load().lbm_batch_get_state(b.handle, int(i), _ptr(h)))
    return h


def lbm_batch_moments(b: Batch, i: int, out_ptr: int):
    _check(_load().lbm_batch_moments(b.handle, int(i), out_ptr))


class BatchRefineInfo(ctypes.Structure):
    _fields_ = [("correction_steps", ctypes.c_long), ("sweeps", ctypes.c_int), ("defect", ctypes.c_double)]


def lbm_batch_refine(b: Batch, tol: float, max_sweeps: int = 3, refine_tol: float = 0.0,
                     max_steps: int = 1_000_000) -> list:
    """Batched mixed-precision refinement of every instance; one dict per instance."""
    info = (BatchRefineInfo * len(b.probs))()
    _check(_load().lbm_batch_refine(b.handle, float(tol), int(max_sweeps), float(refine_tol), int(max_steps),
                                    ctypes.cast(info, ctypes.c_void_p)))
    return [{"correction_steps": r.correction_steps, "sweeps": r.sweeps, "defect": r.defect} for r in info]


def lbm_batch_set_state(b: Batch, i: int, h: np.ndarray):
    h = np.ascontiguousarray(h, dtype=np.float64)
    _check(_load().lbm_batch_set_state(b.handle, int(i), _ptr(h)))


def lbm_batch_warm_start(b: Batch, i: int, m, kn: float, u_w: float):
    _check(_load().lbm_batch_warm_start(b.handle, int(i), m.handle, float(kn), float(u_w)))


def lbm_batch_reset(b: Batch):
    _check(_load().lbm_batch_reset(b.handle))


def lbm_batch_tune(b: Batch, steps_per_trial: int = 20) -> dict:
    g, bp, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    _check(_load().lbm_batch_tune(b.handle, int(steps_per_trial), ctypes.byref(g), ctypes.byref(bp),
                                  ctypes.byref(o), ctypes.byref(ms)))
    return {"warps_per_segment": g.value, "blocks_per_sm": bp.value, "order": o.value, "ms_per_step": ms.value}


class MLP:
    """Owner of an lbm_mlp* (the warm-start network)."""

    def __init__(self, handle: int, keepalive=None):
        self.handle = handle
        self._keepalive = keepalive

    def close(self):
        if self.handle and _lib is not None:
            _lib.lbm_mlp_destroy(self.handle)
        self.handle = None

    def __del__(self):
        self.close()


def _fptr(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def lbm_mlp_param_count() -> int:
    n = ctypes.c_long()
    _check(_load().lbm_mlp_param_count(ctypes.byref(n)))
    return n.value


def lbm_mlp_create(max_batch: int, seed: int = 0, stream=None) -> MLP:
    out = _vp()
    _check(_load().lbm_mlp_create(int(max_batch), int(seed), _stream_handle(stream), ctypes.byref(out)))
    return MLP(out.value, keepalive=stream)


def lbm_mlp_set_params(m: MLP, flat: np.ndarray):
    flat = np.ascontiguousarray(flat, dtype=np.float32)
    assert flat.size == lbm_mlp_param_count()
    _check(_load().lbm_mlp_set_params(m.handle, _fptr(flat)))


def lbm_mlp_get_params(m: MLP) -> np.ndarray:
    flat = np.empty(lbm_mlp_param_count(), dtype=np.float32)
    _check(_load().lbm_mlp_get_params(m.handle, _fptr(flat)))
    return flat


def lbm_mlp_forward(m: MLP, x_ptr: int, rows: int, y_ptr: int):
    _check(_load().lbm_mlp_forward(m.handle, x_ptr, int(rows), y_ptr))


def lbm_mlp_loss_grad(m: MLP, x_ptr: int, t_ptr: int, rows: int, want_grad: bool = True):
    loss = ctypes.c_double()
    g = np.empty(lbm_mlp_param_count(), dtype=np.float32) if want_grad else None
    _check(_load().lbm_mlp_loss_grad(m.handle, x_ptr, t_ptr, int(rows), ctypes.byref(loss),
                                     _fptr(g) if g is not None else None))
    return loss.value, g


def lbm_mlp_train_step(m: MLP, x_ptr: int, t_ptr: int, rows: int, lr: float, want_loss: bool = False):
    loss = ctypes.c_double()
    _check(_load().lbm_mlp_train_step(m.handle, x_ptr, t_ptr, int(rows), float(lr),
                                      ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def lbm_mlp_features(m: MLP, nx: int, ny: int, kn: float, u_w: float, x_ptr: int):
    _check(_load().lbm_mlp_features(m.handle, int(nx), int(ny), float(kn), float(u_w), x_ptr))


def lbm_warm_start(sim: Sim, m: MLP, kn: float, u_w: float):
    _check(_load().lbm_warm_start(sim.handle, m.handle, float(kn), float(u_w)))


def mlp_unflatten(flat: np.ndarray, widths=(4, 256, 256, 256, 6)):
    """Split a flat parameter vector into [(W, b), ...] (float64 copies)."""
    out, o = [], 0
    for i in range(len(widths) - 1):
        nw = widths[i + 1] * widths[i]
        W = np.asarray(flat[o:o + nw], dtype=np.float64).reshape(widths[i + 1], widths[i])
        o += nw
        b = np.asarray(flat[o:o + widths[i + 1]], dtype=np.float64)
        o += widths[i + 1]
        out.append((W, b))
    return out


def mlp_flatten(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)


class Hybrid:
    """Owner of an lbm_hybrid* (hybrid half-range / full-range Couette column or cavity)."""

    def __init__(self, handle: int, nx: int, ny: int, keepalive=None):
        self.handle = handle
        self.nx, self.ny = nx, ny
        self._keepalive = keepalive

    def close(self):
        if self.handle and _lib is not None:
            _lib.lbm_hybrid_destroy(self.handle)
        self.handle = None

    def __del__(self):
        self.close()


def lbm_hybrid_init(geom: int, n_half: int, nx: int, ny: int, kn: float, u_bottom: float, u_top: float,
                    layer: int, cfl: float = 0.9, stream=None) -> Hybrid:
    out = _vp()
    _check(_load().lbm_hybrid_init(int(geom), int(n_half), int(nx), int(ny), float(kn), float(u_bottom),
                                   float(u_top), int(layer), float(cfl), _stream_handle(stream), ctypes.byref(out)))
    return Hybrid(out.value, nx, ny, keepalive=stream)


def lbm_hybrid_query(hb: Hybrid) -> dict:
    n, c, dt = ctypes.c_long(), ctypes.c_int(), ctypes.c_double()
    _check(_load().lbm_hybrid_query(hb.handle, ctypes.byref(n), ctypes.byref(c), ctypes.byref(dt)))
    return {"unknowns": n.value, "half_range_cells": c.value, "dt": dt.value}


def lbm_hybrid_set_state(hb: Hybrid, h: np.ndarray):
    h = np.ascontiguousarray(h, dtype=np.float64)
    if h.size != lbm_hybrid_query(hb)["unknowns"]:
        raise ValueError("state size does not match the hybrid grid")
    _check(_load().lbm_hybrid_set_state(hb.handle, _ptr(h)))


def lbm_hybrid_get_state(hb: Hybrid) -> np.ndarray:
    h = np.empty(lbm_hybrid_query(hb)["unknowns"])
    _check(_load().lbm_hybrid_get_state(hb.handle, _ptr(h)))
    return h


def lbm_hybrid_step(hb: Hybrid, nsteps: int):
    _check(_load().lbm_hybrid_step(hb.handle, int(nsteps)))


def lbm_hybrid_residual(hb: Hybrid) -> float:
    r = ctypes.c_double()
    _check(_load().lbm_hybrid_residual(hb.handle, ctypes.byref(r)))
    return r.value


def lbm_hybrid_solve(hb: Hybrid, tol: float, max_steps: int, every: int = 100) -> dict:
    s, r = ctypes.c_long(), ctypes.c_double()
    _check(_load().lbm_hybrid_solve(hb.handle, float(tol), int(max_steps), int(every), ctypes.byref(s),
                                    ctypes.byref(r)))
    return {"steps": s.value, "residual": r.value}


def lbm_hybrid_set_precision(hb: Hybrid, prec: int):
    _check(_load().lbm_hybrid_set_precision(hb.handle, int(prec)))


def lbm_hybrid_refine(hb: Hybrid, tol: float, max_sweeps: int = 3, refine_tol: float = 0.0,
                      max_steps: int = 2_000_000, every: int = 100) -> dict:
    k, d = ctypes.c_long(), ctypes.c_double()
    _check(_load().lbm_hybrid_refine(hb.handle, float(tol), int(max_sweeps), float(refine_tol), int(max_steps),
                                     int(every), ctypes.byref(k), ctypes.byref(d)))
    return {"correction_steps": k.value, "defect": d.value}


def lbm_hybrid_velocity(hb: Hybrid):
    """(u_x, u_y) per cell, each [ny][nx]."""
    ux, uy = np.empty(hb.nx * hb.ny), np.empty(hb.nx * hb.ny)
    _check(_load().lbm_hybrid_velocity(hb.handle, _ptr(ux), _ptr(uy)))
    return ux.reshape(hb.ny, hb.nx), uy.reshape(hb.ny, hb.nx)


def lbm_hybrid_face_flux(hb: Hybrid) -> np.ndarray:
    """Couette column: x-momentum flux through the ny + 1 faces."""
    pxy = np.empty(hb.ny + 1)
    _check(_load().lbm_hybrid_face_flux(hb.handle, _ptr(pxy)))
    return pxy
