"""Thin ctypes binding of libfdu (include/fdu.h).

Argument marshalling only: every step of the residual and the RK stage runs
in the library's CUDA kernels.  Device buffers are torch CUDA tensors
(passed by data_ptr()); host buffers are numpy arrays.  The library is
loaded lazily and a missing or unbuildable library raises: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

FDU_OK = 0
FDU_BC_PERIODIC = 0
FDU_BC_TRANSMISSIVE = 1
ERRORS = {
    -1: "FDU_ERR_ARG", -2: "FDU_ERR_MESH", -3: "FDU_ERR_STENCIL", -4: "FDU_ERR_RANK_DEFICIENT",
    -5: "FDU_ERR_CUDA", -6: "FDU_ERR_TIMEOUT", -7: "FDU_ERR_NONPHYSICAL", -8: "FDU_ERR_NODEVICE",
}

# Every symbol include/fdu.h declares (checked by the CPU tests).
EXPORTS = (
    "fdu_version", "fdu_last_error", "fdu_default_opts", "fdu_mesh_create", "fdu_mesh_destroy",
    "fdu_mesh_info_get", "fdu_get_edges", "fdu_get_edge_stencils", "fdu_get_div_sizes", "fdu_get_div_stencils",
    "fdu_set_state", "fdu_get_state", "fdu_residual", "fdu_max_dt", "fdu_rk_step", "fdu_rk_steps",
    "fdu_fallback_count", "fdu_profile", "fdu_profile_read", "fdu_probe_fma", "fdu_residual_noalloc",
    "fdu_check_recip64", "fdu_check_rsqrt64", "fdu_check_scale2", "fdu_check_weno_coef32", "fdu_check_dw", "fdu_set_adjoint_precision", "fdu_mesh_create_cells", "fdu_advance", "fdu_limited_count", "fdu_batch_create", "fdu_batch_info",
    "fdu_batch_max_dt", "fdu_batch_set_dt", "fdu_batch_rk_steps", "fdu_batch_set_launch", "fdu_batch_autotune",
    "fdu_batch_barrier_selftest", "fdu_residual_vjp", "fdu_rk_step_vjp", "fdu_adjoint_rk",
)


class FduError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{ERRORS.get(status, status)}: {msg}")
        self.status = status


class MeshOpts(C.Structure):
    _fields_ = [
        ("Lx", C.c_double), ("Ly", C.c_double), ("weno_eps", C.c_double), ("weno_eps32", C.c_double),
        ("gamma", C.c_double), ("lsq_degree", C.c_int), ("lsq_levels", C.c_int), ("bc", C.c_int),
        ("renumber", C.c_int), ("device", C.c_int), ("host_threads", C.c_int),
        ("ghost_donor", C.POINTER(C.c_int32)), ("positivity_alpha", C.c_double), ("f32_coef", C.c_int),
    ]


class MeshInfo(C.Structure):
    _fields_ = [
        ("nv", C.c_int64), ("ne", C.c_int64), ("nt", C.c_int64), ("n_real", C.c_int64),
        ("div_vert_nnz", C.c_int64), ("div_edge_nnz", C.c_int64),
        ("J_min", C.c_int32), ("J_max", C.c_int32), ("K_min", C.c_int32), ("K_max", C.c_int32),
        ("device_bytes", C.c_int64), ("table_bytes_f64", C.c_int64), ("table_bytes_f32", C.c_int64),
        ("sell_width", C.c_int32), ("pad0", C.c_int32),
        ("sell_vert_nnz", C.c_int64), ("sell_edge_nnz", C.c_int64),
        ("sell_vert_nnz64", C.c_int64), ("sell_edge_nnz64", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad0"}


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libfdu.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        lp = C.POINTER(C.c_int64)
        i64 = C.c_int64
        L.fdu_version.restype = C.c_char_p
        L.fdu_last_error.restype = C.c_char_p
        L.fdu_default_opts.argtypes = [C.POINTER(MeshOpts)]
        L.fdu_mesh_create.argtypes = [dp, i64, ip, i64, C.POINTER(MeshOpts), C.POINTER(P)]
        L.fdu_mesh_destroy.argtypes = [P]
        L.fdu_mesh_info_get.argtypes = [P, C.POINTER(MeshInfo)]
        L.fdu_get_edges.argtypes = [P, ip]
        L.fdu_get_edge_stencils.argtypes = [P, ip, dp]
        L.fdu_get_div_sizes.argtypes = [P, lp, lp]
        L.fdu_get_div_stencils.argtypes = [P, lp, ip, dp, dp, lp, ip, dp]
        L.fdu_set_state.argtypes = [P, P, C.c_int, P]
        L.fdu_get_state.argtypes = [P, P, C.c_int, P]
        L.fdu_residual.argtypes = [P, C.c_int, P, C.c_int, P]
        L.fdu_max_dt.argtypes = [P, C.c_double, dp, P]
        L.fdu_rk_step.argtypes = [P, C.c_double, C.c_int, P]
        L.fdu_rk_steps.argtypes = [P, C.c_double, C.c_int, C.c_int, P]
        L.fdu_fallback_count.argtypes = [P, lp, C.c_int, P]
        L.fdu_profile.argtypes = [P, C.c_int]
        L.fdu_probe_fma.argtypes = [C.c_int, C.c_int, dp]
        L.fdu_residual_noalloc.argtypes = [P, P, P, P]
        L.fdu_check_recip64.argtypes = [C.c_int, dp, dp, i64]
        L.fdu_check_rsqrt64.argtypes = [C.c_int, dp, dp, i64]
        L.fdu_check_weno_coef32.argtypes = [C.c_int, dp, dp, i64]
        L.fdu_check_scale2.argtypes = [C.c_int, dp, dp, i64, C.c_int]
        L.fdu_check_dw.argtypes = [C.c_int, C.c_int, dp, dp, dp, i64]
        L.fdu_set_adjoint_precision.argtypes = [C.c_void_p, C.c_int]
        L.fdu_mesh_create_cells.argtypes = [dp, i64, lp, ip, i64, C.c_int, C.POINTER(MeshOpts), C.POINTER(P)]
        L.fdu_advance.argtypes = [P, C.c_double, C.c_double, C.c_int, i64, lp, dp, P]
        L.fdu_limited_count.argtypes = [P, lp, C.c_int, P]
        L.fdu_batch_create.argtypes = [C.c_int32, C.POINTER(dp), lp, C.POINTER(ip), lp, C.POINTER(MeshOpts),
                                       C.POINTER(P)]
        L.fdu_batch_info.argtypes = [P, C.POINTER(C.c_int32), lp]
        L.fdu_batch_max_dt.argtypes = [P, C.c_double, dp, P]
        L.fdu_batch_set_dt.argtypes = [P, dp, P]
        L.fdu_batch_rk_steps.argtypes = [P, C.c_int, C.c_int, P]
        L.fdu_batch_set_launch.argtypes = [P, C.c_int, C.c_int]
        L.fdu_batch_autotune.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
        L.fdu_batch_barrier_selftest.argtypes = [P, C.POINTER(C.c_int)]
        L.fdu_residual_vjp.argtypes = [P, P, P, C.c_int, P]
        L.fdu_rk_step_vjp.argtypes = [P, C.c_double, P, P, C.c_int, P]
        L.fdu_adjoint_rk.argtypes = [P, C.c_double, C.c_int, C.c_int, P, P, C.c_int, P]
        L.fdu_profile_read.argtypes = [P, C.c_int, C.c_int, dp, lp, C.c_int]
        for name in EXPORTS:
            if name not in ("fdu_version", "fdu_last_error"):
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def _check(st):
    if st != FDU_OK:
        raise FduError(st, load().fdu_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _lp(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def default_opts(**kw) -> MeshOpts:
    o = MeshOpts()
    _check(load().fdu_default_opts(C.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _buffer(x, rows, cols=4, writable=False):
    """(pointer, on_device) of a torch CUDA tensor or a numpy array of [rows][cols] float64."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous() or tuple(x.shape) != (rows, cols):
            raise ValueError(f"expected a contiguous float64 tensor of shape ({rows}, {cols})")
        if not x.is_cuda:
            if writable:
                raise ValueError("output tensors must be CUDA tensors or numpy arrays")
            return C.c_void_p(x.data_ptr()), 0
        return C.c_void_p(x.data_ptr()), 1
    a = np.asarray(x)
    if a.dtype != np.float64 or not a.flags.c_contiguous or a.shape != (rows, cols):
        raise ValueError(f"expected a C-contiguous float64 array of shape ({rows}, {cols})")
    if writable and not a.flags.writeable:
        raise ValueError("output array is read-only")
    return C.c_void_p(a.ctypes.data), 0


def probe_fma(device=0, precision=64) -> float:
    """FMA throughput of the device in TFLOP/s (measurement helper)."""
    t = C.c_double()
    _check(load().fdu_probe_fma(int(device), int(precision), C.byref(t)))
    return t.value


def check_recip64(x, device=0):
    """The kernels' FP64 reciprocal of x (accuracy check)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    _check(load().fdu_check_recip64(int(device), _dp(x), _dp(y), x.size))
    return y


def check_scale2(x, up, device=0):
    """The kernels' exact scaling of x by 2 (up) or 1/2 on the integer pipe
    (accuracy check)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    _check(load().fdu_check_scale2(int(device), _dp(x), _dp(y), x.size, 1 if up else 0))
    return y


def check_weno_coef32(xi, device=0):
    """The FP32 edge kernel's NU-WENO5 coefficient block [n, 24] formed from
    stencil coordinates xi [n, 6] (accuracy check)."""
    xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, 6)
    k = np.zeros((xi.shape[0], 24))
    _check(load().fdu_check_weno_coef32(int(device), _dp(xi), _dp(k), xi.shape[0]))
    return k


DW_OPS = {"split": 0, "add": 1, "add_sloppy": 2, "mul": 3, "mul_unnormalised": 4, "recip": 5, "rsqrt": 6,
          "dot8": 7}


def check_dw(op, x, y=None, device=0):
    """A double-word primitive of precision 48 applied to x (and y), the
    result returned exactly as doubles (accuracy check)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x) if y is None else np.ascontiguousarray(y, dtype=np.float64)
    k = DW_OPS[op]
    z = np.zeros(x.size // 8 if k == 7 else x.size)
    _check(load().fdu_check_dw(int(device), k, _dp(x), _dp(y), _dp(z), x.size))
    return z


def check_rsqrt64(x, device=0):
    """The kernels' FP64 reciprocal square root of x (accuracy check)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    _check(load().fdu_check_rsqrt64(int(device), _dp(x), _dp(y), x.size))
    return y


class Mesh:
    """A mesh with its stencils, weights and device state (one fdu_mesh)."""

    def __init__(self, xy, tri, Lx=0.0, Ly=0.0, *, lsq_degree=2, lsq_levels=2, device=0, renumber=1,
                 ghost_donor=None, weno_eps=1e-40, weno_eps32=1e-30, gamma=1.4, host_threads=0,
                 positivity_alpha=0.0, artificial_edges=None, f32_coef=0):
        """`tri` is an (nt, 3) array of triangles, or a pair (cell_off,
        cell_vtx) of a hybrid triangle / quadrilateral mesh in CSR form; then
        `artificial_edges` (0, 1 or 2, default 1) selects the artificial
        edges of fdu_mesh_create_cells.  `f32_coef` selects the FP32 path's
        NU-WENO5 coefficients: 0 the FP64-built block streamed in FP32, 1
        formed in the FP32 edge kernel from the stencil gaps."""
        L = load()
        self._h = None
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        cells = None
        if isinstance(tri, tuple):
            cells = (np.ascontiguousarray(tri[0], dtype=np.int64), np.ascontiguousarray(tri[1], dtype=np.int32))
        else:
            tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
            if artificial_edges is not None:
                raise ValueError("artificial_edges needs a (cell_off, cell_vtx) cell list")
        self._ghost = None
        bc = FDU_BC_PERIODIC
        gp = None
        if ghost_donor is not None:
            self._ghost = np.ascontiguousarray(ghost_donor, dtype=np.int32).reshape(xy.shape[0])
            gp = _ip(self._ghost)
            bc = FDU_BC_TRANSMISSIVE
        o = default_opts(Lx=float(Lx), Ly=float(Ly), lsq_degree=lsq_degree, lsq_levels=lsq_levels, device=device,
                         renumber=renumber, weno_eps=weno_eps, weno_eps32=weno_eps32, gamma=gamma, bc=bc,
                         host_threads=host_threads, positivity_alpha=float(positivity_alpha), f32_coef=int(f32_coef))
        if gp is not None:
            o.ghost_donor = gp
        h = C.c_void_p()
        if cells is not None:
            off, vtx = cells
            art = 1 if artificial_edges is None else int(artificial_edges)
            _check(L.fdu_mesh_create_cells(_dp(xy), xy.shape[0], _lp(off), _ip(vtx), off.shape[0] - 1, art, C.byref(o),
                                           C.byref(h)))
        else:
            _check(L.fdu_mesh_create(_dp(xy), xy.shape[0], _ip(tri), tri.shape[0], C.byref(o), C.byref(h)))
        self._h = h
        self.device = device
        info = self.info()
        self.nv = int(info["nv"])
        self.ne = int(info["ne"])

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().fdu_mesh_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------- host queries
    def info(self) -> dict:
        i = MeshInfo()
        _check(load().fdu_mesh_info_get(self._h, C.byref(i)))
        return i.as_dict()

    def edges(self):
        e = np.zeros((self.ne, 2), np.int32)
        _check(load().fdu_get_edges(self._h, _ip(e)))
        return e

    def edge_stencils(self):
        s = np.zeros((self.ne, 6), np.int32)
        xi = np.zeros((self.ne, 6))
        _check(load().fdu_get_edge_stencils(self._h, _ip(s), _dp(xi)))
        return s, xi

    def div_stencils(self):
        vn, en = C.c_int64(), C.c_int64()
        _check(load().fdu_get_div_sizes(self._h, C.byref(vn), C.byref(en)))
        voff = np.zeros(self.nv + 1, np.int64)
        eoff = np.zeros(self.nv + 1, np.int64)
        vid = np.zeros(vn.value, np.int32)
        eid = np.zeros(en.value, np.int32)
        wf = np.zeros(vn.value)
        wg = np.zeros(vn.value)
        we = np.zeros(en.value)
        _check(load().fdu_get_div_stencils(self._h, _lp(voff), _ip(vid), _dp(wf), _dp(wg), _lp(eoff), _ip(eid),
                                           _dp(we)))
        return voff, vid, wf, wg, eoff, eid, we

    # ---------------------------------------------------------- device calls
    def set_state(self, w, stream=None):
        p, dev = _buffer(w, self.nv)
        _check(load().fdu_set_state(self._h, p, dev, _stream_ptr(stream)))

    def get_state(self, out=None, stream=None):
        if out is None:
            out = np.zeros((self.nv, 4))
        p, dev = _buffer(out, self.nv, writable=True)
        _check(load().fdu_get_state(self._h, p, dev, _stream_ptr(stream)))
        return out

    def residual(self, precision=64, out=None, stream=None):
        """dw/dt of the current state, [nv, 4] in the caller's vertex order
        (edge fluxes by characteristic NU-WENO5 and a Roe flux, Section 2.3.1;
        least-squares divergence, Section 2.2.1).  precision 64: FP64;
        48: the FP64 result with the edge-flux increments in double-word FP32;
        32: FP32 fluxes with FP64 accumulation.  out: a host array or a CUDA
        tensor of that shape (None: a new host array)."""
        if out is None:
            out = np.zeros((self.nv, 4))
        p, dev = _buffer(out, self.nv, writable=True)
        _check(load().fdu_residual(self._h, int(precision), p, dev, _stream_ptr(stream)))
        return out

    def max_dt(self, cfl, stream=None) -> float:
        """CFL time step of the current state: cfl * min over real vertices of
        h_v / (|q_v| + c_v), h_v the shortest edge at v."""
        dt = C.c_double()
        _check(load().fdu_max_dt(self._h, float(cfl), C.byref(dt), _stream_ptr(stream)))
        return dt.value

    def rk_step(self, dt, precision=64, stream=None):
        """One SSP-RK3 step (three stages, Shu-Osher form) of size dt;
        precision as for residual."""
        _check(load().fdu_rk_step(self._h, float(dt), int(precision), _stream_ptr(stream)))

    def rk_steps(self, dt, n_steps, precision=64, stream=None):
        """n_steps SSP-RK3 steps of size dt, replayed from a captured CUDA graph."""
        _check(load().fdu_rk_steps(self._h, float(dt), int(precision), int(n_steps), _stream_ptr(stream)))

    def fallback_count(self, reset=False, stream=None) -> int:
        c = C.c_int64()
        _check(load().fdu_fallback_count(self._h, C.byref(c), 1 if reset else 0, _stream_ptr(stream)))
        return c.value

    def profile(self, enable=True):
        """Record CUDA events around each edge-flux and divergence launch."""
        _check(load().fdu_profile(self._h, 1 if enable else 0))

    def profile_read(self, kernel, precision=64, reset=True):
        """(total device ms, launches) of kernel 'edge' or 'div' since the last reset."""
        k = {"edge": 0, "div": 1}[kernel]
        ms = C.c_double()
        n = C.c_int64()
        _check(load().fdu_profile_read(self._h, k, int(precision), C.byref(ms), C.byref(n), 1 if reset else 0))
        return ms.value, n.value

    def residual_noalloc(self, w, out, stream=None):
        """FP64 residual of the device state `w` into the device tensor `out`
        (both [nv][4] float64, original vertex order) using the library's fixed
        scratch array: no device memory is allocated by this call.  With
        stream=None the call goes to torch's current stream (a null handle,
        torch's default stream, is the legacy default stream in the library),
        so calls made one after the other from one thread are ordered, for
        any mesh.  Every call shares the one scratch array: calls on different
        streams, or from different threads, that overlap on the GPU race on it
        and must be serialised by the caller."""
        pw, dw = _buffer(w, self.nv)
        po, do = _buffer(out, self.nv, writable=True)
        if not (dw and do):
            raise ValueError("residual_noalloc takes CUDA tensors")
        _check(load().fdu_residual_noalloc(self._h, pw, po, _stream_ptr(stream)))
        return out

    def advance(self, cfl, t_end, precision=64, max_steps=10**9, stream=None):
        """SSP-RK3 steps with the device-computed CFL time step until t_end;
        returns (steps taken, time reached)."""
        n = C.c_int64()
        t = C.c_double()
        _check(load().fdu_advance(self._h, float(cfl), float(t_end), int(precision), int(max_steps), C.byref(n),
                                  C.byref(t), _stream_ptr(stream)))
        return n.value, t.value

    def set_adjoint_precision(self, precision):
        """Precision of the adjoint calls: 64 (FP64) or 48 (double-word edge-flux
        VJP and precision-48 steps)."""
        _check(load().fdu_set_adjoint_precision(self._h, int(precision)))
        self._adjoint_precision = int(precision)

    @property
    def adjoint_precision(self):
        return getattr(self, "_adjoint_precision", 64)

    def residual_vjp(self, lam, out=None, stream=None):
        """(dL/dw)^T lam at the current state."""
        if out is None:
            out = np.zeros((self.nv, 4))
        pl, dl = _buffer(lam, self.nv)
        po, do = _buffer(out, self.nv, writable=True)
        if dl != do:
            raise ValueError("lam and out must both be device or both host arrays")
        _check(load().fdu_residual_vjp(self._h, pl, po, do, _stream_ptr(stream)))
        return out

    def rk_step_vjp(self, dt, lam_next, out=None, stream=None):
        """(dw_{n+1}/dw_n)^T lam_next for one SSP-RK3 step from the current state."""
        if out is None:
            out = np.zeros((self.nv, 4))
        pl, dl = _buffer(lam_next, self.nv)
        po, do = _buffer(out, self.nv, writable=True)
        if dl != do:
            raise ValueError("lam_next and out must both be device or both host arrays")
        _check(load().fdu_rk_step_vjp(self._h, float(dt), pl, po, do, _stream_ptr(stream)))
        return out

    def adjoint_rk(self, dt, n_steps, lam_final, out=None, checkpoint_every=10, stream=None):
        """(dw_T/dw0)^T lam_final over n_steps SSP-RK3 steps from the current state w0."""
        if out is None:
            out = np.zeros((self.nv, 4))
        pl, dl = _buffer(lam_final, self.nv)
        po, do = _buffer(out, self.nv, writable=True)
        if dl != do:
            raise ValueError("lam_final and out must both be device or both host arrays")
        _check(load().fdu_adjoint_rk(self._h, float(dt), int(n_steps), int(checkpoint_every), pl, po, do,
                                     _stream_ptr(stream)))
        return out

    def limited_count(self, reset=False, stream=None) -> int:
        """Vertex stage updates scaled by the positivity safeguard since the last reset."""
        c = C.c_int64()
        _check(load().fdu_limited_count(self._h, C.byref(c), 1 if reset else 0, _stream_ptr(stream)))
        return c.value


class Batch(Mesh):
    """Many independent periodic meshes advanced together (one persistent
    launch per RK stage).  States are the meshes' rows concatenated."""

    def __init__(self, meshes, L, *, lsq_degree=2, lsq_levels=2, device=0, renumber=1, gamma=1.4,
                 weno_eps=1e-40, weno_eps32=1e-30, host_threads=0, f32_coef=0):
        Lib = load()
        self._h = None
        xys = [np.ascontiguousarray(m[0], dtype=np.float64).reshape(-1, 2) for m in meshes]
        tris = [np.ascontiguousarray(m[1], dtype=np.int32).reshape(-1, 3) for m in meshes]
        self._keep = (xys, tris)
        n = len(meshes)
        xp = (C.POINTER(C.c_double) * n)(*[_dp(a) for a in xys])
        tp = (C.POINTER(C.c_int32) * n)(*[_ip(a) for a in tris])
        nv = np.array([a.shape[0] for a in xys], np.int64)
        nt = np.array([a.shape[0] for a in tris], np.int64)
        o = default_opts(Lx=float(L), Ly=float(L), lsq_degree=lsq_degree, lsq_levels=lsq_levels, device=device,
                         renumber=renumber, weno_eps=weno_eps, weno_eps32=weno_eps32, gamma=gamma,
                         host_threads=host_threads, f32_coef=int(f32_coef))
        h = C.c_void_p()
        _check(Lib.fdu_batch_create(n, xp, _lp(nv), tp, _lp(nt), C.byref(o), C.byref(h)))
        self._h = h
        self.device = device
        info = self.info()
        self.nv = int(info["nv"])
        self.ne = int(info["ne"])
        k = C.c_int32()
        self.offsets = np.zeros(n + 1, np.int64)
        _check(Lib.fdu_batch_info(self._h, C.byref(k), _lp(self.offsets)))
        self.n_meshes = int(k.value)

    def batch_max_dt(self, cfl, stream=None):
        dt = np.zeros(self.n_meshes)
        _check(load().fdu_batch_max_dt(self._h, float(cfl), _dp(dt), _stream_ptr(stream)))
        return dt

    def set_dt(self, dt, stream=None):
        dt = np.ascontiguousarray(dt, dtype=np.float64).reshape(self.n_meshes)
        _check(load().fdu_batch_set_dt(self._h, _dp(dt), _stream_ptr(stream)))

    def batch_rk_steps(self, n_steps, precision=32, stream=None):
        """n_steps SSP-RK3 steps of every mesh with its own dt (set_dt), one
        persistent launch per stage; precision 32, 48 or 64."""
        _check(load().fdu_batch_rk_steps(self._h, int(precision), int(n_steps), _stream_ptr(stream)))

    def set_launch(self, threads, blocks_per_sm):
        _check(load().fdu_batch_set_launch(self._h, int(threads), int(blocks_per_sm)))

    def autotune(self, precision=32):
        """Pick the fastest persistent launch shape; returns (threads, blocks/SM, ms per step)."""
        t, b = C.c_int(), C.c_int()
        ms = C.c_double()
        _check(load().fdu_batch_autotune(self._h, int(precision), C.byref(t), C.byref(b), C.byref(ms)))
        return t.value, b.value, ms.value

    def barrier_selftest(self):
        st = C.c_int()
        _check(load().fdu_batch_barrier_selftest(self._h, C.byref(st)))
        return st.value
