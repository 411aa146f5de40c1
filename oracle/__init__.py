"""Plain FP64 CPU oracle of the unstructured-mesh FDM (arXiv 2102.12933).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package.  The arithmetic lives in ``fdu_oracle.c`` (plain C,
single thread, no shared code with the CUDA path); this module compiles it
with gcc and wraps it with ctypes and numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdu_oracle.c")
_SRC_STATE = os.path.join(_HERE, "fdu_oracle_state.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libfdu_oracle.so")
_lock = threading.Lock()
_lib = None

EPS = 1e-40  # epsilon of the nonlinear weights (Appendix)
GAMMA = 1.4  # ratio of specific heats (Section 2.1)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_STATE))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            P = C.c_void_p
            i64 = C.c_int64
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            lp = C.POINTER(C.c_int64)
            up = C.POINTER(C.c_uint8)
            L.om_last_error.restype = C.c_char_p
            L.om_create.argtypes = [dp, i64, ip, i64, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, ip,
                                    C.POINTER(P)]
            L.om_create.restype = C.c_int
            L.om_create_cells.argtypes = [dp, i64, lp, ip, i64, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                          C.c_double, ip, C.POINTER(P)]
            L.om_create_cells.restype = C.c_int
            L.om_destroy.argtypes = [P]
            L.om_num_edges.argtypes = [P]
            L.om_num_edges.restype = i64
            L.om_get_edges.argtypes = [P, ip]
            L.om_get_normals.argtypes = [P, dp]
            L.om_get_stencils.argtypes = [P, ip, dp]
            L.om_div_sizes.argtypes = [P, lp, lp]
            L.om_get_div.argtypes = [P, lp, ip, dp, dp, lp, ip, dp]
            L.om_build_weights.argtypes = [P, up]
            L.om_build_weights.restype = C.c_int
            L.om_edge_fluxes.argtypes = [P, dp, C.c_double, up, dp, lp]
            L.om_edge_fluxes.restype = C.c_int
            L.om_residual.argtypes = [P, dp, C.c_double, up, dp, lp]
            L.om_residual.restype = C.c_int
            L.om_rk3_step.argtypes = [P, dp, C.c_double, C.c_double, lp]
            L.om_rk3_step.restype = C.c_int
            L.om_max_dt.argtypes = [P, dp, C.c_double]
            L.om_max_dt.restype = C.c_double
            L.om_fill_ghosts.argtypes = [P, dp]
            # complex-step copies (double complex arrays passed as pointers)
            L.om_residual_cs.argtypes = [P, P, C.c_double, up, P, lp]
            L.om_residual_cs.restype = C.c_int
            L.om_rk3_step_cs.argtypes = [P, P, C.c_double, C.c_double, lp]
            L.om_rk3_step_cs.restype = C.c_int
            L.om_fill_ghosts_cs.argtypes = [P, P]
            L.om_walk_edge.argtypes = [P, i64, ip]
            L.om_walk_edge.restype = C.c_int
            L.om_curve_coords.argtypes = [dp, dp]
            L.om_curve_coords.restype = C.c_int
            L.om_substencil_coeffs.argtypes = [dp, dp]
            L.om_linear_weights.argtypes = [dp, dp]
            L.om_s5_coeffs.argtypes = [dp, dp]
            L.om_nuweno.argtypes = [dp, dp, C.c_double, C.c_int]
            L.om_nuweno.restype = C.c_double
            L.om_eigvec.argtypes = [dp, dp, dp, C.c_double, dp, dp, dp]
            L.om_eigvec.restype = C.c_int
            L.om_roe_flux.argtypes = [dp, dp, dp, C.c_double, dp]
            L.om_roe_flux.restype = C.c_int
            L.om_stage_combine.argtypes = [i64, C.c_int, dp, dp, dp, C.c_double, dp]
            L.om_smoothness_all.argtypes = [dp, dp, dp]
            L.om_set_positivity.argtypes = [P, C.c_double]
            L.om_pos_limited.argtypes = [P]
            L.om_pos_limited.restype = i64
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _l(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _u(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class OracleError(RuntimeError):
    pass


def _check(st):
    if st != 0:
        raise OracleError(f"oracle status {st}: {lib().om_last_error().decode()}")


# ---------------------------------------------------------------- 1D pieces
def substencil_coeffs(x):
    """Coefficients of the sub-stencil interpolants at 0 (Appendix, Eqs. u0-u2) -> [3,3]."""
    x = _f64(x, (5,))
    out = np.zeros(9)
    lib().om_substencil_coeffs(_d(x), _d(out))
    return out.reshape(3, 3)


def linear_weights(x):
    """Linear weights C_0..C_2 (Appendix, Eq. C_K)."""
    x = _f64(x, (5,))
    out = np.zeros(3)
    lib().om_linear_weights(_d(x), _d(out))
    return out


def s5_coeffs(x):
    """Degree-4 Lagrange weights at 0 over all five points (Appendix, Eq. S5)."""
    x = _f64(x, (5,))
    out = np.zeros(5)
    lib().om_s5_coeffs(_d(x), _d(out))
    return out


def nuweno(x, u, eps=EPS, linear=False):
    """Left-state NU-WENO5 value at 0 from x_{i-2..i+2}, u_{i-2..i+2} (Appendix)."""
    x = _f64(x, (5,))
    u = _f64(u, (5,))
    return float(lib().om_nuweno(_d(x), _d(u), float(eps), 1 if linear else 0))


def curve_coords(P):
    """Normalised arc-length coordinates of the six stencil points [6,2] -> [6]."""
    P = _f64(P, (12,))
    out = np.zeros(6)
    _check(lib().om_curve_coords(_d(P), _d(out)))
    return out


def eigvec(wa, wb, n, gamma=GAMMA):
    """Right eigenvectors R (columns), their numeric inverse and eigenvalues at the Roe average."""
    wa, wb, n = _f64(wa, (4,)), _f64(wb, (4,)), _f64(n, (2,))
    R = np.zeros(16)
    Linv = np.zeros(16)
    lam = np.zeros(4)
    _check(lib().om_eigvec(_d(wa), _d(wb), _d(n), gamma, _d(R), _d(Linv), _d(lam)))
    return R.reshape(4, 4), Linv.reshape(4, 4), lam


def roe_flux(wl, wr, n, gamma=GAMMA):
    wl, wr, n = _f64(wl, (4,)), _f64(wr, (4,)), _f64(n, (2,))
    out = np.zeros(4)
    _check(lib().om_roe_flux(_d(wl), _d(wr), _d(n), gamma, _d(out)))
    return out


def stage_combine(stage, wn, ws, L, dt):
    wn, ws, L = _f64(wn), _f64(ws), _f64(L)
    out = np.zeros_like(wn)
    lib().om_stage_combine(wn.size, int(stage), _d(wn), _d(ws), _d(L), float(dt), _d(out))
    return out


# ---------------------------------------------------------------- meshes
class OracleMesh:
    """Oracle mesh: edges, 1D stencils, divergence stencils, LSQ weights."""

    def __init__(self, xy, tri, Lx=0.0, Ly=0.0, degree=2, levels=2, gamma=GAMMA, ghost=None, artificial=None):
        """`tri`: (nt, 3) triangles, or a pair (cell_off, cell_vtx) of
        triangles and quadrilaterals; then `artificial` (0, 1, 2; default 1)
        selects the artificial edges (Section 2.2.2)."""
        xy = _f64(xy, (-1, 2))
        cells = None
        if isinstance(tri, tuple):
            cells = (np.ascontiguousarray(tri[0], dtype=np.int64), np.ascontiguousarray(tri[1], dtype=np.int32))
        else:
            tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        self.nv = xy.shape[0]
        self.gamma = gamma
        gp = None
        self._ghost = None
        if ghost is not None:
            self._ghost = np.ascontiguousarray(ghost, dtype=np.int32).reshape(self.nv)
            gp = _i(self._ghost)
        h = C.c_void_p()
        if cells is not None:
            off, vtx = cells
            _check(lib().om_create_cells(_d(xy), self.nv, off.ctypes.data_as(C.POINTER(C.c_int64)), _i(vtx),
                                         off.shape[0] - 1, 1 if artificial is None else int(artificial), float(Lx),
                                         float(Ly), int(degree), int(levels), float(gamma), gp, C.byref(h)))
        else:
            _check(lib().om_create(_d(xy), self.nv, _i(tri), tri.shape[0], float(Lx), float(Ly), int(degree),
                                   int(levels), float(gamma), gp, C.byref(h)))
        self._h = h
        self.ne = int(lib().om_num_edges(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().om_destroy(h)
            self._h = None

    @property
    def ghost(self):
        return self._ghost

    def edges(self):
        e = np.zeros((self.ne, 2), np.int32)
        lib().om_get_edges(self._h, _i(e))
        return e

    def normals(self):
        n = np.zeros((self.ne, 2))
        lib().om_get_normals(self._h, _d(n))
        return n

    def stencils(self):
        s = np.zeros((self.ne, 6), np.int32)
        xi = np.zeros((self.ne, 6))
        lib().om_get_stencils(self._h, _i(s), _d(xi))
        return s, xi

    def build_weights(self, mask=None):
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        _check(lib().om_build_weights(self._h, None if m is None else _u(m)))

    def div_stencils(self, weights=True):
        """CSR: (voff, vid, wf, wg, eoff, eid, we); weights of vertices not yet built are 0."""
        nvv = C.c_int64()
        nee = C.c_int64()
        lib().om_div_sizes(self._h, C.byref(nvv), C.byref(nee))
        voff = np.zeros(self.nv + 1, np.int64)
        eoff = np.zeros(self.nv + 1, np.int64)
        vid = np.zeros(nvv.value, np.int32)
        eid = np.zeros(nee.value, np.int32)
        wf = np.zeros(nvv.value)
        wg = np.zeros(nvv.value)
        we = np.zeros(nee.value)
        lib().om_get_div(self._h, _l(voff), _i(vid), _d(wf), _d(wg), _l(eoff), _i(eid), _d(we))
        return voff, vid, wf, wg, eoff, eid, we

    def edge_fluxes(self, w, eps=EPS, mask=None):
        w = _f64(w, (self.nv, 4))
        r = np.zeros((self.ne, 4))
        nf = C.c_int64()
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        _check(lib().om_edge_fluxes(self._h, _d(w), float(eps), None if m is None else _u(m), _d(r), C.byref(nf)))
        return r, nf.value

    def residual(self, w, eps=EPS, mask=None, return_fallbacks=False):
        """dw/dt at every real vertex (or at ``mask``ed ones; the rest are left 0)."""
        w = _f64(w, (self.nv, 4)).copy()
        if self._ghost is not None:
            lib().om_fill_ghosts(self._h, _d(w))
        out = np.zeros((self.nv, 4))
        nf = C.c_int64()
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        _check(lib().om_residual(self._h, _d(w), float(eps), None if m is None else _u(m), _d(out), C.byref(nf)))
        return (out, nf.value) if return_fallbacks else out

    def rk3_step(self, w, dt, eps=EPS, return_fallbacks=False):
        w = _f64(w, (self.nv, 4)).copy()
        nf = C.c_int64()
        _check(lib().om_rk3_step(self._h, _d(w), float(dt), float(eps), C.byref(nf)))
        return (w, nf.value) if return_fallbacks else w

    # ---- complex-step tangents (directional derivatives of the same functions)
    # Im F(w + i h d) / h = J d for a function analytic in the state, with no
    # subtraction (Squire & Trapp 1998); the branches are those of F at w.
    CS_STEP = 1e-30

    def _complex_state(self, w, d):
        z = np.ascontiguousarray(_f64(w, (self.nv, 4)) + 1j * self.CS_STEP * _f64(d, (self.nv, 4)))
        return z

    def residual_jvp(self, w, d, eps=EPS, return_value=False):
        """J d, J the Jacobian of ``residual`` at w (ghost fill included)."""
        z = self._complex_state(w, d)
        if self._ghost is not None:
            lib().om_fill_ghosts_cs(self._h, z.ctypes.data)
        out = np.zeros((self.nv, 4), np.complex128)
        nf = C.c_int64()
        _check(lib().om_residual_cs(self._h, z.ctypes.data, float(eps), None, out.ctypes.data, C.byref(nf)))
        jd = out.imag / self.CS_STEP
        return (out.real.copy(), jd) if return_value else jd

    def rk3_steps_jvp(self, w, d, dt, n=1, eps=EPS):
        """(state, J d) after n SSP-RK3 steps of size dt from w, J the
        Jacobian of the n-step map (``rk3_step`` applied n times)."""
        z = self._complex_state(w, d)
        nf = C.c_int64()
        for _ in range(n):
            _check(lib().om_rk3_step_cs(self._h, z.ctypes.data, float(dt), float(eps), C.byref(nf)))
        return z.real.copy(), z.imag / self.CS_STEP

    def set_positivity(self, alpha):
        """Enable the stage positivity safeguard (alpha > 0) or disable it (0)."""
        lib().om_set_positivity(self._h, float(alpha))

    def positivity_limited(self):
        return int(lib().om_pos_limited(self._h))

    def max_dt(self, w, cfl):
        w = _f64(w, (self.nv, 4))
        return float(lib().om_max_dt(self._h, _d(w), float(cfl)))

    def walk(self, k):
        s = np.zeros(6, np.int32)
        _check(lib().om_walk_edge(self._h, int(k), _i(s)))
        return s


def smoothness(x, u):
    """Smoothness indicators beta_0..2 of the left-state sub-stencils (Appendix)."""
    x = _f64(x, (5,))
    u = _f64(u, (5,))
    out = np.zeros(3)
    lib().om_smoothness_all(_d(x), _d(u), _d(out))
    return out
