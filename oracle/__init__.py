"""FP64 CPU oracle for the Biot-Savart velocity on tetrahedral meshes.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The oracle shares no code
with the CUDA path.  ``build()`` compiles ``bs_oracle.c`` with gcc (OpenMP,
no floating-point contraction so x86 and Arm give identical results).

Every function below is a thin ctypes marshalling layer over the C code; the
arithmetic and its citations live in ``bs_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bs_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libbs_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile ``src`` into the shared library ``out`` (skipped when up to date)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class OracleLib:
    """ctypes view of one compiled copy of ``bs_oracle.c``."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        lib.orc_gauss_legendre.argtypes = [ctypes.c_int, _D, _D]
        lib.orc_gauss_jacobi01.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc_tet_rule.argtypes = [ctypes.c_int, _D, _D]
        lib.orc_directions.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc_moller_trumbore.argtypes = [_D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double, _D, _D, _D]
        lib.orc_tet_geometry.argtypes = [_D, _D, _D, _D, _D]
        lib.orc_line_tet.argtypes = [_D, _D, _D, _D, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, _D, _D, _D]
        lib.orc_velocity.argtypes = [_D, ctypes.c_int64, _I32, ctypes.c_int64, _D, _D, ctypes.c_int64,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _I32]
        lib.orc_tet_analytic.argtypes = [_D, _D, _D, _D]
        lib.orc_velocity_dderiv.argtypes = [_D, ctypes.c_int64, _I32, ctypes.c_int64, _D, _D, _D, ctypes.c_int64,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D]
        lib.orc_num_threads.argtypes = []
        lib.orc_set_num_threads.argtypes = [ctypes.c_int]
        self.lib = lib
        self.path = path

    def num_threads(self) -> int:
        return int(self.lib.orc_num_threads())

    def set_num_threads(self, n: int) -> None:
        self.lib.orc_set_num_threads(int(n))

    def gauss_legendre(self, n: int):
        t = np.zeros(n)
        w = np.zeros(n)
        if self.lib.orc_gauss_legendre(n, _dp(t), _dp(w)) != 0:
            raise ValueError("bad order")
        return t, w

    def gauss_jacobi01(self, k: int, alpha: int):
        u = np.zeros(k)
        w = np.zeros(k)
        if self.lib.orc_gauss_jacobi01(k, alpha, _dp(u), _dp(w)) != 0:
            raise ValueError("bad Gauss-Jacobi request")
        return u, w

    def tet_rule(self, order: int):
        bary = np.zeros((max(order, 1), 4))
        w = np.zeros(max(order, 1))
        if self.lib.orc_tet_rule(order, _dp(bary), _dp(w)) != 0:
            raise ValueError(f"unsupported tet rule order {order}")
        return bary, w

    def directions(self, n_phi: int, n_theta: int):
        L = n_phi * n_theta
        s = np.zeros((L, 3))
        k = np.zeros(L)
        if self.lib.orc_directions(n_phi, n_theta, _dp(s), _dp(k)) != 0:
            raise ValueError("bad direction request")
        return s, k

    def moller_trumbore(self, o, d, p0, p1, p2, eps_det=1e-12, eps_b=1e-12):
        o, d, p0, p1, p2 = (_f64(a, (3,)) for a in (o, d, p0, p1, p2))
        t, u, v = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        hit = self.lib.orc_moller_trumbore(_dp(o), _dp(d), _dp(p0), _dp(p1), _dp(p2), eps_det, eps_b,
                                           ctypes.byref(t), ctypes.byref(u), ctypes.byref(v))
        return bool(hit), t.value, u.value, v.value

    def tet_analytic(self, x, verts, om):
        """Exact Eq. 1 over one tet with linear vorticity (the analytic near-field evaluation)."""
        x = _f64(x, (3,))
        v = _f64(verts, (4, 3))
        w = _f64(om, (4, 3))
        out = np.zeros(3)
        rc = self.lib.orc_tet_analytic(_dp(x), _dp(v), _dp(w), _dp(out))
        if rc != 0:
            raise ValueError("degenerate tet")
        return out

    def tet_geometry(self, verts):
        v = _f64(verts, (4, 3))
        c = np.zeros(3)
        r, h, vol = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self.lib.orc_tet_geometry(_dp(v), _dp(c), ctypes.byref(r), ctypes.byref(h), ctypes.byref(vol))
        return c, r.value, h.value, vol.value

    def line_tet(self, x, s, verts, om, use_precheck=False, eps_b=1e-12, tau=1e-9):
        x, s = _f64(x, (3,)), _f64(s, (3,))
        v, w = _f64(verts, (4, 3)), _f64(om, (4, 3))
        _, _, h, _ = self.tet_geometry(v)
        R0, R1 = ctypes.c_double(), ctypes.c_double()
        J = np.zeros(3)
        hit = self.lib.orc_line_tet(_dp(x), _dp(s), _dp(v), _dp(w), h, int(use_precheck), eps_b, tau,
                                    ctypes.byref(R0), ctypes.byref(R1), _dp(J))
        return bool(hit), R0.value, R1.value, J

    def velocity(self, nodes, tets, omega, pts, far_ratio=2.0, tet_order=4, n_theta=8, n_phi=16,
                 use_precheck=True, eps_b=1e-12, tau=1e-9, counts=False, near_rule=0):
        """Velocity [n_pts, 3] (and optionally counts [n_pts, 3] = near, far, ray hits).

        near_rule 0: near tets by the ray rule; 1: by the exact integral (``tet_analytic``)."""
        nodes = _f64(nodes).reshape(-1, 3)
        omega = _f64(omega).reshape(-1, 3)
        pts = _f64(pts).reshape(-1, 3)
        tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
        vel = np.zeros((len(pts), 3))
        cnt = np.zeros((len(pts), 3), dtype=np.int32)
        rc = self.lib.orc_velocity(_dp(nodes), len(nodes), tets.ctypes.data_as(_I32), len(tets), _dp(omega),
                                   _dp(pts), len(pts), float(far_ratio), int(tet_order), int(n_theta),
                                   int(n_phi), int(use_precheck), float(eps_b), float(tau), int(near_rule), _dp(vel),
                                   cnt.ctypes.data_as(_I32))
        if rc != 0:
            raise ValueError(f"oracle rejected arguments (code {rc})")
        return (vel, cnt) if counts else vel


    def velocity_dderiv(self, nodes, tets, omega, pts, dirs, n_theta=8, n_phi=16, eps_b=1e-12, tau=1e-9):
        """All-ray velocity [n_pts, 3] and its derivative along dirs [n_pts, 3] (the stretching term
        (omega . grad) v when dirs = omega at the points)."""
        nodes = _f64(nodes).reshape(-1, 3)
        omega = _f64(omega).reshape(-1, 3)
        pts = _f64(pts).reshape(-1, 3)
        dirs = _f64(dirs).reshape(-1, 3)
        if dirs.shape != pts.shape:
            raise ValueError("one direction per point")
        tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
        vel = np.zeros((len(pts), 3))
        dvel = np.zeros((len(pts), 3))
        rc = self.lib.orc_velocity_dderiv(_dp(nodes), len(nodes), tets.ctypes.data_as(_I32), len(tets), _dp(omega),
                                          _dp(pts), _dp(dirs), len(pts), int(n_theta), int(n_phi), float(eps_b),
                                          float(tau), _dp(vel), _dp(dvel))
        if rc != 0:
            raise ValueError(f"oracle rejected arguments (code {rc})")
        return vel, dvel


def heun_step(orc, nodes, tets, omega, dt, **params):
    """One Heun (RK2) step of the node positions with the oracle's velocity (plain numpy arithmetic).

    v0 = v(x0) at the nodes of the mesh as it is; x* = x0 + dt v0; v1 = v(x*)
    at the nodes of the moved mesh (same tets, same nodal vorticity);
    x1 = x0 + dt (v0 + v1) / 2.
    """
    x0 = np.ascontiguousarray(nodes, dtype=np.float64)
    v0 = orc.velocity(x0, tets, omega, x0, **params)
    xs = x0 + dt * v0
    v1 = orc.velocity(xs, tets, omega, xs, **params)
    return x0 + 0.5 * dt * (v0 + v1)


def heun_step_stretch(orc, nodes, tets, omega, dt, n_theta=8, n_phi=16):
    """One Heun step of node positions and nodal vorticity with vortex stretching (plain numpy arithmetic),
    all-ray velocity: dx/dt = v, d omega/dt = (omega . grad) v at the nodes (orc.velocity_dderiv with the
    nodal vorticity as the directions).  Returns (x1, omega1)."""
    x0 = np.ascontiguousarray(nodes, dtype=np.float64)
    w0 = np.ascontiguousarray(omega, dtype=np.float64)
    v0, s0 = orc.velocity_dderiv(x0, tets, w0, x0, w0, n_theta=n_theta, n_phi=n_phi)
    xs, ws = x0 + dt * v0, w0 + dt * s0
    v1, s1 = orc.velocity_dderiv(xs, tets, ws, xs, ws, n_theta=n_theta, n_phi=n_phi)
    return x0 + 0.5 * dt * (v0 + v1), w0 + 0.5 * dt * (s0 + s1)


def _load() -> OracleLib:
    global _lib
    with _lock:
        if _lib is None:
            _lib = OracleLib(build())
    return _lib


def num_threads() -> int:
    return _load().num_threads()


def set_num_threads(n: int) -> None:
    _load().set_num_threads(n)


def gauss_legendre(n):
    return _load().gauss_legendre(n)


def gauss_jacobi01(k, alpha):
    return _load().gauss_jacobi01(k, alpha)


def tet_rule(order):
    return _load().tet_rule(order)


def directions(n_phi, n_theta):
    return _load().directions(n_phi, n_theta)


def moller_trumbore(*args, **kw):
    return _load().moller_trumbore(*args, **kw)


def tet_geometry(verts):
    return _load().tet_geometry(verts)


def tet_analytic(*args, **kw):
    return _load().tet_analytic(*args, **kw)


def line_tet(*args, **kw):
    return _load().line_tet(*args, **kw)


def velocity(*args, **kw):
    return _load().velocity(*args, **kw)


def velocity_dderiv(*args, **kw):
    return _load().velocity_dderiv(*args, **kw)
