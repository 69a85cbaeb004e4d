"""Thin ctypes binding of libbs (include/bs.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors (float64 [k, 3] points
and outputs, int32 [k, 3] counts); streams are taken from torch.  If the
library is missing, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbs.so")

BS_OK, BS_ERR_ARG, BS_ERR_MESH, BS_ERR_ORDER, BS_ERR_CUDA, BS_ERR_TIMEOUT = range(6)
BS_FP64, BS_FP32 = 0, 1
BS_NEAR_RAY, BS_NEAR_EXACT = 0, 1
EXPORTED = ("bs_create", "bs_update", "bs_velocity", "bs_velocity_host", "bs_status", "bs_destroy",
            "bs_mesh_size", "bs_last_error", "bs_direction_table", "bs_tet_rule", "bs_batch_create",
            "bs_batch_velocity", "bs_batch_destroy", "bs_autotune", "bs_profile", "bs_profile_read",
            "bs_velocity_noalloc", "bs_tuned_variant", "bs_rk2_step", "bs_nodes", "bs_velocity_nodes",
            "bs_velocity_nodes_dderiv", "bs_rk2_step_stretch", "bs_omega", "bs_rk2_steps",
            "bs_graph_steps", "bs_set_wait_limits", "bs_num_variants", "bs_variant_shape", "bs_set_variant", "bs_noalloc_status", "bs_batch_status")


class BSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libbs error {code}: {msg}")
        self.code = code


class bs_params(ctypes.Structure):
    _fields_ = [("far_ratio", ctypes.c_double), ("tet_gauss_order", ctypes.c_int), ("n_theta", ctypes.c_int),
                ("n_phi", ctypes.c_int), ("precision", ctypes.c_int), ("counts", ctypes.c_void_p),
                ("near_rule", ctypes.c_int)]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def load(path: str = LIB_PATH):
    """Load libbs.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libbs.so not built ({path}); run paper_0712_1695_gb300/build.py")
        lib = ctypes.CDLL(path)
        lib.bs_create.argtypes = [_D, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64, _D,
                                  ctypes.POINTER(_P)]
        lib.bs_update.argtypes = [_P, _P, _P, _P]
        lib.bs_velocity.argtypes = [_P, _P, ctypes.c_int64, ctypes.POINTER(bs_params), _P, _P]
        lib.bs_velocity_host.argtypes = [_P, _D, ctypes.c_int64, ctypes.POINTER(bs_params), _D, _P]
        lib.bs_status.argtypes = [_P, _P]
        lib.bs_destroy.argtypes = [_P]
        lib.bs_mesh_size.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        lib.bs_last_error.argtypes = []
        lib.bs_last_error.restype = ctypes.c_char_p
        lib.bs_direction_table.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.bs_tet_rule.argtypes = [ctypes.c_int, _D, _D]
        lib.bs_set_wait_limits.argtypes = [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        lib.bs_num_variants.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.bs_variant_shape.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int32)]
        lib.bs_set_variant.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.bs_rk2_steps.argtypes = [_P, ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(bs_params), _P]
        lib.bs_graph_steps.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
        lib.bs_batch_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)]
        lib.bs_batch_velocity.argtypes = [_P, ctypes.POINTER(bs_params), ctypes.POINTER(_P), _P]
        lib.bs_batch_destroy.argtypes = [_P]
        lib.bs_batch_status.argtypes = [_P, _P]
        lib.bs_autotune.argtypes = [_P, ctypes.POINTER(bs_params), _P]
        lib.bs_velocity_noalloc.argtypes = [_P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P, ctypes.c_int64,
                                            ctypes.POINTER(bs_params), _P, _P]
        lib.bs_noalloc_status.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
        lib.bs_rk2_step.argtypes = [_P, ctypes.c_double, ctypes.POINTER(bs_params), _P]
        lib.bs_nodes.argtypes = [_P, _P, _P]
        lib.bs_velocity_nodes.argtypes = [_P, ctypes.POINTER(bs_params), _P, _P]
        lib.bs_velocity_nodes_dderiv.argtypes = [_P, ctypes.POINTER(bs_params), _P, _P, _P, _P]
        lib.bs_rk2_step_stretch.argtypes = [_P, ctypes.c_double, ctypes.POINTER(bs_params), _P]
        lib.bs_omega.argtypes = [_P, _P, _P]
        lib.bs_tuned_variant.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.bs_profile.argtypes = [_P, ctypes.c_int]
        lib.bs_profile_read.argtypes = [_P, _D, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        _lib = lib
        return lib


def _check(rc: int):
    if rc != BS_OK:
        raise BSError(rc, load().bs_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_params(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16, precision=BS_FP64, counts=None,
                near_rule=0):
    p = bs_params()
    p.near_rule = int(near_rule)
    p.far_ratio = float(far_ratio)
    p.tet_gauss_order = int(tet_gauss_order)
    p.n_theta = int(n_theta)
    p.n_phi = int(n_phi)
    p.precision = int(precision)
    p.counts = None if counts is None else ctypes.c_void_p(counts.data_ptr())
    return p


def _host_f64(a, cols=3):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1, cols)
    return a


class Mesh:
    """A mesh on the device (bs_handle)."""

    def __init__(self, nodes, tets, omega):
        lib = load()
        nodes = _host_f64(nodes)
        omega = _host_f64(omega)
        tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
        h = _P()
        _check(lib.bs_create(nodes.ctypes.data_as(_D), len(nodes), tets.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             len(tets), omega.ctypes.data_as(_D), ctypes.byref(h)))
        self.handle = h
        self.n_nodes = len(nodes)
        self.n_tets = len(tets)

    def close(self):
        if self.handle:
            _check(load().bs_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bs_update(self, nodes_dev=None, omega_dev=None, stream=None):
        for t in (nodes_dev, omega_dev):
            if t is not None:
                _require_dev(t, (self.n_nodes, 3))
        _check(load().bs_update(self.handle, None if nodes_dev is None else nodes_dev.data_ptr(),
                                None if omega_dev is None else omega_dev.data_ptr(), _stream_ptr(stream)))

    def bs_status(self, stream=None):
        _check(load().bs_status(self.handle, _stream_ptr(stream)))

    def bs_set_wait_limits(self, walk_max_steps=0, copy_wait_polls=0, withhold_copies=False):
        """Limits of the bounded device waits (0 = the defaults); withhold_copies tests their give-up path."""
        _check(load().bs_set_wait_limits(self.handle, int(walk_max_steps), int(copy_wait_polls),
                                         int(bool(withhold_copies))))

    def bs_velocity(self, pts_dev, out_dev=None, counts_dev=None, stream=None, **params):
        """Velocity at device points (torch float64 [k, 3]); returns the output tensor."""
        import torch

        k = int(pts_dev.shape[0])
        _require_dev(pts_dev, (k, 3))
        if out_dev is None:
            out_dev = torch.empty((k, 3), dtype=torch.float64, device=pts_dev.device)
        _require_dev(out_dev, (k, 3))
        if counts_dev is not None:
            if not (counts_dev.is_cuda and counts_dev.device == pts_dev.device and counts_dev.dtype == torch.int32
                    and tuple(counts_dev.shape) == (k, 3) and counts_dev.is_contiguous()):
                raise ValueError("counts must be a contiguous int32 [k, 3] CUDA tensor on the points' device")
        p = make_params(counts=counts_dev, **params)
        _check(load().bs_velocity(self.handle, pts_dev.data_ptr(), k, ctypes.byref(p), out_dev.data_ptr(),
                                  _stream_ptr(stream)))
        return out_dev

    def bs_velocity_nodes(self, out_dev=None, counts_dev=None, stream=None, **params):
        """Velocity at the mesh's own nodes (torch float64 [n_nodes, 3] on the device); returns the output."""
        import torch

        n = self.n_nodes
        if out_dev is None:
            out_dev = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        _require_dev(out_dev, (n, 3))
        if counts_dev is not None:
            if not (counts_dev.is_cuda and counts_dev.dtype == torch.int32 and tuple(counts_dev.shape) == (n, 3)
                    and counts_dev.is_contiguous()):
                raise ValueError("counts must be a contiguous int32 [n_nodes, 3] CUDA tensor")
        p = make_params(counts=counts_dev, **params)
        _check(load().bs_velocity_nodes(self.handle, ctypes.byref(p), out_dev.data_ptr(), _stream_ptr(stream)))
        return out_dev

    def bs_velocity_nodes_dderiv(self, dirs_dev=None, out_dev=None, dout_dev=None, stream=None, **params):
        """Velocity at the nodes and its derivative along dirs ([n_nodes, 3] CUDA float64, or None for the
        nodal vorticity: the stretching term); returns (velocity, derivative)."""
        import torch

        n = self.n_nodes
        if out_dev is None:
            out_dev = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        if dout_dev is None:
            dout_dev = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        _require_dev(out_dev, (n, 3))
        _require_dev(dout_dev, (n, 3))
        if dirs_dev is not None:
            _require_dev(dirs_dev, (n, 3))
        p = make_params(**params)
        _check(load().bs_velocity_nodes_dderiv(self.handle, ctypes.byref(p),
                                               None if dirs_dev is None else dirs_dev.data_ptr(),
                                               out_dev.data_ptr(), dout_dev.data_ptr(), _stream_ptr(stream)))
        return out_dev, dout_dev

    def bs_rk2_step_stretch(self, dt: float, stream=None, **params):
        """One Heun step of the nodes and the nodal vorticity with vortex stretching (all-ray method)."""
        p = make_params(**params)
        _check(load().bs_rk2_step_stretch(self.handle, float(dt), ctypes.byref(p), _stream_ptr(stream)))

    def bs_omega(self):
        """Current nodal vorticity as a float64 [n_nodes, 3] CUDA tensor."""
        import torch

        out = torch.empty((self.n_nodes, 3), dtype=torch.float64, device="cuda")
        _check(load().bs_omega(self.handle, out.data_ptr(), None))
        return out

    def bs_velocity_host(self, pts, stream=None, out=None, **params):
        """Velocity at host points (numpy float64 [k, 3]) through host buffers."""
        pts = _host_f64(pts)
        if out is None:
            out = np.empty_like(pts)
        p = make_params(**params)
        _check(load().bs_velocity_host(self.handle, pts.ctypes.data_as(_D), len(pts), ctypes.byref(p),
                                       out.ctypes.data_as(_D), _stream_ptr(stream)))
        return out

    def bs_rk2_step(self, dt: float, stream=None, **params):
        """One Heun step: the mesh nodes move with the velocity (vorticity carried unchanged)."""
        p = make_params(**params)
        _check(load().bs_rk2_step(self.handle, float(dt), ctypes.byref(p), _stream_ptr(stream)))

    def bs_rk2_steps(self, dt: float, n_steps: int, stretch: bool = False, stream=None, **params):
        """n_steps Heun steps (with vortex stretching if ``stretch``), replayed as a CUDA graph after the first."""
        p = make_params(**params)
        _check(load().bs_rk2_steps(self.handle, float(dt), int(n_steps), int(bool(stretch)), ctypes.byref(p),
                                   _stream_ptr(stream)))

    def bs_graph_steps(self) -> int:
        """Steps bs_rk2_steps has run by graph launch on this mesh."""
        n = ctypes.c_int64()
        _check(load().bs_graph_steps(self.handle, ctypes.byref(n)))
        return n.value

    def bs_nodes(self, out_dev=None, stream=None):
        """Current node positions as a float64 [n_nodes, 3] CUDA tensor."""
        import torch

        if out_dev is None:
            out_dev = torch.empty((self.n_nodes, 3), dtype=torch.float64, device="cuda")
        _require_dev(out_dev, (self.n_nodes, 3))
        _check(load().bs_nodes(self.handle, out_dev.data_ptr(), _stream_ptr(stream)))
        return out_dev

    def bs_profile(self, enable: bool):
        _check(load().bs_profile(self.handle, int(bool(enable))))

    def bs_profile_read(self):
        """(summed velocity-kernel ms, velocity-kernel launches, all kernel launches)."""
        ms = ctypes.c_double()
        kl = ctypes.c_int64()
        al = ctypes.c_int64()
        _check(load().bs_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(kl), ctypes.byref(al)))
        return ms.value, kl.value, al.value

    def bs_autotune(self, stream=None, at_nodes=False, **params):
        """Tune the kernel variant for these parameters (both paths); returns the variant of the points path
        (bs_velocity) or, with at_nodes, of the nodes path (bs_velocity_nodes)."""
        p = make_params(**params)
        _check(load().bs_autotune(self.handle, ctypes.byref(p), _stream_ptr(stream)))
        return self.bs_tuned_variant(params.get("precision", BS_FP64), params.get("tet_gauss_order", 4), at_nodes)

    def bs_tuned_variant(self, precision, tet_gauss_order, at_nodes=False):
        v = ctypes.c_int()
        _check(load().bs_tuned_variant(self.handle, int(precision), int(tet_gauss_order), int(bool(at_nodes)),
                                       ctypes.byref(v)))
        return v.value

    def bs_set_variant(self, precision, tet_gauss_order, near_rule, variant):
        """Pin a kernel variant for this mesh's calls with these settings (-1: automatic choice)."""
        _check(load().bs_set_variant(self.handle, int(precision), int(tet_gauss_order), int(near_rule), int(variant)))


def _require_dev(t, shape):
    import torch

    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and tuple(t.shape) == tuple(shape)):
        raise ValueError(f"expected a contiguous float64 CUDA tensor of shape {shape}")


def bs_create(nodes, tets, omega) -> Mesh:
    return Mesh(nodes, tets, omega)


VARIANT_FIELDS = ("points_per_thread", "tile", "stages", "ctas_per_sm", "near_drain", "ray_bundle", "point_pairs",
                  "tet_unroll")


def bs_num_variants(precision: int, tet_gauss_order: int, near_rule: int = BS_NEAR_RAY) -> int:
    n = ctypes.c_int()
    _check(load().bs_num_variants(int(precision), int(tet_gauss_order), int(near_rule), ctypes.byref(n)))
    return n.value


def bs_variant_shape(precision: int, tet_gauss_order: int, near_rule: int, variant: int) -> dict:
    s = (ctypes.c_int32 * 8)()
    _check(load().bs_variant_shape(int(precision), int(tet_gauss_order), int(near_rule), int(variant), s))
    return dict(zip(VARIANT_FIELDS, list(s)))


def bs_direction_table(n_phi: int, n_theta: int):
    L = n_phi * n_theta
    s = np.zeros((L, 3))
    k = np.zeros(L)
    _check(load().bs_direction_table(n_phi, n_theta, s.ctypes.data_as(_D), k.ctypes.data_as(_D)))
    return s, k


def bs_tet_rule(order: int):
    b = np.zeros((order, 4))
    w = np.zeros(order)
    _check(load().bs_tet_rule(order, b.ctypes.data_as(_D), w.ctypes.data_as(_D)))
    return b, w


def bs_velocity_noalloc(nodes_dev, tets_dev, omega_dev, pts_dev, out_dev, counts_dev=None, stream=None, **params):
    """Velocity that allocates no device memory (all arrays are caller-owned torch CUDA tensors).

    For callers that may not let the library allocate GPU memory; the
    library's fixed scratch caps the sizes (8192 tets, 4096 points, 4096
    directions, tet rules 1 and 4).  Calls share that scratch: keep them
    ordered on one stream.  A mesh error found on the device (node index out
    of range, degenerate tet) makes every output NaN and every count -1.
    """
    import torch

    n_nodes = int(nodes_dev.shape[0])
    k = int(pts_dev.shape[0])
    _require_dev(nodes_dev, (n_nodes, 3))
    _require_dev(omega_dev, (n_nodes, 3))
    _require_dev(pts_dev, (k, 3))
    _require_dev(out_dev, (k, 3))
    if not (tets_dev.is_cuda and tets_dev.dtype == torch.int32 and tets_dev.is_contiguous() and tets_dev.dim() == 2
            and tets_dev.shape[1] == 4):
        raise ValueError("tets must be a contiguous int32 [n_tets, 4] CUDA tensor")
    for t in (nodes_dev, omega_dev, tets_dev, out_dev):
        if t.device != pts_dev.device:
            raise ValueError("all arrays must be on the same CUDA device")
    if counts_dev is not None:
        if not (counts_dev.is_cuda and counts_dev.device == pts_dev.device and counts_dev.dtype == torch.int32
                and counts_dev.is_contiguous() and tuple(counts_dev.shape) == (k, 3)):
            raise ValueError("counts must be a contiguous int32 [k, 3] CUDA tensor on the points' device")
    p = make_params(counts=counts_dev, **params)
    _check(load().bs_velocity_noalloc(nodes_dev.data_ptr(), n_nodes, tets_dev.data_ptr(), int(tets_dev.shape[0]),
                                      omega_dev.data_ptr(), pts_dev.data_ptr(), k, ctypes.byref(p),
                                      out_dev.data_ptr(), _stream_ptr(stream)))
    return out_dev


def bs_noalloc_status(stream=None):
    """Error state of the last bs_velocity_noalloc call on the current device (synchronises the stream).

    Returns None when that call found nothing wrong; raises BSError (code
    BS_ERR_MESH or BS_ERR_TIMEOUT) otherwise, with the lowest bad tet in the
    exception's `first_bad_tet` attribute (-1 if not a mesh error).
    """
    bad = ctypes.c_int64(-1)
    rc = load().bs_noalloc_status(_stream_ptr(stream), ctypes.byref(bad))
    if rc != BS_OK:
        err = BSError(rc, load().bs_last_error().decode())
        err.first_bad_tet = bad.value
        raise err


class Batch:
    """Many meshes evaluated in one persistent launch (bs_batch)."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        arr = (_P * len(self.meshes))(*[m.handle for m in self.meshes])
        h = _P()
        _check(load().bs_batch_create(arr, len(self.meshes), ctypes.byref(h)))
        self.handle = h

    def bs_batch_velocity(self, outs, stream=None, **params):
        ptrs = (_P * len(outs))(*[o.data_ptr() for o in outs])
        for o, m in zip(outs, self.meshes):
            _require_dev(o, (m.n_nodes, 3))
        p = make_params(**params)
        _check(load().bs_batch_velocity(self.handle, ctypes.byref(p), ptrs, _stream_ptr(stream)))
        return outs

    def bs_batch_status(self, stream=None):
        """Synchronise and raise BSError if a launch of this batch raised a device error (clears the flags)."""
        _check(load().bs_batch_status(self.handle, _stream_ptr(stream)))

    def close(self):
        if self.handle:
            _check(load().bs_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


INF = math.inf
