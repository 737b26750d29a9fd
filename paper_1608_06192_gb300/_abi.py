"""ctypes binding of libdcrf.so: argument marshalling only.

Every function here checks shapes and dtypes, passes raw device pointers and
the current CUDA stream to the C ABI declared in include/dcrf.h, and raises
DcrfError on a non-zero status.  All arithmetic runs in the library's CUDA
kernels; there is no CPU fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

STORAGE = {"f32": 0, "f16": 1}

_lib = None


class DcrfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().dcrf_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


class FwRecord(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("gap", ctypes.c_double), ("alpha", ctypes.c_double),
                ("A", ctypes.c_double), ("B", ctypes.c_double)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_F = ctypes.c_float
_D = ctypes.c_double

_SIGS = {
    "dcrf_status_string": ([_I], ctypes.c_char_p),
    "dcrf_version": ([], _I),
    "dcrf_features": ([_P, _P, _P, _I, _F, _F, _F, _P, _P, _P], _I),
    "dcrf_lattice_build": ([_P, _I64, _I, _P, _P], _I),
    "dcrf_lattice_build_batch": ([_P, _P, _I, _I, _P, _P], _I),
    "dcrf_lattice_destroy": ([_P], _I),
    "dcrf_lattice_info": ([_P, _P, _P, _P, _P], _I),
    "dcrf_lattice_vertex_offsets": ([_P, _P], _I),
    "dcrf_lattice_status": ([_P, _P], _I),
    "dcrf_lattice_export": ([_P, _P, _P, _P, _P, _P], _I),
    "dcrf_filter": ([_P, _P, _I, _P, _I, _P], _I),
    "dcrf_filter_adjoint": ([_P, _P, _I, _P, _I, _P], _I),
    "dcrf_filter_static": ([_P, _P, _I, _P, _I, _P], _I),
    "dcrf_filter_static_capacity": ([], ctypes.c_size_t),
    "dcrf_qp_fw": ([_P, _P, _P, _I, _P, _I, _I, _P, _P, _I, _P], _I),
    "dcrf_dc_cccp": ([_P, _P, _P, _I, _P, _I, _I, _I, _P, _P, _I, _P], _I),
    "dcrf_dc_cccp_trace": ([_P, _P, _P, _I, _P, _I, _I, _I, _P, _P, _P, _I, _P], _I),
    "dcrf_dc_neg": ([_P, _P, _P, _I, _P, _I, _I, _I, _P, _P, _I, _P], _I),
    "dcrf_mean_field": ([_P, _P, _P, _I, _P, _I, _I, _P, _P, _I, _P], _I),
    "dcrf_round": ([_P, ctypes.c_int64, _I, _P, _P, _P], _I),
    "dcrf_labelling_energy": ([_P, _P, _P, _I, _P, _I, _P, _P, _I, _P], _I),
    "dcrf_qp_fw_trace": ([_P, _P, _P, _I, _P, _I, _I, _P, _P, _P, _I, _P], _I),
    "dcrf_qp_fw_backward": ([_P, _P, _P, _I, _P, _I, _I, _P, _P, _P, _P, _P, _P, _P], _I),
    "dcrf_lp_subgrad": ([_P, _P, _P, _P, _I, _I, _P, _P, _P], _I),
    "dcrf_lp_solve": ([_P, _P, _P, _I, _I, _I, _D, _P, _P, _P], _I),
    "dcrf_lp_subgrad_tree": ([_P, _P, _P, _P, _I, _I, _I, _P, _P, _P, _P, _P], _I),
    "dcrf_lp_solve_tree": ([_P, _P, _P, _I, _I, _I, _P, _P, _I, _D, _P, _P, _P], _I),
    "dcrf_qp_fw_host": ([_P, _P, _P, _P, _P, _P, _I, _I, _F, _F, _F, _P, _P, _I, _P, _I, _P], _I),
    "dcrf_pool_trim": ([], _I),
    "dcrf_round_kt": ([_P, _I64, _I, _I, _P, _P, _I, _P, _P, _P], _I),
    "dcrf_simplex_project": ([_P, _I64, _I, _P, _P], _I),
    "dcrf_selftest_bounded_wait": ([_P, _I64, _I, _P], _I),
    "dcrf_check_lattice_tables": ([_P, _P, _I64, _I, _P, _I64, _P, _P, _I, _P, _P], _I),
    "dcrf_lattice_validate": ([_P, _P, _P], _I),
    "dcrf_profile_enable": ([_I], _I),
    "dcrf_profile_reset": ([], _I),
    "dcrf_profile_read": ([_P, _P, _P, _I], _I),
}


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not path.exists():
            raise RuntimeError(f"{path} is missing: build it with paper_1608_06192_gb300.build.build()")
        handle = ctypes.CDLL(str(path))
        for name, (args, res) in _SIGS.items():
            fn = getattr(handle, name)   # a missing export is an error
            fn.argtypes = args
            fn.restype = res
        _lib = handle
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise DcrfError(status, where)


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream: torch.cuda.Stream | None = None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, dtype: torch.dtype, name: str, ndim: int | None = None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class Lattice:
    """Owns a dcrf_lattice handle (destroyed with the object)."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle
        n, d, m, b = _I64(), _I(), _I64(), _I()
        _check(lib().dcrf_lattice_info(handle, ctypes.byref(n), ctypes.byref(d), ctypes.byref(m),
                                       ctypes.byref(b)), "dcrf_lattice_info")
        self.n, self.d, self.m, self.batch = n.value, d.value, m.value, b.value
        off = (_I64 * (self.batch + 1))()
        _check(lib().dcrf_lattice_vertex_offsets(handle, off), "dcrf_lattice_vertex_offsets")
        self.vertex_offsets = np.array(off[:], dtype=np.int64)

    def close(self):
        if self.handle:
            lib().dcrf_lattice_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None):
        _check(lib().dcrf_lattice_status(self.handle, _stream(stream)), "device status")


def _handles(lattices):
    arr = (ctypes.c_void_p * len(lattices))(*[lt.handle for lt in lattices])
    return arr


def _floats(values):
    vals = [float(v) for v in values]
    return (ctypes.c_float * len(vals))(*vals)


def _compat(compat, L):
    if compat is None:
        return None
    a = np.ascontiguousarray(np.asarray(compat, dtype=np.float32).reshape(L, L))
    return a, a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------

def dcrf_features(rgb: torch.Tensor, widths, heights, theta_alpha: float, theta_beta: float,
                  theta_gamma: float, stream=None):
    """Step a1: (f_bil [N,5], f_sp [N,2]) from concatenated RGB images [N,3]."""
    rgb = _dev(rgb, torch.float32, "rgb", 2)
    w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
    h = np.ascontiguousarray(np.asarray(heights, dtype=np.int32))
    n = rgb.shape[0]
    fb = torch.empty((n, 5), dtype=torch.float32, device=rgb.device)
    fs = torch.empty((n, 2), dtype=torch.float32, device=rgb.device)
    _check(lib().dcrf_features(_ptr(rgb), w.ctypes.data_as(_P), h.ctypes.data_as(_P), len(w),
                               theta_alpha, theta_beta, theta_gamma, _ptr(fb), _ptr(fs), _stream(stream)),
           "dcrf_features")
    return fb, fs


def dcrf_lattice_build(features: torch.Tensor, offsets=None, stream=None) -> Lattice:
    """Step a2: the lattice of one kernel over [N, d] pre-scaled features."""
    features = _dev(features, torch.float32, "features", 2)
    n, d = features.shape
    h = ctypes.c_void_p()
    if offsets is None:
        st = lib().dcrf_lattice_build(_ptr(features), n, d, _stream(stream), ctypes.byref(h))
    else:
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        st = lib().dcrf_lattice_build_batch(_ptr(features), off.ctypes.data_as(_P), len(off) - 1, d,
                                            _stream(stream), ctypes.byref(h))
    _check(st, "dcrf_lattice_build")
    return Lattice(h)


def dcrf_lattice_export(lat: Lattice, stream=None) -> dict:
    dev = torch.device("cuda")
    d1 = lat.d + 1
    keys = torch.empty((lat.m, lat.d), dtype=torch.int32, device=dev)
    pv = torch.empty((lat.n, d1), dtype=torch.int32, device=dev)
    pw = torch.empty((lat.n, d1), dtype=torch.float32, device=dev)
    nb = torch.empty((lat.m, d1, 2), dtype=torch.int32, device=dev)
    _check(lib().dcrf_lattice_export(lat.handle, _ptr(keys), _ptr(pv), _ptr(pw), _ptr(nb), _stream(stream)),
           "dcrf_lattice_export")
    return {"keys": keys, "point_vertex": pv, "point_weight": pw, "neighbours": nb}


def dcrf_filter(lat: Lattice, Y: torch.Tensor, storage: str = "f32", stream=None, out=None) -> torch.Tensor:
    """K~ Y through the lattice (Eq. 6), Y [N, L] float32."""
    Y = _dev(Y, torch.float32, "Y", 2)
    out = torch.empty_like(Y) if out is None else _dev(out, torch.float32, "out", 2)
    _check(lib().dcrf_filter(lat.handle, _ptr(Y), Y.shape[1], _ptr(out), STORAGE[storage], _stream(stream)),
           "dcrf_filter")
    return out


def dcrf_filter_static(lat: Lattice, Y: torch.Tensor, storage: str = "f32", stream=None, out=None):
    """dcrf_filter without device allocation in the library (fixed static scratch)."""
    Y = _dev(Y, torch.float32, "Y", 2)
    out = torch.empty_like(Y) if out is None else _dev(out, torch.float32, "out", 2)
    _check(lib().dcrf_filter_static(lat.handle, _ptr(Y), Y.shape[1], _ptr(out), STORAGE[storage],
                                    _stream(stream)), "dcrf_filter_static")
    return out


def dcrf_filter_adjoint(lat: Lattice, U: torch.Tensor, storage: str = "f32", stream=None, out=None):
    U = _dev(U, torch.float32, "U", 2)
    out = torch.empty_like(U) if out is None else _dev(out, torch.float32, "out", 2)
    _check(lib().dcrf_filter_adjoint(lat.handle, _ptr(U), U.shape[1], _ptr(out), STORAGE[storage],
                                     _stream(stream)), "dcrf_filter_adjoint")
    return out


def dcrf_qp_fw(unaries: torch.Tensor, lattices, weights, Y: torch.Tensor, iters: int, compat=None,
               storage: str = "f32", records: bool = True, stream=None):
    """Frank-Wolfe on S_cvx; Y is updated in place.  Returns records [iters, batch] or None."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Y = _dev(Y, torch.float32, "Y", 2)
    L = unaries.shape[1]
    batch = lattices[0].batch
    rec = (FwRecord * max(1, iters * batch))() if records else None
    cm = _compat(compat, L)
    _check(lib().dcrf_qp_fw(_ptr(unaries), _handles(lattices), _floats(weights), len(lattices),
                            None if cm is None else cm[1], L, iters, _ptr(Y), rec, STORAGE[storage],
                            _stream(stream)), "dcrf_qp_fw")
    if not records:
        return None
    arr = np.array([(r.energy, r.gap, r.alpha, r.A, r.B) for r in rec[:iters * batch]], dtype=np.float64)
    return arr.reshape(iters, batch, 5)


def dcrf_qp_fw_trace(unaries: torch.Tensor, lattices, weights, Y: torch.Tensor, iters: int, compat=None,
                     storage: str = "f32", stream=None):
    """dcrf_qp_fw that also returns the decisions: (records [iters, batch, 5],
    s_trace uint8 [iters, N] on the device, row t = s^t of iteration t)."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Y = _dev(Y, torch.float32, "Y", 2)
    L = unaries.shape[1]
    batch = lattices[0].batch
    rec = (FwRecord * max(1, iters * batch))()
    trace = torch.empty((iters, Y.shape[0]), dtype=torch.uint8, device=Y.device)
    cm = _compat(compat, L)
    _check(lib().dcrf_qp_fw_trace(_ptr(unaries), _handles(lattices), _floats(weights), len(lattices),
                                  None if cm is None else cm[1], L, iters, _ptr(Y), rec, _ptr(trace),
                                  STORAGE[storage], _stream(stream)), "dcrf_qp_fw_trace")
    arr = np.array([(r.energy, r.gap, r.alpha, r.A, r.B) for r in rec[:iters * batch]], dtype=np.float64)
    return arr.reshape(iters, batch, 5), trace


def _host(a, name: str, cols: int | None = None):
    """A C-contiguous float32 host array (numpy, or a CPU tensor, pinned or not) and its address."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError(f"{name}: contiguous float32 host tensor required")
        arr, ptr = a, ctypes.c_void_p(a.data_ptr())
    else:
        arr = np.asarray(a)
        if arr.dtype != np.float32 or not arr.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: C-contiguous float32 array required")
        ptr = arr.ctypes.data_as(_P)
    if arr.ndim != 2 or (cols is not None and arr.shape[1] != cols):
        raise ValueError(f"{name}: shape [N, {cols if cols is not None else 'L'}] required")
    return arr, ptr


def dcrf_qp_fw_host(rgb, unaries, Y0, widths, heights, thetas, weights, iters: int, Y=None, compat=None,
                    storage: str = "f16", records: bool = False, stream=None):
    """The QP path from host buffers: features, both lattices, Frank-Wolfe, y back
    in `Y` (a new numpy array unless given; may be Y0).  Returns (Y, records or None)."""
    w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
    h = np.ascontiguousarray(np.asarray(heights, dtype=np.int32))
    rgb, prgb = _host(rgb, "rgb", 3)
    unaries, pphi = _host(unaries, "unaries")
    L = unaries.shape[1]
    Y0, py0 = _host(Y0, "Y0", L)
    if Y is None:
        Y = np.empty(tuple(Y0.shape), dtype=np.float32)
    Y, py = _host(Y, "Y", L)
    n = int((w.astype(np.int64) * h).sum())
    if not (rgb.shape[0] == unaries.shape[0] == Y0.shape[0] == Y.shape[0] == n):
        raise ValueError("rgb, unaries, Y0 and Y must have one row per pixel of the batch")
    batch = len(w)
    rec = (FwRecord * max(1, iters * batch))() if records else None
    cm = _compat(compat, L)
    ta, tb, tg = thetas
    _check(lib().dcrf_qp_fw_host(prgb, pphi, py0, py, w.ctypes.data_as(_P), h.ctypes.data_as(_P), batch, L,
                                 ta, tb, tg, _floats(weights), None if cm is None else cm[1], iters, rec,
                                 STORAGE[storage], _stream(stream)), "dcrf_qp_fw_host")
    if not records:
        return Y, None
    arr = np.array([(r.energy, r.gap, r.alpha, r.A, r.B) for r in rec[:iters * batch]], dtype=np.float64)
    return Y, arr.reshape(iters, batch, 5)


def dcrf_qp_fw_backward(unaries, lattices, weights, Y0, dYT, iters: int, compat=None, need_dy0: bool = False,
                        tape: bool = False, stream=None):
    """(dphi [N, L], dweights [n_kernels] float64, dY0 or None) of <dYT, y^T>;
    with tape=True a fourth item, the recomputed forward's decisions uint8 [iters, N]."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Y0 = _dev(Y0, torch.float32, "Y0", 2)
    dYT = _dev(dYT, torch.float32, "dYT", 2)
    L = unaries.shape[1]
    dphi = torch.empty_like(unaries)
    dy0 = torch.empty_like(Y0) if need_dy0 else None
    dw = np.zeros(len(lattices), dtype=np.float64)
    st = torch.empty((iters, Y0.shape[0]), dtype=torch.uint8, device=Y0.device) if tape else None
    cm = _compat(compat, L)
    _check(lib().dcrf_qp_fw_backward(_ptr(unaries), _handles(lattices), _floats(weights), len(lattices),
                                     None if cm is None else cm[1], L, iters, _ptr(Y0), _ptr(dYT), _ptr(dphi),
                                     _ptr(dy0), dw.ctypes.data_as(_P), _ptr(st), _stream(stream)),
           "dcrf_qp_fw_backward")
    return (dphi, dw, dy0, st) if tape else (dphi, dw, dy0)


def dcrf_dc_cccp(unaries, lattices, weights, Y, outer: int, inner: int, compat=None, storage="f32",
                 energies: bool = True, stream=None):
    """CCCP (generic DC); Y updated in place.  Returns S_QP [outer+1, batch] or None."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Y = _dev(Y, torch.float32, "Y", 2)
    L = unaries.shape[1]
    batch = lattices[0].batch
    qe = np.zeros((outer + 1) * batch, dtype=np.float64) if energies else None
    cm = _compat(compat, L)
    _check(lib().dcrf_dc_cccp(_ptr(unaries), _handles(lattices), _floats(weights), len(lattices),
                              None if cm is None else cm[1], L, outer, inner, _ptr(Y),
                              None if qe is None else qe.ctypes.data_as(_P), STORAGE[storage],
                              _stream(stream)), "dcrf_dc_cccp")
    return None if qe is None else qe.reshape(outer + 1, batch)


def dcrf_dc_cccp_trace(unaries, lattices, weights, Y, outer: int, inner: int, compat=None, storage="f32",
                       stream=None):
    """dcrf_dc_cccp that also returns the decisions: (S_QP [outer+1, batch],
    s_trace uint8 [outer * inner, N] on the device)."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Y = _dev(Y, torch.float32, "Y", 2)
    L = unaries.shape[1]
    batch = lattices[0].batch
    qe = np.zeros((outer + 1) * batch, dtype=np.float64)
    trace = torch.empty((outer * inner, Y.shape[0]), dtype=torch.uint8, device=Y.device)
    cm = _compat(compat, L)
    _check(lib().dcrf_dc_cccp_trace(_ptr(unaries), _handles(lattices), _floats(weights), len(lattices),
                                    None if cm is None else cm[1], L, outer, inner, _ptr(Y), qe.ctypes.data_as(_P),
                                    _ptr(trace), STORAGE[storage], _stream(stream)), "dcrf_dc_cccp_trace")
    return qe.reshape(outer + 1, batch), trace


def dcrf_dc_neg(unaries, lattices, weights, Y, outer: int, inner: int, compat=None, storage="f32",
                 energies: bool = True, stream=None):
    """CCCP for negative semi-definite mu (Section 5.2, Appendix C); Y updated in place.

    Returns S_QP [outer+1, batch] or None.  `inner` is used for a non-Potts mu only.
    """
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Y = _dev(Y, torch.float32, "Y", 2)
    L = unaries.shape[1]
    batch = lattices[0].batch
    qe = np.zeros((outer + 1) * batch, dtype=np.float64) if energies else None
    cm = _compat(compat, L)
    _check(lib().dcrf_dc_neg(_ptr(unaries), _handles(lattices), _floats(weights), len(lattices),
                             None if cm is None else cm[1], L, outer, inner, _ptr(Y),
                             None if qe is None else qe.ctypes.data_as(_P), STORAGE[storage],
                             _stream(stream)), "dcrf_dc_neg")
    return None if qe is None else qe.reshape(outer + 1, batch)


def dcrf_mean_field(unaries, lattices, weights, Q, iters: int, compat=None, storage="f32", energies: bool = True,
                    stream=None):
    """Parallel mean field (the MF baseline); Q updated in place.  Returns S_QP [iters+1, batch] or None."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Q = _dev(Q, torch.float32, "Q", 2)
    L = unaries.shape[1]
    batch = lattices[0].batch
    qe = np.zeros((iters + 1) * batch, dtype=np.float64) if energies else None
    cm = _compat(compat, L)
    _check(lib().dcrf_mean_field(_ptr(unaries), _handles(lattices), _floats(weights), len(lattices),
                                 None if cm is None else cm[1], L, iters, _ptr(Q),
                                 None if qe is None else qe.ctypes.data_as(_P), STORAGE[storage],
                                 _stream(stream)), "dcrf_mean_field")
    return None if qe is None else qe.reshape(iters + 1, batch)


def dcrf_round(Y, onehot: bool = False, stream=None):
    """Most probable label per pixel (int32), and the one-hot rows when asked."""
    Y = _dev(Y, torch.float32, "Y", 2)
    labels = torch.empty(Y.shape[0], dtype=torch.int32, device=Y.device)
    oh = torch.empty_like(Y) if onehot else None
    _check(lib().dcrf_round(_ptr(Y), Y.shape[0], Y.shape[1], _ptr(labels), None if oh is None else _ptr(oh),
                            _stream(stream)), "dcrf_round")
    return (labels, oh) if onehot else labels


def pool_trim():
    """Return the library's unused cached device memory to the driver."""
    _check(lib().dcrf_pool_trim(), "dcrf_pool_trim")


def dcrf_round_kt(Y, phase_labels, phase_thresholds, labels=None, count: bool = True, stream=None):
    """Kleinberg-Tardos rounding with the given phases (host int32 labels, float32
    thresholds in [0, 1)).  Continues from `labels` when given (entries >= 0
    kept, updated in place).  Returns (labels int32 [N], pixels left at -1 or None)."""
    Y = _dev(Y, torch.float32, "Y", 2)
    pl = np.ascontiguousarray(np.asarray(phase_labels, dtype=np.int32))
    pt = np.ascontiguousarray(np.asarray(phase_thresholds, dtype=np.float32))
    if pl.shape != pt.shape or pl.ndim != 1:
        raise ValueError("one threshold per phase label")
    resume = labels is not None
    if resume:
        labels = _dev(labels, torch.int32, "labels", 1)
    else:
        labels = torch.empty(Y.shape[0], dtype=torch.int32, device=Y.device)
    left = np.zeros(1, dtype=np.int64) if count else None
    _check(lib().dcrf_round_kt(_ptr(Y), Y.shape[0], Y.shape[1], len(pl), pl.ctypes.data_as(_P),
                               pt.ctypes.data_as(_P), int(resume), _ptr(labels),
                               None if left is None else left.ctypes.data_as(_P), _stream(stream)),
           "dcrf_round_kt")
    return labels, (None if left is None else int(left[0]))


def dcrf_labelling_energy(unaries, lattices, weights, labels, compat=None, storage="f32", stream=None):
    """E(x) of Eq. 1 per image (host float64 [batch])."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    labels = _dev(labels, torch.int32, "labels", 1)
    L = unaries.shape[1]
    out = np.zeros(lattices[0].batch, dtype=np.float64)
    cm = _compat(compat, L)
    _check(lib().dcrf_labelling_energy(_ptr(unaries), _handles(lattices), _floats(weights), len(lattices),
                                       None if cm is None else cm[1], L, _ptr(labels),
                                       out.ctypes.data_as(_P), STORAGE[storage], _stream(stream)),
           "dcrf_labelling_energy")
    return out


def dcrf_lp_subgrad(unaries, Y, lattices, weights, energy: bool = True, stream=None):
    """LP subgradient G [N, L] and S_LP = <y, G> per image."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Y = _dev(Y, torch.float32, "Y", 2)
    L = unaries.shape[1]
    G = torch.empty_like(Y)
    e = np.zeros(lattices[0].batch, dtype=np.float64) if energy else None
    _check(lib().dcrf_lp_subgrad(_ptr(unaries), _ptr(Y), _handles(lattices), _floats(weights), len(lattices),
                                 L, _ptr(G), None if e is None else e.ctypes.data_as(_P), _stream(stream)),
           "dcrf_lp_subgrad")
    return G, e


def _tree(members, c_t, L):
    """Subtree label sets as uint64 bit masks (from a 0/1 [subtrees][labels] matrix) and float32 weights."""
    m = np.asarray(members)
    if m.ndim != 2 or m.shape[1] != L:
        raise ValueError("members must be [subtrees, L]")
    masks = np.zeros(m.shape[0], dtype=np.uint64)
    for t in range(m.shape[0]):
        for i in np.nonzero(m[t])[0]:
            masks[t] |= np.uint64(1) << np.uint64(i)
    w = np.ascontiguousarray(np.asarray(c_t, dtype=np.float32))
    if w.shape != (m.shape[0],):
        raise ValueError("one weight per subtree")
    return masks, w


def dcrf_lp_subgrad_tree(unaries, Y, lattices, weights, members, c_t, energy: bool = True, stream=None):
    """Tree-metric (r-HST) LP subgradient G [N, L] and objective <y, G> per image (Appendix F)."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Y = _dev(Y, torch.float32, "Y", 2)
    L = unaries.shape[1]
    masks, w = _tree(members, c_t, L)
    G = torch.empty_like(Y)
    e = np.zeros(lattices[0].batch, dtype=np.float64) if energy else None
    _check(lib().dcrf_lp_subgrad_tree(_ptr(unaries), _ptr(Y), _handles(lattices), _floats(weights), len(lattices),
                                      L, len(masks), masks.ctypes.data_as(_P), w.ctypes.data_as(_P), _ptr(G),
                                      None if e is None else e.ctypes.data_as(_P), _stream(stream)),
           "dcrf_lp_subgrad_tree")
    return G, e


def dcrf_lp_solve_tree(unaries, lattices, weights, Y, members, c_t, steps: int, beta0: float = 0.0,
                       energies: bool = True, stream=None):
    """Projected subgradient on the tree-metric LP; Y updated in place (best iterate)."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Y = _dev(Y, torch.float32, "Y", 2)
    L = unaries.shape[1]
    masks, w = _tree(members, c_t, L)
    batch = lattices[0].batch
    e = np.zeros((steps + 1) * batch, dtype=np.float64) if energies else None
    _check(lib().dcrf_lp_solve_tree(_ptr(unaries), _handles(lattices), _floats(weights), len(lattices), L,
                                    len(masks), masks.ctypes.data_as(_P), w.ctypes.data_as(_P), steps,
                                    float(beta0), _ptr(Y), None if e is None else e.ctypes.data_as(_P),
                                    _stream(stream)), "dcrf_lp_solve_tree")
    return None if e is None else e.reshape(steps + 1, batch)


def dcrf_lp_solve(unaries, lattices, weights, Y, steps: int, beta0: float = 0.0, energies: bool = True,
                  stream=None):
    """Projected subgradient on the LP; Y updated in place (best iterate)."""
    unaries = _dev(unaries, torch.float32, "unaries", 2)
    Y = _dev(Y, torch.float32, "Y", 2)
    L = unaries.shape[1]
    batch = lattices[0].batch
    e = np.zeros((steps + 1) * batch, dtype=np.float64) if energies else None
    _check(lib().dcrf_lp_solve(_ptr(unaries), _handles(lattices), _floats(weights), len(lattices), L, steps,
                               float(beta0), _ptr(Y), None if e is None else e.ctypes.data_as(_P),
                               _stream(stream)), "dcrf_lp_solve")
    return None if e is None else e.reshape(steps + 1, batch)


def dcrf_simplex_project(V: torch.Tensor, stream=None) -> torch.Tensor:
    V = _dev(V, torch.float32, "V", 2)
    Y = torch.empty_like(V)
    _check(lib().dcrf_simplex_project(_ptr(V), V.shape[0], V.shape[1], _ptr(Y), _stream(stream)),
           "dcrf_simplex_project")
    return Y


def dcrf_check_lattice_tables(point_vertex, point_weight, neighbours, point_offsets, vertex_offsets, stream=None):
    """Check mode of the lattice tables (device tensors as dcrf_lattice_export
    returns them, host offsets).  Returns the number of failing entries (0 = valid)."""
    pv = _dev(point_vertex, torch.int32, "point_vertex", 2)
    pw = _dev(point_weight, torch.float32, "point_weight", 2)
    nb = _dev(neighbours, torch.int32, "neighbours", 3)
    po = np.ascontiguousarray(np.asarray(point_offsets, dtype=np.int64))
    vo = np.ascontiguousarray(np.asarray(vertex_offsets, dtype=np.int64))
    bad = np.zeros(1, dtype=np.int64)
    st = lib().dcrf_check_lattice_tables(_ptr(pv), _ptr(pw), pv.shape[0], pv.shape[1] - 1, _ptr(nb), nb.shape[0],
                                         po.ctypes.data_as(_P), vo.ctypes.data_as(_P), len(po) - 1,
                                         bad.ctypes.data_as(_P), _stream(stream))
    if st not in (0, -1) or (st == -1 and bad[0] == 0):
        _check(st, "dcrf_check_lattice_tables")
    return int(bad[0])


def dcrf_lattice_validate(lat: Lattice, stream=None) -> int:
    """Check mode on a lattice's own tables: the number of failing entries (0 = valid)."""
    bad = np.zeros(1, dtype=np.int64)
    st = lib().dcrf_lattice_validate(lat.handle, bad.ctypes.data_as(_P), _stream(stream))
    if st not in (0, -1) or (st == -1 and bad[0] == 0):
        _check(st, "dcrf_lattice_validate")
    return int(bad[0])


def dcrf_selftest_bounded_wait(lat: Lattice, polls: int, never_complete: bool, stream=None):
    """Launches the bounded-wait self-test; the outcome lands in lat's status word."""
    _check(lib().dcrf_selftest_bounded_wait(lat.handle, int(polls), 1 if never_complete else 0, _stream(stream)),
           "dcrf_selftest_bounded_wait")


def exported_symbols() -> list[str]:
    return list(_SIGS)


def profile_enable(on: bool = True):
    _check(lib().dcrf_profile_enable(1 if on else 0), "dcrf_profile_enable")
    _check(lib().dcrf_profile_reset(), "dcrf_profile_reset")


def profile_read() -> dict:
    """{kernel name: (launches, milliseconds)} since the last reset (synchronises)."""
    cap = 64
    names = (ctypes.c_char_p * cap)()
    cnt = (_I64 * cap)()
    ms = (_D * cap)()
    k = lib().dcrf_profile_read(names, cnt, ms, cap)
    return {names[i].decode(): (int(cnt[i]), float(ms[i])) for i in range(k)}
