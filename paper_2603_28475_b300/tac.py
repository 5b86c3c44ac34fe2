"""Thin Python binding of the C ABI in include/tac.h (ctypes + torch tensors).

Only argument marshalling lives here: every step of the solve runs in the
CUDA kernels of ``libtac.so``. Device memory and streams come from PyTorch.
Importing this module without a built library raises immediately, and every
call needs a CUDA device; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtac.so")

TAC_OK = 0
PAD_STATUS = {0: "converged", 1: "maxiter", 2: "nonfinite", 3: "linesearch", 4: "pair_overflow"}

SYMBOLS = ("tac_create_batch", "tac_destroy_batch", "tac_reset", "tac_set_indenter", "tac_step", "tac_markers",
           "tac_adjoint", "tac_adjoint_frame", "tac_set_frame",
           "tac_get_state", "tac_set_state", "tac_set_params", "tac_get_params", "tac_broadphase",
           "tac_broadphase_static",
           "tac_debug_eval", "tac_stats",
           "tac_pad_norms", "tac_sizes", "tac_marker_map", "tac_mesh_info", "tac_last_error",
           "tac_set_block_shape", "tac_autotune_block_shape")


class PadDesc(ctypes.Structure):
    _fields_ = [("n_verts", ctypes.c_int), ("n_tets", ctypes.c_int), ("n_fixed", ctypes.c_int),
                ("n_markers", ctypes.c_int), ("rest_xyz", ctypes.c_void_p), ("tets", ctypes.c_void_p),
                ("fixed_idx", ctypes.c_void_p), ("marker_xy", ctypes.c_void_p)]


class IndenterDesc(ctypes.Structure):
    _fields_ = [("n_verts", ctypes.c_int), ("n_tris", ctypes.c_int), ("verts", ctypes.c_void_p),
                ("tris", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("E", ctypes.c_float), ("nu", ctypes.c_float), ("rho", ctypes.c_float), ("h", ctypes.c_float),
                ("dhat", ctypes.c_float), ("kappa", ctypes.c_float), ("mu_f", ctypes.c_float),
                ("eps_v", ctypes.c_float), ("tol_rel_grad", ctypes.c_float), ("tol_advance", ctypes.c_float),
                ("max_iter", ctypes.c_int), ("precond_mode", ctypes.c_int), ("step_mode", ctypes.c_int),
                ("marker_mode", ctypes.c_int), ("precision_mode", ctypes.c_int), ("floor_ulps", ctypes.c_float)]


class Options(ctypes.Structure):
    _fields_ = [("pair_capacity", ctypes.c_int), ("share_meshes", ctypes.c_int), ("no_dm_table", ctypes.c_int)]


def load_library(path=_LIB_PATH):
    """Load libtac.so and declare the C signatures."""
    if not os.path.exists(path):
        raise ImportError(f"libtac.so not built ({path}); run python -m paper_2603_28475_b300.build")
    lib = ctypes.CDLL(path)
    vp, i, f, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
    sig = {
        "tac_create_batch": [ctypes.POINTER(PadDesc), ctypes.POINTER(Params), i, ctypes.POINTER(IndenterDesc), i, i,
                             ctypes.POINTER(Options), vp, ctypes.POINTER(vp)],
        "tac_destroy_batch": [vp],
        "tac_reset": [vp, vp, vp],
        "tac_set_indenter": [vp, vp, vp, vp],
        "tac_step": [vp, vp, vp, vp],
        "tac_markers": [vp, vp, vp],
        "tac_adjoint": [vp, vp, vp, vp, vp, i, f, vp],
        "tac_adjoint_frame": [vp, vp, vp, vp, vp, vp, vp, vp, i, f, i, vp],
        "tac_set_frame": [vp, vp, vp, vp, vp, vp, vp],
        "tac_get_state": [vp, vp, vp, vp],
        "tac_set_state": [vp, vp, vp, vp],
        "tac_set_params": [vp, ctypes.POINTER(Params), i],
        "tac_get_params": [vp, ctypes.POINTER(Params), i],
        "tac_broadphase": [vp, i, vp, vp, d, vp, i, vp, vp],
        "tac_broadphase_static": [vp, vp, i, vp, i, vp, i, vp, i, vp, i, vp, i, d, vp, i, vp, vp],
        "tac_debug_eval": [vp, vp, vp, f, vp, vp, vp, vp],
        "tac_stats": [vp, vp, vp],
        "tac_pad_norms": [vp, vp, vp],
        "tac_sizes": [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)],
        "tac_set_block_shape": [vp, i],
        "tac_autotune_block_shape": [vp, vp, i, ctypes.POINTER(i), vp, vp],
        "tac_marker_map": [ctypes.POINTER(PadDesc), i, vp, vp],
        "tac_mesh_info": [ctypes.POINTER(PadDesc), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                          ctypes.POINTER(d), ctypes.POINTER(i), ctypes.POINTER(i)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.tac_last_error.argtypes = []
    lib.tac_last_error.restype = ctypes.c_char_p
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class TacError(RuntimeError):
    pass


def _check(rc):
    if rc != TAC_OK:
        raise TacError(f"tac error {rc}: {lib().tac_last_error().decode()}")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_params(mat, tol=1e-6, tol_advance=1e-2, max_iter=10000, precond=0, kappa=0.0, eps_v=0.0, step=0, marker=0,
                precision=0, floor_ulps=0.0):
    """tac_params of one pad. precond: 0 block Jacobi, 1 scalar Jacobi;
    step: 0 bounded (CCD + Armijo), 1 Eq. (step_size) as printed; marker: 0
    barycentric, 1 kNN inverse distance; precision: 0 the float32/float64
    split, 1 the plain FP32 form; floor_ulps: the float32 resolution floor
    of the stopping target in ulps of the largest corner force (0: 256)."""
    return Params(E=mat.E, nu=mat.nu, rho=mat.rho, h=mat.h, dhat=mat.dhat, kappa=kappa, mu_f=mat.mu_f,
                  eps_v=eps_v, tol_rel_grad=tol, tol_advance=tol_advance, max_iter=max_iter, precond_mode=precond,
                  step_mode=step, marker_mode=marker, precision_mode=precision, floor_ulps=floor_ulps)


def _host_desc(pad):
    arrs = (np.ascontiguousarray(pad.rest, dtype=np.float32), np.ascontiguousarray(pad.tets, dtype=np.int32),
            np.ascontiguousarray(pad.fixed, dtype=np.int32), np.ascontiguousarray(pad.markers, dtype=np.float32))
    rest, tets, fixed, mk = arrs
    d = PadDesc(rest.shape[0], tets.shape[0], fixed.shape[0], mk.shape[0], rest.ctypes.data, tets.ctypes.data,
                fixed.ctypes.data if fixed.size else 0, mk.ctypes.data if mk.size else 0)
    return d, arrs


def mesh_info(pad):
    """Host-side layout of one pad's mesh: dict(patches, colours, dm_types,
    dm_dev, rounds, conflicts) (dm_types 0: per-tet Dm^-1; dm_dev: largest
    relative deviation of a tet's Dm^-1 from its table class; rounds: warp
    rounds of a scatter pass; conflicts: vertices shared within a colour
    class, 0 for a valid layout)."""
    d, keep = _host_desc(pad)
    a, b, c, e = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    r, k = ctypes.c_int(), ctypes.c_int()
    _check(lib().tac_mesh_info(ctypes.byref(d), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(e),
                               ctypes.byref(r), ctypes.byref(k)))
    del keep
    return {"patches": a.value, "colours": b.value, "dm_types": c.value, "dm_dev": e.value, "rounds": r.value,
            "conflicts": k.value}


def marker_map(pad, marker_mode=0):
    """The library's marker map of one pad (host only): (ids [M, 4] input
    vertex ids, weights [M, 4] float32)."""
    d, (rest, tets, fixed, mk) = _host_desc(pad)
    ids = np.zeros((mk.shape[0], 4), dtype=np.int32)
    w = np.zeros((mk.shape[0], 4), dtype=np.float32)
    _check(lib().tac_marker_map(ctypes.byref(d), int(marker_mode), ids.ctypes.data, w.ctypes.data))
    return ids, w


class TacBatch:
    """A batch of gel pads on the current CUDA device.

    ``pads``: list of objects with rest/tets/fixed/markers arrays (one per
    pad; pads that share the same numpy arrays share device mesh data);
    ``params``: list of ``Params``; ``indenters``: list of objects with
    verts/tris (one per environment)."""

    def __init__(self, pads, params, indenters, pads_per_env=1, pair_capacity=0, share_meshes=True, stream=None,
                 dm_table=True):
        if not torch.cuda.is_available():
            raise TacError("TacBatch needs a CUDA device")
        self._keep = []
        n = len(pads)
        pd = (PadDesc * n)()
        for k, p in enumerate(pads):
            rest = np.ascontiguousarray(p.rest, dtype=np.float32)
            tets = np.ascontiguousarray(p.tets, dtype=np.int32)
            fixed = np.ascontiguousarray(p.fixed, dtype=np.int32)
            mk = np.ascontiguousarray(p.markers, dtype=np.float32)
            # keep identical host arrays identical so that the library can share them
            key = id(p)
            cached = getattr(p, "_tac_cache", None)
            if cached is None:
                cached = (rest, tets, fixed, mk)
                try:
                    p._tac_cache = cached
                except AttributeError:
                    self._keep.append(cached)
            rest, tets, fixed, mk = cached
            self._keep.append(cached)
            pd[k] = PadDesc(rest.shape[0], tets.shape[0], fixed.shape[0], mk.shape[0], rest.ctypes.data,
                            tets.ctypes.data, fixed.ctypes.data if fixed.size else 0, mk.ctypes.data if mk.size else 0)
            del key
        ne = len(indenters)
        idesc = (IndenterDesc * ne)()
        for e, ind in enumerate(indenters):
            cached = getattr(ind, "_tac_cache", None)
            if cached is None:
                cached = (np.ascontiguousarray(ind.verts, dtype=np.float32), np.ascontiguousarray(ind.tris, dtype=np.int32))
                try:
                    ind._tac_cache = cached
                except AttributeError:
                    pass
            self._keep.append(cached)
            idesc[e] = IndenterDesc(cached[0].shape[0], cached[1].shape[0], cached[0].ctypes.data, cached[1].ctypes.data)
        prm = (Params * n)(*params)
        opts = Options(pair_capacity, 1 if share_meshes else 0, 0 if dm_table else 1)
        h = ctypes.c_void_p()
        _check(lib().tac_create_batch(pd, prm, n, idesc, ne, pads_per_env, ctypes.byref(opts), _stream(stream),
                                      ctypes.byref(h)))
        self._h = h
        self.n_pads = n
        tv, tm, cap, gr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().tac_sizes(h, ctypes.byref(tv), ctypes.byref(tm), ctypes.byref(cap), ctypes.byref(gr)))
        self.total_verts, self.total_markers, self.pair_capacity = tv.value, tm.value, cap.value
        self.grid_ctas = gr.value
        self.vert_offsets = np.cumsum([0] + [int(np.asarray(p.rest).shape[0]) for p in pads])
        self.marker_offsets = np.cumsum([0] + [int(np.asarray(p.markers).shape[0]) for p in pads])
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            lib().tac_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f32(self, a):
        t = torch.as_tensor(a, dtype=torch.float32, device=self.device)
        return t.contiguous()

    def reset(self, poses, stream=None):
        p = self._f32(poses).reshape(self.n_pads, 6)
        _check(lib().tac_reset(self._h, _ptr(p), _stream(stream)))
        self._hold = p

    def set_indenter(self, poses=None, twists=None, stream=None):
        p = self._f32(poses).reshape(self.n_pads, 6) if poses is not None else None
        w = self._f32(twists).reshape(self.n_pads, 6) if twists is not None else None
        _check(lib().tac_set_indenter(self._h, _ptr(p), _ptr(w), _stream(stream)))
        self._hold = (p, w)

    def step(self, status=None, iters=None, stream=None):
        status = status if status is not None else torch.empty(self.n_pads, dtype=torch.int32, device=self.device)
        iters = iters if iters is not None else torch.empty(self.n_pads, dtype=torch.int32, device=self.device)
        _check(lib().tac_step(self._h, _ptr(status), _ptr(iters), _stream(stream)))
        return status, iters

    def set_block_shape(self, threads):
        """tac_set_block_shape: 256 or 512 threads per pad's CTA."""
        _check(lib().tac_set_block_shape(self._h, int(threads)))
        self._sync_grid()

    def autotune_block_shape(self, poses, reps=1, stream=None):
        """tac_autotune_block_shape toward the next frame's poses: returns
        (chosen threads, [mean ms of the 256- and 512-thread solves])."""
        p = self._f32(poses).reshape(self.n_pads, 6)
        th = ctypes.c_int()
        ms = (ctypes.c_float * 2)()
        _check(lib().tac_autotune_block_shape(self._h, _ptr(p), int(reps), ctypes.byref(th), ms, _stream(stream)))
        self._sync_grid()
        return th.value, [float(ms[0]), float(ms[1])]

    def _sync_grid(self):
        gr = ctypes.c_int()
        _check(lib().tac_sizes(self._h, None, None, None, ctypes.byref(gr)))
        self.grid_ctas = gr.value

    def markers(self, out=None, stream=None):
        out = out if out is not None else torch.empty(self.total_markers, 2, dtype=torch.float32, device=self.device)
        _check(lib().tac_markers(self._h, _ptr(out), _stream(stream)))
        return out

    def adjoint(self, dL_dmarkers, max_iter=4000, tol=1e-6, stream=None):
        """dL/dtheta [n_pads, 9] (Lame lambda, Lame mu, mu_f, rotation vector,
        translation) of the last frame for dL/d(markers); also the PCG status
        and iterations per pad."""
        g = self._f32(dL_dmarkers).reshape(self.total_markers, 2)
        out = torch.empty(self.n_pads, 9, dtype=torch.float64, device=self.device)
        st = torch.empty(self.n_pads, dtype=torch.int32, device=self.device)
        it = torch.empty(self.n_pads, dtype=torch.int32, device=self.device)
        _check(lib().tac_adjoint(self._h, _ptr(g), _ptr(out), _ptr(st), _ptr(it), int(max_iter), float(tol),
                                 _stream(stream)))
        self._hold = g
        return out, st, it

    def adjoint_frame(self, dL_dmarkers=None, dL_dx=None, max_iter=4000, tol=1e-6, relag=False, stream=None):
        """Adjoint of the last frame for a reverse sweep (tac_adjoint_frame):
        returns dL/dtheta [n_pads, 15] (Lame lambda, Lame mu, mu_f, end pose
        rotation vector and translation, start pose rotation vector and
        translation), dL/dx^t and dL/dv^t [total_verts, 3] (caller order),
        and the PCG status and iterations per pad. dL_dmarkers [total_markers,
        2] and dL_dx [total_verts, 3] (gradient of the end positions beyond
        the markers) may be None. relag differentiates the frame's friction
        lag as a function of its start state and start pose (lag_mode 1)."""
        gm = None if dL_dmarkers is None else self._f32(dL_dmarkers).reshape(self.total_markers, 2)
        gx = None if dL_dx is None else self._f32(dL_dx).reshape(self.total_verts, 3)
        out = torch.empty(self.n_pads, 15, dtype=torch.float64, device=self.device)
        dx0 = torch.empty(self.total_verts, 3, dtype=torch.float32, device=self.device)
        dv0 = torch.empty_like(dx0)
        st = torch.empty(self.n_pads, dtype=torch.int32, device=self.device)
        it = torch.empty(self.n_pads, dtype=torch.int32, device=self.device)
        _check(lib().tac_adjoint_frame(self._h, None if gm is None else _ptr(gm), None if gx is None else _ptr(gx),
                                       _ptr(out), _ptr(dx0), _ptr(dv0), _ptr(st), _ptr(it), int(max_iter),
                                       float(tol), 1 if relag else 0, _stream(stream)))
        self._hold = (gm, gx)
        return out, dx0, dv0, st, it

    def set_frame(self, x0, v0, pose_start, x1, pose_end, stream=None):
        """Install a solved frame for the adjoint without re-solving it
        (tac_set_frame): start state x0, v0 and end positions x1
        [total_verts, 3], poses [n_pads, 6]."""
        a = [self._f32(t).reshape(-1, 3) for t in (x0, v0, x1)]
        ps = self._f32(pose_start).reshape(self.n_pads, 6)
        pe = self._f32(pose_end).reshape(self.n_pads, 6)
        _check(lib().tac_set_frame(self._h, _ptr(a[0]), _ptr(a[1]), _ptr(ps), _ptr(a[2]), _ptr(pe),
                                   _stream(stream)))
        self._hold = (a, ps, pe)

    def get_state(self, stream=None):
        x = torch.empty(self.total_verts, 3, dtype=torch.float32, device=self.device)
        v = torch.empty_like(x)
        _check(lib().tac_get_state(self._h, _ptr(x), _ptr(v), _stream(stream)))
        return x, v

    def set_state(self, x, v, stream=None):
        x, v = self._f32(x).reshape(-1, 3), self._f32(v).reshape(-1, 3)
        _check(lib().tac_set_state(self._h, _ptr(x), _ptr(v), _stream(stream)))
        self._hold = (x, v)

    def set_params(self, params):
        prm = (Params * self.n_pads)(*params)
        _check(lib().tac_set_params(self._h, prm, self.n_pads))

    def get_params(self):
        prm = (Params * self.n_pads)()
        _check(lib().tac_get_params(self._h, prm, self.n_pads))
        return list(prm)

    def broadphase(self, pad, x, y, r, capacity=1 << 16, stream=None):
        x, y = self._f32(x).reshape(-1, 3), self._f32(y).reshape(-1, 3)
        out = torch.zeros(capacity, 3, dtype=torch.int32, device=self.device)
        cnt = torch.zeros(1, dtype=torch.int32, device=self.device)
        _check(lib().tac_broadphase(self._h, pad, _ptr(x), _ptr(y), float(r), _ptr(out), capacity, _ptr(cnt),
                                    _stream(stream)))
        n = int(cnt.item())
        return out[:min(n, capacity)], n

    def debug_eval(self, u, p, alpha, stream=None):
        u, p = self._f32(u).reshape(-1, 3), self._f32(p).reshape(-1, 3)
        g = torch.empty(self.total_verts, 3, dtype=torch.float32, device=self.device)
        k = torch.empty(self.total_verts, 6, dtype=torch.float32, device=self.device)
        sc = torch.empty(self.n_pads, 8, dtype=torch.float64, device=self.device)
        _check(lib().tac_debug_eval(self._h, _ptr(u), _ptr(p), float(alpha), _ptr(g), _ptr(k), _ptr(sc),
                                    _stream(stream)))
        return g, k, sc

    def norms(self, stream=None):
        out = torch.empty(self.n_pads, 4, dtype=torch.float64, device=self.device)
        _check(lib().tac_pad_norms(self._h, _ptr(out), _stream(stream)))
        return out

    def stats(self, stream=None):
        out = torch.empty(self.n_pads, 16, dtype=torch.int64, device=self.device)
        _check(lib().tac_stats(self._h, _ptr(out), _stream(stream)))
        return out


def broadphase_static(x, surf_verts, surf_tris, surf_edges, y, ind_tris, ind_edges, r, capacity=1 << 16,
                      stream=None):
    """Allocation-free candidate search (tac_broadphase_static): every array
    is a caller-owned CUDA tensor; the call allocates nothing itself. The
    output tensors are created here by torch, outside the library."""
    dev = x.device
    i32 = lambda a: torch.as_tensor(a, dtype=torch.int32, device=dev).contiguous()
    f32 = lambda a: torch.as_tensor(a, dtype=torch.float32, device=dev).contiguous()
    x, y = f32(x).reshape(-1, 3), f32(y).reshape(-1, 3)
    sv, st, se = i32(surf_verts).reshape(-1), i32(surf_tris).reshape(-1, 3), i32(surf_edges).reshape(-1, 2)
    it, ie = i32(ind_tris).reshape(-1, 3), i32(ind_edges).reshape(-1, 2)
    out = torch.zeros(capacity, 3, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(lib().tac_broadphase_static(_ptr(x), _ptr(sv), sv.numel(), _ptr(st), st.shape[0], _ptr(se), se.shape[0],
                                       _ptr(y), y.shape[0], _ptr(it), it.shape[0], _ptr(ie), ie.shape[0], float(r),
                                       _ptr(out), capacity, _ptr(cnt), _stream(stream)))
    n = int(cnt.item())
    return out[:min(n, capacity)], n


def batch_from_workload(w, tol=1e-6, tol_advance=1e-2, max_iter=10000, precond=0, pair_capacity=0,
                        share_meshes=True, stream=None, step=0, marker=0, dm_table=True, precision=0,
                        floor_ulps=0.0):
    params = [make_params(m, tol=tol, tol_advance=tol_advance, max_iter=max_iter, precond=precond, step=step,
                          marker=marker, precision=precision, floor_ulps=floor_ulps) for m in w.materials]
    return TacBatch(w.pads, params, w.indenters, w.pads_per_env, pair_capacity=pair_capacity,
                    share_meshes=share_meshes, stream=stream, dm_table=dm_table)
