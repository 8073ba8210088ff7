"""ctypes binding of libp3t (the tree side of the P3T scheme on one B300).

Thin Python binding over ``libp3t.so`` (the C ABI declared in
``include/p3t.h``).  It only marshals arguments: device pointers of torch
tensors, the current CUDA stream, and status codes turned into exceptions.
Every step of the computation runs in the library's CUDA kernels; there is no
CPU fallback, and importing without the built library raises.

Conventions: particle vectors are ``(3, n)`` float64 CUDA tensors
(structure of arrays, the caller's particle order), masses ``(n,)`` float64,
accelerations ``(3, n)`` float32.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, fields

import numpy as np

from . import build as _build

__all__ = ["Params", "Context", "P3TError", "kick", "drift", "library_path",
           "launch_count", "FLAG_NO_SYNC"]

FLAG_NO_SYNC = 1  # build without allocation or host synchronisation

_STATUS = {0: "ok", 1: "invalid argument or input", 2: "capacity exceeded",
           3: "CUDA error", 4: "device wait timed out", 5: "call out of order"}


class P3TError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {_STATUS.get(code, 'unknown')} (status {code})")
        self.code = code


def library_path() -> str:
    return _build.LIB


def _load_lib():
    path = _build.LIB
    if not os.path.exists(path):
        if os.environ.get("P3T_AUTOBUILD", "1") == "1":
            _build.build()
        else:
            raise ImportError(f"libp3t.so not built at {path}")
    return C.CDLL(path)


class _CParams(C.Structure):
    _fields_ = [("theta", C.c_double), ("r_out", C.c_double),
                ("gamma", C.c_double), ("eps", C.c_double), ("h", C.c_double),
                ("G", C.c_double), ("n_leaf", C.c_int32),
                ("n_group", C.c_int32), ("flags", C.c_int32),
                ("reserved", C.c_int32)]


class _CStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "n", "n_cells", "n_groups", "n_levels", "list_pc", "list_pp_near",
        "list_pp_far", "int_pc", "int_pp", "int_pp_near", "max_walk_stack",
        "nnz", "herm_block_steps", "herm_particle_steps", "herm_pairs",
        "herm_capped", "herm_components", "herm_max_component",
        "herm_max_block_steps", "need_cells")]


class _CHermite(C.Structure):
    _fields_ = [("eta", C.c_double), ("alpha", C.c_double),
                ("dt_soft", C.c_double), ("log2_soft_over_max", C.c_int32),
                ("kmax", C.c_int32)]


class _CTune(C.Structure):
    _fields_ = [("n_group", C.c_int32), ("n_leaf", C.c_int32),
                ("force_warps", C.c_int32), ("vjp_warps", C.c_int32),
                ("ms", C.c_double), ("err_median", C.c_double),
                ("err_max", C.c_double), ("base_err_median", C.c_double),
                ("base_err_max", C.c_double), ("evaluated", C.c_int32),
                ("rejected", C.c_int32), ("cand_ms", C.c_double * 9),
                ("cand_err_median", C.c_double * 9),
                ("cand_err_max", C.c_double * 9)]


class _CProfile(C.Structure):
    _fields_ = [("build_ms", C.c_double), ("walk_ms", C.c_double),
                ("force_ms", C.c_double), ("ngb_ms", C.c_double),
                ("builds", C.c_int64), ("walks", C.c_int64),
                ("forces", C.c_int64), ("ngbs", C.c_int64),
                ("int_pc", C.c_int64), ("int_pp", C.c_int64),
                ("int_pp_near", C.c_int64), ("vjp_walk_ms", C.c_double),
                ("vjp_walks", C.c_int64), ("build_keys_ms", C.c_double),
                ("build_sort_ms", C.c_double), ("build_split_ms", C.c_double),
                ("build_moments_ms", C.c_double),
                ("build_groups_ms", C.c_double)]


_lib = _load_lib()
_vp = C.c_void_p
_i64 = C.c_int64
_sigs = {
    "p3t_default_params": [_vp],
    "p3t_create": [_vp, _vp],
    "p3t_destroy": [_vp],
    "p3t_set_params": [_vp, _vp],
    "p3t_build_tree": [_vp, _i64, _vp, _vp, _vp],
    "p3t_long_force": [_vp, _vp, _vp, _vp],
    "p3t_neighbours": [_vp, _vp, _vp, _i64, _vp, _vp],
    "p3t_kick": [_i64, _vp, _vp, C.c_double, _vp],
    "p3t_drift": [_i64, _vp, _vp, C.c_double, _vp],
    "p3t_energy": [_vp, _i64, _vp, _vp, _vp, _vp, _vp],
    "p3t_get_stats": [_vp, _vp],
    "p3t_get_order": [_vp, _vp, _vp],
    "p3t_get_root": [_vp, _vp, _vp],
    "p3t_get_cells": [_vp] + [_vp] * 10,
    "p3t_get_groups": [_vp, _vp, _vp, _vp, _vp],
    "p3t_get_lists": [_vp] + [_vp] * 6,
    "p3t_force_lists": [_vp, _vp, _vp, _i64, _vp, _vp],
    "p3t_set_limits": [_vp, _vp],
    "p3t_profile_enable": [_vp, C.c_int],
    "p3t_check": [_vp, _vp],
    "p3t_long_force_vjp": [_vp, _vp, _vp, _vp, _vp],
    "p3t_set_ensemble": [_vp, C.c_int32, _vp, _vp, _vp, _vp],
    "p3t_set_species": [_vp, C.c_int64, C.c_int64, _vp],
    "p3t_autotune": [_vp, _i64, _vp, _vp, _vp, C.c_int, _vp, _vp],
    "p3t_get_profile": [_vp, _vp, C.c_int],
    "p3t_alu_peaks": [_vp, _vp, _vp],
    "p3t_fp64_peaks": [_vp, _vp, _vp, _vp],
    "p3t_hard_force": [_i64, _vp, _vp, _vp, _vp, _vp, C.c_double, C.c_double,
                       C.c_double, C.c_double, _vp, _vp, _vp],
    "p3t_hard_step": [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
}
for _name, _args in _sigs.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.p3t_status_string.argtypes = [C.c_int]
_lib.p3t_status_string.restype = C.c_char_p
_lib.p3t_launch_count.argtypes = []
_lib.p3t_launch_count.restype = C.c_int64


def launch_count() -> int:
    """Kernels launched by libp3t since it was loaded."""
    return int(_lib.p3t_launch_count())


def alu_peaks() -> dict:
    """Measured FP32 FMA (scalar and FP32x2) flop/s and rsqrt/s of the
    current device (p3t_alu_peaks)."""
    v = [C.c_double(), C.c_double(), C.c_double()]
    _check(_lib.p3t_alu_peaks(*[C.byref(x) for x in v]), "p3t_alu_peaks")
    return {"fma_flops": v[0].value, "fma2_flops": v[1].value,
            "rsqrt_ops": v[2].value}


def fp64_peaks() -> dict:
    """Measured FP64 FMA/s and the latencies (SM cycles) of one dependent
    add, division and square root on the current device (p3t_fp64_peaks)."""
    v = [C.c_double() for _ in range(4)]
    _check(_lib.p3t_fp64_peaks(*[C.byref(x) for x in v]), "p3t_fp64_peaks")
    return {"dfma_ops": v[0].value, "add_cycles": v[1].value,
            "div_cycles": v[2].value, "sqrt_cycles": v[3].value}


def _check(code: int, where: str):
    if code != 0:
        raise P3TError(code, where)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t, dtype, shape, name):
    """Device pointer of a contiguous CUDA tensor with the given dtype/shape."""
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    return C.c_void_p(t.data_ptr()) if t.numel() else None


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class Params:
    """Parameters of one context (names after the paper: r_out is r_cut of
    Eq. 12-15, gamma = r_in/r_cut, eps the Plummer softening of Eq. 2, theta
    the opening criterion, h the neighbour radius of Sect. 2.2)."""
    theta: float = 0.4
    r_out: float = 1.0 / 64.0
    gamma: float = 0.1
    eps: float = 0.0
    h: float = 0.0
    G: float = 1.0
    n_leaf: int = 16
    n_group: int = 64
    flags: int = 0

    def _c(self) -> _CParams:
        p = _CParams()
        for f in fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


class Context:
    """One tree-side context on the current CUDA device (libp3t p3t_ctx)."""

    def __init__(self, params: Params | None = None):
        self.params = params or Params()
        self._h = C.c_void_p()
        cp = self.params._c()
        _check(_lib.p3t_create(C.byref(self._h), C.byref(cp)), "p3t_create")
        self.n = 0

    def close(self):
        if self._h:
            _lib.p3t_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: Params):
        cp = params._c()
        _check(_lib.p3t_set_params(self._h, C.byref(cp)), "p3t_set_params")
        self.params = params

    def set_ensemble(self, offsets, r_out=None, eps=None, h=None):
        """Independent clusters: cluster k holds particles
        [offsets[k], offsets[k+1]); optional per-cluster r_out, eps, h."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        nc = off.size - 1
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64)
                for a in (r_out, eps, h)]
        _check(_lib.p3t_set_ensemble(
            self._h, nc, _np_ptr(off) if nc > 0 else None,
            *[None if a is None else _np_ptr(a) for a in arrs]),
            "p3t_set_ensemble")
        self._ens = (off, arrs)  # keep the host arrays alive

    def set_species(self, n, n_bh, r_cut_bh=0.0, eps_bh=0.0, h_bh=0.0,
                    eta_bh=0.03):
        """Two species (p3t_set_species, Sect. 3.2.2): the last n_bh of the
        n particles are black holes with their own cut-off, softening and
        neighbour radius against stars and their own eta; n_bh = 0 turns
        species off."""
        sp = _Species(r_cut_bh, eps_bh, h_bh, eta_bh)
        _check(_lib.p3t_set_species(self._h, int(n), int(n_bh),
                                    C.byref(sp) if n_bh else None),
               "p3t_set_species")

    def autotune(self, pos, mass, w=None, reps=2, stream=None) -> dict:
        """p3t_autotune: n_group x n_leaf, then the walk kernels' warps per
        block, timed on build + force (+ backward with weights w, (3, n)
        float32), keeping only sizes whose force stays within the accuracy
        check against the theta/2 reference.  Returns the p3t_tune record as
        a dict; the context keeps the chosen configuration."""
        import torch
        n = int(mass.shape[0])
        t = _CTune()
        wp = _dptr(w, torch.float32, (3, n), "w") if w is not None else None
        _check(_lib.p3t_autotune(
            self._h, n, _dptr(pos, torch.float64, (3, n), "pos"),
            _dptr(mass, torch.float64, (n,), "mass"), wp, reps, _stream(stream),
            C.byref(t)), "p3t_autotune")
        self.params.n_group, self.params.n_leaf = int(t.n_group), int(t.n_leaf)
        self.n = n
        self.build_id = getattr(self, "build_id", 0) + 1
        out = {}
        for f, ty in _CTune._fields_:
            v = getattr(t, f)
            out[f] = [float(x) for x in v] if f.startswith("cand_") else (
                float(v) if ty is C.c_double else int(v))
        return out

    # ---- hot path ----
    def build_tree(self, pos, mass, stream=None):
        import torch
        n = int(mass.shape[0])
        p = _dptr(pos, torch.float64, (3, n), "pos")
        m = _dptr(mass, torch.float64, (n,), "mass")
        _check(_lib.p3t_build_tree(self._h, n, p, m, _stream(stream)),
               "p3t_build_tree")
        self.n = n
        self.build_id = getattr(self, "build_id", 0) + 1

    def long_force(self, acc=None, pot=None, want_potential=False, stream=None,
                   check=True):
        """Soft acceleration (3, n) float32; with ``want_potential`` also the
        soft potential (n,) float64.  Returns acc or (acc, pot).  With
        ``check`` the stream is synchronised and device-side errors raise."""
        import torch
        n = self.n
        if acc is None:
            acc = torch.empty((3, n), dtype=torch.float32, device="cuda")
        if want_potential and pot is None:
            pot = torch.empty((n,), dtype=torch.float64, device="cuda")
        a = _dptr(acc, torch.float32, (3, n), "acc")
        q = _dptr(pot, torch.float64, (n,), "pot") if pot is not None else None
        _check(_lib.p3t_long_force(self._h, a, q, _stream(stream)),
               "p3t_long_force")
        if check:
            self.check(stream)
        return (acc, pot) if pot is not None else acc

    def long_force_vjp(self, w, grad_pos=None, grad_mass=None, stream=None,
                       check=True):
        """dL/dx (3, n) float64 and dL/dm (n,) float64 of L = sum_i w_i . a_i
        for the current tree (structure and interaction sets held fixed);
        w is (3, n) float32."""
        import torch
        n = self.n
        if grad_pos is None:
            grad_pos = torch.empty((3, n), dtype=torch.float64, device="cuda")
        if grad_mass is None:
            grad_mass = torch.empty((n,), dtype=torch.float64, device="cuda")
        _check(_lib.p3t_long_force_vjp(
            self._h, _dptr(w, torch.float32, (3, n), "w"),
            _dptr(grad_pos, torch.float64, (3, n), "grad_pos"),
            _dptr(grad_mass, torch.float64, (n,), "grad_mass"),
            _stream(stream)), "p3t_long_force_vjp")
        if check:
            self.check(stream)
        return grad_pos, grad_mass

    def hard_step(self, pos, vel, mass, offsets, idx, hp: "HermiteParams",
                  stream=None, check=True):
        """One hard step (p3t_hard_step): isolated particles drift, the others
        are Hermite-integrated over hp.dt_soft under H_hard; pos and vel
        (3, n) float64 are updated in place."""
        import torch
        n = int(pos.shape[1])
        ip, keep = _idx_ptr(idx)
        c = hp._c()
        _check(_lib.p3t_hard_step(
            self._h, n, _dptr(pos, torch.float64, (3, n), "pos"),
            _dptr(vel, torch.float64, (3, n), "vel"),
            _dptr(mass, torch.float64, (n,), "mass"),
            _dptr(offsets, torch.int64, (n + 1,), "offsets"), ip,
            C.byref(c), _stream(stream)), "p3t_hard_step")
        if check:
            self.check(stream)
        else:
            # keep the dummy index buffer alive until the work has run
            self._keep = keep
        return pos, vel

    def check(self, stream=None):
        """Synchronise and raise the first error latched on the device."""
        _check(_lib.p3t_check(self._h, _stream(stream)), "p3t_check")

    def neighbours(self, stream=None):
        """CSR neighbour lists (offsets int64[n+1], idx int32[nnz]) on the
        device, rows in the caller's order, ascending indices."""
        import torch
        n = self.n
        off = torch.empty((n + 1,), dtype=torch.int64, device="cuda")
        need = C.c_int64(0)
        code = _lib.p3t_neighbours(self._h, C.c_void_p(off.data_ptr()), None, 0,
                                   C.byref(need), _stream(stream))
        if code not in (0, 2):
            _check(code, "p3t_neighbours")
        nnz = int(need.value)
        idx = torch.empty((max(nnz, 1),), dtype=torch.int32, device="cuda")
        _check(_lib.p3t_neighbours(self._h, C.c_void_p(off.data_ptr()),
                                   C.c_void_p(idx.data_ptr()), idx.numel(),
                                   C.byref(need), _stream(stream)),
               "p3t_neighbours")
        return off, idx[:nnz]

    def neighbours_into(self, offsets, idx, stream=None, sync=True):
        """Fill caller buffers; returns nnz (or None when sync=False)."""
        import torch
        n = self.n
        o = _dptr(offsets, torch.int64, (n + 1,), "offsets")
        i = C.c_void_p(idx.data_ptr()) if idx.numel() else None
        need = C.c_int64(0)
        _check(_lib.p3t_neighbours(self._h, o, i, idx.numel(),
                                   C.byref(need) if sync else None,
                                   _stream(stream)), "p3t_neighbours")
        return int(need.value) if sync else None

    def energy(self, mass, vel, pot=None, out=None, stream=None):
        import torch
        n = int(mass.shape[0])
        if out is None:
            out = torch.zeros((2,), dtype=torch.float64, device="cuda")
        _check(_lib.p3t_energy(
            self._h, n, _dptr(mass, torch.float64, (n,), "mass"),
            _dptr(vel, torch.float64, (3, n), "vel"),
            _dptr(pot, torch.float64, (n,), "pot") if pot is not None else None,
            _dptr(out, torch.float64, (2,), "out"), _stream(stream)),
            "p3t_energy")
        return out

    # ---- profiling ----
    def profile_enable(self, on: bool = True):
        _check(_lib.p3t_profile_enable(self._h, 1 if on else 0),
               "p3t_profile_enable")

    def profile(self, reset: bool = True) -> dict:
        p = _CProfile()
        _check(_lib.p3t_get_profile(self._h, C.byref(p), 1 if reset else 0),
               "p3t_get_profile")
        return {f: (float(getattr(p, f)) if t is C.c_double else int(getattr(p, f)))
                for f, t in _CProfile._fields_}

    # ---- inspection ----
    def stats(self) -> dict:
        s = _CStats()
        _check(_lib.p3t_get_stats(self._h, C.byref(s)), "p3t_get_stats")
        return {f: int(getattr(s, f)) for f, _ in _CStats._fields_}

    def order(self):
        n = self.n
        key = np.zeros(n, np.uint64)
        order = np.zeros(n, np.int32)
        _check(_lib.p3t_get_order(self._h, _np_ptr(key), _np_ptr(order)),
               "p3t_get_order")
        return key, order

    def root(self):
        lo = np.zeros(3)
        size = np.zeros(1)
        _check(_lib.p3t_get_root(self._h, _np_ptr(lo), _np_ptr(size)),
               "p3t_get_root")
        return lo, float(size[0])

    def cells(self) -> dict:
        c = self.stats()["n_cells"]
        out = dict(level=np.zeros(c, np.int32), first=np.zeros(c, np.int32),
                   count=np.zeros(c, np.int32), child=np.zeros(c, np.int32),
                   nchild=np.zeros(c, np.int32), M=np.zeros(c),
                   com=np.zeros((c, 3)), Q=np.zeros((c, 6)),
                   fmin=np.zeros((c, 3), np.float32),
                   fmax=np.zeros((c, 3), np.float32))
        if c:
            _check(_lib.p3t_get_cells(self._h, *[_np_ptr(out[k]) for k in (
                "level", "first", "count", "child", "nchild", "M", "com", "Q",
                "fmin", "fmax")]), "p3t_get_cells")
        return out

    def groups(self) -> dict:
        g = self.stats()["n_groups"]
        out = dict(first=np.zeros(g, np.int32), count=np.zeros(g, np.int32),
                   fmin=np.zeros((g, 3), np.float32),
                   fmax=np.zeros((g, 3), np.float32))
        if g:
            _check(_lib.p3t_get_groups(self._h, *[_np_ptr(out[k]) for k in (
                "first", "count", "fmin", "fmax")]), "p3t_get_groups")
        return out

    def lists(self) -> dict:
        """Interaction lists (CSR per group) from the inspection walk."""
        g = self.stats()["n_groups"]
        offs = {k: np.zeros(g + 1, np.int64) for k in ("pc_off", "ppn_off", "ppf_off")}
        if g == 0:
            return dict(**offs, pc=np.zeros(0, np.int32), ppn=np.zeros(0, np.int32),
                        ppf=np.zeros(0, np.int32))
        _check(_lib.p3t_get_lists(self._h, _np_ptr(offs["pc_off"]), None,
                                  _np_ptr(offs["ppn_off"]), None,
                                  _np_ptr(offs["ppf_off"]), None), "p3t_get_lists")
        out = dict(offs)
        for k in ("pc", "ppn", "ppf"):
            out[k] = np.zeros(max(int(offs[k + "_off"][-1]), 1), np.int32)
        _check(_lib.p3t_get_lists(self._h, *[_np_ptr(out[k]) for k in (
            "pc_off", "pc", "ppn_off", "ppn", "ppf_off", "ppf")]), "p3t_get_lists")
        for k in ("pc", "ppn", "ppf"):
            out[k] = out[k][: int(offs[k + "_off"][-1])]
        return out


    def set_limits(self, walk_iters=0, uf_rounds=0, block_steps=0, max_cells=0):
        """Bounds of the kernels' loops and waits and of the cells a build may
        allocate (p3t_set_limits; 0 = the default)."""
        lim = (C.c_int64 * 4)(walk_iters, uf_rounds, block_steps, max_cells)
        _check(_lib.p3t_set_limits(self._h, lim), "p3t_set_limits")

    def force_lists(self, stream=None) -> dict:
        """The sources the fused walk + force kernel evaluated, per group, as
        recorded by the kernel itself (p3t_force_lists): sorted arrays of
        cell ids ("pc"), near-leaf and far-leaf sorted particle ids ("ppn",
        "ppf") in CSR per group (numbering of groups() and cells())."""
        import torch
        n = self.stats()["n"]
        acc = torch.empty((3, max(n, 1)), dtype=torch.float32, device="cuda")
        cnt = C.c_int64(0)
        cap = 1 << 16
        for _ in range(2):
            rec = torch.empty((cap,), dtype=torch.int64, device="cuda")
            code = _lib.p3t_force_lists(self._h, _vp(acc.data_ptr()),
                                        _vp(rec.data_ptr()), cap,
                                        C.byref(cnt), _stream(stream))
            if code != 2:
                break
            cap = cnt.value
        _check(code, "p3t_force_lists")
        r = rec[: cnt.value].cpu().numpy()
        g = (r >> 33).astype(np.int64)
        kind = (r >> 31) & 3
        ident = (r & ((1 << 31) - 1)).astype(np.int64)
        ng = self.stats()["n_groups"]
        out = {}
        for k, name in enumerate(("pc", "ppn", "ppf")):
            sel = kind == k
            o = np.lexsort((ident[sel], g[sel]))
            gs, ids = g[sel][o], ident[sel][o]
            out[name + "_off"] = np.searchsorted(gs, np.arange(ng + 1))
            out[name] = ids
        return out


class _Species(C.Structure):
    _fields_ = [("r_cut_bh", C.c_double), ("eps_bh", C.c_double),
                ("h_bh", C.c_double), ("eta_bh", C.c_double)]


@dataclass
class HermiteParams:
    """Hard-part integration (p3t_hermite_params): eta and alpha of
    Eq. 18-20, the soft step, dt_max = dt_soft 2^-log2_soft_over_max
    and the finest level kmax."""
    dt_soft: float
    eta: float = 0.1
    alpha: float = 0.1
    log2_soft_over_max: int = 2
    kmax: int = 30

    def _c(self):
        return _CHermite(self.eta, self.alpha, self.dt_soft,
                         self.log2_soft_over_max, self.kmax)


def _idx_ptr(idx):
    """idx may be empty (no neighbour anywhere): pass a one-element dummy,
    never read since every row is then empty."""
    import torch
    if not isinstance(idx, torch.Tensor) or not idx.is_cuda or idx.dtype != torch.int32:
        raise TypeError("idx: expected a CUDA int32 tensor")
    if idx.dim() != 1 or not idx.is_contiguous():
        raise ValueError("idx: expected a contiguous 1-D tensor")
    if idx.numel() == 0:
        idx = torch.zeros((1,), dtype=torch.int32, device=idx.device)
    return C.c_void_p(idx.data_ptr()), idx


def hard_force(pos, vel, mass, offsets, idx, *, r_cut, G=1.0, eps=0.0,
               gamma=0.1, acc=None, jerk=None, stream=None):
    """Hard acceleration and jerk (3, n) float64 of every particle from its
    neighbour row (p3t_hard_force)."""
    import torch
    n = int(pos.shape[1])
    if acc is None:
        acc = torch.empty((3, n), dtype=torch.float64, device="cuda")
    if jerk is None:
        jerk = torch.empty((3, n), dtype=torch.float64, device="cuda")
    ip, keep = _idx_ptr(idx)
    _check(_lib.p3t_hard_force(
        n, _dptr(pos, torch.float64, (3, n), "pos"),
        _dptr(vel, torch.float64, (3, n), "vel"),
        _dptr(mass, torch.float64, (n,), "mass"),
        _dptr(offsets, torch.int64, (n + 1,), "offsets"), ip, float(G),
        float(eps), float(r_cut), float(gamma),
        _dptr(acc, torch.float64, (3, n), "acc"),
        _dptr(jerk, torch.float64, (3, n), "jerk"), _stream(stream)),
        "p3t_hard_force")
    del keep
    return acc, jerk


def kick(vel, acc, dt, stream=None):
    """v <- v + dt * a in place (FP64; Eq. 11 / Sect. 2.2)."""
    import torch
    n = int(vel.shape[1])
    _check(_lib.p3t_kick(n, _dptr(vel, torch.float64, (3, n), "vel"),
                         _dptr(acc, torch.float32, (3, n), "acc"), float(dt),
                         _stream(stream)), "p3t_kick")
    return vel


def drift(pos, vel, dt, stream=None):
    """x <- x + dt * v in place (FP64; Sect. 2.2 step 5)."""
    import torch
    n = int(pos.shape[1])
    _check(_lib.p3t_drift(n, _dptr(pos, torch.float64, (3, n), "pos"),
                          _dptr(vel, torch.float64, (3, n), "vel"), float(dt),
                          _stream(stream)), "p3t_drift")
    return pos
