"""FP64 CPU oracle for the tree side of the P3T scheme (arXiv:1506.04553).

TEST INFRASTRUCTURE ONLY: the independent reference that the CUDA library is
checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library never does, and it
shares no code with the CUDA path.  The arithmetic lives in ``p3t_oracle.c``
(plain C, FP64, compiled with ``-ffp-contract=off``); this module builds that
file with gcc on first use and wraps it with ctypes.

Functions and the passages they follow:

* ``K``, ``W``, ``W_inner_slope`` -- Eq. 12-17 (Sect. 2.1); W uses G with its
  numerator's sign reversed, the reading under which Eq. 9 holds.
* ``direct`` -- Eq. 7-9 with the softened distance of Eq. 2-3 (soft, hard
  and Newtonian weights) and the pair potentials of Eq. 5-6.
* ``Tree`` -- the Barnes-Hut tree to quadrupole order of Sect. 2.2: Morton
  keys, octree, moments, groups, opening test, interaction lists, forces.
* ``neighbours`` -- the per-particle list of particles within h (Sect. 2.2).
* ``kick`` / ``drift`` -- the leapfrog pieces of Eq. 11 and Sect. 2.2.
* ``direct_vjp`` / ``Tree.vjp`` -- gradients of sum_i w_i . a_i (no
  counterpart in the paper; derived from Eq. 8 and the quadrupole expansion).

Parity status of each function (what pins it) is listed in the test files
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "p3t_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_THREADS = os.cpu_count() or 1


def build(force: bool = False) -> str:
    """Compile p3t_oracle.c into a shared library (gcc, FP64, no implicit
    FMA contraction; where the hard part fuses a multiply-add it calls fma()
    explicitly)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            _declare(lib)
            _lib = lib
    return _lib


_d = C.c_double
_i64 = C.c_int64
_i32 = C.c_int32
_p = C.c_void_p


def _declare(lib):
    lib.orc_K.restype = _d
    lib.orc_K.argtypes = [_d]
    lib.orc_dKdx.restype = _d
    lib.orc_dKdx.argtypes = [_d]
    lib.orc_K_of_s.restype = _d
    lib.orc_K_of_s.argtypes = [_d, _d, _d]
    lib.orc_W.restype = _d
    lib.orc_W.argtypes = [_d, _d]
    lib.orc_W_inner_slope.restype = _d
    lib.orc_W_inner_slope.argtypes = [_d]
    lib.orc_direct.restype = None
    lib.orc_direct.argtypes = [_i64, _p, _p, _d, _d, _d, _d, C.c_int, _p, _i64,
                               _p, _p, C.c_int]
    lib.orc_neighbours_count.restype = None
    lib.orc_neighbours_count.argtypes = [_i64, _p, _d, _p, _i64, _p, C.c_int]
    lib.orc_neighbours_fill.restype = None
    lib.orc_neighbours_fill.argtypes = [_i64, _p, _d, _p, _i64, _p, _p, _p,
                                        C.c_int]
    lib.orc_is_neighbour.restype = C.c_int
    lib.orc_is_neighbour.argtypes = [_p, _p, _d]
    lib.orc_kick.restype = None
    lib.orc_kick.argtypes = [_i64, _p, _p, _d]
    lib.orc_drift.restype = None
    lib.orc_drift.argtypes = [_i64, _p, _p, _d]
    lib.orc_morton_key.restype = C.c_uint64
    lib.orc_morton_key.argtypes = [_d, _d, _d, _p, _d]
    lib.orc_root_box.restype = None
    lib.orc_root_box.argtypes = [_i64, _p, _p, _p]
    lib.orc_tree_build.restype = _p
    lib.orc_tree_build.argtypes = [_i64, _p, _p, C.c_int, C.c_int]
    lib.orc_tree_free.restype = None
    lib.orc_tree_free.argtypes = [_p]
    for f in ("orc_tree_n", "orc_tree_ncell", "orc_tree_ngroup"):
        getattr(lib, f).restype = _i64
        getattr(lib, f).argtypes = [_p]
    lib.orc_tree_root.restype = None
    lib.orc_tree_root.argtypes = [_p, _p, _p]
    lib.orc_tree_particles.restype = None
    lib.orc_tree_particles.argtypes = [_p, _p, _p]
    lib.orc_tree_cells.restype = None
    lib.orc_tree_cells.argtypes = [_p] + [_p] * 11
    lib.orc_tree_groups.restype = None
    lib.orc_tree_groups.argtypes = [_p, _p, _p, _p, _p]
    lib.orc_tree_walk.restype = None
    lib.orc_tree_walk.argtypes = [_p, _d, _d, _d, C.c_int, _p]
    lib.orc_tree_lists.restype = None
    lib.orc_tree_lists.argtypes = [_p] + [_p] * 6
    lib.orc_tree_force.restype = C.c_int
    lib.orc_tree_force.argtypes = [_p, _d, _d, _d, _d, _p, _i64, _p, _p,
                                   C.c_int]
    lib.orc_tree_group_of.restype = _i64
    lib.orc_tree_group_of.argtypes = [_p, _i64]
    lib.orc_direct_vjp.restype = None
    lib.orc_direct_vjp.argtypes = [_i64, _p, _p, _d, _d, _d, _d, _p, _p, _p,
                                   C.c_int]
    lib.orc_tree_vjp.restype = C.c_int
    lib.orc_tree_vjp.argtypes = [_p, _d, _d, _d, _d, _p, _p, _p, C.c_int]
    lib.orc_tree_update.restype = None
    lib.orc_tree_update.argtypes = [_p, _p, _p]
    lib.orc_tree_force_particles.restype = C.c_int
    lib.orc_tree_force_particles.argtypes = [_p, _d, _d, _d, _d, _p, _p, _i64,
                                             _p, _p, C.c_int]
    for pre in ("orc_", "orc_mirror_"):
        f = getattr(lib, pre + "hard_force")
        f.restype = None
        f.argtypes = [_i64, _p, _p, _p, _p, _p, _d, _d, _d, _d, _p, _p]
        f = getattr(lib, pre + "hard_force_species")
        f.restype = None
        f.argtypes = [_i64, _i64, _p, _p, _p, _p, _p, _d, _p, _p, _d, _p, _p]
    lib.orc_hermite.restype = C.c_int
    lib.orc_hermite.argtypes = [_i64, _p, _p, _p, _p, _p, _d, _d, _d, _d, _d,
                                _d, _d, C.c_int, C.c_int, _p, _p, _p, _p]
    lib.orc_mirror_hermite.restype = C.c_int
    lib.orc_mirror_hermite.argtypes = [_i64, _p, _p, _p, _p, _p, _d, _d, _d,
                                       _d, _d, _d, _d, C.c_int, C.c_int, _p]
    lib.orc_direct_species.restype = None
    lib.orc_direct_species.argtypes = [_i64, _i64, _p, _p, _d, _p, _p, _d,
                                       C.c_int, _p, _i64, _p, _p, C.c_int]
    lib.orc_neighbours_species.restype = None
    lib.orc_neighbours_species.argtypes = [_i64, _i64, _p, _p, _p, _i64, _p,
                                           _p, _p, C.c_int]
    lib.orc_hermite_species.restype = C.c_int
    lib.orc_hermite_species.argtypes = [_i64, _i64, _p, _p, _p, _p, _p, _d,
                                        _p, _p, _d, _p, _d, _d, C.c_int,
                                        C.c_int, _p, _p, _p, _p]
    lib.orc_mirror_hermite_species.restype = C.c_int
    lib.orc_mirror_hermite_species.argtypes = [_i64, _i64, _p, _p, _p, _p, _p,
                                               _d, _p, _p, _d, _p, _d, _d,
                                               C.c_int, C.c_int, _p]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


KINDS = {"soft": 0, "hard": 1, "newton": 2}


# --------------------------------------------------------------------------
# Eq. 12-17
# --------------------------------------------------------------------------

def K(x):
    """Cut-off function K(x) of Eq. 12 (elementwise)."""
    lib = _load()
    x = np.asarray(x, dtype=np.float64)
    return np.vectorize(lib.orc_K, otypes=[np.float64])(x)


def dKdx(x):
    lib = _load()
    x = np.asarray(x, dtype=np.float64)
    return np.vectorize(lib.orc_dKdx, otypes=[np.float64])(x)


def K_of_s(s, r_cut, gamma):
    """K as a function of the softened distance (Eq. 12-15)."""
    lib = _load()
    s = np.asarray(s, dtype=np.float64)
    return np.vectorize(lambda v: lib.orc_K_of_s(v, r_cut, gamma),
                        otypes=[np.float64])(s)


def W(y, gamma):
    """Potential transition function W(y; gamma) of Eq. 16-17 (sign of G's
    numerator reversed, see the module docstring)."""
    lib = _load()
    y = np.asarray(y, dtype=np.float64)
    return np.vectorize(lambda v: lib.orc_W(v, gamma), otypes=[np.float64])(y)


def W_inner_slope(gamma):
    return _load().orc_W_inner_slope(gamma)


# --------------------------------------------------------------------------
# Direct summation
# --------------------------------------------------------------------------

def direct(pos, mass, *, G=1.0, eps=0.0, r_cut=1.0, gamma=0.1, kind="soft",
           rows=None, potential=False, threads=None):
    """Acceleration a_i = -sum_{j!=i} G m_j w(s_ij) q_ij / s_ij^3 with
    w = K (soft, Eq. 8), 1-K (hard, Eq. 7) or 1 (Newton); optionally the
    matching potential.  ``rows`` restricts the evaluation to those i."""
    lib = _load()
    pos = _f64(pos, (-1, 3))
    mass = _f64(mass)
    n = pos.shape[0]
    rws = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = n if rws is None else rws.shape[0]
    acc = np.zeros((nr, 3))
    pot = np.zeros(nr) if potential else None
    lib.orc_direct(n, _ptr(pos), _ptr(mass), G, eps, r_cut, gamma,
                   KINDS[kind], None if rws is None else _ptr(rws), nr,
                   _ptr(acc), None if pot is None else _ptr(pot),
                   threads or DEFAULT_THREADS)
    return (acc, pot) if potential else acc


def direct_vjp(pos, mass, w, *, G=1.0, eps=0.0, r_cut=1.0, gamma=0.1):
    """Gradient of sum_i w_i . a_soft,i (direct summation) with respect to
    positions (n x 3) and masses (n)."""
    lib = _load()
    pos = _f64(pos, (-1, 3))
    mass = _f64(mass)
    w = _f64(w, (-1, 3))
    n = pos.shape[0]
    gx = np.zeros((n, 3))
    gm = np.zeros(n)
    lib.orc_direct_vjp(n, _ptr(pos), _ptr(mass), G, eps, r_cut, gamma, _ptr(w),
                       _ptr(gx), _ptr(gm), 1)
    return gx, gm


# --------------------------------------------------------------------------
# Neighbour lists
# --------------------------------------------------------------------------

def neighbours(pos, h, rows=None, threads=None):
    """CSR neighbour lists: for each row i, every j != i with
    ((dx*dx + dy*dy) + dz*dz) < h*h (FP64, unsoftened), ascending j.
    Returns (offsets int64[nr+1], indices int32[nnz])."""
    lib = _load()
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    rws = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = n if rws is None else rws.shape[0]
    cnt = np.zeros(nr, dtype=np.int64)
    th = threads or DEFAULT_THREADS
    rp = None if rws is None else _ptr(rws)
    lib.orc_neighbours_count(n, _ptr(pos), h, rp, nr, _ptr(cnt), th)
    off = np.zeros(nr + 1, dtype=np.int64)
    np.cumsum(cnt, out=off[1:])
    idx = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
    cnt2 = np.zeros(nr, dtype=np.int64)
    lib.orc_neighbours_fill(n, _ptr(pos), h, rp, nr, _ptr(off), _ptr(idx),
                            _ptr(cnt2), th)
    return off, idx[: int(off[-1])]


# --------------------------------------------------------------------------
# Hard part: F_hard over neighbour rows and the Hermite integrator
# --------------------------------------------------------------------------

def _csr(off, idx, n):
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if off.shape != (n + 1,):
        raise ValueError("offsets must have n + 1 entries")
    if idx.size == 0:
        idx = np.zeros(1, dtype=np.int32)
    return off, idx


def hard_force(pos, vel, mass, off, idx, *, G=1.0, eps=0.0, r_cut=1.0,
               gamma=0.1, mirror=False):
    """Hard acceleration and jerk of every particle from its neighbour row
    (Eq. 7 with the pair weight 1 - K and its time derivative); returns
    (a, jerk), each n x 3.  mirror=True evaluates the fused-order mirror of
    the GPU kernels instead of the plain formulas (a separate check, not
    the oracle)."""
    lib = _load()
    pos = _f64(pos, (-1, 3))
    vel = _f64(vel, (-1, 3))
    mass = _f64(mass)
    n = pos.shape[0]
    off, idx = _csr(off, idx, n)
    a = np.zeros((n, 3))
    jk = np.zeros((n, 3))
    f = lib.orc_mirror_hard_force if mirror else lib.orc_hard_force
    f(n, _ptr(pos), _ptr(vel), _ptr(mass), _ptr(off), _ptr(idx), G, eps,
      r_cut, gamma, _ptr(a), _ptr(jk))
    return a, jk


def hard_force_mirror(pos, vel, mass, off, idx, **kw):
    """hard_force() in the GPU kernels' fused order (bit-exact check)."""
    return hard_force(pos, vel, mass, off, idx, mirror=True, **kw)


def hermite(pos, vel, mass, off, idx, *, dt_soft, G=1.0, eps=0.0, r_cut=1.0,
            gamma=0.1, eta=0.1, alpha=0.1, p=2, kmax=30, detail=False):
    """Fourth-order Hermite integration with block timesteps over dt_soft of
    every particle with a non-empty neighbour row (dt_max = dt_soft 2^-p,
    levels down to dt_max 2^-kmax); particles with an empty row drift.  The
    formulas and the timestep criteria of Eq. 18-20 as printed.
    Returns (pos, vel, stats) with stats = (block steps, particle steps,
    pair evaluations, steps capped at kmax); with detail=True also a dict of
    per-particle arrays: nstep (steps taken), lev0 (first level) and margin
    (least relative distance of a level decision from a tie)."""
    lib = _load()
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    mass = _f64(mass)
    n = pos.shape[0]
    off, idx = _csr(off, idx, n)
    st = np.zeros(4, dtype=np.int64)
    ns = np.zeros(max(n, 1), dtype=np.int64)
    l0 = np.zeros(max(n, 1), dtype=np.int32)
    mg = np.zeros(max(n, 1))
    rc = lib.orc_hermite(n, _ptr(pos), _ptr(vel), _ptr(mass), _ptr(off),
                         _ptr(idx), G, eps, r_cut, gamma, eta, alpha, dt_soft,
                         p, kmax, _ptr(st), _ptr(ns), _ptr(l0), _ptr(mg))
    if rc != 0:
        raise ValueError("orc_hermite: bad arguments")
    out = (pos, vel, tuple(int(v) for v in st))
    if detail:
        out += (dict(nstep=ns[:n], lev0=l0[:n], margin=mg[:n]),)
    return out


def hermite_mirror(pos, vel, mass, off, idx, *, dt_soft, G=1.0, eps=0.0,
                   r_cut=1.0, gamma=0.1, eta=0.1, alpha=0.1, p=2, kmax=30):
    """hermite() in the GPU kernels' fused order, criteria tested in squares:
    a separate bit-exact check of the GPU, not the oracle.  Returns (pos,
    vel, stats)."""
    lib = _load()
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    mass = _f64(mass)
    n = pos.shape[0]
    off, idx = _csr(off, idx, n)
    st = np.zeros(4, dtype=np.int64)
    rc = lib.orc_mirror_hermite(n, _ptr(pos), _ptr(vel), _ptr(mass),
                                _ptr(off), _ptr(idx), G, eps, r_cut, gamma,
                                eta, alpha, dt_soft, p, kmax, _ptr(st))
    if rc != 0:
        raise ValueError("orc_mirror_hermite: bad arguments")
    return pos, vel, tuple(int(v) for v in st)


def is_neighbour(pi, pj, h) -> bool:
    lib = _load()
    a = _f64(pi, (3,))
    b = _f64(pj, (3,))
    return bool(lib.orc_is_neighbour(_ptr(a), _ptr(b), h))


# --------------------------------------------------------------------------
# Leapfrog pieces
# --------------------------------------------------------------------------

def kick(vel, acc32, dt_half):
    """v <- v + dt_half * a (FP64 update with an FP32 acceleration)."""
    lib = _load()
    v = _f64(vel).copy()
    a = np.ascontiguousarray(acc32, dtype=np.float32)
    assert a.size == v.size
    lib.orc_kick(v.size, _ptr(v), _ptr(a), dt_half)
    return v


def drift(pos, vel, dt):
    """x <- x + dt * v (FP64)."""
    lib = _load()
    x = _f64(pos).copy()
    v = _f64(vel)
    assert x.size == v.size
    lib.orc_drift(x.size, _ptr(x), _ptr(v), dt)
    return x


# --------------------------------------------------------------------------
# Tree
# --------------------------------------------------------------------------

def morton_key(p, lo, size) -> int:
    lib = _load()
    lo = _f64(lo, (3,))
    return int(lib.orc_morton_key(float(p[0]), float(p[1]), float(p[2]),
                                  _ptr(lo), float(size)))


def root_box(pos):
    lib = _load()
    pos = _f64(pos, (-1, 3))
    lo = np.zeros(3)
    size = np.zeros(1)
    lib.orc_root_box(pos.shape[0], _ptr(pos), _ptr(lo), _ptr(size))
    return lo, float(size[0])


class Tree:
    """The oracle's octree over (pos, mass) with leaf size n_leaf and group
    size n_group; see p3t_oracle.c for the exact rules."""

    def __init__(self, pos, mass, n_leaf=16, n_group=64):
        self._lib = _load()
        self.pos = _f64(pos, (-1, 3))
        self.mass = _f64(mass)
        self.n = self.pos.shape[0]
        self.n_leaf = n_leaf
        self.n_group = n_group
        self._h = self._lib.orc_tree_build(self.n, _ptr(self.pos),
                                           _ptr(self.mass), n_leaf, n_group)
        self._walk = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_tree_free(h)
            self._h = None

    # ---- structure ----
    @property
    def ncell(self):
        return int(self._lib.orc_tree_ncell(self._h))

    @property
    def ngroup(self):
        return int(self._lib.orc_tree_ngroup(self._h))

    def root(self):
        lo = np.zeros(3)
        size = np.zeros(1)
        self._lib.orc_tree_root(self._h, _ptr(lo), _ptr(size))
        return lo, float(size[0])

    def particles(self):
        """(keys in sorted order, order[k] = original index)."""
        key = np.zeros(self.n, dtype=np.uint64)
        order = np.zeros(self.n, dtype=np.int64)
        if self.n:
            self._lib.orc_tree_particles(self._h, _ptr(key), _ptr(order))
        return key, order

    def cells(self):
        c = self.ncell
        out = dict(level=np.zeros(c, np.int32), first=np.zeros(c, np.int64),
                   count=np.zeros(c, np.int64), parent=np.zeros(c, np.int64),
                   child_first=np.zeros(c, np.int64),
                   nchild=np.zeros(c, np.int32), M=np.zeros(c),
                   com=np.zeros((c, 3)), Q=np.zeros((c, 6)),
                   fmin=np.zeros((c, 3), np.float32),
                   fmax=np.zeros((c, 3), np.float32))
        if c:
            self._lib.orc_tree_cells(self._h, *[_ptr(out[k]) for k in (
                "level", "first", "count", "parent", "child_first", "nchild",
                "M", "com", "Q", "fmin", "fmax")])
        return out

    def groups(self):
        g = self.ngroup
        first = np.zeros(g, np.int64)
        count = np.zeros(g, np.int64)
        fmin = np.zeros((g, 3), np.float32)
        fmax = np.zeros((g, 3), np.float32)
        if g:
            self._lib.orc_tree_groups(self._h, _ptr(first), _ptr(count),
                                      _ptr(fmin), _ptr(fmax))
        return dict(first=first, count=count, fmin=fmin, fmax=fmax)

    # ---- walk / lists ----
    def walk(self, theta, h, r_cut, threads=None):
        out = np.zeros(3, np.int64)
        self._lib.orc_tree_walk(self._h, theta, h, r_cut,
                                threads or DEFAULT_THREADS, _ptr(out))
        self._walk = (theta, h, r_cut)
        self._tot = [int(v) for v in out]
        return dict(n_pc=int(out[0]), n_ppn=int(out[1]), n_ppf=int(out[2]))

    def lists(self):
        """Per-group interaction lists in CSR form: pc (cell ids), ppn
        (near particles, sorted ids), ppf (far particles, sorted ids)."""
        assert self._walk is not None, "walk() first"
        g = self.ngroup
        offs = [np.zeros(g + 1, np.int64) for _ in range(3)]
        tot = self._tot
        pc = np.zeros(max(tot[0], 1), np.int64)
        ppn = np.zeros(max(tot[1], 1), np.int64)
        ppf = np.zeros(max(tot[2], 1), np.int64)
        self._lib.orc_tree_lists(self._h, _ptr(offs[0]), _ptr(pc),
                                 _ptr(offs[1]), _ptr(ppn), _ptr(offs[2]),
                                 _ptr(ppf))
        return dict(pc_off=offs[0], pc=pc[: tot[0]], ppn_off=offs[1],
                    ppn=ppn[: tot[1]], ppf_off=offs[2], ppf=ppf[: tot[2]])

    def group_of_sorted(self, k):
        return int(self._lib.orc_tree_group_of(self._h, int(k)))

    # ---- forces ----
    def force(self, *, G=1.0, eps=0.0, r_cut, gamma=0.1, groups=None,
              potential=False, threads=None):
        """FP64 tree acceleration (n x 3, original order) and soft potential
        over the current lists; ``groups`` restricts to those groups (other
        rows stay zero)."""
        assert self._walk is not None, "walk() first"
        acc = np.zeros((self.n, 3))
        pot = np.zeros(self.n)
        gr = None if groups is None else np.ascontiguousarray(groups, np.int64)
        rc = self._lib.orc_tree_force(
            self._h, G, eps, r_cut, gamma, None if gr is None else _ptr(gr),
            0 if gr is None else gr.shape[0], _ptr(acc), _ptr(pot),
            threads or DEFAULT_THREADS)
        assert rc == 0
        return (acc, pot) if potential else acc

    def force_particles(self, particles, *, G=1.0, eps=0.0, r_cut, gamma=0.1,
                        potential=False, threads=None):
        """force() for the listed particles only (ORIGINAL indices); returns
        acc (len x 3) (and pot) in the order listed."""
        assert self._walk is not None, "walk() first"
        particles = np.asarray(particles, dtype=np.int64)
        _, order = self.particles()
        inv = np.empty(self.n, np.int64)
        inv[order] = np.arange(self.n)
        g = self.groups()
        # group of every sorted particle (groups are disjoint ranges)
        cnt = g["count"]
        start = np.cumsum(cnt) - cnt
        gof = np.empty(self.n, np.int64)
        gof[np.repeat(g["first"] - start, cnt) + np.arange(cnt.sum())] = \
            np.repeat(np.arange(self.ngroup), cnt)
        ids = np.ascontiguousarray(inv[particles])
        grp = np.ascontiguousarray(gof[ids])
        acc = np.zeros((self.n, 3))
        pot = np.zeros(self.n)
        rc = self._lib.orc_tree_force_particles(
            self._h, G, eps, r_cut, gamma, _ptr(ids), _ptr(grp), ids.shape[0],
            _ptr(acc), _ptr(pot), threads or DEFAULT_THREADS)
        assert rc == 0
        return (acc[particles], pot[particles]) if potential else acc[particles]

    # ---- gradients (structure frozen) ----
    def update(self, pos, mass):
        """New positions/masses with the same keys, cells, groups and lists;
        moments are recomputed."""
        self.pos = _f64(pos, (-1, 3))
        self.mass = _f64(mass)
        self._lib.orc_tree_update(self._h, _ptr(self.pos), _ptr(self.mass))

    def vjp(self, w, *, G=1.0, eps=0.0, r_cut, gamma=0.1, threads=None):
        """Gradient of sum_i w_i . a_i over the current lists with respect
        to positions (n x 3) and masses (n), original order."""
        assert self._walk is not None, "walk() first"
        w = _f64(w, (-1, 3))
        gx = np.zeros((self.n, 3))
        gm = np.zeros(self.n)
        rc = self._lib.orc_tree_vjp(self._h, G, eps, r_cut, gamma, _ptr(w),
                                    _ptr(gx), _ptr(gm),
                                    threads or DEFAULT_THREADS)
        assert rc == 0
        return gx, gm


# --------------------------------------------------------------------------
# Two species (Sect. 3.2.2): stars and black holes
# --------------------------------------------------------------------------
# The last n_bh particles are black holes.  A pair of type t (0 star-star,
# 1 black hole-star, 2 black hole-black hole) takes eps[t], r_cut[t] and the
# neighbour radius h[t]; r_cut = h = inf for the black hole pair, whose force
# is not split (F_soft = 0, all of it hard, always a neighbour pair).

def _three(v):
    a = np.ascontiguousarray(v, dtype=np.float64)
    if a.shape != (3,):
        raise ValueError("one value per pair type (3)")
    return a


def direct_species(pos, mass, n_bh, *, eps, r_cut, G=1.0, gamma=0.1,
                   kind="soft", rows=None, potential=False, threads=None):
    """direct() with per-pair-type eps and r_cut."""
    lib = _load()
    pos = _f64(pos, (-1, 3))
    mass = _f64(mass)
    n = pos.shape[0]
    e3, r3 = _three(eps), _three(r_cut)
    rws = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = n if rws is None else rws.shape[0]
    acc = np.zeros((nr, 3))
    pot = np.zeros(nr) if potential else None
    lib.orc_direct_species(n, int(n_bh), _ptr(pos), _ptr(mass), G, _ptr(e3),
                           _ptr(r3), gamma, KINDS[kind],
                           None if rws is None else _ptr(rws), nr, _ptr(acc),
                           None if pot is None else _ptr(pot),
                           threads or DEFAULT_THREADS)
    return (acc, pot) if potential else acc


def neighbours_species(pos, n_bh, h, rows=None, threads=None):
    """neighbours() with a radius per pair type; ``rows`` restricts the
    rows; returns (offsets, idx)."""
    lib = _load()
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    h3 = _three(h)
    th = threads or DEFAULT_THREADS
    rws = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = n if rws is None else rws.shape[0]
    rp = None if rws is None else _ptr(rws)
    cnt = np.zeros(nr, dtype=np.int64)
    lib.orc_neighbours_species(n, int(n_bh), _ptr(pos), _ptr(h3), rp, nr, None,
                               None, _ptr(cnt), th)
    off = np.zeros(nr + 1, dtype=np.int64)
    np.cumsum(cnt, out=off[1:])
    idx = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
    lib.orc_neighbours_species(n, int(n_bh), _ptr(pos), _ptr(h3), rp, nr,
                               _ptr(off), _ptr(idx), _ptr(cnt), th)
    return off, idx[: int(off[-1])]


def hard_force_species(pos, vel, mass, off, idx, n_bh, *, eps, r_cut, G=1.0,
                       gamma=0.1, mirror=False):
    """hard_force() with per-pair-type eps and r_cut."""
    lib = _load()
    pos = _f64(pos, (-1, 3))
    vel = _f64(vel, (-1, 3))
    mass = _f64(mass)
    n = pos.shape[0]
    off, idx = _csr(off, idx, n)
    e3, r3 = _three(eps), _three(r_cut)
    a = np.zeros((n, 3))
    jk = np.zeros((n, 3))
    f = (lib.orc_mirror_hard_force_species if mirror
         else lib.orc_hard_force_species)
    f(n, int(n_bh), _ptr(pos), _ptr(vel), _ptr(mass), _ptr(off), _ptr(idx),
      G, _ptr(e3), _ptr(r3), gamma, _ptr(a), _ptr(jk))
    return a, jk


def hermite_species(pos, vel, mass, off, idx, n_bh, *, dt_soft, eps, r_cut,
                    eta, G=1.0, gamma=0.1, alpha=0.1, p=2, kmax=30,
                    detail=False, mirror=False):
    """hermite() with per-pair-type eps and r_cut and eta per species
    (eta[0] stars, eta[1] black holes); a_0 of a black hole takes the
    black hole-star cut-off.  Returns (pos, vel, stats) (+ the detail dict
    of hermite() with detail=True).  mirror=True runs the GPU kernels'
    fused-order mirror instead (no detail)."""
    lib = _load()
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    mass = _f64(mass)
    n = pos.shape[0]
    off, idx = _csr(off, idx, n)
    e3, r3 = _three(eps), _three(r_cut)
    et = np.ascontiguousarray(eta, dtype=np.float64)
    if et.shape != (2,):
        raise ValueError("one eta per species (2)")
    st = np.zeros(4, dtype=np.int64)
    args = (n, int(n_bh), _ptr(pos), _ptr(vel), _ptr(mass), _ptr(off),
            _ptr(idx), G, _ptr(e3), _ptr(r3), gamma, _ptr(et), alpha, dt_soft,
            p, kmax, _ptr(st))
    if mirror:
        rc = lib.orc_mirror_hermite_species(*args)
    else:
        ns = np.zeros(max(n, 1), dtype=np.int64)
        l0 = np.zeros(max(n, 1), dtype=np.int32)
        mg = np.zeros(max(n, 1))
        rc = lib.orc_hermite_species(*args, _ptr(ns), _ptr(l0), _ptr(mg))
    if rc != 0:
        raise ValueError("orc_hermite_species: bad arguments")
    out = (pos, vel, tuple(int(v) for v in st))
    if detail and not mirror:
        out += (dict(nstep=ns[:n], lev0=l0[:n], margin=mg[:n]),)
    return out
