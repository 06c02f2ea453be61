"""Python face of the CPU oracle (``bh_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  The C file is compiled
here with gcc (``-ffp-contract=off`` so that every binary32 operation of the
acceptance test is one rounding, as the oracle's header specifies).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bh_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OR_OK, OR_ERR_ARG, OR_ERR_GEOMETRY, OR_ERR_OOM = 0, 1, 2, 3


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle shared library (a second or two) and return its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                        "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.or_build.argtypes = [i32, P, P, P, P, dbl, ctypes.POINTER(P)]
            lib.or_build.restype = i32
            lib.or_free.argtypes = [P]
            lib.or_num_nodes.argtypes = [P]
            lib.or_num_nodes.restype = i64
            lib.or_export.argtypes = [P] + [P] * 8
            lib.or_export.restype = i32
            lib.or_walk.argtypes = [P, dbl, dbl, i32, i64, P, P, P, P, i32]
            lib.or_walk.restype = i32
            lib.or_walk_list.argtypes = [P, dbl, i64, P, i64]
            lib.or_walk_list.restype = i64
            lib.or_walk_vote.argtypes = [P, dbl, dbl, i32, i64, P, P, P, P, i32]
            lib.or_quadrupoles.argtypes = [P]
            lib.or_quadrupoles.restype = i32
            lib.or_export_quad.argtypes = [P, P]
            lib.or_export_quad.restype = i32
            lib.or_walk_vote.restype = i32
            lib.or_direct.argtypes = [P, dbl, i64, P, P, i32]
            lib.or_direct.restype = i32
            lib.or_direct_points.argtypes = [i64, P, P, dbl, i64, P, P]
            lib.or_direct_points.restype = i32
            lib.or_max_threads.restype = i32
            lib.or_learn_pairs.argtypes = [P, dbl, i64, i64, P, P, P]
            lib.or_learn_pairs.restype = i64
            lib.or_walk_learned.argtypes = [P, dbl, dbl, P, dbl, i64, P, P, i32]
            lib.or_walk_learned.restype = i32
            lib.or_ewald_sum.argtypes = [i64, P, dbl, i32, i32, P]
            lib.or_ewald_sum.restype = i32
            lib.or_ewald_table.argtypes = [i32, i32, P]
            lib.or_ewald_table.restype = i32
            lib.or_ewald_interp.argtypes = [P, i32, i64, P, P]
            lib.or_ewald_interp.restype = i32
            lib.or_walk_periodic.argtypes = [P, dbl, dbl, P, i32, i64, P, P, P, P, i32]
            lib.or_walk_periodic.restype = i32
            lib.or_direct_periodic.argtypes = [P, dbl, P, i32, i32, i64, P, P, i32]
            lib.or_direct_periodic.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().or_max_threads())


class Tree:
    """The oracle's octree over one AMR mesh, with FP64 moments (Eq. 5)."""

    def __init__(self, level, ijk, density, box_lo=(0.0, 0.0, 0.0), box_len=1.0):
        lib = _load()
        self._level = np.ascontiguousarray(level, dtype=np.int32)
        self._ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        rho = np.ascontiguousarray(density, dtype=np.float64).reshape(-1)
        lo = np.ascontiguousarray(box_lo, dtype=np.float64)
        self.nblocks = int(self._level.shape[0])
        if rho.shape[0] != 512 * self.nblocks:
            raise ValueError("density must hold 512 values per block")
        h = ctypes.c_void_p()
        st = lib.or_build(self.nblocks, _ptr(self._level), _ptr(self._ijk), _ptr(rho),
                          _ptr(lo), float(box_len), ctypes.byref(h))
        if st != OR_OK:
            raise OracleError(st, "or_build")
        self._h = h
        self.box_len = float(box_len)
        self.ncells = 512 * self.nblocks

    @classmethod
    def from_workload(cls, w):
        m = w.mesh
        return cls(m.level, m.ijk, w.density, m.box_lo, m.box_len)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().or_free(h)
            self._h = None

    @property
    def nnodes(self) -> int:
        return int(_load().or_num_nodes(self._h))

    def export(self) -> dict:
        """Node table in pre-order (the order of a depth-first visit in octant
        order): level, ijk, is_leaf, cell, M, R (box units), delta, parent."""
        n = self.nnodes
        out = dict(level=np.empty(n, np.int32), ijk=np.empty((n, 3), np.int64),
                   is_leaf=np.empty(n, np.int32), cell=np.empty(n, np.int64),
                   M=np.empty(n), R=np.empty((n, 3)), delta=np.empty(n),
                   parent=np.empty(n, np.int32))
        _load().or_export(self._h, *[_ptr(out[k]) for k in
                                     ("level", "ijk", "is_leaf", "cell", "M", "R",
                                      "delta", "parent")])
        return out

    def _targets(self, targets):
        if targets is None:
            targets = np.arange(self.ncells, dtype=np.int64)
        return np.ascontiguousarray(targets, dtype=np.int64)

    def quadrupoles(self) -> np.ndarray:
        """Traceless quadrupole of every node about its centre of mass,
        columns xx, yy, zz, xy, xz, yz (box units; zero for cells)."""
        lib = _load()
        st = lib.or_quadrupoles(self._h)
        if st != OR_OK:
            raise OracleError(st, "or_quadrupoles")
        q = np.empty((self.nnodes, 6))
        lib.or_export_quad(self._h, _ptr(q))
        return q

    def walk(self, theta: float, G: float = 1.0, targets=None, threads: int = 0,
             quad: bool = False):
        """Per-cell Barnes-Hut potential (Eqs. 3-4) at the given caller cell
        indices (default: every cell), monopole or with the quadrupole term.
        Returns (phi, n_int, n_test)."""
        if quad:
            self.quadrupoles()
        t = self._targets(targets)
        phi = np.empty(t.shape[0])
        ni = np.empty(t.shape[0], np.int64)
        nt = np.empty(t.shape[0], np.int64)
        st = _load().or_walk(self._h, float(theta), float(G), int(bool(quad)), t.shape[0],
                             _ptr(t), _ptr(phi), _ptr(ni), _ptr(nt), int(threads))
        if st != OR_OK:
            raise OracleError(st, "or_walk")
        return phi, ni, nt

    def walk_list(self, theta: float, target: int) -> np.ndarray:
        """Node indices of the accepted set of one target cell."""
        lib = _load()
        n = lib.or_walk_list(self._h, float(theta), int(target), None, 0)
        if n < 0:
            raise OracleError(OR_ERR_ARG, "or_walk_list")
        buf = np.empty(max(n, 1), np.int64)
        lib.or_walk_list(self._h, float(theta), int(target), _ptr(buf), n)
        return buf[:n]

    def walk_vote(self, theta: float, G: float = 1.0, bricks=None, threads: int = 0,
                  quad: bool = False):
        """Paper-mode walk (all() vote over 32-cell bricks).  bricks are
        block*16 + brick; results come 32 per brick in local Morton order."""
        if quad:
            self.quadrupoles()
        if bricks is None:
            bricks = np.arange(16 * self.nblocks, dtype=np.int64)
        b = np.ascontiguousarray(bricks, dtype=np.int64)
        phi = np.empty(32 * b.shape[0])
        ni = np.empty(32 * b.shape[0], np.int64)
        nt = np.empty(32 * b.shape[0], np.int64)
        st = _load().or_walk_vote(self._h, float(theta), float(G), int(bool(quad)), b.shape[0],
                                  _ptr(b), _ptr(phi), _ptr(ni), _ptr(nt), int(threads))
        if st != OR_OK:
            raise OracleError(st, "or_walk_vote")
        return phi, ni, nt

    def learn_pairs(self, theta: float, target: int):
        """Features, residual eps and node index of every accepted internal
        node of one target's walk (the learned correction's training pairs)."""
        self.quadrupoles()
        lib = _load()
        n = lib.or_learn_pairs(self._h, float(theta), int(target), 0, None, None, None)
        if n < 0:
            raise OracleError(OR_ERR_ARG, "or_learn_pairs")
        f = np.empty((max(n, 1), 10))
        e = np.empty(max(n, 1))
        nd = np.empty(max(n, 1), np.int64)
        lib.or_learn_pairs(self._h, float(theta), int(target), n, _ptr(f), _ptr(e), _ptr(nd))
        return f[:n], e[:n], nd[:n]

    def walk_learned(self, theta: float, weights, G: float = 1.0, targets=None,
                     threads: int = 0, s_min: float = 0.0) -> np.ndarray:
        """Per-cell walk with each accepted node's term times (1 + s^2 MLP(x));
        weights: flat FP64 vector in the layout of mlp_unflatten.  s_min > 0:
        only nodes with s = l/d >= s_min get the network (gate_f32)."""
        self.quadrupoles()
        t = self._targets(targets)
        w = np.ascontiguousarray(weights, dtype=np.float64)
        phi = np.empty(t.shape[0])
        st = _load().or_walk_learned(self._h, float(theta), float(G), _ptr(w), float(s_min),
                                     t.shape[0], _ptr(t), _ptr(phi), int(threads))
        if st != OR_OK:
            raise OracleError(st, "or_walk_learned")
        return phi

    def walk_periodic(self, theta: float, G: float = 1.0, targets=None, threads: int = 0,
                      ng: int = 64, nseries: int = 3):
        """Per-cell walk with periodic boundaries (App. A): minimum-image
        opening test, terms M (1/d + chi) with chi interpolated from the
        Ewald table (ng, nseries).  Returns (phi, n_int, n_test)."""
        T = ewald_table(ng, nseries)
        t = self._targets(targets)
        phi = np.empty(t.shape[0])
        ni = np.empty(t.shape[0], np.int64)
        nt = np.empty(t.shape[0], np.int64)
        st = _load().or_walk_periodic(self._h, float(theta), float(G), _ptr(T), int(ng),
                                      t.shape[0], _ptr(t), _ptr(phi), _ptr(ni), _ptr(nt),
                                      int(threads))
        if st != OR_OK:
            raise OracleError(st, "or_walk_periodic")
        return phi, ni, nt

    def direct_periodic(self, G: float = 1.0, targets=None, threads: int = 0,
                        ng: int | None = 64, nseries: int = 3) -> np.ndarray:
        """Direct periodic potential: every other cell's mass times the Ewald
        field psi, plus the copies of the cell's own mass.  psi from the table
        (ng) or, with ng=None, from the Ewald sum itself (range nseries)."""
        t = self._targets(targets)
        phi = np.empty(t.shape[0])
        T = ewald_table(ng, nseries) if ng else None
        st = _load().or_direct_periodic(self._h, float(G), None if T is None else _ptr(T),
                                        int(ng or 0), int(nseries), t.shape[0], _ptr(t),
                                        _ptr(phi), int(threads))
        if st != OR_OK:
            raise OracleError(st, "or_direct_periodic")
        return phi

    def direct(self, G: float = 1.0, targets=None, threads: int = 0) -> np.ndarray:
        """Direct O(N^2) potential (Eq. 2 without the 1/2) at the given cells."""
        t = self._targets(targets)
        phi = np.empty(t.shape[0])
        st = _load().or_direct(self._h, float(G), t.shape[0], _ptr(t), _ptr(phi),
                               int(threads))
        if st != OR_OK:
            raise OracleError(st, "or_direct")
        return phi


def direct_points(pos, m, G=1.0, targets=None) -> np.ndarray:
    """Direct-sum potential of point masses at the given point indices."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    m = np.ascontiguousarray(m, dtype=np.float64)
    n = pos.shape[0]
    t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(
        targets, dtype=np.int64)
    phi = np.empty(t.shape[0])
    st = _load().or_direct_points(n, _ptr(pos), _ptr(m), float(G), t.shape[0], _ptr(t),
                                  _ptr(phi))
    if st != OR_OK:
        raise OracleError(st, "or_direct_points")
    return phi


# ------------------------------------------------ periodic boundaries --
EWALD_ALPHA = 2.0
_tables: dict = {}


def ewald_sum(r, alpha: float = EWALD_ALPHA, nseries: int = 3, chi: bool = False):
    """Ewald field psi(r) of a unit mass in the unit-period box, mean density
    subtracted (chi=True: psi - 1/|r|), at points r[..., 3], FP64."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    shape = r.shape[:-1]
    r = r.reshape(-1, 3)
    out = np.empty(r.shape[0])
    st = _load().or_ewald_sum(r.shape[0], _ptr(r), float(alpha), int(nseries), int(bool(chi)),
                              _ptr(out))
    if st != OR_OK:
        raise OracleError(st, "or_ewald_sum")
    return out.reshape(shape)


def ewald_table(ng: int = 64, nseries: int = 3) -> np.ndarray:
    """chi on the (ng+2)^3 grid of the octant [0, 1/2 + h]^3, h = 1/(2 ng),
    x fastest (cached per (ng, nseries))."""
    key = (int(ng), int(nseries))
    if key not in _tables:
        T = np.empty((ng + 2) ** 3)
        st = _load().or_ewald_table(int(ng), int(nseries), _ptr(T))
        if st != OR_OK:
            raise OracleError(st, "or_ewald_table")
        _tables[key] = T
    return _tables[key]


def ewald_interp(u, ng: int = 64, nseries: int = 3) -> np.ndarray:
    """chi at displacements u[..., 3] (|u_i| <= 1/2) by the table's quadratic
    interpolation."""
    T = ewald_table(ng, nseries)
    u = np.ascontiguousarray(u, dtype=np.float64)
    shape = u.shape[:-1]
    u = u.reshape(-1, 3)
    out = np.empty(u.shape[0])
    st = _load().or_ewald_interp(_ptr(T), int(ng), u.shape[0], _ptr(u), _ptr(out))
    if st != OR_OK:
        raise OracleError(st, "or_ewald_interp")
    return out.reshape(shape)


def local_morton_order() -> np.ndarray:
    """Caller-layout offset (cz*64 + cy*8 + cx) of the cell with local Morton
    index m = 0..511 inside a block (x in the lowest bit)."""
    m = np.arange(512)
    cx = sum(((m >> (3 * b)) & 1) << b for b in range(3))
    cy = sum(((m >> (3 * b + 1)) & 1) << b for b in range(3))
    cz = sum(((m >> (3 * b + 2)) & 1) << b for b in range(3))
    return cz * 64 + cy * 8 + cx


# ------------------------------------------------------------------ MLP --
MLP_IN, MLP_H = 10, 64
MLP_NW = MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1


def mlp_unflatten(w):
    """Flat weights -> (W1[10,64], b1[64], W2[64,64], b2[64], W3[64], b3)."""
    w = np.asarray(w, dtype=np.float64)
    i = 0
    out = []
    for shape in ((MLP_IN, MLP_H), (MLP_H,), (MLP_H, MLP_H), (MLP_H,), (MLP_H,), (1,)):
        k = int(np.prod(shape))
        out.append(w[i:i + k].reshape(shape))
        i += k
    return out


def gelu(a):
    """tanh form of GELU."""
    c = np.sqrt(2.0 / np.pi)
    return 0.5 * a * (1.0 + np.tanh(c * (a + 0.044715 * a ** 3)))


def gelu_grad(a):
    c = np.sqrt(2.0 / np.pi)
    t = np.tanh(c * (a + 0.044715 * a ** 3))
    return 0.5 * (1.0 + t) + 0.5 * a * (1.0 - t * t) * c * (1.0 + 3 * 0.044715 * a * a)


def mlp_forward(w, x):
    W1, b1, W2, b2, W3, b3 = mlp_unflatten(w)
    a1 = x @ W1 + b1
    h1 = gelu(a1)
    a2 = h1 @ W2 + b2
    h2 = gelu(a2)
    return h2 @ W3 + b3[0], (a1, h1, a2, h2)


def mlp_loss_grad(w, x, z):
    """Mean squared error of MLP(x) against z and its gradient (flat), FP64."""
    y, (a1, h1, a2, h2) = mlp_forward(w, x)
    W1, b1, W2, b2, W3, b3 = mlp_unflatten(w)
    n = x.shape[0]
    r = y - z
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    gW3 = h2.T @ dy
    gb3 = np.array([dy.sum()])
    d2 = np.outer(dy, W3) * gelu_grad(a2)
    gW2 = h1.T @ d2
    gb2 = d2.sum(0)
    d1 = (d2 @ W2.T) * gelu_grad(a1)
    gW1 = x.T @ d1
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return loss, g
