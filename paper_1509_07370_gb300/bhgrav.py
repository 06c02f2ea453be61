"""Thin ctypes binding of libbhgrav (the C-ABI declared in include/bhgrav.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names; device arrays are passed as torch CUDA
tensors (their data pointers), host arrays as numpy arrays.  There is no CPU
fallback: if the library cannot be built or loaded, or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

BH_OK, BH_ERR_ARG, BH_ERR_GEOMETRY, BH_ERR_OOM, BH_ERR_CUDA, BH_ERR_DEVICE_TIMEOUT, \
    BH_ERR_STATE = range(7)
BH_PREC_F32, BH_PREC_F64 = 0, 1
BH_CRIT_PER_CELL, BH_CRIT_WARP_VOTE = 0, 1

EXPORTED = ("bh_default_options", "bh_create", "bh_build", "bh_build_batch",
            "bh_update_density", "bh_sync_status", "bh_autotune", "bh_set_walk_shape",
            "bh_solve_graph",
            "bh_potential", "bh_walk_counts", "bh_tree_size", "bh_export_nodes",
            "bh_export_quadrupoles", "bh_solve_host", "bh_solve_noalloc", "bh_learn_pairs",
            "bh_learn_targets",
            "bh_mlp_grad", "bh_mlp_adam", "bh_set_mlp", "bh_get_mlp", "bh_set_mlp_gate",
            "bh_mlp_eval", "bh_stats",
            "bh_set_ewald", "bh_ewald_eval", "bh_last_error", "bh_destroy")


class bh_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("criterion", ctypes.c_int),
                ("kahan", ctypes.c_int), ("quadrupole", ctypes.c_int),
                ("learned", ctypes.c_int), ("timing", ctypes.c_int),
                ("periodic", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


class bh_stats_t(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_nodes", ctypes.c_int64),
                ("n_blocks", ctypes.c_int32), ("n_fields", ctypes.c_int32),
                ("max_level", ctypes.c_int32), ("built", ctypes.c_int32),
                ("last_theta", ctypes.c_double), ("build_ms", ctypes.c_double),
                ("potential_ms", ctypes.c_double), ("interactions", ctypes.c_int64),
                ("tests", ctypes.c_int64), ("cell_interactions", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64)]


class BHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[bh status {status}] {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libbhgrav.so (building it with nvcc first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libbhgrav not built ({path} missing)")
        lib = ctypes.CDLL(path)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.bh_default_options.argtypes = [ctypes.POINTER(bh_options)]
        lib.bh_default_options.restype = None
        lib.bh_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(bh_options), I, P]
        lib.bh_build.argtypes = [P, I, P, P, P, D, P, I]
        lib.bh_potential.argtypes = [P, D, D, P]
        lib.bh_build_batch.argtypes = [P, I, P, P, P, P, P, P, I]
        lib.bh_update_density.argtypes = [P, P, I]
        lib.bh_sync_status.argtypes = [P]
        lib.bh_autotune.argtypes = [P, D, P]
        lib.bh_set_walk_shape.argtypes = [P, I, I, I, I]
        lib.bh_solve_graph.argtypes = [P, P, I, D, D, P]
        lib.bh_walk_counts.argtypes = [P, D, P, P, P]
        lib.bh_tree_size.argtypes = [P, P, P, P]
        lib.bh_export_nodes.argtypes = [P, P, P, P, P, P]
        lib.bh_export_quadrupoles.argtypes = [P, P]
        lib.bh_solve_host.argtypes = [P, I, P, P, P, D, P, I, D, D, P]
        lib.bh_solve_noalloc.argtypes = [I, P, P, P, D, P, I, D, D, P, P]
        lib.bh_learn_pairs.argtypes = [P, D, ctypes.c_int64, P, ctypes.c_int64, P, P, P, P]
        lib.bh_mlp_grad.argtypes = [ctypes.c_int64, P, P, P, P, P, P]
        lib.bh_learn_targets.argtypes = [ctypes.c_int64, P, P, P, P]
        lib.bh_mlp_adam.argtypes = [P, P, P, P, I, ctypes.c_float, P]
        lib.bh_set_mlp.argtypes = [P, P]
        lib.bh_get_mlp.argtypes = [P, P]
        lib.bh_set_mlp_gate.argtypes = [P, D]
        lib.bh_stats.argtypes = [P, ctypes.POINTER(bh_stats_t)]
        lib.bh_mlp_eval.argtypes = [P, ctypes.c_int64, P, P]
        lib.bh_set_ewald.argtypes = [P, I, I]
        lib.bh_ewald_eval.argtypes = [P, ctypes.c_int64, P, P]
        lib.bh_last_error.argtypes = [P]
        lib.bh_last_error.restype = ctypes.c_char_p
        lib.bh_destroy.argtypes = [P]
        lib.bh_destroy.restype = None
        for name in ("bh_create", "bh_build", "bh_build_batch", "bh_update_density",
                     "bh_sync_status", "bh_autotune", "bh_set_walk_shape", "bh_solve_graph",
                     "bh_potential",
                     "bh_walk_counts",
                     "bh_tree_size", "bh_export_nodes", "bh_export_quadrupoles", "bh_solve_host",
                     "bh_solve_noalloc", "bh_learn_pairs", "bh_learn_targets", "bh_mlp_grad",
                     "bh_mlp_adam",
                     "bh_set_mlp", "bh_get_mlp", "bh_set_mlp_gate", "bh_mlp_eval", "bh_stats",
                     "bh_set_ewald",
                     "bh_ewald_eval"):
            getattr(lib, name).restype = I
        _lib = lib
        return lib


def _check(ctx, st: int, what: str):
    if st != BH_OK:
        msg = load().bh_last_error(ctx).decode() if ctx else ""
        raise BHError(st, f"{what}: {msg}")


def _dev_ptr(t, dtype=None) -> int:
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return t.data_ptr()


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- C names --
def bh_default_options() -> bh_options:
    o = bh_options()
    load().bh_default_options(ctypes.byref(o))
    return o


def bh_create(opt: bh_options | None = None, device: int = 0, stream: int = 0):
    h = ctypes.c_void_p()
    st = load().bh_create(ctypes.byref(h), ctypes.byref(opt) if opt is not None else None,
                          int(device), ctypes.c_void_p(int(stream)))
    _check(None, st, "bh_create")
    return h


def bh_build(ctx, level, ijk, box_lo, box_len, density) -> None:
    """level, ijk: host int arrays; density: CUDA float32/float64 tensor."""
    import torch
    level = np.ascontiguousarray(level, dtype=np.int32)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    lo = np.ascontiguousarray(box_lo, dtype=np.float64)
    if density.dtype not in (torch.float32, torch.float64):
        raise ValueError("density must be float32 or float64")
    if density.numel() != 512 * level.shape[0]:
        raise ValueError("density must hold 512 values per block")
    st = load().bh_build(ctx, int(level.shape[0]), _np_ptr(level), _np_ptr(ijk), _np_ptr(lo),
                         float(box_len), ctypes.c_void_p(_dev_ptr(density)),
                         int(density.dtype == torch.float64))
    _check(ctx, st, "bh_build")


def bh_build_batch(ctx, nblocks, level, ijk, box_lo, box_len, density) -> None:
    """nblocks: blocks per field; level/ijk: all fields' blocks concatenated;
    box_lo [nfields, 3], box_len [nfields] host arrays; density: CUDA tensor."""
    import torch
    nb = np.ascontiguousarray(nblocks, dtype=np.int32)
    level = np.ascontiguousarray(level, dtype=np.int32)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    lo = np.ascontiguousarray(box_lo, dtype=np.float64).reshape(-1, 3)
    ln = np.ascontiguousarray(box_len, dtype=np.float64)
    if density.numel() != 512 * level.shape[0] or nb.sum() != level.shape[0]:
        raise ValueError("density must hold 512 values per block; nblocks must sum to the blocks")
    st = load().bh_build_batch(ctx, int(nb.shape[0]), _np_ptr(nb), _np_ptr(level), _np_ptr(ijk),
                               _np_ptr(lo), _np_ptr(ln), ctypes.c_void_p(_dev_ptr(density)),
                               int(density.dtype == torch.float64))
    _check(ctx, st, "bh_build_batch")


def bh_update_density(ctx, density) -> None:
    import torch
    st = load().bh_update_density(ctx, ctypes.c_void_p(_dev_ptr(density)),
                                  int(density.dtype == torch.float64))
    _check(ctx, st, "bh_update_density")


def bh_sync_status(ctx) -> None:
    _check(ctx, load().bh_sync_status(ctx), "bh_sync_status")


def bh_autotune(ctx, theta: float) -> tuple:
    """Returns the chosen (warps per CTA, target pairs per lane, groups per
    take of the persistent walk or 0 for a plain grid, longest first 0/1)."""
    sh = (ctypes.c_int * 4)()
    _check(ctx, load().bh_autotune(ctx, float(theta), sh), "bh_autotune")
    return int(sh[0]), int(sh[1]), int(sh[2]), int(sh[3])


def bh_set_walk_shape(ctx, warps: int, pairs: int, groups_per_take: int,
                      longest_first: int = 0) -> None:
    _check(ctx, load().bh_set_walk_shape(ctx, int(warps), int(pairs), int(groups_per_take),
                                         int(longest_first)), "bh_set_walk_shape")


def bh_solve_graph(ctx, density, theta: float, G: float, out) -> None:
    import torch
    st = load().bh_solve_graph(ctx, ctypes.c_void_p(_dev_ptr(density)),
                               int(density.dtype == torch.float64), float(theta), float(G),
                               ctypes.c_void_p(_dev_ptr(out)))
    _check(ctx, st, "bh_solve_graph")


def bh_potential(ctx, theta: float, G: float, out) -> None:
    st = load().bh_potential(ctx, float(theta), float(G), ctypes.c_void_p(_dev_ptr(out)))
    _check(ctx, st, "bh_potential")


def bh_walk_counts(ctx, theta: float, n_int, n_test, n_cell=None) -> None:
    import torch
    st = load().bh_walk_counts(ctx, float(theta),
                               ctypes.c_void_p(_dev_ptr(n_int, torch.int32)),
                               ctypes.c_void_p(_dev_ptr(n_test, torch.int32)),
                               ctypes.c_void_p(_dev_ptr(n_cell, torch.int32))
                               if n_cell is not None else None)
    _check(ctx, st, "bh_walk_counts")


def bh_tree_size(ctx):
    nc, nn, ml = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    st = load().bh_tree_size(ctx, ctypes.byref(nc), ctypes.byref(nn), ctypes.byref(ml))
    _check(ctx, st, "bh_tree_size")
    return nc.value, nn.value, ml.value


def bh_export_nodes(ctx, M=None, R=None, delta=None, skip=None, level=None) -> None:
    def p(t):
        return ctypes.c_void_p(_dev_ptr(t)) if t is not None else None
    st = load().bh_export_nodes(ctx, p(M), p(R), p(delta), p(skip), p(level))
    _check(ctx, st, "bh_export_nodes")


def bh_export_quadrupoles(ctx, Q) -> None:
    """Q: CUDA float64 tensor of 6 * n_nodes values (xx, yy, zz, xy, xz, yz)."""
    import torch
    st = load().bh_export_quadrupoles(ctx, ctypes.c_void_p(_dev_ptr(Q, torch.float64)))
    _check(ctx, st, "bh_export_quadrupoles")


def bh_solve_host(ctx, level, ijk, box_lo, box_len, density_host: np.ndarray, theta: float,
                  G: float, out_host: np.ndarray) -> None:
    """Host-memory form: density_host and out_host are (ideally pinned) host
    arrays; copies to and from the device happen inside the call."""
    level = np.ascontiguousarray(level, dtype=np.int32)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    lo = np.ascontiguousarray(box_lo, dtype=np.float64)
    if not (density_host.flags.c_contiguous and out_host.flags.c_contiguous):
        raise ValueError("host buffers must be C-contiguous")
    if density_host.dtype not in (np.float32, np.float64):
        raise ValueError("density must be float32 or float64")
    st = load().bh_solve_host(ctx, int(level.shape[0]), _np_ptr(level), _np_ptr(ijk),
                              _np_ptr(lo), float(box_len), _np_ptr(density_host),
                              int(density_host.dtype == np.float64), float(theta), float(G),
                              _np_ptr(out_host))
    _check(ctx, st, "bh_solve_host")


def bh_solve_noalloc(level, ijk, box_lo, box_len, density, theta: float, G: float, out,
                     stream: int = 0) -> None:
    """Allocation-free solve of a mesh of at most 64 blocks, for callers that
    cannot allocate device memory (the library keeps the tree in a fixed
    device array).  density: CUDA float32/float64 tensor; out: CUDA float32
    tensor; both on the current device.  Calls sharing the fixed array must
    not overlap on the GPU."""
    import torch
    level = np.ascontiguousarray(level, dtype=np.int32)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    lo = np.ascontiguousarray(box_lo, dtype=np.float64)
    st = load().bh_solve_noalloc(int(level.shape[0]), _np_ptr(level), _np_ptr(ijk), _np_ptr(lo),
                                 float(box_len), ctypes.c_void_p(_dev_ptr(density)),
                                 int(density.dtype == torch.float64), float(theta), float(G),
                                 ctypes.c_void_p(_dev_ptr(out, torch.float32)),
                                 ctypes.c_void_p(int(stream)))
    _check(None, st, "bh_solve_noalloc")


MLP_NW = 10 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def bh_learn_pairs(ctx, theta: float, targets, cap: int, with_nodes: bool = False):
    """Training pairs of the learned correction for the DEVICE int64 target
    cell indices; returns (feat [n,10], eps [n], count[, node [n]]) (CUDA)."""
    import torch
    dev = targets.device
    feat = torch.empty((max(cap, 1), 10), dtype=torch.float32, device=dev)
    eps = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
    node = torch.empty(max(cap, 1), dtype=torch.int64, device=dev) if with_nodes else None
    cnt = ctypes.c_int64()
    st = load().bh_learn_pairs(ctx, float(theta), int(targets.numel()),
                               ctypes.c_void_p(_dev_ptr(targets, torch.int64)), int(cap),
                               ctypes.c_void_p(feat.data_ptr()), ctypes.c_void_p(eps.data_ptr()),
                               ctypes.c_void_p(node.data_ptr()) if with_nodes else None,
                               ctypes.byref(cnt))
    _check(ctx, st, "bh_learn_pairs")
    n = min(cnt.value, cap)
    if with_nodes:
        return feat[:n], eps[:n], cnt.value, node[:n]
    return feat[:n], eps[:n], cnt.value


def bh_learn_targets(feat, eps, stream: int = 0):
    """z = eps / s^2 of every pair (s = feat[:, 3]), on the device."""
    import torch
    z = torch.empty_like(eps)
    st = load().bh_learn_targets(int(eps.numel()), ctypes.c_void_p(_dev_ptr(feat, torch.float32)),
                                 ctypes.c_void_p(_dev_ptr(eps, torch.float32)),
                                 ctypes.c_void_p(_dev_ptr(z, torch.float32)),
                                 ctypes.c_void_p(int(stream)))
    _check(None, st, "bh_learn_targets")
    return z


def bh_mlp_grad(x, z, w, grad, loss, stream: int = 0) -> None:
    import torch
    st = load().bh_mlp_grad(int(z.numel()), ctypes.c_void_p(_dev_ptr(x, torch.float32)),
                            ctypes.c_void_p(_dev_ptr(z, torch.float32)),
                            ctypes.c_void_p(_dev_ptr(w, torch.float32)),
                            ctypes.c_void_p(_dev_ptr(grad, torch.float32)),
                            ctypes.c_void_p(_dev_ptr(loss, torch.float32)),
                            ctypes.c_void_p(int(stream)))
    _check(None, st, "bh_mlp_grad")


def bh_mlp_adam(grad, w, m, v, step: int, lr: float, stream: int = 0) -> None:
    import torch
    st = load().bh_mlp_adam(*[ctypes.c_void_p(_dev_ptr(t, torch.float32)) for t in (grad, w, m, v)],
                            int(step), ctypes.c_float(lr), ctypes.c_void_p(int(stream)))
    _check(None, st, "bh_mlp_adam")


def bh_set_mlp(ctx, w_host: np.ndarray) -> None:
    w = np.ascontiguousarray(w_host, dtype=np.float32)
    if w.size != MLP_NW:
        raise ValueError(f"expected {MLP_NW} weights")
    _check(ctx, load().bh_set_mlp(ctx, _np_ptr(w)), "bh_set_mlp")


def bh_set_mlp_gate(ctx, s_min: float) -> None:
    _check(ctx, load().bh_set_mlp_gate(ctx, float(s_min)), "bh_set_mlp_gate")


def bh_get_mlp(ctx) -> np.ndarray:
    w = np.empty(MLP_NW, dtype=np.float32)
    _check(ctx, load().bh_get_mlp(ctx, _np_ptr(w)), "bh_get_mlp")
    return w


def bh_mlp_eval(ctx, x, y) -> None:
    """The context's network on DEVICE float32 features x[n, 10] -> y[n],
    on the tensor cores (tcgen05)."""
    import torch
    if x.dim() != 2 or x.shape[1] != 10 or y.numel() != x.shape[0]:
        raise ValueError("expected x[n, 10] and y[n]")
    st = load().bh_mlp_eval(ctx, int(x.shape[0]), ctypes.c_void_p(_dev_ptr(x, torch.float32)),
                            ctypes.c_void_p(_dev_ptr(y, torch.float32)))
    _check(ctx, st, "bh_mlp_eval")


def bh_stats(ctx) -> dict:
    """Tree sizes, device times of the last build / potential (timing option,
    else -1) and work totals of the last bh_walk_counts (else -1)."""
    out = bh_stats_t()
    _check(ctx, load().bh_stats(ctx, ctypes.byref(out)), "bh_stats")
    return {name: getattr(out, name) for name, _ in bh_stats_t._fields_}


def bh_set_ewald(ctx, n_grid: int, n_series: int) -> None:
    _check(ctx, load().bh_set_ewald(ctx, int(n_grid), int(n_series)), "bh_set_ewald")


def bh_ewald_eval(ctx, r, chi) -> None:
    """chi (smooth part of the Ewald field) at DEVICE float32 displacements
    r[n, 3] (box units, |component| <= 1/2) -> chi[n], by the table."""
    import torch
    if r.dim() != 2 or r.shape[1] != 3 or chi.numel() != r.shape[0]:
        raise ValueError("expected r[n, 3] and chi[n]")
    st = load().bh_ewald_eval(ctx, int(r.shape[0]), ctypes.c_void_p(_dev_ptr(r, torch.float32)),
                              ctypes.c_void_p(_dev_ptr(chi, torch.float32)))
    _check(ctx, st, "bh_ewald_eval")


def bh_last_error(ctx) -> str:
    return load().bh_last_error(ctx).decode()


def bh_destroy(ctx) -> None:
    if ctx:
        load().bh_destroy(ctx)


# ------------------------------------------------------------ convenience --
class Solver:
    """Owns one bh_ctx.  Example::

        s = Solver(precision=BH_PREC_F32)
        s.build(mesh.level, mesh.ijk, density_cuda)       # tree + FP64 moments
        phi = s.potential(theta=0.5, G=1.0)               # CUDA tensor, density layout
    """

    def __init__(self, precision=BH_PREC_F32, criterion=BH_CRIT_PER_CELL, kahan=True,
                 quadrupole=False, learned=False, timing=False, periodic=False, device=0,
                 stream=None):
        import torch
        o = bh_default_options()
        o.precision, o.criterion, o.kahan = int(precision), int(criterion), int(bool(kahan))
        o.quadrupole = int(bool(quadrupole))
        o.learned = int(learned)  # 1: mma.sync network in the walk; 2: tcgen05
        o.timing = int(bool(timing))
        o.periodic = int(bool(periodic))
        self.options = o
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self._ctx = bh_create(o, device, stream.cuda_stream)
        self.ncells = 0

    def _handoff(self, *tensors):
        """Outputs are written on the library's stream: tie them to it and make
        the caller's current stream wait for it."""
        import torch
        cur = torch.cuda.current_stream(self.device)
        for t in tensors:
            if t is not None:
                t.record_stream(self.stream)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)

    def _keep(self, density):
        """The build's kernels read the density on the library's stream after
        the call returns: keep its memory from being reused before that."""
        if hasattr(density, "record_stream"):
            density.record_stream(self.stream)

    def build(self, level, ijk, density, box_lo=(0.0, 0.0, 0.0), box_len=1.0):
        bh_build(self._ctx, level, ijk, box_lo, box_len, density)
        self._keep(density)
        self.ncells = 512 * len(level)
        return self

    def build_batch(self, nblocks, level, ijk, density, box_lo=None, box_len=None):
        """Several fields at once (see bh_build_batch)."""
        nf = len(nblocks)
        box_lo = np.zeros((nf, 3)) if box_lo is None else box_lo
        box_len = np.ones(nf) if box_len is None else box_len
        bh_build_batch(self._ctx, nblocks, level, ijk, box_lo, box_len, density)
        self._keep(density)
        self.ncells = 512 * int(np.sum(nblocks))
        return self

    def update_density(self, density):
        bh_update_density(self._ctx, density)
        self._keep(density)

    def sync_status(self):
        bh_sync_status(self._ctx)

    def autotune(self, theta: float) -> tuple:
        """Tunes the walk's launch shape: (warps per CTA, target pairs per lane,
        groups per take of the persistent walk or 0, longest first 0/1)."""
        return bh_autotune(self._ctx, theta)

    def set_walk_shape(self, warps: int, pairs: int = 0, groups_per_take: int = 0,
                       longest_first: int = 0):
        """Pins the walk's launch shape (see bh_set_walk_shape)."""
        bh_set_walk_shape(self._ctx, warps, pairs, groups_per_take, longest_first)

    def solve_graph(self, density, theta: float, G: float = 1.0, out=None):
        import torch
        if out is None:
            dt = torch.float64 if self.options.precision == BH_PREC_F64 else torch.float32
            out = torch.empty(self.ncells, dtype=dt, device=self.device)
        bh_solve_graph(self._ctx, density, theta, G, out)
        self._handoff(out)
        return out

    def potential(self, theta: float, G: float = 1.0, out=None):
        import torch
        if out is None:
            dt = torch.float64 if self.options.precision == BH_PREC_F64 else torch.float32
            out = torch.empty(self.ncells, dtype=dt, device=self.device)
        bh_potential(self._ctx, theta, G, out)
        self._handoff(out)
        return out

    def walk_counts(self, theta: float, with_cells: bool = False):
        """Per-cell interaction and opening-test counts (and, with_cells, the
        interactions with single cells)."""
        import torch
        ni = torch.empty(self.ncells, dtype=torch.int32, device=self.device)
        nt = torch.empty(self.ncells, dtype=torch.int32, device=self.device)
        nc = torch.empty(self.ncells, dtype=torch.int32, device=self.device) if with_cells else None
        bh_walk_counts(self._ctx, theta, ni, nt, nc)
        self._handoff(ni, nt, nc)
        return (ni, nt, nc) if with_cells else (ni, nt)

    def tree_size(self):
        return bh_tree_size(self._ctx)

    def export_nodes(self):
        import torch
        _, n, _ = self.tree_size()
        d = self.device
        out = dict(M=torch.empty(n, dtype=torch.float64, device=d),
                   R=torch.empty((n, 3), dtype=torch.float64, device=d),
                   delta=torch.empty(n, dtype=torch.float32, device=d),
                   skip=torch.empty(n, dtype=torch.int32, device=d),
                   level=torch.empty(n, dtype=torch.int32, device=d))
        bh_export_nodes(self._ctx, **out)
        self._handoff(*out.values())
        return out

    def learn_pairs(self, theta: float, targets, cap: int, with_nodes: bool = False):
        out = bh_learn_pairs(self._ctx, theta, targets, cap, with_nodes)
        self._handoff(*[t for t in out if hasattr(t, "record_stream")])
        return out

    def set_mlp(self, w):
        bh_set_mlp(self._ctx, w)

    def set_mlp_gate(self, s_min: float):
        """Network only for accepted nodes with s = l/d >= s_min (0: all)."""
        bh_set_mlp_gate(self._ctx, s_min)

    def set_ewald(self, n_grid: int = 64, n_series: int = 3):
        """Recompute the periodic walk's Ewald table (grid, series range)."""
        bh_set_ewald(self._ctx, n_grid, n_series)

    def ewald_eval(self, r):
        """chi at DEVICE float32 displacements r[n, 3] by the table."""
        import torch
        chi = torch.empty(r.shape[0], dtype=torch.float32, device=self.device)
        bh_ewald_eval(self._ctx, r, chi)
        self._handoff(chi)
        return chi

    def stats(self) -> dict:
        return bh_stats(self._ctx)

    def mlp_eval(self, x):
        import torch
        x = x.contiguous()
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        bh_mlp_eval(self._ctx, x, y)
        self._handoff(y)
        return y

    def get_mlp(self):
        return bh_get_mlp(self._ctx)

    def export_quadrupoles(self):
        import torch
        _, n, _ = self.tree_size()
        q = torch.empty((n, 6), dtype=torch.float64, device=self.device)
        bh_export_quadrupoles(self._ctx, q)
        self._handoff(q)
        return q

    def solve_host(self, level, ijk, density_host, theta, G=1.0, out_host=None,
                   box_lo=(0.0, 0.0, 0.0), box_len=1.0):
        if out_host is None:
            dt = np.float64 if self.options.precision == BH_PREC_F64 else np.float32
            out_host = np.empty(512 * len(level), dtype=dt)
        bh_solve_host(self._ctx, level, ijk, box_lo, box_len, density_host, theta, G, out_host)
        self.ncells = 512 * len(level)
        return out_host

    def close(self):
        if getattr(self, "_ctx", None):
            bh_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
