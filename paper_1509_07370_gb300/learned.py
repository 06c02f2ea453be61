"""Training of the learned residual correction on the GPU.

The walk accepts a node and adds its monopole M/d; the learned walk adds
(M/d)(1 + s^2 y) with y = MLP(x) of ten pair features (see include/bhgrav.h).
The network learns z = eps / s^2, where eps is the node's exact error against
its monopole.  Everything runs in the library's own kernels:
  * bh_learn_pairs lists, for sampled target cells of seeded training fields,
    every internal node their walk accepts and the exact residual of each pair;
  * bh_mlp_grad / bh_mlp_adam run the forward and backward passes and the
    optimiser steps.
Training fields: homogeneous oblate spheroids (the Maclaurin family of the
accuracy test) with seeded semi-axis a1 in [0.12, 0.3] and eccentricity in
[0.3, 0.95], on meshes of 32^3 cells refined twice at the surface.  Each
field's targets: random cells and the cells where the plain walk at the
training theta errs most against the exhaustive direct sum (computed by the
library itself at a theta below which no node is accepted) -- the pairs
that decide the largest errors.  (Measured over every cell of the 2M-cell
spheroid, two trainings each: 32 random + 32 worst cells per field gave a
max error of 1.66e-3 - 1.70e-3 at theta 0.8; 32 random + 32 in the densest
blocks 2.82e-3 - 2.86e-3; adding dense-block cells to the worst ones did
not help.)
"""
from __future__ import annotations

import numpy as np

from . import bhgrav as bh
from . import meshgen as mg

NW = bh.MLP_NW


def training_field(seed: int) -> mg.Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    a1 = float(rng.uniform(0.12, 0.3))
    e = float(rng.uniform(0.3, 0.95))
    return mg.maclaurin(base_level=2, extra_levels=2, a1=a1, e=e, rho_out=1e-4)


def init_weights(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases, in the flat layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_in, fan_out in ((10, 64), (64, 64), (64, 1)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, fan_in * fan_out))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def dense_cells(density: np.ndarray, nblocks: int = 8) -> np.ndarray:
    """Cell indices of the densest blocks (by mean density)."""
    mean = density.reshape(-1, 512).mean(axis=1)
    top = np.argsort(-mean, kind="stable")[:nblocks]
    return (top[:, None] * 512 + np.arange(512)[None, :]).reshape(-1)


def worst_cells(w: mg.Workload, density, theta: float, k: int, device: int = 0) -> np.ndarray:
    """The k cells where the plain monopole walk at theta has the largest
    relative error against the exhaustive direct sum, which the library
    computes at theta = 2^-(deepest cell level): there the smallest internal
    node has l/theta = 2, more than any box-unit distance, so no node is
    accepted and every cell meets every other cell singly."""
    plain = bh.Solver(device=device)
    plain.build(w.mesh.level, w.mesh.ijk, density, w.mesh.box_lo, w.mesh.box_len)
    _, _, maxlev = plain.tree_size()
    direct = plain.potential(2.0 ** -maxlev).double()
    err = (plain.potential(theta).double() / direct - 1.0).abs()
    plain.close()
    return np.sort(err.argsort(descending=True)[:k].cpu().numpy())


def pairs_of(solver: bh.Solver, ncells: int, theta: float, ntargets: int, seed: int,
             cap: int = 1 << 20, dense=None, extra=None):
    """(features, z) of the accepted pairs of `ntargets` cells: random ones,
    or half random and half drawn from `dense` (cell indices) if given; plus
    the cells in `extra`, if given."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    n = min(ntargets, ncells)
    if dense is None:
        cells = rng.choice(ncells, n, replace=False)
    else:
        cells = np.unique(np.concatenate([rng.choice(ncells, n - n // 2, replace=False),
                                          rng.choice(dense, min(n // 2, len(dense)),
                                                     replace=False)]))
    if extra is not None:
        cells = np.unique(np.concatenate([cells, np.asarray(extra, dtype=cells.dtype)]))
    tg = torch.as_tensor(cells, dtype=torch.int64, device=solver.device)
    feat, eps, _ = solver.learn_pairs(theta, tg, cap)
    with torch.cuda.stream(solver.stream):
        z = bh.bh_learn_targets(feat, eps, solver.stream.cuda_stream)
    solver.stream.synchronize()
    return feat, z


def make_dataset(nfields: int = 200, theta: float = 0.8, targets_per_field: int = 32,
                 seed0: int = 9000, device: int = 0, worst_per_field: int = 32,
                 dense: bool = False):
    """Method-generated training pairs from `nfields` seeded fields: per
    field, `targets_per_field` random cells (half of them from the densest
    blocks with dense=True) plus the `worst_per_field` cells where the plain
    walk errs most."""
    import torch
    xs, zs = [], []
    for i in range(nfields):
        w = training_field(seed0 + i)
        s = bh.Solver(quadrupole=True, device=device)
        rho = torch.as_tensor(w.density.reshape(-1), dtype=torch.float32, device=s.device)
        s.build(w.mesh.level, w.mesh.ijk, rho)
        worst = (worst_cells(w, rho, theta, worst_per_field, device)
                 if worst_per_field > 0 else None)
        x, z = pairs_of(s, w.ncells, theta, targets_per_field, seed0 + 100000 + i,
                        dense=dense_cells(w.density) if dense else None, extra=worst)
        xs.append(x)
        zs.append(z)
        s.close()
    return torch.cat(xs), torch.cat(zs)


def train(x, z, epochs: int = 16, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          w0: np.ndarray | None = None, stream: int = 0):
    """Adam on the mean squared error of MLP(x) against z, the learning rate
    halved after half and after three quarters of the epochs; returns the
    FP32 weights and the per-epoch mean losses."""
    import torch
    dev = x.device
    w = torch.as_tensor(init_weights(seed) if w0 is None else w0, device=dev).contiguous()
    m = torch.zeros(NW, device=dev)
    v = torch.zeros(NW, device=dev)
    g = torch.empty(NW, device=dev)
    loss = torch.empty(1, device=dev)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = z.numel()
    step = 0
    history = []
    for ep in range(epochs):
        rate = lr * (0.5 if ep >= epochs // 2 else 1.0) * (0.5 if ep >= (3 * epochs) // 4 else 1.0)
        perm = torch.randperm(n, generator=gen).to(dev)
        tot = 0.0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            xb, zb = x[idx].contiguous(), z[idx].contiguous()
            bh.bh_mlp_grad(xb, zb, w, g, loss, stream)
            step += 1
            bh.bh_mlp_adam(g, w, m, v, step, rate, stream)
            tot += float(loss.item()) * idx.numel()
        history.append(tot / n)
    return w.cpu().numpy(), history
