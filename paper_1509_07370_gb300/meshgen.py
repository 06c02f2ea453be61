"""Seeded synthetic AMR meshes and density fields.

This module only *makes inputs*: block geometry of an octree AMR mesh made of
8^3-cell blocks (the PARAMESH layout the paper's solver reads, Sec. 3.1.1) and
cell densities on it.  It holds none of the Barnes-Hut arithmetic; both the
CUDA library and the CPU oracle consume what it produces.

Conventions (shared by every consumer):
  * The box is the cube [lo, lo + L)^3; by default lo = 0, L = 1.
  * A block has a level lb >= 0 and integer coordinates (bi, bj, bk) in
    [0, 2^lb); it covers the cube of side L / 2^lb at that position and holds
    8^3 cells of side L / 2^(lb+3).
  * Densities are float arrays of shape [nblocks, 8, 8, 8] indexed
    [block, cz, cy, cx] -- x fastest in memory.
  * Blocks are returned sorted by the Morton key of their lower corner, the
    space-filling-curve order FLASH uses for its domain decomposition
    (Sec. 2.1).  The library accepts any order; sorting is a convenience.

Workloads (the paper's FLASH test problems are not available; these are
synthetic stand-ins with the same structure):
  * ``uniform_sphere``: a top-hat sphere on a uniform mesh (Eq. topeq shape).
  * ``maclaurin``: an oblate spheroid of eccentricity 0.9 on a mesh refined
    at its surface (Sec. 4.1).
  * ``cloud_core``: a centrally concentrated, perturbed, Jeans-refined cloud
    core (the collapsing-core setups of Sec. 4.2).
"""
from __future__ import annotations

import dataclasses
import functools

import numpy as np

MAX_BLOCK_LEVEL = 18          # cells then sit at level <= 21: 63-bit Morton keys
CELLS_PER_BLOCK = 512


# ----------------------------------------------------------------------------
# Morton keys (input ordering only)
# ----------------------------------------------------------------------------
def _spread3(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def corner_keys(level: np.ndarray, ijk: np.ndarray) -> np.ndarray:
    """Morton key of each block's lower corner on the level-21 cell lattice."""
    sh = (np.uint64(21) - (level.astype(np.uint64) + np.uint64(3)))
    ijk = ijk.astype(np.uint64) << (sh[:, None] + np.uint64(3))
    return _spread3(ijk[:, 0]) | (_spread3(ijk[:, 1]) << np.uint64(1)) | (
        _spread3(ijk[:, 2]) << np.uint64(2))


@dataclasses.dataclass
class Mesh:
    """Leaf blocks of an AMR mesh in the unit-of-blocks description above."""

    level: np.ndarray          # int32 [nb]
    ijk: np.ndarray            # int32 [nb, 3]
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_len: float = 1.0
    name: str = "mesh"

    @property
    def nblocks(self) -> int:
        return int(self.level.shape[0])

    @property
    def ncells(self) -> int:
        return CELLS_PER_BLOCK * self.nblocks

    def cell_centres(self) -> np.ndarray:
        """Physical cell-centre coordinates, shape [nb, 8, 8, 8, 3] (x, y, z)."""
        c = np.arange(8, dtype=np.float64) + 0.5
        h = self.box_len / np.exp2(self.level.astype(np.float64) + 3)  # cell side
        base = self.ijk.astype(np.float64) * 8.0
        x = (base[:, 0, None] + c[None, :]) * h[:, None] + self.box_lo[0]
        y = (base[:, 1, None] + c[None, :]) * h[:, None] + self.box_lo[1]
        z = (base[:, 2, None] + c[None, :]) * h[:, None] + self.box_lo[2]
        nb = self.nblocks
        out = np.empty((nb, 8, 8, 8, 3))
        out[..., 0] = x[:, None, None, :]
        out[..., 1] = y[:, None, :, None]
        out[..., 2] = z[:, :, None, None]
        return out

    def cell_side(self) -> np.ndarray:
        """Physical side of the cells of each block, shape [nb]."""
        return self.box_len / np.exp2(self.level.astype(np.float64) + 3)

    def level_histogram(self) -> dict:
        lv, n = np.unique(self.level, return_counts=True)
        return {int(a): int(b) for a, b in zip(lv, n)}


def _sorted_mesh(levels: list, ijks: list, **kw) -> Mesh:
    level = np.concatenate(levels).astype(np.int32)
    ijk = np.concatenate(ijks).astype(np.int32).reshape(-1, 3)
    order = np.argsort(corner_keys(level, ijk), kind="stable")
    return Mesh(level=level[order], ijk=np.ascontiguousarray(ijk[order]), **kw)


def uniform_mesh(block_level: int, **kw) -> Mesh:
    n = 1 << block_level
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n),
                             indexing="ij"), -1).reshape(-1, 3)
    return _sorted_mesh([np.full(len(g), block_level)], [g], **kw)


# ----------------------------------------------------------------------------
# Refinement with 2:1 balance
# ----------------------------------------------------------------------------
def _code(level: int, ijk: np.ndarray) -> np.ndarray:
    """Unique integer id of a dyadic cube (level, ijk)."""
    ijk = ijk.astype(np.int64)
    return (np.int64(level) << np.int64(57)) | (ijk[:, 0] << np.int64(38)) | (
        ijk[:, 1] << np.int64(19)) | ijk[:, 2]


_NEIGH = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1)
                   for c in (-1, 0, 1) if (a, b, c) != (0, 0, 0)], dtype=np.int64)


def _children(ijk: np.ndarray) -> np.ndarray:
    o = np.array([(x, y, z) for z in (0, 1) for y in (0, 1) for x in (0, 1)],
                 dtype=np.int64)
    return (2 * ijk.astype(np.int64)[:, None, :] + o[None, :, :]).reshape(-1, 3)


def _balance(leaves: dict) -> dict:
    """Refine leaves until face/edge/corner neighbours differ by <= 1 level."""
    while True:
        deep = set()
        for lev, ijk in leaves.items():
            for a in range(0, lev - 1):
                deep.update(_code(a, ijk >> (lev - a)).tolist())
        if not deep:
            return leaves
        deep_arr = np.fromiter(deep, dtype=np.int64)
        changed = False
        new = {}
        for lev, ijk in sorted(leaves.items()):
            n = 1 << lev
            nb = ijk.astype(np.int64)[:, None, :] + _NEIGH[None, :, :]
            ok = np.all((nb >= 0) & (nb < n), axis=2)
            codes = _code(lev, nb.reshape(-1, 3)).reshape(nb.shape[:2])
            bad = np.any(np.isin(codes, deep_arr) & ok, axis=1)
            if bad.any():
                changed = True
                new.setdefault(lev + 1, []).append(_children(ijk[bad]))
            new.setdefault(lev, []).append(ijk[~bad])
        leaves = {k: np.concatenate(v) for k, v in new.items()
                  if sum(len(x) for x in v)}
        if not changed:
            return leaves


def refined_mesh(base_level: int, max_level: int, needs_refine, name="amr",
                 **kw) -> Mesh:
    """Refine a uniform block mesh level by level.

    ``needs_refine(level, ijk) -> bool[n]`` flags blocks (at ``level``) to be
    split into 8 children; the mesh is 2:1 balanced after every level.
    """
    assert 0 <= base_level <= max_level <= MAX_BLOCK_LEVEL
    n = 1 << base_level
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n),
                             indexing="ij"), -1).reshape(-1, 3)
    leaves = {base_level: g.astype(np.int64)}
    for lev in range(base_level, max_level):
        cur = leaves.get(lev)
        if cur is None or len(cur) == 0:
            continue
        flag = np.asarray(needs_refine(lev, cur), dtype=bool)
        if flag.any():
            leaves[lev + 1] = np.concatenate(
                [leaves.get(lev + 1, np.zeros((0, 3), np.int64)),
                 _children(cur[flag])])
            leaves[lev] = cur[~flag]
        leaves = _balance(leaves)
    lv = [np.full(len(v), k) for k, v in leaves.items() if len(v)]
    ij = [v for v in leaves.values() if len(v)]
    return _sorted_mesh(lv, ij, name=name, **kw)


def block_bounds(mesh_level: int, ijk: np.ndarray, box_len=1.0, box_lo=(0, 0, 0)):
    h = box_len / (1 << mesh_level)
    lo = ijk.astype(np.float64) * h + np.asarray(box_lo, dtype=np.float64)
    return lo, lo + h


# ----------------------------------------------------------------------------
# Densities
# ----------------------------------------------------------------------------
def _volume_fraction(mesh: Mesh, inside, sdist, sub: int = 4) -> np.ndarray:
    """Fraction of each cell's volume for which ``inside(x,y,z)`` holds.

    Cells whose centre lies farther than 1.5 half-diagonals from the surface
    (by the approximate signed distance ``sdist``) are taken as fully in or
    out; the others are sampled on a sub^3 lattice.
    """
    xc = mesh.cell_centres()
    h = mesh.cell_side()[:, None, None, None]
    d = sdist(xc[..., 0], xc[..., 1], xc[..., 2])
    frac = (d < 0).astype(np.float64)
    near = np.abs(d) < 1.5 * 0.8660254 * h
    idx = np.nonzero(near)
    if len(idx[0]):
        pts = xc[idx]                                  # [m, 3]
        hs = np.broadcast_to(h, near.shape)[idx]       # [m]
        o = (np.arange(sub) + 0.5) / sub - 0.5
        off = np.stack(np.meshgrid(o, o, o, indexing="ij"), -1).reshape(-1, 3)
        acc = np.zeros(len(pts))
        for k in range(len(off)):
            q = pts + off[k][None, :] * hs[:, None]
            acc += inside(q[:, 0], q[:, 1], q[:, 2])
        frac[idx] = acc / len(off)
    return frac


def sphere_density(mesh: Mesh, centre, radius, rho_in, rho_out, sub=4):
    cx, cy, cz = centre

    def inside(x, y, z):
        return ((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) < radius ** 2

    def sdist(x, y, z):
        return np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - radius

    f = _volume_fraction(mesh, inside, sdist, sub)
    return rho_out + (rho_in - rho_out) * f


def spheroid_density(mesh: Mesh, centre, a1, a3, rho_in, rho_out, sub=4):
    cx, cy, cz = centre

    def fimp(x, y, z):
        return ((x - cx) ** 2 + (y - cy) ** 2) / a1 ** 2 + (z - cz) ** 2 / a3 ** 2

    def inside(x, y, z):
        return fimp(x, y, z) < 1.0

    def sdist(x, y, z):
        # first-order distance to the surface f = 1
        g = 2.0 * np.sqrt(((x - cx) ** 2 + (y - cy) ** 2) / a1 ** 4 +
                          (z - cz) ** 2 / a3 ** 4) + 1e-300
        return (fimp(x, y, z) - 1.0) / g

    f = _volume_fraction(mesh, inside, sdist, sub)
    return rho_out + (rho_in - rho_out) * f


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    density: np.ndarray            # float64 [nb, 8, 8, 8]
    thetas: tuple
    G: float = 1.0
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return self.mesh.ncells


def uniform_sphere(block_level=2, radius=0.5, rho_in=1.0, rho_out=1e-3) -> Workload:
    """Top-hat sphere (r = 0.5, contrast 1e-3) on a uniform mesh.

    block_level 2 gives 4^3 blocks = 32^3 cells, the plain FP64 test case.
    """
    m = uniform_mesh(block_level, name=f"uniform_sphere_{8 << block_level}^3")
    rho = sphere_density(m, (0.5, 0.5, 0.5), radius, rho_in, rho_out)
    return Workload(m.name, m, rho, (0.5,), meta=dict(
        centre=(0.5, 0.5, 0.5), radius=radius, rho_in=rho_in, rho_out=rho_out))


MACLAURIN_A1 = 0.25
MACLAURIN_E = 0.9


def maclaurin(base_level=2, extra_levels=3, a1=MACLAURIN_A1, e=MACLAURIN_E,
              rho_in=1.0, rho_out=1e-5) -> Workload:
    """Oblate spheroid (a1 = a2 = 0.25, eccentricity 0.9) refined at its surface.

    Base mesh 4^3 blocks (32^3 cells); blocks within about one block
    half-diagonal of the surface are refined ``extra_levels`` times (finest
    cell 1/256 by default, 2,039,808 cells) and the mesh is 2:1 balanced.
    """
    a3 = a1 * np.sqrt(1.0 - e * e)
    c = 0.5

    def fimp(x, y, z):
        return ((x - c) ** 2 + (y - c) ** 2) / a1 ** 2 + (z - c) ** 2 / a3 ** 2

    def crosses(lev, ijk):
        lo, hi = block_bounds(lev, ijk)
        s = np.linspace(0.0, 1.0, 5)
        fs = []
        for u in s:
            for v in s:
                for w in s:
                    p = lo + (hi - lo) * np.array([u, v, w])
                    fs.append(fimp(p[:, 0], p[:, 1], p[:, 2]))
        fs = np.stack(fs, 1)
        ctr = 0.5 * (lo + hi)
        g = 2.0 * np.sqrt(((ctr[:, 0] - c) ** 2 + (ctr[:, 1] - c) ** 2) / a1 ** 4
                          + (ctr[:, 2] - c) ** 2 / a3 ** 4) + 1e-300
        dist = np.abs(fimp(ctr[:, 0], ctr[:, 1], ctr[:, 2]) - 1.0) / g
        halfdiag = 0.5 * np.sqrt(3.0) * (hi[:, 0] - lo[:, 0])
        return ((fs.min(1) < 1.0) & (fs.max(1) > 1.0)) | (dist < 1.0 * halfdiag)

    m = refined_mesh(base_level, base_level + extra_levels, crosses,
                     name=f"maclaurin_e{e}_L{base_level}+{extra_levels}")
    rho = spheroid_density(m, (c, c, c), a1, a3, rho_in, rho_out)
    return Workload(m.name, m, rho, (0.3, 0.5, 0.7), meta=dict(
        centre=(c, c, c), a1=a1, a3=a3, e=e, rho_in=rho_in, rho_out=rho_out))


@functools.lru_cache(maxsize=4)
def _noise_lattice(n=128, seed=3) -> np.ndarray:
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((n, n, n))


def _trilinear(lat: np.ndarray, x, y, z):
    n = lat.shape[0]
    u = np.clip(np.stack([x, y, z], -1) * (n - 1), 0, n - 1 - 1e-9)
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    out = 0.0
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (np.where(dx, f[..., 0], 1 - f[..., 0]) *
                     np.where(dy, f[..., 1], 1 - f[..., 1]) *
                     np.where(dz, f[..., 2], 1 - f[..., 2]))
                out = out + w * lat[i0[..., 0] + dx, i0[..., 1] + dy, i0[..., 2] + dz]
    return out


def cloud_core_profile(x, y, z, rho_c=1.0, r0=0.05, amp_m2=0.1, sigma=0.1,
                       seed=3):
    """rho_c / (1 + (r/r0)^2), cut to an ambient of rho_c*1e-4 where it falls
    below rho_c/100, times a 10 % m=2 azimuthal mode and lognormal noise."""
    dx, dy, dz = x - 0.5, y - 0.5, z - 0.5
    r2 = dx * dx + dy * dy + dz * dz
    base = rho_c / (1.0 + r2 / (r0 * r0))
    phi = np.arctan2(dy, dx)
    g = _trilinear(_noise_lattice(seed=seed), x, y, z)
    pert = (1.0 + amp_m2 * np.cos(2.0 * phi)) * np.exp(sigma * g - 0.5 * sigma ** 2)
    return np.where(base >= rho_c / 100.0, base * pert, rho_c * 1e-4)


def _cloud_mesh(c_jeans: float, base_level: int, max_level: int, r0: float) -> Mesh:
    def jeans(lev, ijk):
        lo, hi = block_bounds(lev, ijk)
        near = np.clip(0.5, lo, hi)                  # point nearest the centre
        r2 = np.sum((near - 0.5) ** 2, axis=1)
        rho_max = 1.1 * 1.0 / (1.0 + r2 / (r0 * r0))
        dx_cell = (hi[:, 0] - lo[:, 0]) / 8.0
        return dx_cell * np.sqrt(rho_max) > c_jeans
    return refined_mesh(base_level, max_level, jeans, name="cloud_core")


CLOUD_CORE_C_JEANS = 0.0010273507681793025   # gives 16,289,792 cells


def calibrate_cloud_core(target_cells, base_level=2, extra_levels=6, r0=0.05):
    """Bisect the Jeans refinement constant so the cell count lands within
    10 % of ``target_cells``; returns (constant, mesh)."""
    lo_c, hi_c = 1e-5, 1.0
    best = None
    for _ in range(40):
        mid = np.sqrt(lo_c * hi_c)
        m = _cloud_mesh(mid, base_level, base_level + extra_levels, r0)
        if best is None or abs(m.ncells - target_cells) < abs(best[1].ncells - target_cells):
            best = (mid, m)
        if abs(m.ncells - target_cells) <= 0.1 * target_cells:
            break
        if m.ncells > target_cells:
            lo_c = mid
        else:
            hi_c = mid
    return best


def cloud_core(c_jeans=CLOUD_CORE_C_JEANS, base_level=2, extra_levels=6, r0=0.05,
               seed=3) -> Workload:
    """Jeans-refined collapsing cloud core (16,289,792 cells by default).

    A block is refined while its cell side exceeds c_jeans / sqrt(rho_max)
    (rho_max: the smooth profile at the block point nearest the centre, with
    a 10 % margin for the m=2 mode), i.e. a fixed number of cells per Jeans
    length lambda_J ~ rho^-1/2 (Truelove-style refinement, Sec. 4.2.1).
    """
    m = _cloud_mesh(c_jeans, base_level, base_level + extra_levels, r0)
    x = m.cell_centres()
    rho = cloud_core_profile(x[..., 0], x[..., 1], x[..., 2], r0=r0, seed=seed)
    return Workload(f"cloud_core_{m.ncells}", m, rho, (0.5,), meta=dict(
        c_jeans=float(c_jeans), r0=r0, seed=seed, levels=m.level_histogram()))


def random_blob_field(seed: int, block_level: int, nblobs=None) -> Workload:
    """Uniform mesh with a mixture of 1-8 Gaussian blobs of lognormal mass
    (sigma = 1) and width 0.02-0.2; used for many small independent fields."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = uniform_mesh(block_level, name=f"blobs_s{seed}_{8 << block_level}^3")
    k = int(rng.integers(1, 9)) if nblobs is None else nblobs
    ctr = rng.uniform(0.2, 0.8, size=(k, 3))
    w = rng.uniform(0.02, 0.2, size=k)
    mass = rng.lognormal(0.0, 1.0, size=k)
    x = m.cell_centres()
    rho = np.full(x.shape[:-1], 1e-3)
    for i in range(k):
        r2 = np.sum((x - ctr[i]) ** 2, axis=-1)
        rho += mass[i] / (2 * np.pi * w[i] ** 2) ** 1.5 * np.exp(-0.5 * r2 / w[i] ** 2)
    return Workload(m.name, m, rho, (0.5,), meta=dict(seed=seed, nblobs=k))


def batch_fields(nfields=64, seed0=5000, levels=(1, 2, 3, 4)):
    """Independent fields of uneven size for the batched solve: field i is a
    uniform mesh of 16^3, 32^3, 64^3 or 128^3 cells (block level drawn from
    ``levels`` with seed seed0 + i) holding 1-8 Gaussian blobs of lognormal
    mass (sigma 1) and width 0.02-0.2.  Returns the list of Workloads."""
    out = []
    for i in range(nfields):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        lev = int(rng.choice(levels))
        out.append(random_blob_field(seed0 + i, lev))
    return out


def concat_fields(workloads):
    """Concatenated block geometry and densities of several fields, as the
    batched build takes them: (nblocks, level, ijk, box_lo, box_len, density)."""
    nb = np.array([w.mesh.nblocks for w in workloads], dtype=np.int32)
    level = np.concatenate([w.mesh.level for w in workloads]).astype(np.int32)
    ijk = np.concatenate([w.mesh.ijk for w in workloads]).astype(np.int32)
    lo = np.array([w.mesh.box_lo for w in workloads], dtype=np.float64)
    ln = np.array([w.mesh.box_len for w in workloads], dtype=np.float64)
    rho = np.concatenate([w.density.reshape(-1) for w in workloads])
    return nb, level, ijk, lo, ln, rho


def tiny_meshes() -> dict:
    """Small meshes for exhaustive checks: 1 block, 8 blocks, and mixed-level
    meshes (one octant refined once / twice) with ragged level structure."""
    out = {"one_block": uniform_mesh(0, name="one_block"),
           "eight_blocks": uniform_mesh(1, name="eight_blocks")}

    def corner(lev, ijk):
        return np.all(ijk == 0, axis=1)

    out["refined_corner"] = refined_mesh(1, 2, corner, name="refined_corner")
    out["refined_twice"] = refined_mesh(1, 3, corner, name="refined_twice")

    def diag(lev, ijk):
        return (ijk[:, 0] == ijk[:, 1]) & (ijk[:, 1] == ijk[:, 2])

    out["diag_refined"] = refined_mesh(1, 3, diag, name="diag_refined")
    return out


def random_density(mesh: Mesh, seed: int, lo=0.1, hi=2.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(mesh.nblocks, 8, 8, 8))


def shuffled(mesh: Mesh, density: np.ndarray, seed: int):
    """The same mesh with its blocks listed in a random order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = rng.permutation(mesh.nblocks)
    m2 = Mesh(level=mesh.level[p].copy(), ijk=mesh.ijk[p].copy(),
              box_lo=mesh.box_lo, box_len=mesh.box_len, name=mesh.name + "_shuffled")
    return m2, density[p].copy()
