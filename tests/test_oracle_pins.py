"""Pins of the CPU oracle against facts it does not itself produce.

Each check is chosen so that a plausible slip in the oracle -- a dropped or
double-counted term, a wrong sign, a swapped axis or octant, a wrong scale, a
wrong child order -- fails at least one of them:

* closed forms: uniform sphere (textbook), corrected Maclaurin spheroid
  (Sec. 4.1), uniform prism, and their Laplacian / continuity / far field;
* special cases: two point masses, two massive cells, theta -> 0 equals the
  direct sum, linearity in rho, scaling with the box;
* invariants: node count of a full octree, octant topology, moments against
  a separate numpy sum over the cells of each subtree, and the accepted set
  of every target partitioning all other cells exactly once;
* the paper's printed accuracy curve (Fig. Errors) as an order-of-magnitude
  and monotonicity check.
"""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import oracle as O
from paper_1509_07370_gb300 import meshgen as mg


# ---------------------------------------------------------------- helpers --
def _tree(mesh, rho, **kw):
    return O.Tree(mesh.level, mesh.ijk, rho, mesh.box_lo, mesh.box_len, **kw)


def _cell_geometry(mesh):
    """Box-unit centres, levels and masses of the caller-layout cells."""
    x = mesh.cell_centres().reshape(-1, 3)
    u = (x - np.asarray(mesh.box_lo)) / mesh.box_len
    lev = np.repeat(mesh.level.astype(np.int64) + 3, 512)
    return u, lev


def _subtree_end(parent):
    """Pre-order index one past the end of each node's subtree."""
    n = len(parent)
    end = np.arange(1, n + 1)
    for i in range(n - 1, 0, -1):
        p = parent[i]
        end[p] = max(end[p], end[i])
    return end


@pytest.fixture(scope="module")
def tiny():
    out = {}
    for i, (name, m) in enumerate(sorted(mg.tiny_meshes().items())):
        out[name] = (m, mg.random_density(m, seed=100 + i))
    return out


# ------------------------------------------------------------ closed forms --
def test_cube_centre_constant():
    # integral of 1/r over a unit cube from its centre: 8 * (1/2)^2 times the
    # classical corner integral 3 ln(1+sqrt3) - (3/2) ln 2 - pi/4 = 1.19003...
    s3 = np.sqrt(3.0)
    exact = 2.0 * (3.0 * np.log(1.0 + s3) - 1.5 * np.log(2.0) - np.pi / 4.0)
    assert abs(A.cube_centre_factor() - exact) < 1e-12


def test_prism_against_quadrature():
    n = 48
    g = (np.arange(n) + 0.5) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    for p in [(1.7, 0.3, -0.4), (-0.6, 1.4, 2.2), (0.5, 0.5, 3.0)]:
        q = -np.sum(1.0 / np.sqrt((X - p[0]) ** 2 + (Y - p[1]) ** 2 + (Z - p[2]) ** 2)) / n ** 3
        assert abs(A.prism(*p, (0, 0, 0), (1, 1, 1), 1.0) / q - 1.0) < 1e-5


def _laplacian(f, x, y, z, h=1e-4):
    return (f(x + h, y, z) + f(x - h, y, z) + f(x, y + h, z) + f(x, y - h, z)
            + f(x, y, z + h) + f(x, y, z - h) - 6.0 * f(x, y, z)) / (h * h)


@pytest.mark.parametrize("kind", ["sphere", "maclaurin", "prism"])
def test_poisson_equation(kind):
    """Laplacian Phi = 4 pi G rho inside the body and 0 outside."""
    if kind == "sphere":
        f = lambda x, y, z: A.uniform_sphere(x, y, z, (0, 0, 0), 0.3, 1.0)
        pin, pout = (0.1, -0.05, 0.12), (0.25, 0.3, -0.2)
    elif kind == "maclaurin":
        f = lambda x, y, z: A.maclaurin(x, y, z, (0, 0, 0), 0.25, 0.9, 1.0)
        pin, pout = (0.12, 0.08, 0.03), (0.2, 0.15, 0.1)
    else:
        f = lambda x, y, z: A.prism(x, y, z, (0, 0, 0), (1, 0.5, 0.25), 1.0)
        pin, pout = (0.3, 0.2, 0.1), (1.3, 0.2, 0.6)
    assert abs(_laplacian(f, *pin) / (4.0 * np.pi) - 1.0) < 1e-5
    assert abs(_laplacian(f, *pout) / (4.0 * np.pi)) < 1e-5


def test_maclaurin_coefficients_sum_to_two():
    for e in (0.1, 0.5, 0.9, 0.99):
        A1, A3 = A.maclaurin_coefficients(e)
        assert abs(2.0 * A1 + A3 - 2.0) < 1e-12


def test_maclaurin_continuous_at_surface_and_far_field():
    a1, e = 0.25, 0.9
    a3 = a1 * np.sqrt(1 - e * e)
    f = lambda x, y, z: A.maclaurin(x, y, z, (0, 0, 0), a1, e, 1.0)
    for d in [(1, 0, 0), (0, 0, 1), (0.6, 0.5, 0.62)]:
        d = np.asarray(d) / np.sqrt((d[0] ** 2 + d[1] ** 2) / a1 ** 2 + d[2] ** 2 / a3 ** 2)
        v_in, v_out = f(*(d * (1 - 1e-9))), f(*(d * (1 + 1e-9)))
        assert abs(v_in / v_out - 1.0) < 1e-7
        # the normal derivative is continuous too (no surface mass)
        g_in = (f(*(d * (1 - 1e-6))) - f(*(d * (1 - 2e-6)))) / 1e-6
        g_out = (f(*(d * (1 + 2e-6))) - f(*(d * (1 + 1e-6)))) / 1e-6
        assert abs(g_in / g_out - 1.0) < 1e-3
    M = 4.0 / 3.0 * np.pi * a1 * a1 * a3
    for p in [(80.0, 0, 0), (0, 0, 80.0), (40.0, 50.0, 30.0)]:
        r = np.sqrt(sum(c * c for c in p))
        assert abs(f(*p) * r / (-M) - 1.0) < 1e-5


def test_maclaurin_sphere_limit():
    for p in [(0.1, 0.0, 0.05), (0.4, 0.3, 0.0)]:
        assert abs(A.maclaurin(*p, (0, 0, 0), 0.25, 1e-4, 1.0)
                   / A.uniform_sphere(*p, (0, 0, 0), 0.25, 1.0) - 1.0) < 1e-6


# --------------------------------------------------------- direct sums -----
def test_direct_points_two_and_three_bodies():
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    phi = O.direct_points(pos, [2.0, 5.0], G=0.5)
    assert phi[0] == -0.5 * 5.0 / 5.0 and phi[1] == -0.5 * 2.0 / 5.0
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    phi = O.direct_points(pos, [1.0, 1.0, 1.0])
    assert np.allclose(phi, [-(1 + 0.5), -(1 + 1 / np.sqrt(5)), -(0.5 + 1 / np.sqrt(5))],
                       rtol=1e-15)


def test_two_massive_cells_direct_and_walk():
    """All mass in two cells: every method must give -G m_other / r."""
    m = mg.uniform_mesh(1)
    rho = np.zeros((8, 8, 8, 8))
    rho[0, 1, 2, 3] = 3.0            # block 0, cz=1, cy=2, cx=3
    rho[7, 6, 5, 4] = 5.0
    t = _tree(m, rho)
    u, lev = _cell_geometry(m)
    a = 0 * 512 + 1 * 64 + 2 * 8 + 3
    b = 7 * 512 + 6 * 64 + 5 * 8 + 4
    r = np.linalg.norm(u[a] - u[b])
    vol = (1.0 / 16) ** 3
    G = 2.0
    want = np.array([-G * 5.0 * vol / r, -G * 3.0 * vol / r])
    assert np.allclose(t.direct(G=G, targets=[a, b]), want, rtol=1e-14)
    for theta in (0.2, 0.5, 1.0):
        assert np.allclose(t.walk(theta, G=G, targets=[a, b])[0], want, rtol=1e-13)


def test_self_term_excluded_and_sign():
    m = mg.uniform_mesh(0)
    rho = np.zeros((1, 8, 8, 8))
    rho[0, 4, 4, 4] = 1.0
    t = _tree(m, rho)
    c = 4 * 64 + 4 * 8 + 4
    assert t.direct(targets=[c])[0] == 0.0
    assert t.walk(0.5, targets=[c])[0][0] == 0.0
    other = t.direct(targets=[c + 1])[0]
    assert other < 0.0 and abs(other / (-(1 / 8) ** 3 / (1 / 8)) - 1.0) < 1e-14


# ------------------------------------------------------------- the tree ---
def test_full_octree_node_count(tiny):
    for name, (m, rho) in tiny.items():
        t = _tree(m, rho)
        n = m.ncells
        assert t.nnodes == n + (n - 1) // 7, name


def test_octant_topology_and_preorder(tiny):
    m, rho = tiny["refined_twice"]
    e = _tree(m, rho).export()
    lev, ijk, par, leaf = e["level"], e["ijk"], e["parent"], e["is_leaf"]
    assert par[0] == -1 and lev[0] == 0
    kids = {}
    for i in range(1, len(par)):
        assert par[i] < i                                   # pre-order
        assert lev[i] == lev[par[i]] + 1
        assert np.all(ijk[i] // 2 == ijk[par[i]])          # inside the parent cube
        kids.setdefault(par[i], []).append(i)
    for p, ch in kids.items():
        assert len(ch) == 8 and not leaf[p]
        o = [int((ijk[c][0] & 1) + 2 * (ijk[c][1] & 1) + 4 * (ijk[c][2] & 1)) for c in ch]
        assert o == list(range(8))                          # octant order x, y, z
    # leaves are exactly the caller cells, each once
    cells = np.sort(e["cell"][leaf == 1])
    assert np.array_equal(cells, np.arange(m.ncells))


def test_moments_against_cell_sums(tiny):
    """M and R of every node equal the mass and mass-weighted mean of the
    cells inside its cube (numpy, independent of the recursion)."""
    m, rho = tiny["diag_refined"]
    e = _tree(m, rho).export()
    u, lev = _cell_geometry(m)
    mass = rho.reshape(-1) * (m.box_len / np.exp2(lev)) ** 3
    rng = np.random.default_rng(1)
    internal = np.nonzero(e["is_leaf"] == 0)[0]
    for nid in np.concatenate([[0], rng.choice(internal, 40, replace=False)]):
        L = e["level"][nid]
        inside = np.all(np.floor(u * (1 << L)).astype(np.int64) == e["ijk"][nid], axis=1)
        Mw = mass[inside].sum()
        Rw = (mass[inside, None] * u[inside]).sum(0) / Mw
        assert abs(e["M"][nid] / Mw - 1.0) < 1e-13
        assert np.allclose(e["R"][nid], Rw, rtol=0, atol=1e-14)
        c = (e["ijk"][nid] + 0.5) / (1 << L)
        assert abs(e["delta"][nid] - np.linalg.norm(Rw - c)) < 1e-14


def test_geometry_errors():
    m = mg.uniform_mesh(1)
    rho = np.ones((8, 8, 8, 8))
    with pytest.raises(O.OracleError) as ex:          # gap: one block missing
        O.Tree(m.level[:7], m.ijk[:7], rho[:7])
    assert ex.value.code == O.OR_ERR_GEOMETRY
    lv = np.concatenate([m.level, [2]])
    ij = np.concatenate([m.ijk, [[0, 0, 0]]])
    with pytest.raises(O.OracleError):                 # overlap: a finer block inside
        O.Tree(lv, ij, np.ones((9, 8, 8, 8)))
    with pytest.raises(O.OracleError):                 # duplicate block
        O.Tree(np.concatenate([m.level, [1]]), np.concatenate([m.ijk, [[1, 1, 1]]]),
               np.ones((9, 8, 8, 8)))
    with pytest.raises(O.OracleError):                 # coordinate outside its level
        O.Tree([0], [[1, 0, 0]], np.ones((1, 8, 8, 8)))
    bad = rho.copy()
    bad[3, 1, 1, 1] = -1.0
    with pytest.raises(O.OracleError) as ex:
        O.Tree(m.level, m.ijk, bad)
    assert ex.value.code == O.OR_ERR_ARG


def test_block_order_does_not_matter(tiny):
    m, rho = tiny["refined_corner"]
    t1 = _tree(m, rho)
    m2, rho2 = mg.shuffled(m, rho, seed=5)
    t2 = _tree(m2, rho2)
    e1, e2 = t1.export(), t2.export()
    assert np.array_equal(e1["M"], e2["M"]) and np.array_equal(e1["R"], e2["R"])
    p = np.random.default_rng(5).permutation(m.nblocks)      # same as mg.shuffled
    inv = np.argsort(p)
    tg = np.arange(m.ncells)
    tg2 = inv[tg // 512] * 512 + tg % 512
    assert np.array_equal(t1.walk(0.5, targets=tg)[0], t2.walk(0.5, targets=tg2)[0])


# ------------------------------------------------------------- the walk ---
def test_theta_to_zero_is_direct_sum(tiny):
    for name, (m, rho) in tiny.items():
        t = _tree(m, rho)
        tg = np.arange(0, m.ncells, 7)
        walk, ni, nt = t.walk(1e-6, targets=tg)
        d = t.direct(targets=tg)
        assert np.allclose(walk, d, rtol=1e-13, atol=0), name
        assert np.all(ni == m.ncells - 1)                 # every other cell, once


@pytest.mark.parametrize("theta", [0.3, 0.5, 1.0])
def test_accepted_set_partitions_all_other_cells(tiny, theta):
    """Every cell other than the target is covered by exactly one accepted
    node (or is itself an accepted leaf); the target is covered by none."""
    for name in ("refined_corner", "diag_refined"):
        m, rho = tiny[name]
        t = _tree(m, rho)
        e = t.export()
        end = _subtree_end(e["parent"])
        leaf_pos = np.nonzero(e["is_leaf"])[0]
        cell_at = e["cell"][leaf_pos]
        rng = np.random.default_rng(int(theta * 10))
        for tgt in rng.choice(m.ncells, 25, replace=False):
            acc = t.walk_list(theta, tgt)
            cover = np.zeros(m.ncells, np.int64)
            for nid in acc:
                sel = (leaf_pos >= nid) & (leaf_pos < end[nid])
                cover[cell_at[sel]] += 1
            want = np.ones(m.ncells, np.int64)
            want[tgt] = 0
            assert np.array_equal(cover, want), (name, tgt)


@pytest.mark.parametrize("theta", [0.3, 0.7, 1.0])
def test_accepted_nodes_pass_criterion_and_opened_ancestors_fail(tiny, theta):
    """Eq. 4 in FP64 (allowing for the binary32 evaluation of the test)."""
    m, rho = tiny["diag_refined"]
    t = _tree(m, rho)
    e = t.export()
    u, _ = _cell_geometry(m)
    rng = np.random.default_rng(3)
    for tgt in rng.choice(m.ncells, 15, replace=False):
        for nid in t.walk_list(theta, tgt):
            chain = [nid]
            while e["parent"][chain[-1]] >= 0:
                chain.append(e["parent"][chain[-1]])
            for k, a in enumerate(chain):
                if e["is_leaf"][a]:
                    continue
                s = np.exp2(-e["level"][a]) / theta + e["delta"][a]
                d = np.linalg.norm(u[tgt] - e["R"][a])
                if k == 0:
                    assert d > s * (1 - 1e-6)                 # accepted
                else:
                    assert d <= s * (1 + 1e-6)                # opened on the way


def test_interactions_fall_as_theta_grows(tiny):
    m, rho = tiny["diag_refined"]
    t = _tree(m, rho)
    tg = np.arange(0, m.ncells, 5)
    counts = [t.walk(th, targets=tg)[1].sum() for th in (0.2, 0.4, 0.6, 0.8, 1.0)]
    assert all(a > b for a, b in zip(counts, counts[1:]))


def test_linearity_and_box_scaling(tiny):
    m, rho = tiny["refined_corner"]
    tg = np.arange(0, m.ncells, 3)
    base = _tree(m, rho).walk(0.5, targets=tg)[0]
    assert np.array_equal(_tree(m, 2.0 * rho).walk(0.5, targets=tg)[0], 2.0 * base)
    # L -> 4L, lo shifted: m ~ L^3, 1/r ~ 1/L, so Phi ~ L^2 (exact for L = 4)
    m4 = mg.Mesh(m.level, m.ijk, box_lo=(-3.0, 5.0, 0.25), box_len=4.0)
    assert np.allclose(_tree(m4, rho).walk(0.5, targets=tg)[0], 16.0 * base,
                       rtol=1e-15, atol=0)


def test_mirror_symmetry():
    """x -> 1-x maps the mesh and density onto themselves: the direct sum is
    symmetric to rounding, the walk to its truncation error."""
    m = mg.uniform_mesh(1)
    u, _ = _cell_geometry(m)
    rho = (1.0 + np.sin(7 * u[:, 1]) ** 2 + u[:, 2] + np.cos(3 * (u[:, 0] - 0.5)) ** 2)
    t = _tree(m, rho.reshape(-1, 8, 8, 8))
    key = {tuple(np.round(p * 64).astype(int)): i for i, p in enumerate(u)}
    mirror = np.array([key[tuple(np.round(np.array([1 - p[0], p[1], p[2]]) * 64).astype(int))]
                       for p in u])
    tg = np.arange(0, m.ncells, 11)
    d = t.direct(targets=tg)
    dm = t.direct(targets=mirror[tg])
    assert np.allclose(d, dm, rtol=1e-13, atol=0)
    w = t.walk(0.5, targets=tg)[0]
    wm = t.walk(0.5, targets=mirror[tg])[0]
    assert np.allclose(w, wm, rtol=5e-3, atol=0)
    assert not np.allclose(w, np.roll(wm, 1), rtol=5e-3, atol=0)


def test_paper_mode_refines_per_cell_sets(tiny):
    """The all() vote opens every node any brick member opens, so each cell
    interacts with at least as many nodes and tests at least as many."""
    m, rho = tiny["diag_refined"]
    t = _tree(m, rho)
    bricks = np.arange(0, 16 * m.nblocks, 9)
    pv, niv, ntv = t.walk_vote(0.6, bricks=bricks)
    lm = O.local_morton_order()
    cells = ((bricks[:, None] // 16) * 512 + lm[32 * (bricks[:, None] % 16)
                                                 + np.arange(32)[None, :]]).reshape(-1)
    pc, nic, ntc = t.walk(0.6, targets=cells)
    assert np.all(niv >= nic) and np.all(ntv >= ntc) and np.any(niv > nic)
    d = t.direct(targets=cells)
    assert np.abs(pv / d - 1).max() <= np.abs(pc / d - 1).max() * 1.0001
    pv0, _, _ = t.walk_vote(1e-6, bricks=bricks)
    assert np.allclose(pv0, d, rtol=1e-13, atol=0)


# --------------------------------------------- closed forms on the mesh ---
@pytest.mark.slow
def test_direct_sum_converges_to_sphere_closed_form():
    """Discretisation error of the direct sum against the top-hat sphere in
    its ambient box falls with resolution and is below 1e-2 at 32^3."""
    errs = []
    for bl in (1, 2, 3):
        w = mg.uniform_sphere(block_level=bl)
        t = O.Tree.from_workload(w)
        x = w.mesh.cell_centres().reshape(-1, 3)
        tg = np.random.default_rng(7).choice(w.ncells, min(w.ncells, 1500), replace=False)
        ref = A.sphere_in_box(x[tg, 0], x[tg, 1], x[tg, 2], (0.5,) * 3, 0.5, 1.0, 1e-3)
        errs.append(np.abs(t.direct(targets=tg) / ref - 1.0).max())
    assert errs[0] > errs[1] > errs[2] and errs[1] < 1e-2


@pytest.mark.slow
def test_error_curve_matches_paper_figure(golden_dir):
    """Max relative error vs the analytic Maclaurin potential, on a coarser
    stand-in of the paper's mesh: same order of magnitude as Fig. Errors and
    falling with theta."""
    tab = np.loadtxt(f"{golden_dir}/fig_errors_maclaurin.txt")
    paper = {float(r[0]): float(r[1]) for r in tab}
    w = mg.maclaurin(base_level=2, extra_levels=2)
    t = O.Tree.from_workload(w)
    x = w.mesh.cell_centres().reshape(-1, 3)
    ref = A.maclaurin_in_box(x[:, 0], x[:, 1], x[:, 2], (0.5,) * 3, mg.MACLAURIN_A1,
                             mg.MACLAURIN_E, 1.0, 1e-5)
    tg = np.sort(np.random.default_rng(0).choice(w.ncells, 1500, replace=False))
    errs = {}
    for th in (1.0, 0.75, 0.5, 0.25):
        errs[th] = np.abs(t.walk(th, targets=tg)[0] / ref[tg] - 1.0).max()
        assert paper[th] / 10.0 < errs[th] < paper[th] * 10.0, (th, errs[th])
    assert errs[1.0] > errs[0.75] > errs[0.5] > errs[0.25]


# ------------------------------------------------- quadrupole extension ---
def test_quadrupole_traceless_and_zero_for_a_point_mass(tiny):
    m, rho = tiny["refined_corner"]
    t = _tree(m, rho)
    e = t.export()
    Q = t.quadrupoles()
    scale = e["M"] * np.exp2(-2.0 * e["level"]) + 1e-300
    assert np.all(np.abs(Q[:, 0] + Q[:, 1] + Q[:, 2]) <= 1e-13 * scale)
    assert np.all(Q[e["is_leaf"] == 1] == 0.0)
    # all mass in one cell: every node is that point mass about its own
    # centre of mass, so Q = 0 and the quadrupole walk equals the monopole walk
    one = np.zeros_like(rho)
    one[3, 2, 5, 1] = 4.0
    t1 = _tree(m, one)
    assert np.abs(t1.quadrupoles()).max() <= 1e-15
    tg = np.arange(0, m.ncells, 13)
    assert np.allclose(t1.walk(0.7, targets=tg, quad=True)[0], t1.walk(0.7, targets=tg)[0],
                       rtol=1e-15, atol=0)


def test_quadrupole_of_two_masses_far_field():
    """Two equal masses 2a apart seen from distance r along their axis: the
    monopole errs by ~(a/r)^2, the quadrupole term removes that order."""
    m = mg.uniform_mesh(2)                     # 32^3 cells of side 1/32
    rho = np.zeros((m.nblocks, 8, 8, 8))
    u, _ = _cell_geometry(m)
    key = {tuple(np.round(p * 64).astype(int)): i for i, p in enumerate(u)}
    a = key[(1, 1, 1)]                         # cell centres (1,1,1)/64 and (5,1,1)/64
    b = key[(5, 1, 1)]
    rho.reshape(-1)[a] = rho.reshape(-1)[b] = 1.0
    t = _tree(m, rho)
    far = [key[(k, 1, 1)] for k in (41, 51, 61)]   # along the axis
    d = t.direct(targets=far)
    mono = t.walk(1.0, targets=far)[0]
    quad = t.walk(1.0, targets=far, quad=True)[0]
    em, eq = np.abs(mono / d - 1), np.abs(quad / d - 1)
    assert np.all(em > 1e-4) and np.all(eq < 0.05 * em)


def test_quadrupole_reduces_walk_error():
    w = mg.uniform_sphere(block_level=2)
    t = O.Tree.from_workload(w)
    tg = np.random.default_rng(2).choice(w.ncells, 600, replace=False)
    d = t.direct(targets=tg)
    for th, factor in ((0.3, 8.0), (0.5, 8.0), (0.8, 3.0)):
        em = np.abs(t.walk(th, targets=tg)[0] / d - 1).max()
        eq = np.abs(t.walk(th, targets=tg, quad=True)[0] / d - 1).max()
        assert eq < em / factor, (th, em, eq)
    # the opening decisions do not depend on the quadrupole term
    assert np.array_equal(t.walk(0.6, targets=tg)[1], t.walk(0.6, targets=tg, quad=True)[1])


# ---------------------------------------------- learned correction (MLP) ---
def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = rng.normal(0, 0.3, O.MLP_NW)
    x = rng.normal(0, 1, (7, O.MLP_IN))
    z = rng.normal(0, 1, 7)
    loss, g = O.mlp_loss_grad(w, x, z)
    idx = rng.choice(O.MLP_NW, 60, replace=False)
    for i in idx:
        e = np.zeros_like(w)
        e[i] = 1e-6
        fd = (O.mlp_loss_grad(w + e, x, z)[0] - O.mlp_loss_grad(w - e, x, z)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_gelu_is_the_tanh_form():
    a = np.linspace(-4, 4, 9)
    assert np.allclose(O.gelu(a), 0.5 * a * (1 + np.tanh(np.sqrt(2 / np.pi) * (a + 0.044715 * a ** 3))))
    h = 1e-6
    assert np.allclose(O.gelu_grad(a), (O.gelu(a + h) - O.gelu(a - h)) / (2 * h), atol=1e-8)


def test_learned_walk_with_zero_network_is_the_monopole_walk(tiny):
    m, rho = tiny["refined_twice"]
    t = _tree(m, rho)
    tg = np.arange(0, m.ncells, 17)
    mono = t.walk(0.8, targets=tg)[0]
    assert np.allclose(t.walk_learned(0.8, np.zeros(O.MLP_NW), targets=tg), mono, rtol=1e-14,
                       atol=0)
    w = np.zeros(O.MLP_NW)
    w[-1] = 0.5                                    # y = 0.5 for every pair
    lw = t.walk_learned(0.8, w, targets=tg)
    assert np.all(np.abs(lw) > np.abs(mono))      # every node term grows by s^2/2


def test_learned_gate_corrects_exactly_the_pairs_with_s_at_least_s_min(tiny):
    """The gate (no network for accepted nodes with s = l/d < s_min): s_min
    = 0 is the ungated walk; s_min near 1 gates every accepted node off (an
    accepted node has d > l/theta >= l, so s < 1), which is the monopole walk;
    in between, with a constant network (y = 1/2 for every pair), the
    correction is (M/d) s^2/2 summed over exactly the accepted pairs with s
    >= s_min, which the pair listing gives independently of the walk."""
    m, rho = tiny["diag_refined"]
    t = _tree(m, rho)
    tg = np.arange(0, m.ncells, 151)
    rng = np.random.default_rng(4)
    w = rng.normal(0, 0.2, O.MLP_NW)
    assert np.array_equal(t.walk_learned(0.8, w, targets=tg, s_min=0.0),
                          t.walk_learned(0.8, w, targets=tg))
    mono = t.walk(0.8, targets=tg)[0]
    assert np.allclose(t.walk_learned(0.8, w, targets=tg, s_min=0.999), mono, rtol=1e-14, atol=0)
    e = t.export()
    u, _ = _cell_geometry(m)
    c = np.zeros(O.MLP_NW)
    c[-1] = 0.5
    s_all = np.concatenate([t.learn_pairs(0.8, q)[0][:, 3] for q in tg])
    # s_min halfway across the widest relative gap between distinct s values
    # in the middle 80 % of them: no pair lies near the boundary, where the
    # gate's binary32 d^2 (from binary32 centres of mass) and the listing's
    # FP64 s could disagree (relative differences of order 1e-6)
    sv = np.unique(s_all)
    lo, hi = len(sv) // 10, 9 * len(sv) // 10
    k = lo + int(np.argmax(np.diff(sv[lo:hi + 1]) / sv[lo:hi]))
    s_min = 0.5 * (sv[k] + sv[k + 1])
    gap = np.min(np.abs(s_all - s_min)) / s_min
    assert gap > 1e-4, gap
    got = t.walk_learned(0.8, c, targets=tg, s_min=s_min)
    for k, q in enumerate(tg):
        f, _, nodes = t.learn_pairs(0.8, q)
        mn = e["M"][nodes] / np.linalg.norm(u[q] - e["R"][nodes], axis=1)
        on = f[:, 3] >= s_min
        want = mono[k] - np.sum(mn[on] * 0.5 * f[on, 3] ** 2)   # Phi = -G (sum), G = 1
        assert abs(got[k] / want - 1.0) < 1e-12, (q, got[k], want)
    assert np.any(got != mono)


def test_exact_residuals_turn_the_walk_into_the_direct_sum(tiny):
    """walk + sum over accepted nodes of (M/d) eps = direct sum, per target:
    eps is each node's exact error against its monopole."""
    m, rho = tiny["diag_refined"]
    t = _tree(m, rho)
    e = t.export()
    u, _ = _cell_geometry(m)
    for tgt in np.random.default_rng(9).choice(m.ncells, 12, replace=False):
        f, eps, nodes = t.learn_pairs(0.8, tgt)
        assert len(nodes) > 0 and np.allclose(np.linalg.norm(f[:, :3], axis=1), 1.0)
        mono = e["M"][nodes] / np.linalg.norm(u[tgt] - e["R"][nodes], axis=1)
        walk = t.walk(0.8, targets=[tgt])[0][0]
        d = t.direct(targets=[tgt])[0]
        assert abs((walk - np.sum(mono * eps)) / d - 1.0) < 1e-12
        far = f[:, 3] < 0.25                          # small s: eps ~ s^2 uQu/(2 M l^2)
        if far.any():
            assert np.all(np.abs(eps[far] - 0.5 * f[far, 9]) <= 0.2 * np.abs(eps[far]) + 1e-9)
