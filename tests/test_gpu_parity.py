"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Bars, as written in each test:
  * tree and moments: bit-exact (same pre-order, levels, skips; FP64 masses
    and centres of mass identical; delta identical after rounding to binary32);
  * opening decisions: bit-exact, checked through the per-cell counts of
    interactions and tests;
  * potential, binary32 walk: max relative difference 1e-5 per cell; binary64
    walk: 1e-12 per cell.
Small meshes are compared cell by cell in full; the 2.0M-cell Maclaurin mesh
(the benchmark workload, same launch configuration) and the 16.3M-cell cloud
core are compared on sampled cells, where the oracle computes each one alone.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1509_07370_gb300 import bhgrav as B  # noqa: E402
from paper_1509_07370_gb300 import meshgen as mg  # noqa: E402

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
F64_TOL = 1e-12


def _cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def _solver(prec=B.BH_PREC_F32, crit=B.BH_CRIT_PER_CELL, kahan=True):
    return B.Solver(precision=prec, criterion=crit, kahan=kahan)


def _build(s, mesh, rho, dtype=torch.float64):
    s.build(mesh.level, mesh.ijk, _cuda(rho.reshape(-1), dtype), mesh.box_lo, mesh.box_len)
    return s


def _oracle(mesh, rho):
    return O.Tree(mesh.level, mesh.ijk, rho, mesh.box_lo, mesh.box_len)


def _rel(a, b):
    return np.abs(np.asarray(a, np.float64) / np.asarray(b, np.float64) - 1.0)


def _subtree_end(parent):
    n = len(parent)
    end = np.arange(1, n + 1)
    for i in range(n - 1, 0, -1):
        end[parent[i]] = max(end[parent[i]], end[i])
    return end


MESHES = {}


def _mesh(name):
    if name not in MESHES:
        if name == "c1":
            w = mg.uniform_sphere()
            MESHES[name] = (w.mesh, w.density)
        elif name == "maclaurin_small":
            w = mg.maclaurin(base_level=2, extra_levels=2)
            MESHES[name] = (w.mesh, w.density)
        elif name == "maclaurin":
            w = mg.maclaurin()
            MESHES[name] = (w.mesh, w.density)
        elif name == "cloud_core":
            w = mg.cloud_core()
            MESHES[name] = (w.mesh, w.density)
        elif name.endswith("_shuffled"):
            m, r = _mesh(name[: -len("_shuffled")])
            MESHES[name] = mg.shuffled(m, r, seed=11)
        else:
            m = mg.tiny_meshes()[name]
            MESHES[name] = (m, mg.random_density(m, seed=len(name)))
    return MESHES[name]


TINY = ["one_block", "eight_blocks", "refined_corner", "refined_twice", "diag_refined"]


# ------------------------------------------------------------- the tree ---
@pytest.mark.parametrize("name", TINY + ["c1", "diag_refined_shuffled", "maclaurin_small"])
def test_tree_and_moments_bit_exact(name):
    mesh, rho = _mesh(name)
    s = _build(_solver(), mesh, rho)
    e = _oracle(mesh, rho).export()
    nc, nn, ml = s.tree_size()
    assert nc == mesh.ncells and nn == len(e["M"]) and ml == int(mesh.level.max()) + 3
    g = {k: v.cpu().numpy() for k, v in s.export_nodes().items()}
    assert np.array_equal(g["level"], e["level"])
    assert np.array_equal(g["skip"], _subtree_end(e["parent"]))
    assert np.array_equal(g["M"], e["M"])
    assert np.array_equal(g["R"], e["R"])
    assert np.array_equal(g["delta"], e["delta"].astype(np.float32))


def test_density_fp32_input_equals_rounded_fp64_input():
    mesh, rho = _mesh("refined_corner")
    r32 = rho.astype(np.float32)
    a = _build(_solver(), mesh, r32, torch.float32).export_nodes()["M"].cpu().numpy()
    b = _build(_solver(), mesh, r32.astype(np.float64)).export_nodes()["M"].cpu().numpy()
    assert np.array_equal(a, b)


# ------------------------------------------------------- the decisions ----
@pytest.mark.parametrize("name", TINY + ["c1", "diag_refined_shuffled"])
@pytest.mark.parametrize("theta", [0.3, 0.5, 1.0])
def test_opening_decisions_bit_exact(name, theta):
    mesh, rho = _mesh(name)
    s = _build(_solver(), mesh, rho)
    ni, nt = (x.cpu().numpy() for x in s.walk_counts(theta))
    _, oi, ot = _oracle(mesh, rho).walk(theta)
    assert np.array_equal(ni, oi) and np.array_equal(nt, ot)


def test_cell_interaction_counts_match_accepted_sets():
    mesh, rho = _mesh("diag_refined")
    s = _build(_solver(), mesh, rho)
    ni, nt, nc = (x.cpu().numpy() for x in s.walk_counts(0.6, with_cells=True))
    t = _oracle(mesh, rho)
    leaf = t.export()["is_leaf"]
    for tgt in np.random.default_rng(4).choice(mesh.ncells, 40, replace=False):
        acc = t.walk_list(0.6, tgt)
        assert nc[tgt] == int(leaf[acc].sum()) and ni[tgt] == len(acc)


@pytest.mark.parametrize("name", ["refined_twice", "c1"])
def test_paper_mode_decisions_bit_exact(name):
    mesh, rho = _mesh(name)
    s = _build(_solver(crit=B.BH_CRIT_WARP_VOTE), mesh, rho)
    ni, nt = (x.cpu().numpy() for x in s.walk_counts(0.6))
    _, oi, ot = _oracle(mesh, rho).walk_vote(0.6)
    perm = _vote_to_caller(mesh)
    assert np.array_equal(ni[perm], oi) and np.array_equal(nt[perm], ot)


def _vote_to_caller(mesh):
    """Caller cell index of each entry of the oracle's brick-ordered output."""
    lm = O.local_morton_order()
    b = np.arange(16 * mesh.nblocks)
    return ((b[:, None] // 16) * 512 + lm[32 * (b[:, None] % 16) + np.arange(32)]).reshape(-1)


# -------------------------------------------------------- the potential ---
@pytest.mark.parametrize("name", TINY + ["c1", "diag_refined_shuffled"])
@pytest.mark.parametrize("theta", [0.3, 0.5, 1.0])
def test_potential_f32_matches_oracle_walk(name, theta):
    mesh, rho = _mesh(name)
    s = _build(_solver(), mesh, rho)
    phi = s.potential(theta, G=1.0).cpu().numpy()
    ref, _, _ = _oracle(mesh, rho).walk(theta)
    assert _rel(phi, ref).max() <= F32_TOL


@pytest.mark.parametrize("name", ["refined_corner", "c1"])
def test_potential_f64_matches_oracle_walk(name):
    mesh, rho = _mesh(name)
    s = _build(_solver(prec=B.BH_PREC_F64), mesh, rho)
    phi = s.potential(0.5, G=1.0).cpu().numpy()
    assert phi.dtype == np.float64
    ref, _, _ = _oracle(mesh, rho).walk(0.5)
    assert _rel(phi, ref).max() <= F64_TOL


@pytest.mark.parametrize("prec,tol", [(B.BH_PREC_F32, F32_TOL), (B.BH_PREC_F64, F64_TOL)])
def test_paper_mode_potential_matches_oracle(prec, tol):
    mesh, rho = _mesh("c1")
    s = _build(_solver(prec=prec, crit=B.BH_CRIT_WARP_VOTE), mesh, rho)
    phi = s.potential(0.6, G=2.0).cpu().numpy()
    ref, _, _ = _oracle(mesh, rho).walk_vote(0.6, G=2.0)
    assert _rel(phi[_vote_to_caller(mesh)], ref).max() <= tol


def test_theta_to_small_is_direct_sum():
    mesh, rho = _mesh("refined_corner")
    s = _build(_solver(prec=B.BH_PREC_F64), mesh, rho)
    phi = s.potential(1e-6, G=1.0).cpu().numpy()
    d = _oracle(mesh, rho).direct()
    assert _rel(phi, d).max() <= F64_TOL


def test_box_scaling_and_G():
    mesh, rho = _mesh("refined_corner")
    m4 = mg.Mesh(mesh.level, mesh.ijk, box_lo=(-3.0, 5.0, 0.25), box_len=4.0)
    a = _build(_solver(prec=B.BH_PREC_F64), mesh, rho).potential(0.5, G=1.0).cpu().numpy()
    b = _build(_solver(prec=B.BH_PREC_F64), m4, rho).potential(0.5, G=3.0).cpu().numpy()
    assert _rel(b, 48.0 * a).max() <= F64_TOL


def test_kahan_sum_not_worse_than_plain():
    mesh, rho = _mesh("c1")
    ref, _, _ = _oracle(mesh, rho).walk(0.3)
    k = _build(_solver(kahan=True), mesh, rho).potential(0.3).cpu().numpy()
    p = _build(_solver(kahan=False), mesh, rho).potential(0.3).cpu().numpy()
    assert _rel(k, ref).max() <= F32_TOL
    assert _rel(k, ref).mean() <= _rel(p, ref).mean()


def test_deterministic_and_host_path_identical():
    mesh, rho = _mesh("refined_twice")
    s = _build(_solver(), mesh, rho)
    a = s.potential(0.5).cpu().numpy()
    b = s.potential(0.5).cpu().numpy()
    assert np.array_equal(a, b)
    h = _solver().solve_host(mesh.level, mesh.ijk, rho.reshape(-1).copy(), 0.5)
    assert np.array_equal(a, h)
    # a pinned output buffer: written by the walk through its device address
    pinned = torch.empty(mesh.ncells, dtype=torch.float32).pin_memory()
    pinned.fill_(float("nan"))
    q = _solver()
    B.bh_solve_host(q._ctx, mesh.level, mesh.ijk, (0.0, 0.0, 0.0), 1.0,
                    torch.as_tensor(rho.reshape(-1).copy()).pin_memory().numpy(), 0.5, 1.0,
                    pinned.numpy())
    assert np.array_equal(a, pinned.numpy())


def test_host_path_keeps_every_bit_at_full_size():
    """bh_solve_host with a pinned and with a pageable density, into a pinned
    output (written by the walk through its device address): bit-identical
    to bh_build + bh_potential on the device, in either density precision,
    at full size; a bad value in the density is still reported."""
    mesh, rho = _mesh("maclaurin")
    for dt, npdt in ((torch.float32, np.float32), (torch.float64, np.float64)):
        r = rho.reshape(-1).astype(npdt)
        want = _build(_solver(), mesh, r, dt).potential(0.75).cpu().numpy()
        s = _solver()
        out = torch.empty(mesh.ncells, dtype=torch.float32).pin_memory()
        for dens in (torch.as_tensor(r).pin_memory().numpy(), r.copy()):
            out.fill_(float("nan"))
            s.solve_host(mesh.level, mesh.ijk, dens, 0.75, 1.0, out.numpy(),
                         mesh.box_lo, mesh.box_len)
            assert np.array_equal(out.numpy(), want), (dt, dens.flags)
    bad = torch.as_tensor(rho.reshape(-1).astype(np.float32)).pin_memory()
    bad[mesh.ncells // 2] = float("nan")
    with pytest.raises(B.BHError) as e:
        _solver().solve_host(mesh.level, mesh.ijk, bad.numpy(), 0.75, 1.0, None,
                             mesh.box_lo, mesh.box_len)
    assert e.value.status == B.BH_ERR_ARG


# ----------------------------------------------------- full-size meshes ---
def _sample(ncells, k, seed):
    rng = np.random.default_rng(seed)
    return np.sort(np.concatenate([rng.choice(ncells, k, replace=False),
                                   [0, ncells - 1]]))


@pytest.mark.parametrize("theta", [0.24, 0.3, 0.5, 0.7])
def test_maclaurin_full_size_sampled(theta):
    """The benchmark workload (2,039,808 cells), benchmark launch config."""
    mesh, rho = _mesh("maclaurin")
    s = _build(_solver(), mesh, rho)
    phi = s.potential(theta).cpu().numpy()
    ni, nt = (x.cpu().numpy() for x in s.walk_counts(theta))
    t = _oracle(mesh, rho)
    tg = _sample(mesh.ncells, 3000, seed=int(theta * 100))
    ref, oi, ot = t.walk(theta, targets=tg)
    assert _rel(phi[tg], ref).max() <= F32_TOL
    assert np.array_equal(ni[tg], oi) and np.array_equal(nt[tg], ot)
    assert np.all(np.isfinite(phi)) and np.all(phi < 0)


def test_autotuned_walk_at_full_size_keeps_every_bit():
    """The benchmark's tuning at full size: bh_autotune times every launch
    shape and, for the longest-first order, walks the tree once recording
    each group's time; whatever shape and order it keeps, and the
    longest-first persistent walk pinned directly, give the default walk's
    potentials bit for bit (monopole at theta 0.24, the plain comparison,
    and with the quadrupole term at theta 0.75, the headline)."""
    mesh, rho = _mesh("maclaurin")
    for quad, theta in ((False, 0.24), (True, 0.75)):
        ref = _build(B.Solver(quadrupole=quad), mesh, rho)
        want = ref.potential(theta).cpu().numpy()
        ref.close()
        s = _build(B.Solver(quadrupole=quad), mesh, rho)
        shape = s.autotune(theta)
        assert shape[3] in (0, 1)
        assert np.array_equal(s.potential(theta).cpu().numpy(), want), shape
        s.set_walk_shape(16, 1, 1, 1)
        assert np.array_equal(s.potential(theta).cpu().numpy(), want)
        s.close()


@pytest.mark.parametrize("theta", [0.72, 0.75])
def test_against_the_analytic_potentials(theta):
    """The two configurations that state an analytic reference: the 32^3
    top-hat sphere (FP64 walk, monopole, theta 0.5) against the uniform
    sphere in its ambient box, and the 2,039,808-cell Maclaurin spheroid at
    the benchmark's setting (binary32 walk, quadrupole, theta 0.75) and at
    theta 0.72 against
    the corrected Maclaurin potential, on 3,000 sampled cells.  What remains
    is the mesh's discretisation (the oracle's direct sum is off by 2.1e-3
    and 9.7e-4) plus the walk's error; the oracle's own walks reach 1.8e-3
    and 9.3e-4."""
    from oracle import analytic as A
    w = mg.uniform_sphere()
    s = _build(_solver(prec=B.BH_PREC_F64), w.mesh, w.density)
    x = w.mesh.cell_centres().reshape(-1, 3)
    ref = A.sphere_in_box(x[:, 0], x[:, 1], x[:, 2], (0.5,) * 3, 0.5, 1.0, 1e-3)
    assert _rel(s.potential(0.5).cpu().numpy(), ref).max() <= 2.5e-3
    mesh, rho = _mesh("maclaurin")
    s = _build(B.Solver(quadrupole=True), mesh, rho)
    phi = s.potential(theta).cpu().numpy()
    tg = _sample(mesh.ncells, 3000, seed=9)
    x = mesh.cell_centres().reshape(-1, 3)[tg]
    ref = A.maclaurin_in_box(x[:, 0], x[:, 1], x[:, 2], (0.5,) * 3, mg.MACLAURIN_A1,
                             mg.MACLAURIN_E, 1.0, 1e-5)
    assert _rel(phi[tg], ref).max() <= 1.2e-3


@pytest.mark.parametrize("quad,theta", [(False, 0.5), (True, 0.75)])
def test_maclaurin_full_size_shuffled_blocks(quad, theta):
    """The 2,039,808-cell spheroid with its 3,984 blocks in a random order,
    so that the build really sorts them (a single-CTA radix sort of the block
    keys).  The potentials come back in the caller's (shuffled) layout,
    identical bit for bit to the solve of the Morton-ordered list; opening
    decisions and potentials also match the oracle, which builds its own tree
    from the shuffled list, on 2,000 sampled cells."""
    mesh, rho = _mesh("maclaurin")
    rng = np.random.Generator(np.random.PCG64(23))
    p = rng.permutation(mesh.nblocks)
    sm = mg.Mesh(level=mesh.level[p].copy(), ijk=mesh.ijk[p].copy(), box_lo=mesh.box_lo,
                 box_len=mesh.box_len)
    srho = rho[p].copy()
    ordered = _build(B.Solver(quadrupole=quad), mesh, rho).potential(theta).cpu().numpy()
    s = _build(B.Solver(quadrupole=quad), sm, srho)
    phi = s.potential(theta).cpu().numpy()
    assert np.array_equal(phi.reshape(-1, 512), ordered.reshape(-1, 512)[p])
    ni, nt = (x.cpu().numpy() for x in s.walk_counts(theta))
    tg = _sample(sm.ncells, 2000, seed=31)
    ref, oi, ot = _oracle(sm, srho).walk(theta, targets=tg, quad=quad)
    assert np.array_equal(ni[tg], oi) and np.array_equal(nt[tg], ot)
    assert _rel(phi[tg], ref).max() <= F32_TOL


def test_cloud_core_compensated_sum_beats_plain():
    """The compensated binary32 sum against plain binary32 addition on the
    16,289,792-cell cloud core (monopole, theta 0.5, about 1,350 terms per
    cell), both against the oracle's FP64 walk on 1,502 sampled cells: the
    compensated sum stays within the 1e-5 bar and the plain one is measurably
    worse, on average and at its worst cell."""
    mesh, rho = _mesh("cloud_core")
    r32 = rho.astype(np.float32)
    t = _oracle(mesh, r32.astype(np.float64))
    tg = _sample(mesh.ncells, 1500, seed=12)
    ref, _, _ = t.walk(0.5, targets=tg)
    err = {}
    for kahan in (True, False):
        s = _build(_solver(kahan=kahan), mesh, r32, torch.float32)
        err[kahan] = _rel(s.potential(0.5).cpu().numpy()[tg], ref)
        s.close()
    assert err[True].max() <= F32_TOL
    assert err[False].mean() >= 2.0 * err[True].mean()
    assert err[False].max() > err[True].max()


def test_cloud_core_full_size_sampled():
    mesh, rho = _mesh("cloud_core")
    s = _build(_solver(), mesh, rho.astype(np.float32), torch.float32)
    phi = s.potential(0.5).cpu().numpy()
    t = _oracle(mesh, rho.astype(np.float32).astype(np.float64))
    tg = _sample(mesh.ncells, 1500, seed=5)
    ref, _, _ = t.walk(0.5, targets=tg)
    assert _rel(phi[tg], ref).max() <= F32_TOL
    assert np.all(np.isfinite(phi)) and np.all(phi < 0)


def test_cloud_core_quadrupole_autotuned_full_size_sampled():
    """The 16.3M-cell cloud core with quadrupole nodes at the headline's
    theta, in the launch shape and group order bh_autotune picks for it:
    decisions bit-exact and potentials within 1e-5 of the oracle's walk on
    sampled cells."""
    mesh, rho = _mesh("cloud_core")
    s = _build(B.Solver(quadrupole=True), mesh, rho.astype(np.float32), torch.float32)
    s.autotune(0.75)
    phi = s.potential(0.75).cpu().numpy()
    ni, nt = (x.cpu().numpy() for x in s.walk_counts(0.75))
    tg = _sample(mesh.ncells, 1500, seed=75)
    t = _oracle(mesh, rho.astype(np.float32).astype(np.float64))
    ref, oi, ot = t.walk(0.75, targets=tg, quad=True)
    assert _rel(phi[tg], ref).max() <= F32_TOL
    assert np.array_equal(ni[tg], oi) and np.array_equal(nt[tg], ot)
    assert np.all(np.isfinite(phi)) and np.all(phi < 0)


# ----------------------------------------------------- quadrupole term ---
@pytest.mark.parametrize("name", ["refined_twice", "c1", "maclaurin_small"])
@pytest.mark.parametrize("prec,tol", [(B.BH_PREC_F64, 1e-12), (B.BH_PREC_F32, 1e-5)])
def test_quadrupole_moments_match_oracle(name, prec, tol):
    """FP64 quadrupoles (FP64 walk) to 1e-12 and binary32 ones (binary32 walk)
    to 1e-5 of M l^2, the natural scale of a node's quadrupole."""
    mesh, rho = _mesh(name)
    s = _build(B.Solver(precision=prec, quadrupole=True), mesh, rho)
    q = s.export_quadrupoles().cpu().numpy()
    t = _oracle(mesh, rho)
    qo = t.quadrupoles()
    e = t.export()
    scale = e["M"] * np.exp2(-2.0 * e["level"]) + 1e-300     # M l^2 of each node
    assert np.all(np.abs(q - qo) <= tol * scale[:, None])


@pytest.mark.parametrize("name", ["refined_twice", "c1", "diag_refined_shuffled"])
@pytest.mark.parametrize("theta", [0.5, 0.8])
def test_quadrupole_potential_f32_matches_oracle(name, theta):
    mesh, rho = _mesh(name)
    s = _build(B.Solver(quadrupole=True), mesh, rho)
    phi = s.potential(theta).cpu().numpy()
    ref, _, _ = _oracle(mesh, rho).walk(theta, quad=True)
    assert _rel(phi, ref).max() <= F32_TOL


def test_quadrupole_potential_f64_and_paper_mode():
    mesh, rho = _mesh("c1")
    t = _oracle(mesh, rho)
    s = _build(B.Solver(precision=B.BH_PREC_F64, quadrupole=True), mesh, rho)
    ref, _, _ = t.walk(0.7, quad=True)
    assert _rel(s.potential(0.7).cpu().numpy(), ref).max() <= F64_TOL
    for prec, tol in ((B.BH_PREC_F32, F32_TOL), (B.BH_PREC_F64, F64_TOL)):
        s = _build(B.Solver(precision=prec, criterion=B.BH_CRIT_WARP_VOTE, quadrupole=True),
                   mesh, rho)
        refv, _, _ = t.walk_vote(0.7, quad=True)
        assert _rel(s.potential(0.7).cpu().numpy()[_vote_to_caller(mesh)], refv).max() <= tol


@pytest.mark.parametrize("theta", [0.7, 0.72, 0.75, 0.8])
def test_quadrupole_maclaurin_full_size_sampled(theta):
    """The benchmark's headline setting (theta 0.75) and its neighbours:
    potentials within 1e-5 and decisions bit-exact on sampled cells."""
    mesh, rho = _mesh("maclaurin")
    s = _build(B.Solver(quadrupole=True), mesh, rho)
    phi = s.potential(theta).cpu().numpy()
    ni, nt = (x.cpu().numpy() for x in s.walk_counts(theta))
    tg = _sample(mesh.ncells, 3000, seed=int(theta * 100))
    ref, oi, ot = _oracle(mesh, rho).walk(theta, targets=tg, quad=True)
    assert _rel(phi[tg], ref).max() <= F32_TOL
    assert np.array_equal(ni[tg], oi) and np.array_equal(nt[tg], ot)
    assert np.all(np.isfinite(phi)) and np.all(phi < 0)


def test_paper_mode_and_fp64_full_size_sampled():
    """The 2,039,808-cell spheroid in the two other walk kernels: the paper's
    warp vote (binary32, quadrupole, theta 0.8) on 120 sampled 32-cell
    bricks, decisions bit-exact and potentials within 1e-5; and the binary64
    walk (monopole, theta 0.5) on 1,500 sampled cells within 1e-12."""
    mesh, rho = _mesh("maclaurin")
    t = _oracle(mesh, rho)
    s = _build(B.Solver(criterion=B.BH_CRIT_WARP_VOTE, quadrupole=True), mesh, rho)
    phi = s.potential(0.8).cpu().numpy()
    ni, _ = s.walk_counts(0.8)
    bricks = np.sort(np.random.default_rng(12).choice(16 * mesh.nblocks, 120, replace=False))
    ref, oi, _ = t.walk_vote(0.8, bricks=bricks, quad=True)
    lm = O.local_morton_order()
    cells = ((bricks[:, None] // 16) * 512 + lm[32 * (bricks[:, None] % 16)
                                               + np.arange(32)]).reshape(-1)
    assert _rel(phi[cells], ref).max() <= F32_TOL
    assert np.array_equal(ni.cpu().numpy()[cells], oi)
    s = _build(_solver(prec=B.BH_PREC_F64), mesh, rho)
    phi = s.potential(0.5).cpu().numpy()
    tg = _sample(mesh.ncells, 1500, seed=13)
    ref, _, _ = t.walk(0.5, targets=tg)
    assert _rel(phi[tg], ref).max() <= F64_TOL


def test_quadrupole_export_needs_the_option():
    mesh, rho = _mesh("one_block")
    s = _build(_solver(), mesh, rho)
    with pytest.raises(B.BHError) as e:
        s.export_quadrupoles()
    assert e.value.status == B.BH_ERR_STATE


# --------------------------------------------------------------- errors ---
@pytest.mark.parametrize("n", [0, 3, 9, 14])
def test_out_of_memory_reported_and_recoverable(monkeypatch, n):
    """Fault injection on the host: with BHGRAV_FAIL_ALLOC_AFTER=n the
    library's device allocations after the first n fail as out of memory
    (nothing is allocated; no device fault).  bh_build reports BH_ERR_OOM
    with a reason and keeps no tree (bh_potential: BH_ERR_STATE); once the
    variable is cleared the same context builds and gives the potentials of
    a fresh one, bit for bit."""
    mesh, rho = _mesh("refined_corner")
    s = _solver()
    monkeypatch.setenv("BHGRAV_FAIL_ALLOC_AFTER", str(n))
    with pytest.raises(B.BHError) as e:
        _build(s, mesh, rho)
    assert e.value.status == B.BH_ERR_OOM and "out of memory" in str(e.value).lower()
    with pytest.raises(B.BHError) as e:
        s.potential(0.5)
    assert e.value.status == B.BH_ERR_STATE
    monkeypatch.delenv("BHGRAV_FAIL_ALLOC_AFTER")
    got = _build(s, mesh, rho).potential(0.5).cpu().numpy()
    want = _build(_solver(), mesh, rho).potential(0.5).cpu().numpy()
    assert np.array_equal(got, want)


def test_errors_reported():
    mesh, rho = _mesh("eight_blocks")
    s = _solver()
    with pytest.raises(B.BHError) as e:
        s.potential(0.5)                                   # no tree yet
    assert e.value.status == B.BH_ERR_STATE
    d = _cuda(rho.reshape(-1))
    with pytest.raises(B.BHError) as e:                    # gap: 7 of 8 blocks
        s.build(mesh.level[:7], mesh.ijk[:7], d[: 7 * 512])
    assert e.value.status == B.BH_ERR_GEOMETRY
    ij = mesh.ijk.copy()
    ij[3] = ij[2]                                          # duplicate + gap
    with pytest.raises(B.BHError) as e:
        s.build(mesh.level, ij, d)
    assert e.value.status == B.BH_ERR_GEOMETRY
    lv = mesh.level.copy()
    lv[0] = 2                                              # block moved to a finer level
    with pytest.raises(B.BHError) as e:
        s.build(lv, mesh.ijk, d)
    assert e.value.status == B.BH_ERR_GEOMETRY
    bad = d.clone()
    bad[100] = -1.0
    with pytest.raises(B.BHError) as e:
        s.build(mesh.level, mesh.ijk, bad)
    assert e.value.status == B.BH_ERR_ARG
    bad[100] = float("nan")
    with pytest.raises(B.BHError):
        s.build(mesh.level, mesh.ijk, bad)
    with pytest.raises(B.BHError) as e:                    # failed build leaves no tree
        s.potential(0.5)
    assert e.value.status == B.BH_ERR_STATE
    s.build(mesh.level, mesh.ijk, d)
    for th in (0.0, -0.5, 1.5, float("nan")):
        with pytest.raises(B.BHError) as e:
            s.potential(th)
        assert e.value.status == B.BH_ERR_ARG
    with pytest.raises(B.BHError) as e:
        s.potential(0.5, G=float("inf"))
    assert e.value.status == B.BH_ERR_ARG
    assert np.all(np.isfinite(s.potential(0.5).cpu().numpy()))   # still usable


def test_build_reports_every_bad_density_before_its_moments():
    """bh_build returns once its first kernels have checked the input, with
    the moments still running: a bad value anywhere (the last cell of the
    last block, either precision, a field of a batch) is still reported by
    the call itself, and the tree that follows a good build is complete."""
    import torch
    mesh, rho = _mesh("eight_blocks")
    s = _solver()
    for dt in (torch.float32, torch.float64):
        for bad_v in (-1e-30, float("inf"), float("-inf"), float("nan")):
            d = torch.as_tensor(rho.reshape(-1), dtype=dt, device="cuda").clone()
            d[-1] = bad_v
            with pytest.raises(B.BHError) as e:
                s.build(mesh.level, mesh.ijk, d, mesh.box_lo, mesh.box_len)
            assert e.value.status == B.BH_ERR_ARG, (dt, bad_v)
        got = _build(s, mesh, rho, dt).potential(0.5).cpu().numpy()    # after the failures
        want = _build(_solver(), mesh, rho, dt).potential(0.5).cpu().numpy()
        assert np.array_equal(got, want)
    two = _cuda(np.concatenate([rho.reshape(-1), rho.reshape(-1)]))
    two[512 * len(mesh.level) + 3] = float("nan")          # a cell of the second field
    nb = np.array([len(mesh.level)] * 2, dtype=np.int32)
    with pytest.raises(B.BHError) as e:
        s.build_batch(nb, np.concatenate([mesh.level] * 2), np.concatenate([mesh.ijk] * 2), two)
    assert e.value.status == B.BH_ERR_ARG


def test_stats_sizes_timings_and_work_totals():
    """bh_stats: tree sizes equal bh_tree_size, device times with the timing
    option are positive (and -1 without it), the work totals equal the sums
    of bh_walk_counts' per-cell arrays."""
    mesh, rho = _mesh("refined_twice")
    s = B.Solver(timing=True)
    assert s.stats()["built"] == 0 and s.stats()["build_ms"] == -1.0
    _build(s, mesh, rho)
    out = s.potential(0.5)
    torch.cuda.synchronize()
    st = s.stats()
    nc, nn, ml = s.tree_size()
    assert (st["n_cells"], st["n_nodes"], st["max_level"]) == (nc, nn, ml)
    assert st["n_blocks"] == len(mesh.level) and st["n_fields"] == 1 and st["built"] == 1
    assert st["build_ms"] > 0.0 and st["potential_ms"] > 0.0 and st["last_theta"] == 0.5
    assert st["interactions"] == -1 and st["device_bytes"] > 0
    ni, nt, ncell = s.walk_counts(0.5, with_cells=True)
    st = s.stats()
    assert st["interactions"] == int(ni.sum(dtype=torch.int64))
    assert st["tests"] == int(nt.sum(dtype=torch.int64))
    assert st["cell_interactions"] == int(ncell.sum(dtype=torch.int64))
    plain = _build(B.Solver(), mesh, rho)
    plain.potential(0.5, out=out)
    assert plain.stats()["build_ms"] == -1.0 and plain.stats()["potential_ms"] == -1.0


# ------------------------------------------------ units and extreme depths ---
def test_physical_units_do_not_overflow_the_binary32_walk():
    """cgs units: rho ~ 1e-18 g/cm^3 in a 10 pc box holds ~3e40 g, beyond the
    binary32 range (3.4e38): the binary32 records carry masses in a per-field
    power-of-two unit, so the binary32 walks still match the FP64 oracle."""
    mesh, rho = _mesh("refined_twice")
    L, G = 3.0857e19, 6.674e-8
    m = mg.Mesh(mesh.level, mesh.ijk, box_lo=(-L / 2, -L / 2, -L / 2), box_len=L)
    rho_cgs = rho * 1e-18
    t = _oracle(m, rho_cgs)
    ref, _, _ = t.walk(0.5, G=G)
    assert np.abs(t.export()["M"][0]) > 1e39
    for quad in (False, True):
        s = B.Solver(quadrupole=quad)
        _build(s, m, rho_cgs)
        phi = s.potential(0.5, G=G).cpu().numpy()
        want = t.walk(0.5, G=G, quad=True)[0] if quad else ref
        assert np.all(np.isfinite(phi)) and _rel(phi, want).max() <= F32_TOL
    s = _build(_solver(prec=B.BH_PREC_F64), m, rho_cgs)
    assert _rel(s.potential(0.5, G=G).cpu().numpy(), ref).max() <= F64_TOL


def _chain18():
    if "chain18" not in MESHES:
        m = mg.refined_mesh(1, 18, lambda lev, ijk: np.all(ijk == 0, axis=1), name="chain18")
        MESHES["chain18"] = (m, mg.random_density(m, seed=18))
    return MESHES["chain18"]


def test_deepest_levels_tree_decisions_and_potentials():
    """One corner refined down to block level 18 (cells of 2^-21 of the box,
    the end of the 63-bit key lattice; 911 blocks): tree and moments
    bit-exact, decisions bit-exact, monopole and quadrupole binary32 walks
    within 1e-5 of the oracle on the deepest cells and a random sample (the
    binary32 mass unit keeps ½ d^T Q d of nodes 2^-20 wide far from the
    binary32 underflow)."""
    mesh, rho = _chain18()
    assert int(mesh.level.max()) == 18
    s = _build(_solver(), mesh, rho)
    t = _oracle(mesh, rho)
    e = t.export()
    g = {k: v.cpu().numpy() for k, v in s.export_nodes().items()}
    assert np.array_equal(g["M"], e["M"]) and np.array_equal(g["R"], e["R"])
    assert np.array_equal(g["skip"], _subtree_end(e["parent"]))
    deep = np.flatnonzero(np.repeat(mesh.level == 18, 512))
    tg = np.unique(np.concatenate([deep, np.random.default_rng(5).choice(mesh.ncells, 3000,
                                                                         replace=False)]))
    ni, nt = (x.cpu().numpy() for x in s.walk_counts(0.6))
    ref, oi, ot = t.walk(0.6, targets=tg)
    assert np.array_equal(ni[tg], oi) and np.array_equal(nt[tg], ot)
    phi = s.potential(0.6).cpu().numpy()
    assert _rel(phi[tg], ref).max() <= F32_TOL
    sq = B.Solver(quadrupole=True)
    _build(sq, mesh, rho)
    refq = t.walk(0.6, targets=tg, quad=True)[0]
    assert _rel(sq.potential(0.6).cpu().numpy()[tg], refq).max() <= F32_TOL


def test_zero_density_regions_and_all_zero_field():
    """Massless blocks and cells (nodes of zero mass sit at their geometric
    centre): bit-exact tree, potentials within 1e-5; an all-zero field gives
    zero potential."""
    mesh, rho = _mesh("diag_refined")
    z = rho.copy()
    rng = np.random.default_rng(3)
    z[rng.random(mesh.nblocks) < 0.4] = 0.0
    z[rng.random(z.shape) < 0.3] = 0.0
    s = _build(_solver(), mesh, z)
    t = _oracle(mesh, z)
    e = t.export()
    g = {k: v.cpu().numpy() for k, v in s.export_nodes().items()}
    assert np.array_equal(g["M"], e["M"]) and np.array_equal(g["R"], e["R"])
    ref, _, _ = t.walk(0.5)
    phi = s.potential(0.5).cpu().numpy()
    assert _rel(phi, ref).max() <= F32_TOL
    sq = _build(B.Solver(quadrupole=True), mesh, z)
    assert _rel(sq.potential(0.5).cpu().numpy(), t.walk(0.5, quad=True)[0]).max() <= F32_TOL
    s0 = _build(_solver(), mesh, np.zeros_like(rho))
    assert np.all(s0.potential(0.5).cpu().numpy() == 0.0)
