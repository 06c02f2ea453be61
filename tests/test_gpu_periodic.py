"""Periodic boundaries (App. A) on the GPU, against the CPU oracle.

Bars:
  * the Ewald table: bh_ewald_eval against the oracle's interpolation of its
    own FP64 table within 1e-6 (binary32 table values and arithmetic; chi is
    about 3 in size), against the Ewald sum itself within the interpolation
    error (4e-6 at 64 points per half box);
  * opening decisions bit-exact: per-cell interaction and test counts equal
    the oracle's periodic walk (the minimum-image wrap is exact in binary32);
  * potentials: the periodic potential has zero mean and changes sign, so the
    bar is relative to the field's largest magnitude: within 1e-5 of
    max |Phi| per cell;
  * a uniform density: Phi = -G rho h^2 chi(0) (the lattice sum) within the
    table's interpolation error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1509_07370_gb300 import bhgrav as B  # noqa: E402
from paper_1509_07370_gb300 import meshgen as mg  # noqa: E402

pytestmark = pytest.mark.gpu

XI = -2.837297479480619


def _solver(mesh, rho, **kw):
    s = B.Solver(periodic=True, **kw)
    s.build(mesh.level, mesh.ijk, torch.as_tensor(np.asarray(rho, np.float32).reshape(-1)).cuda(),
            mesh.box_lo, mesh.box_len)
    return s


def _oracle(mesh, rho):
    return O.Tree(mesh.level, mesh.ijk, np.asarray(rho, np.float32).astype(np.float64),
                  mesh.box_lo, mesh.box_len)


def test_ewald_table_matches_oracle():
    s = B.Solver(periodic=True)
    rng = np.random.default_rng(1)
    u = rng.uniform(-0.5, 0.5, (5000, 3)).astype(np.float32)
    chi = s.ewald_eval(torch.as_tensor(u).cuda()).cpu().numpy()
    ref = O.ewald_interp(u.astype(np.float64), 64)
    assert np.abs(chi - ref).max() < 1e-6
    assert np.abs(chi - O.ewald_sum(u.astype(np.float64), chi=True)).max() < 4e-6
    # at the grid points the table itself, and chi(0) the lattice constant
    g = (rng.integers(0, 65, (500, 3)) / 128.0).astype(np.float32)
    chi_g = s.ewald_eval(torch.as_tensor(g).cuda()).cpu().numpy()
    assert np.abs(chi_g - O.ewald_sum(g.astype(np.float64), chi=True)).max() < 1e-6
    z = s.ewald_eval(torch.zeros((1, 3), device="cuda")).cpu().numpy()[0]
    assert abs(z - XI) < 5e-7
    # another table: 32 points, series range 2
    s.set_ewald(32, 2)
    chi32 = s.ewald_eval(torch.as_tensor(u).cuda()).cpu().numpy()
    assert np.abs(chi32 - O.ewald_interp(u.astype(np.float64), 32, 2)).max() < 1e-6


def test_ewald_arguments():
    s = B.Solver(periodic=True)
    for n, ns in ((1, 3), (513, 3), (64, 0), (64, 9)):
        with pytest.raises(B.BHError):
            s.set_ewald(n, ns)
    for kw in (dict(quadrupole=True), dict(learned=1), dict(precision=B.BH_PREC_F64),
               dict(criterion=B.BH_CRIT_WARP_VOTE)):
        with pytest.raises(B.BHError):
            B.Solver(periodic=True, **kw)
    plain = B.Solver()
    with pytest.raises(B.BHError):
        plain.ewald_eval(torch.zeros((4, 3), device="cuda"))


@pytest.mark.parametrize("theta", [0.3, 0.6, 1.0])
def test_counts_and_potential_match_oracle_on_small_meshes(theta):
    for i, (name, m) in enumerate(sorted(mg.tiny_meshes().items())):
        rho = mg.random_density(m, seed=40 + i)
        for mesh, r in ((m, rho), mg.shuffled(m, rho, seed=i)):
            s = _solver(mesh, r)
            phi = s.potential(theta, G=1.3).cpu().numpy()
            ni, nt = (x.cpu().numpy() for x in s.walk_counts(theta))
            t = _oracle(mesh, r)
            po, nio, nto = t.walk_periodic(theta, G=1.3)
            assert np.array_equal(ni, nio) and np.array_equal(nt, nto), name
            assert np.abs(phi - po).max() <= 1e-5 * np.abs(po).max(), name


def test_sphere_in_a_periodic_box():
    w = mg.uniform_sphere(block_level=2, radius=0.3, rho_out=1e-2)
    s = _solver(w.mesh, w.density)
    phi = s.potential(0.5).cpu().numpy()
    t = _oracle(w.mesh, w.density)
    po, nio, _ = t.walk_periodic(0.5)
    ni, _ = s.walk_counts(0.5)
    assert np.array_equal(ni.cpu().numpy(), nio)
    assert np.abs(phi - po).max() <= 1e-5 * np.abs(po).max()
    # and close to the direct periodic sum (the method's own error, theta 0.5)
    tg = np.random.default_rng(2).choice(t.ncells, 400, replace=False)
    d = t.direct_periodic(targets=tg)
    assert np.abs(phi[tg] - d).max() <= 2e-2 * np.abs(d).max()


def test_uniform_density_is_the_lattice_sum():
    """At theta 0.05 every cell meets every other one (a direct sum); a
    uniform density is then a lattice whose sum is -G rho h^2 chi(0).  The
    displacements fall on table points, so the interpolation is exact; what
    remains is binary32 rounding of terms that nearly cancel (the field has
    zero mean), hence the 2e-4 bar."""
    m = mg.uniform_mesh(1)
    s = _solver(m, np.full((8, 8, 8, 8), 2.0))
    phi = s.potential(0.05, G=1.0).cpu().numpy()
    ni, _ = s.walk_counts(0.05)
    assert np.all(ni.cpu().numpy() == 8 * 512 - 1)
    want = -1.0 * 2.0 * (1.0 / 16) ** 2 * XI
    assert np.abs(phi / want - 1).max() < 2e-4


def test_graph_and_batch_equal_single_solves():
    fields = [mg.uniform_sphere(block_level=1, radius=0.3),
              mg.maclaurin(base_level=1, extra_levels=1)]
    single = []
    for f in fields:
        s = _solver(f.mesh, f.density)
        single.append(s.potential(0.6).cpu().numpy())
    nb, level, ijk, lo, ln, rho = mg.concat_fields(fields)
    st = torch.cuda.Stream()
    s = B.Solver(periodic=True, stream=st)
    d_rho = torch.as_tensor(rho.astype(np.float32)).cuda()
    s.build_batch(nb, level, ijk, d_rho, lo, ln)
    out = torch.empty(d_rho.numel(), device="cuda")
    with torch.cuda.stream(st):
        s.solve_graph(d_rho, 0.6, 1.0, out)
        s.solve_graph(d_rho, 0.6, 1.0, out)
    st.synchronize()
    assert np.array_equal(out.cpu().numpy(), np.concatenate(single))


def test_full_size_sampled_against_oracle():
    w = mg.maclaurin()
    s = _solver(w.mesh, w.density)
    phi = s.potential(0.7).cpu().numpy()
    ni, nt = (x.cpu().numpy() for x in s.walk_counts(0.7))
    t = _oracle(w.mesh, w.density)
    tg = np.random.default_rng(3).choice(t.ncells, 1500, replace=False)
    po, nio, nto = t.walk_periodic(0.7, targets=tg)
    assert np.array_equal(ni[tg], nio) and np.array_equal(nt[tg], nto)
    assert np.abs(phi[tg] - po).max() <= 1e-5 * np.abs(po).max()
    assert np.all(np.isfinite(phi))


def test_autotuned_order_keeps_every_bit():
    """bh_autotune times the periodic walk once per octant and may run the
    octants longest first: every CTA width, in either order, gives the
    potentials and counts of the octants' own order, bit for bit, at full
    size."""
    w = mg.maclaurin()
    s = _solver(w.mesh, w.density)
    want = s.potential(0.7).cpu().numpy()
    wi, wt = (x.cpu().numpy() for x in s.walk_counts(0.7))
    shape = s.autotune(0.7)
    assert shape[1:3] == (1, 0) and shape[3] in (0, 1), shape
    for warps in (2, 4, 8, 16):
        for longest in (0, 1):
            s.set_walk_shape(warps, 1, 0, longest)
            assert np.array_equal(s.potential(0.7).cpu().numpy(), want), (warps, longest)
    s.set_walk_shape(4, 1, 0, 1)
    gi, gt = (x.cpu().numpy() for x in s.walk_counts(0.7))
    assert np.array_equal(gi, wi) and np.array_equal(gt, wt)


def test_zero_field_and_one_block():
    """Edge cases: an all-zero density gives exactly zero (every term carries
    its mass), and a mesh of one block (the whole box one 8^3 block, every
    displacement wrapped) matches the oracle."""
    m = mg.uniform_mesh(0)
    s = _solver(m, np.zeros((1, 8, 8, 8)))
    assert np.all(s.potential(0.5).cpu().numpy() == 0.0)
    rho = mg.random_density(m, seed=77)
    s = _solver(m, rho)
    for theta in (0.2, 0.5, 1.0):
        phi = s.potential(theta).cpu().numpy()
        po, nio, _ = _oracle(m, rho).walk_periodic(theta)
        ni, _ = s.walk_counts(theta)
        assert np.array_equal(ni.cpu().numpy(), nio)
        assert np.abs(phi - po).max() <= 1e-5 * np.abs(po).max()


def test_physical_box_and_G():
    """A box of side 2.5 at (1, -2, 0.5) and G = 3: the walk works in box
    units and scales by -G/L like the oracle (which takes the same box)."""
    m = mg.refined_mesh(1, 2, lambda lev, ijk: np.all(ijk == 1, axis=1), name="corner11")
    rho = mg.random_density(m, seed=21)
    lo, L = (1.0, -2.0, 0.5), 2.5
    s = B.Solver(periodic=True)
    s.build(m.level, m.ijk, torch.as_tensor(np.asarray(rho, np.float32).reshape(-1)).cuda(), lo, L)
    phi = s.potential(0.6, G=3.0).cpu().numpy()
    t = O.Tree(m.level, m.ijk, np.asarray(rho, np.float32).astype(np.float64), lo, L)
    po = t.walk_periodic(0.6, G=3.0)[0]
    assert np.abs(phi - po).max() <= 1e-5 * np.abs(po).max()
    # and the unit box scales: Phi_L = Phi_1 * L^2 (masses ~ L^3, distances ~ L)
    s1 = _solver(m, rho)
    phi1 = s1.potential(0.6, G=3.0).cpu().numpy()
    assert np.abs(phi - phi1 * L * L).max() <= 1e-5 * np.abs(phi).max()


def test_batch_of_periodic_boxes_of_different_sizes():
    """Three fields in boxes of sides 1, 3 and 0.5 at different corners, built
    as one batch: each field's potentials equal the oracle's periodic walk in
    its own box (the wrap and chi act in each field's box units)."""
    from dataclasses import replace
    ms = [mg.uniform_mesh(0), mg.uniform_mesh(1),
          mg.refined_mesh(1, 2, lambda lev, ijk: np.all(ijk == 0, axis=1), name="c0")]
    boxes = [((0.0, 0.0, 0.0), 1.0), ((-1.0, 2.0, 0.5), 3.0), ((4.0, 4.0, 4.0), 0.5)]
    fields = [mg.Workload(name=f"box{i}", mesh=replace(m, box_lo=lo, box_len=L),
                          density=mg.random_density(m, seed=60 + i), thetas=(0.5,))
              for i, (m, (lo, L)) in enumerate(zip(ms, boxes))]
    nb, level, ijk, lo, ln, rho = mg.concat_fields(fields)
    s = B.Solver(periodic=True)
    d_rho = torch.as_tensor(rho.astype(np.float32)).cuda()
    s.build_batch(nb, level, ijk, d_rho, lo, ln)
    phi = s.potential(0.5, G=2.0).cpu().numpy()
    off = 0
    for f in fields:
        t = _oracle(f.mesh, f.density)
        po = t.walk_periodic(0.5, G=2.0)[0]
        got = phi[off:off + f.ncells]
        assert np.abs(got - po).max() <= 1e-5 * np.abs(po).max()
        off += f.ncells
