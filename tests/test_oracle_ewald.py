"""Pins of the oracle's periodic boundaries (App. A, the Ewald field).

Facts the oracle does not produce itself:

* the field's value at the origin, chi(0) = psi(r) - 1/r at r -> 0, is the
  Madelung-type constant of a simple cubic lattice in a neutralising
  background, -2.837297479480619 (Nijboer & De Wette 1957; the usual Ewald
  self term of a cubic box);
* the result does not depend on the split parameter alpha (a wrong
  Fourier-space factor, exponent or constant term changes with alpha);
* psi is periodic with period 1, even, and symmetric under axis swaps;
* Poisson: chi = psi - 1/r has Laplacian 4 pi (a unit mass per unit volume
  subtracted) everywhere in the box around the origin;
* zero mean: the integral of psi over the box is 0, i.e. the integral of chi
  equals minus the integral of 1/r over the unit cube from its centre (the
  closed form pinned in test_oracle_pins.py);
* a uniform density: every cell sees a lattice of spacing h, so
  Phi = -G rho h^2 chi(0) exactly;
* the quadratic interpolation reproduces the table at its points, and its
  error falls about 8x per halving of the spacing (third order);
* the periodic walk: one massive cell gives -G m psi(minimum image) for every
  theta; theta -> 0 gives the direct periodic sum; a cyclic shift of the
  density shifts the direct periodic potential.
"""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import oracle as O
from paper_1509_07370_gb300 import meshgen as mg

XI = -2.837297479480619


def test_value_at_origin_is_the_cubic_lattice_constant():
    assert abs(O.ewald_sum(np.zeros(3), chi=True) - XI) < 1e-12


def test_independent_of_the_split_parameter():
    r = np.random.default_rng(0).uniform(-0.5, 0.5, (40, 3))
    ref = O.ewald_sum(r, 2.0, 4)
    for a in (1.3, 1.7, 2.6):
        assert np.abs(O.ewald_sum(r, a, 4) - ref).max() < 1e-12


def test_series_range_three_is_converged():
    r = np.random.default_rng(1).uniform(-0.5, 0.5, (40, 3))
    ref = O.ewald_sum(r, nseries=5, chi=True)
    assert np.abs(O.ewald_sum(r, nseries=3, chi=True) - ref).max() < 1e-13
    assert np.abs(O.ewald_sum(r, nseries=1, chi=True) - ref).max() > 1e-6


def test_periodic_even_and_axis_symmetric():
    r = np.random.default_rng(2).uniform(-0.5, 0.5, (40, 3))
    p = O.ewald_sum(r, nseries=4)
    for e in np.eye(3):
        assert np.abs(O.ewald_sum(r + e, nseries=4) - p).max() < 1e-11
    assert np.abs(O.ewald_sum(-r, nseries=4) - p).max() < 1e-13
    assert np.abs(O.ewald_sum(r[:, [2, 0, 1]], nseries=4) - p).max() < 1e-13
    assert np.abs(O.ewald_sum(r[:, [1, 0, 2]], nseries=4) - p).max() < 1e-13


def test_laplacian_is_four_pi():
    r = np.random.default_rng(3).uniform(-0.5, 0.5, (30, 3))
    h = 1e-3
    lap = -6.0 * O.ewald_sum(r, chi=True)
    for a in range(3):
        for s in (1.0, -1.0):
            q = r.copy()
            q[:, a] += s * h
            lap += O.ewald_sum(q, chi=True)
    assert np.abs(lap / h ** 2 - 4 * np.pi).max() < 1e-3


def test_zero_mean_over_the_box():
    x, w = np.polynomial.legendre.leggauss(10)
    xs = np.concatenate([-0.25 + 0.25 * x, 0.25 + 0.25 * x])
    ws = np.concatenate([0.25 * w, 0.25 * w])
    X, Y, Z = np.meshgrid(xs, xs, xs, indexing="ij")
    W = ws[:, None, None] * ws[None, :, None] * ws[None, None, :]
    integral = (O.ewald_sum(np.stack([X, Y, Z], -1), chi=True) * W).sum()
    assert abs(integral + A.cube_centre_factor()) < 1e-10


def test_table_interpolation():
    ng = 32
    T = O.ewald_table(ng).reshape(ng + 2, ng + 2, ng + 2)       # [k][j][i]
    h = 1.0 / (2 * ng)
    idx = np.random.default_rng(4).integers(0, ng + 1, (50, 3))
    u = idx * h
    assert np.abs(O.ewald_interp(u, ng) - T[idx[:, 2], idx[:, 1], idx[:, 0]]).max() < 1e-14
    assert np.abs(T[idx[:, 2], idx[:, 1], idx[:, 0]] - O.ewald_sum(u, chi=True)).max() < 1e-14
    pts = np.random.default_rng(5).uniform(0.0, 0.5, (3000, 3))
    exact = O.ewald_sum(pts, chi=True)
    err = [np.abs(O.ewald_interp(pts, n) - exact).max() for n in (16, 32, 64)]
    assert err[2] < 4e-6
    assert 5.0 < err[0] / err[1] < 11.0 and 5.0 < err[1] / err[2] < 11.0
    # the minimum-image argument: |u| per component, the sign does not matter
    s = pts * np.array([-1.0, 1.0, -1.0])
    assert np.array_equal(O.ewald_interp(s, 64), O.ewald_interp(pts, 64))


def test_uniform_density_is_the_lattice_sum():
    m = mg.uniform_mesh(0)
    rho = np.full((1, 8, 8, 8), 1.7)
    t = O.Tree(m.level, m.ijk, rho, m.box_lo, m.box_len)
    G, h = 0.8, 1.0 / 8
    want = -G * 1.7 * h * h * XI
    tg = np.array([0, 7, 73, 292, 511])
    exact = t.direct_periodic(G=G, targets=tg, ng=None)
    assert np.abs(exact / want - 1).max() < 1e-11
    table = t.direct_periodic(G=G, targets=tg, ng=64)
    assert np.abs(table / want - 1).max() < 1e-4


def test_one_massive_cell_every_theta():
    m = mg.uniform_mesh(1)
    rho = np.zeros((8, 8, 8, 8))
    rho[5, 7, 6, 7] = 4.0          # a cell near the far corner of block 5
    t = O.Tree(m.level, m.ijk, rho, m.box_lo, m.box_len)
    tg = np.random.default_rng(6).choice(8 * 512, 60, replace=False)
    want = t.direct_periodic(G=1.5, targets=tg)
    for theta in (0.3, 0.7, 1.0):
        got = t.walk_periodic(theta, G=1.5, targets=tg)[0]
        assert np.allclose(got, want, rtol=1e-12, atol=0)
    # against the Ewald sum itself (table error only), through the wrap
    exact = t.direct_periodic(G=1.5, targets=tg, ng=None)
    assert np.abs(want - exact).max() < 1e-5 * np.abs(exact).max()
    # by hand for a cell across the box edge: minimum image
    u, _ = _centres(m)
    a = 5 * 512 + 7 * 64 + 6 * 8 + 7
    b = 0                           # block 0, cell (0, 0, 0): the corner opposite
    d = u[b] - u[a]
    d -= np.round(d)
    psi = O.ewald_sum(d, chi=False)
    mass = 4.0 / 16 ** 3
    got = t.direct_periodic(G=1.0, targets=[b], ng=None)[0]
    assert abs(got / (-mass * psi) - 1) < 1e-12


def _centres(mesh):
    x = mesh.cell_centres().reshape(-1, 3)
    return (x - np.asarray(mesh.box_lo)) / mesh.box_len, None


def test_small_theta_is_the_direct_periodic_sum():
    for name, m in sorted(mg.tiny_meshes().items()):
        rho = mg.random_density(m, seed=7)
        t = O.Tree(m.level, m.ijk, rho, m.box_lo, m.box_len)
        tg = np.random.default_rng(8).choice(t.ncells, 40, replace=False)
        phi, ni, _ = t.walk_periodic(1e-3, targets=tg)
        assert np.all(ni == t.ncells - 1), name
        d = t.direct_periodic(targets=tg)
        assert np.abs(phi - d).max() < 1e-12 * np.abs(d).max(), name


def test_error_falls_with_theta_and_is_small():
    w = mg.uniform_sphere(block_level=1, radius=0.3, rho_out=1e-2)
    t = O.Tree.from_workload(w)
    tg = np.random.default_rng(9).choice(t.ncells, 300, replace=False)
    d = t.direct_periodic(targets=tg)
    scale = np.abs(d).max()
    errs = [np.abs(t.walk_periodic(th, targets=tg)[0] - d).max() / scale
            for th in (0.9, 0.6, 0.3)]
    assert errs[0] > errs[1] > errs[2] and errs[0] < 0.05


def test_cyclic_shift_shifts_the_potential():
    m = mg.uniform_mesh(1)
    rho = mg.random_density(m, seed=10)
    ijk = m.ijk.copy()
    ijk[:, 0] = (ijk[:, 0] + 1) % 2                     # every block one block along x
    t0 = O.Tree(m.level, m.ijk, rho, m.box_lo, m.box_len)
    t1 = O.Tree(m.level, ijk, rho, m.box_lo, m.box_len)
    tg = np.random.default_rng(11).choice(t0.ncells, 50, replace=False)
    a = t0.direct_periodic(targets=tg)
    b = t1.direct_periodic(targets=tg)                   # the same cells, moved
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    iso_a, iso_b = t0.direct(targets=tg), t1.direct(targets=tg)
    assert np.abs(iso_a - iso_b).max() > 1e-3 * np.abs(iso_a).max()
