"""Batched solves (several independent fields in one build and one walk) and
the CUDA-graph replay, through the C-ABI.

Bars: a field solved inside a batch gives bit-identical potentials to the
same field solved alone (same tree, same arithmetic, same warp grouping);
the graph replay and the tuned launch shape change nothing either; per-cell
decisions match the oracle for every field.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1509_07370_gb300 import bhgrav as B  # noqa: E402
from paper_1509_07370_gb300 import meshgen as mg  # noqa: E402

pytestmark = pytest.mark.gpu


def _fields():
    t = mg.tiny_meshes()
    ws = []
    for i, (name, lo, ln) in enumerate([("refined_corner", (0, 0, 0), 1.0),
                                        ("one_block", (-2.0, 1.0, 0.5), 3.0),
                                        ("diag_refined", (0, 0, 0), 0.5),
                                        ("eight_blocks", (1.0, 1.0, 1.0), 2.0)]):
        m = t[name]
        m2, rho = mg.shuffled(m, mg.random_density(m, 40 + i), seed=i)
        m2 = mg.Mesh(m2.level, m2.ijk, box_lo=lo, box_len=ln, name=name)
        ws.append(mg.Workload(name, m2, rho, (0.5,)))
    ws += mg.batch_fields(3, seed0=7000, levels=(1, 2))
    return ws


def _solver(**kw):
    return B.Solver(stream=torch.cuda.Stream(), **kw)


@pytest.mark.parametrize("quad", [False, True])
def test_batch_equals_fields_solved_alone(quad):
    ws = _fields()
    nb, level, ijk, lo, ln, rho = mg.concat_fields(ws)
    s = _solver(quadrupole=quad)
    s.build_batch(nb, level, ijk, torch.as_tensor(rho).cuda(), lo, ln)
    with torch.cuda.stream(s.stream):
        phi = s.potential(0.6, G=1.5)
    s.stream.synchronize()
    phi = phi.cpu().numpy()
    off = 0
    for w in ws:
        a = _solver(quadrupole=quad)
        a.build(w.mesh.level, w.mesh.ijk, torch.as_tensor(w.density.reshape(-1)).cuda(),
                w.mesh.box_lo, w.mesh.box_len)
        with torch.cuda.stream(a.stream):
            want = a.potential(0.6, G=1.5)
        a.stream.synchronize()
        n = w.ncells
        assert np.array_equal(phi[off:off + n], want.cpu().numpy()), w.name
        off += n


def test_batch_decisions_match_oracle_per_field():
    ws = _fields()
    nb, level, ijk, lo, ln, rho = mg.concat_fields(ws)
    s = _solver()
    s.build_batch(nb, level, ijk, torch.as_tensor(rho).cuda(), lo, ln)
    ni, nt = (x.cpu().numpy() for x in s.walk_counts(0.5))
    off = 0
    for w in ws:
        t = O.Tree(w.mesh.level, w.mesh.ijk, w.density, w.mesh.box_lo, w.mesh.box_len)
        _, oi, ot = t.walk(0.5)
        n = w.ncells
        assert np.array_equal(ni[off:off + n], oi) and np.array_equal(nt[off:off + n], ot)
        off += n


def test_update_density_graph_replay_and_autotune():
    ws = _fields()
    nb, level, ijk, lo, ln, rho = mg.concat_fields(ws)
    s = _solver(quadrupole=True)
    d0 = torch.as_tensor(rho, dtype=torch.float32).cuda()
    s.build_batch(nb, level, ijk, d0, lo, ln)
    rho2 = rho * np.random.default_rng(1).uniform(0.5, 2.0, size=rho.shape)
    d1 = torch.as_tensor(rho2, dtype=torch.float32).cuda()
    ref = _solver(quadrupole=True)
    ref.build_batch(nb, level, ijk, d1, lo, ln)
    with torch.cuda.stream(ref.stream):
        want = ref.potential(0.7).cpu().numpy()
    s.update_density(d1)
    s.sync_status()
    with torch.cuda.stream(s.stream):
        got = s.potential(0.7)
    s.stream.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)
    w, npairs, ticket, longest = s.autotune(0.7)
    assert w in (2, 4, 8, 16) and npairs in (1, 2) and ticket in (0, 1, 2, 4)
    assert longest in (0, 1)
    out = torch.empty(s.ncells, device="cuda")
    for _ in range(3):                                  # capture once, replay twice
        out.fill_(float("nan"))
        s.solve_graph(d1, 0.7, 1.0, out)
        s.stream.synchronize()
        assert np.array_equal(out.cpu().numpy(), want)
    s.solve_graph(d0, 0.7, 1.0, out)                    # new density: recaptured
    s.stream.synchronize()
    with torch.cuda.stream(ref.stream):
        ref.update_density(d0)
        want0 = ref.potential(0.7).cpu().numpy()
    assert np.array_equal(out.cpu().numpy(), want0)
    s.sync_status()


def test_batch_errors():
    ws = _fields()
    nb, level, ijk, lo, ln, rho = mg.concat_fields(ws)
    s = _solver()
    lv = level.copy()
    lv[0] = lv[0] + 1                                           # a gap in field 0
    with pytest.raises(B.BHError) as e:
        s.build_batch(nb, lv, ijk, torch.as_tensor(rho).cuda(), lo, ln)
    assert e.value.status == B.BH_ERR_GEOMETRY
    s.build_batch(nb, level, ijk, torch.as_tensor(rho).cuda(), lo, ln)
    neg = torch.as_tensor(rho).cuda()
    neg[5] = -1.0
    s.update_density(neg)
    with pytest.raises(B.BHError) as e:
        s.sync_status()
    assert e.value.status == B.BH_ERR_ARG
    plain = B.Solver()                                          # legacy default stream
    plain.build(ws[0].mesh.level, ws[0].mesh.ijk, torch.as_tensor(ws[0].density.reshape(-1)).cuda())
    with pytest.raises(B.BHError) as e:
        plain.solve_graph(torch.as_tensor(ws[0].density.reshape(-1)).cuda(), 0.5)
    assert e.value.status == B.BH_ERR_ARG


SHAPES = [(4, 1, 0), (2, 1, 0), (16, 1, 0), (8, 2, 0), (4, 1, 1), (8, 1, 4), (4, 2, 2),
          (1, 2, 64), (16, 1, 1), (16, 2, 0)]


@pytest.mark.parametrize("quad", [False, True])
def test_every_walk_shape_gives_identical_potentials(quad):
    """Every launch shape the autotuner can choose -- CTA width, 64- or
    128-target groups, plain or persistent grid with 1-64 groups per take --
    gives the potentials of the default shape bit for bit (the same
    decisions and the same additions in the same order, a masked target's
    zero term changing nothing), on the batch of uneven fields and through
    the graph replay; the counting walk gives the same counts."""
    ws = _fields()
    nb, level, ijk, lo, ln, rho = mg.concat_fields(ws)
    d = torch.as_tensor(rho).cuda()
    s = _solver(quadrupole=quad)
    s.build_batch(nb, level, ijk, d, lo, ln)
    with torch.cuda.stream(s.stream):
        want = s.potential(0.6).cpu().numpy()
        wi, wt = (x.cpu().numpy() for x in s.walk_counts(0.6))
    out = torch.empty(s.ncells, device="cuda")
    for shape in SHAPES:
        s.set_walk_shape(*shape)
        with torch.cuda.stream(s.stream):
            got = s.potential(0.6).cpu().numpy()
            gi, gt = (x.cpu().numpy() for x in s.walk_counts(0.6))
        assert np.array_equal(got, want), shape
        assert np.array_equal(gi, wi) and np.array_equal(gt, wt), shape
        out.fill_(float("nan"))
        s.solve_graph(d, 0.6, 1.0, out)
        s.stream.synchronize()
        assert np.array_equal(out.cpu().numpy(), want), shape


@pytest.mark.parametrize("quad", [False, True])
def test_walk_order_keeps_every_bit(quad):
    """bh_autotune also sorts the groups by the length of their walks
    (longest first) for the plain and persistent grids; walking them in that
    order changes which warp takes which group and when, not what any group
    computes: the potentials and counts of every shape stay those of the
    groups' own order, bit for bit."""
    ws = _fields()
    nb, level, ijk, lo, ln, rho = mg.concat_fields(ws)
    d = torch.as_tensor(rho).cuda()
    s = _solver(quadrupole=quad)
    s.build_batch(nb, level, ijk, d, lo, ln)
    with torch.cuda.stream(s.stream):
        want = s.potential(0.6).cpu().numpy()
        wi, wt = (x.cpu().numpy() for x in s.walk_counts(0.6))
    s.autotune(0.6)
    for shape in SHAPES:
        s.set_walk_shape(*shape, 1)
        with torch.cuda.stream(s.stream):
            got = s.potential(0.6).cpu().numpy()
            gi, gt = (x.cpu().numpy() for x in s.walk_counts(0.6))
        assert np.array_equal(got, want), shape
        assert np.array_equal(gi, wi) and np.array_equal(gt, wt), shape


def test_walk_shape_arguments_checked():
    s = _solver()
    for bad in [(17, 1, 0), (4, 3, 0), (4, 1, 65), (-1, 1, 0), (4, 1, 0, 2)]:
        with pytest.raises(B.BHError) as e:
            s.set_walk_shape(*bad)
        assert e.value.status == B.BH_ERR_ARG
    with pytest.raises(B.BHError) as e:                        # no order before bh_autotune
        s.set_walk_shape(4, 1, 1, 1)
    assert e.value.status == B.BH_ERR_STATE
    p = B.Solver(periodic=True)
    for bad in [(4, 2, 0), (4, 1, 1)]:
        with pytest.raises(B.BHError) as e:
            p.set_walk_shape(*bad)
        assert e.value.status == B.BH_ERR_ARG
    with pytest.raises(B.BHError) as e:                        # no order before bh_autotune
        p.set_walk_shape(4, 1, 0, 1)
    assert e.value.status == B.BH_ERR_STATE
    p.set_walk_shape(16, 1, 0)
