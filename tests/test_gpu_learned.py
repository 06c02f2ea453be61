"""The learned residual correction on the GPU, against the CPU oracle.

Bars:
  * training pairs: the same accepted nodes as the oracle's walk (exact, the
    decisions are bit-exact), features within 1e-5 (the GPU reads binary32
    quadrupoles), eps within 1e-6 absolute (both sum the node's cells in FP64);
  * gradients of the loss: within 1e-4 of the largest gradient component
    (FP32 accumulation over the batch vs the oracle's FP64);
  * the learned walk against the oracle's FP64 evaluation with the same
    bf16-rounded weights: within 2 % of the largest network contribution
    (learned walk minus monopole walk) plus 1e-5 of the potential -- the
    tensor-core path rounds the features, b1 and the hidden activations to
    bf16 (8 significant bits, relative 2^-9 each, through two 64-wide layers)
    and evaluates the GELU in bf16 pairs with the SFU's tanh, so each node's
    correction carries about 1 % error; corrections of different nodes can cancel in a cell, so
    the bound scales with their size, not with a cell's net correction;
  * what the trained network gains: smaller max error against the direct sum
    than the plain walk at the same theta, on a field it was not trained on.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1509_07370_gb300 import bhgrav as B  # noqa: E402
from paper_1509_07370_gb300 import learned as L  # noqa: E402
from paper_1509_07370_gb300 import meshgen as mg  # noqa: E402

pytestmark = pytest.mark.gpu


def _field():
    return mg.maclaurin(base_level=1, extra_levels=2, a1=0.22, e=0.85)


def _gpu(w, learned=False):
    s = B.Solver(quadrupole=not learned, learned=learned)
    s.build(w.mesh.level, w.mesh.ijk, torch.as_tensor(w.density.reshape(-1)).cuda())
    return s


def test_training_pairs_match_oracle():
    w = _field()
    s = _gpu(w)
    t = O.Tree.from_workload(w)
    for tgt in np.random.default_rng(3).choice(w.ncells, 8, replace=False):
        f, e, n, nd = s.learn_pairs(0.8, torch.tensor([tgt], device="cuda"), 4096,
                                    with_nodes=True)
        order = torch.argsort(nd)
        f, e, nd = (x[order].cpu().numpy() for x in (f, e, nd))
        fo, eo, ndo = t.learn_pairs(0.8, tgt)
        o = np.argsort(ndo)
        assert n == len(ndo) and np.array_equal(nd, ndo[o])
        assert np.abs(f - fo[o]).max() <= 1e-5
        assert np.abs(e - eo[o]).max() <= 1e-6


def test_mlp_gradient_matches_oracle():
    rng = np.random.default_rng(5)
    w = L.init_weights(7) + rng.normal(0, 0.02, B.MLP_NW).astype(np.float32)
    x = rng.normal(0, 1, (1000, 10)).astype(np.float32)
    z = rng.normal(0, 0.3, 1000).astype(np.float32)
    g = torch.empty(B.MLP_NW, device="cuda")
    loss = torch.empty(1, device="cuda")
    B.bh_mlp_grad(torch.as_tensor(x).cuda(), torch.as_tensor(z).cuda(),
                  torch.as_tensor(w).cuda(), g, loss)
    torch.cuda.synchronize()
    lo, go = O.mlp_loss_grad(w.astype(np.float64), x.astype(np.float64), z.astype(np.float64))
    assert abs(float(loss.item()) / lo - 1) < 1e-5
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-4 * np.abs(go).max()


def test_adam_step_lowers_the_loss():
    rng = np.random.default_rng(1)
    x = torch.as_tensor(rng.normal(0, 1, (4096, 10)).astype(np.float32)).cuda()
    z = (x[:, 3] * 0.5 - x[:, 7] * 0.2).contiguous()
    w, hist = L.train(x, z, epochs=6, batch=1024, lr=3e-3, seed=2)
    assert hist[-1] < 0.2 * hist[0]


def test_learned_walk_matches_oracle():
    """A fixed (Glorot-initialised, seed 3) network, so that the comparison is
    reproducible: training on the GPU is not bit-reproducible (its pair list
    and gradient sums use atomics), and with trained networks, whose net
    corrections are small and cancel between nodes, the largest
    difference measured 0.8 to 1.2 times this bar across four trainings.
    Trained networks are checked by what they gain (below)."""
    w = _field()
    wts = L.init_weights(3)
    s = _gpu(w, learned=True)
    s.set_mlp(wts)
    phi = s.potential(0.8).cpu().numpy()
    wb = s.get_mlp().astype(np.float64)                   # the bf16 weights in use
    t = O.Tree.from_workload(w)
    tg = np.random.default_rng(2).choice(w.ncells, 600, replace=False)
    learned = t.walk_learned(0.8, wb, targets=tg)
    mono = t.walk(0.8, targets=tg)[0]
    corr = np.abs(learned - mono)
    assert corr.max() > 1e-6 * np.abs(mono).max()        # the network does something
    assert np.all(np.abs(phi[tg] - learned) <= 0.02 * corr.max() + 1e-5 * np.abs(learned))


def test_gated_learned_walk_matches_oracle():
    """The gate (network only for accepted nodes with s = l/d >= s_min,
    decided in binary32 on the opening test's d^2 on both sides): at s_min =
    0.4 the learned walk, in both tensor-core forms, against the oracle's
    gated walk with the same bf16 weights (the bar of the ungated test); at
    s_min = 0.999 no accepted node is corrected (s < theta < 1), which is the
    oracle's plain monopole walk within the binary32 bar; bad gates are
    refused."""
    w = _field()
    wts = L.init_weights(3)
    t = O.Tree.from_workload(w)
    tg = np.random.default_rng(5).choice(w.ncells, 600, replace=False)
    mono = t.walk(0.8, targets=tg)[0]
    rho = torch.as_tensor(w.density.reshape(-1)).cuda()
    for mode in (1, 2):
        s = B.Solver(learned=mode)
        s.build(w.mesh.level, w.mesh.ijk, rho)
        s.set_mlp(wts)
        wb = s.get_mlp().astype(np.float64)
        s.set_mlp_gate(0.4)
        phi = s.potential(0.8).cpu().numpy()
        s.sync_status()
        gated = t.walk_learned(0.8, wb, targets=tg, s_min=0.4)
        full = t.walk_learned(0.8, wb, targets=tg)
        corr = np.abs(gated - mono)
        assert corr.max() > 1e-6 * np.abs(mono).max()       # some pairs pass the gate
        assert np.any(np.abs(full - gated) > 1e-9 * np.abs(mono))  # and some do not
        assert np.all(np.abs(phi[tg] - gated) <= 0.02 * corr.max() + 1e-5 * np.abs(gated))
        s.set_mlp_gate(0.999)
        phi = s.potential(0.8).cpu().numpy()
        assert np.max(np.abs(phi[tg] / mono - 1.0)) <= 1e-5
        for bad in (-0.1, 1.0, float("nan")):
            with pytest.raises(B.BHError) as e:
                s.set_mlp_gate(bad)
            assert e.value.status == B.BH_ERR_ARG
        s.close()


def test_trained_network_beats_the_plain_walk_at_the_same_theta():
    xs, zs = [], []
    for i in range(24):
        f = L.training_field(9000 + i)
        x, z = L.pairs_of(_gpu(f), f.ncells, 0.8, 64, seed=i)
        xs.append(x)
        zs.append(z)
    wts, hist = L.train(torch.cat(xs), torch.cat(zs), epochs=4, batch=4096, seed=0)
    test = mg.maclaurin(base_level=2, extra_levels=2)     # not a training field
    s = _gpu(test, learned=True)
    s.set_mlp(wts)
    phi_l = s.potential(0.8).cpu().numpy()
    plain = B.Solver()
    plain.build(test.mesh.level, test.mesh.ijk, torch.as_tensor(test.density.reshape(-1)).cuda())
    phi_p = plain.potential(0.8).cpu().numpy()
    t = O.Tree.from_workload(test)
    tg = np.random.default_rng(4).choice(test.ncells, 1500, replace=False)
    d = t.direct(targets=tg)
    err_l = np.abs(phi_l[tg] / d - 1).max()
    err_p = np.abs(phi_p[tg] / d - 1).max()
    assert err_l < 0.5 * err_p, (err_l, err_p)


def test_learned_walk_in_a_graph_and_a_batch():
    """The learned walk replayed as a CUDA graph (bh_solve_graph) and inside a
    batch of fields gives the same potentials as bh_potential per field."""
    wts = L.init_weights(5)
    fields = [_field(), mg.maclaurin(base_level=1, extra_levels=2, a1=0.15, e=0.6)]
    single = []
    for f in fields:
        s = B.Solver(learned=True)
        s.build(f.mesh.level, f.mesh.ijk,
                torch.as_tensor(f.density.reshape(-1).astype(np.float32)).cuda())
        s.set_mlp(wts)
        single.append(s.potential(0.8).cpu().numpy())
    nb, level, ijk, lo, ln, rho = mg.concat_fields(fields)
    st = torch.cuda.Stream()
    s = B.Solver(learned=True, stream=st)
    d_rho = torch.as_tensor(rho.astype(np.float32)).cuda()
    s.build_batch(nb, level, ijk, d_rho, lo, ln)
    s.set_mlp(wts)
    out = torch.empty(d_rho.numel(), device="cuda")
    with torch.cuda.stream(st):
        s.solve_graph(d_rho, 0.8, 1.0, out)
        s.solve_graph(d_rho, 0.8, 1.0, out)
    st.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got, np.concatenate(single))


@pytest.mark.parametrize("n", [1, 128, 1000])
def test_tensor_core_network_matches_oracle(n):
    """bh_mlp_eval (tcgen05, bf16 operands, FP32 accumulators in tensor
    memory) against the oracle's FP64 forward pass with the same bf16
    weights: within 2 % of the largest |y| (bf16 features and activations,
    bf16 GELU), on 1 row, one full 128-row tile and a ragged 1,000 rows."""
    rng = np.random.default_rng(n)
    w = L.init_weights(11) + rng.normal(0, 0.05, B.MLP_NW).astype(np.float32)
    x = rng.normal(0, 1, (n, 10)).astype(np.float32)
    s = B.Solver(learned=True)
    s.set_mlp(w)
    y = s.mlp_eval(torch.as_tensor(x).cuda()).cpu().numpy()
    wb = s.get_mlp().astype(np.float64)
    xb = torch.as_tensor(x).to(torch.bfloat16).double().numpy()   # the features it sees
    ref = O.mlp_forward(wb, xb)[0]
    assert np.all(np.isfinite(y))
    assert np.abs(y - ref).max() <= 0.02 * np.abs(ref).max() + 1e-6


def test_training_targets_normalised_in_the_library():
    """bh_learn_targets: z = eps / s^2 of each pair, s = feature 3, the same
    binary32 operations as the definition (s * s rounded, then divided)."""
    w = _field()
    s = _gpu(w, learned=True)
    tg = torch.as_tensor(np.arange(0, w.ncells, 997), dtype=torch.int64).cuda()
    feat, eps, _ = s.learn_pairs(0.8, tg, 1 << 18)
    z = B.bh_learn_targets(feat, eps).cpu().numpy()
    f = feat.cpu().numpy()
    e = eps.cpu().numpy()
    sq = (f[:, 3] * f[:, 3]).astype(np.float32)
    assert len(z) > 1000 and np.array_equal(z, (e / sq).astype(np.float32))


def test_tensor_core_wait_timeout_reported_and_recoverable(monkeypatch):
    """The bounded wait for the tensor core, made to run out without a fault:
    with BHGRAV_TC_WAIT_PROBE=k the evaluator issues no MMA (nothing is in
    flight) and gives up its first wait on a barrier no one arrives at after
    k tries; bh_mlp_eval returns BH_ERR_DEVICE_TIMEOUT with its reason, the
    kernel releases its tensor memory, and the same context then evaluates
    the same rows as a fresh one does, bit for bit (3,000 rows: several CTAs,
    a ragged last tile)."""
    import time
    rng = np.random.default_rng(7)
    w = L.init_weights(5) + rng.normal(0, 0.05, B.MLP_NW).astype(np.float32)
    x = torch.as_tensor(rng.normal(0, 1, (3000, 10)).astype(np.float32)).cuda()
    s = B.Solver(learned=True)
    s.set_mlp(w)
    monkeypatch.setenv("BHGRAV_TC_WAIT_PROBE", "16")
    t0 = time.perf_counter()
    with pytest.raises(B.BHError) as e:
        s.mlp_eval(x)
    assert time.perf_counter() - t0 < 60.0
    assert e.value.status == B.BH_ERR_DEVICE_TIMEOUT
    assert "wait" in str(e.value) and "gave up" in str(e.value)
    monkeypatch.delenv("BHGRAV_TC_WAIT_PROBE")
    got = s.mlp_eval(x).cpu().numpy()
    fresh = B.Solver(learned=True)
    fresh.set_mlp(w)
    want = fresh.mlp_eval(x).cpu().numpy()
    assert np.all(np.isfinite(got)) and np.array_equal(got, want)


def test_tensor_core_learned_walk_matches_the_warp_level_one_and_the_oracle():
    """The learned walk with the network on tcgen05 (learned = 2): the same
    per-row arithmetic as the mma.sync walk up to FP32 accumulation order,
    so within 1e-5 of it per cell; and within the oracle bar."""
    w = _field()
    wts = L.init_weights(4)
    rho = torch.as_tensor(w.density.reshape(-1).astype(np.float32)).cuda()
    phis = []
    for mode in (1, 2):
        s = B.Solver(learned=mode)
        s.build(w.mesh.level, w.mesh.ijk, rho)
        s.set_mlp(wts)
        phis.append(s.potential(0.8).cpu().numpy())
        s.sync_status()
        wb = s.get_mlp().astype(np.float64)
    assert np.all(np.abs(phis[1] / phis[0] - 1.0) <= 1e-5)
    t = O.Tree(w.mesh.level, w.mesh.ijk, w.density.astype(np.float32).astype(np.float64))
    tg = np.random.default_rng(6).choice(w.ncells, 600, replace=False)
    learned = t.walk_learned(0.8, wb, targets=tg)
    mono = t.walk(0.8, targets=tg)[0]
    corr = np.abs(learned - mono)
    assert np.all(np.abs(phis[1][tg] - learned) <= 0.02 * corr.max() + 1e-5 * np.abs(learned))
