"""The allocation-free entry point, bh_solve_noalloc.

It serves callers that cannot allocate device memory (their GPU memory is
reserved by their own allocator, or they must keep the library out of
cudaMalloc/cudaFree, which may synchronise the device): the tree of a mesh of
up to 64 blocks lives in a fixed device array inside the library.  Here it is
called through the C-ABI and compared with the regular entry points
(bh_build + bh_potential) on two calls in a row (with a differently sized mesh
in between, so the second call runs over a scratch array the previous calls
left filled).  Both paths launch the same kernels with the same arguments on
the same inputs, only with the tree in a different place, so their
potentials must agree bit for bit; the first round of calls is also checked
against the CPU oracle's walk within the binary32 parity tolerance of the
other tests.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1509_07370_gb300 import bhgrav as B  # noqa: E402
from paper_1509_07370_gb300 import meshgen as mg  # noqa: E402

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _noalloc(mesh, rho_dev, theta, G, out):
    """One call of bh_solve_noalloc through the C-ABI (raw pointers)."""
    lib = B.load()
    level = np.ascontiguousarray(mesh.level, dtype=np.int32)
    ijk = np.ascontiguousarray(mesh.ijk, dtype=np.int32)
    lo = np.ascontiguousarray(mesh.box_lo, dtype=np.float64)
    P = ctypes.c_void_p
    return lib.bh_solve_noalloc(
        int(mesh.nblocks), level.ctypes.data_as(P), ijk.ctypes.data_as(P), lo.ctypes.data_as(P),
        float(mesh.box_len), P(rho_dev.data_ptr()), int(rho_dev.dtype == torch.float64),
        float(theta), float(G), P(out.data_ptr()),
        P(torch.cuda.current_stream().cuda_stream))


def _regular(mesh, rho_dev, theta, G):
    s = B.Solver()
    s.build(mesh.level, mesh.ijk, rho_dev, mesh.box_lo, mesh.box_len)
    phi = s.potential(theta, G).cpu().numpy()
    s.close()
    return phi


def test_noalloc_matches_regular_entry_points_on_consecutive_calls():
    big = mg.uniform_sphere()                                # 64 blocks: the maximum
    small = mg.tiny_meshes()["refined_corner"]               # 15 blocks, two levels
    cases = [
        (big.mesh, torch.as_tensor(big.density.reshape(-1), dtype=torch.float32).cuda(), 0.5),
        (small, torch.as_tensor(mg.random_density(small, 3).reshape(-1)).cuda(), 0.7),
        (big.mesh, torch.as_tensor(big.density.reshape(-1), dtype=torch.float32).cuda(), 0.3),
    ]
    for k in range(2):                                       # twice in a row
        for mesh, rho, theta in cases:
            want = _regular(mesh, rho, theta, 2.0)
            out = torch.full((mesh.ncells,), float("nan"), dtype=torch.float32, device="cuda")
            st = _noalloc(mesh, rho, theta, 2.0, out)
            assert st == B.BH_OK, st
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            # same kernels, same arguments: identical bits
            assert np.array_equal(got, want), (k, mesh.nblocks, theta)
            if k == 0:                                       # and the oracle's walk
                rho64 = rho.cpu().numpy().astype(np.float64)
                ref = O.Tree(mesh.level, mesh.ijk, rho64, mesh.box_lo,
                             mesh.box_len).walk(theta, G=2.0)[0]
                assert np.max(np.abs(got / ref - 1.0)) <= F32_TOL, (mesh.nblocks, theta)


def test_noalloc_rejects_what_does_not_fit_or_is_invalid():
    m = mg.uniform_mesh(2)
    rho = torch.ones(m.ncells, dtype=torch.float32, device="cuda")
    out = torch.empty(m.ncells, dtype=torch.float32, device="cuda")
    assert _noalloc(m, rho, 0.5, 1.0, out) == B.BH_OK
    too_big = mg.refined_mesh(2, 3, lambda lev, ijk: np.all(ijk == 0, axis=1))   # 71 blocks
    assert too_big.nblocks > 64
    rho2 = torch.ones(too_big.ncells, dtype=torch.float32, device="cuda")
    out2 = torch.empty(too_big.ncells, dtype=torch.float32, device="cuda")
    assert _noalloc(too_big, rho2, 0.5, 1.0, out2) == B.BH_ERR_ARG
    assert _noalloc(m, rho, 1.5, 1.0, out) == B.BH_ERR_ARG
    gap = mg.Mesh(m.level[:57], m.ijk[:57])                  # 57 = 1 + 7*8 blocks, with a gap
    assert _noalloc(gap, rho[: 57 * 512], 0.5, 1.0, out) == B.BH_ERR_GEOMETRY
    bad = rho.clone()
    bad[7] = -1.0
    assert _noalloc(m, bad, 0.5, 1.0, out) == B.BH_ERR_ARG
    for lo in ((float("nan"), 0.0, 0.0), (0.0, float("inf"), 0.0)):
        shifted = mg.Mesh(m.level, m.ijk, box_lo=np.array(lo), box_len=m.box_len)
        assert _noalloc(shifted, rho, 0.5, 1.0, out) == B.BH_ERR_ARG
    assert _noalloc(m, rho, 0.5, 1.0, out) == B.BH_OK        # still usable afterwards
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out.cpu().numpy()))
