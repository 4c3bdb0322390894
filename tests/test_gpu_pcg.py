"""The batched Jacobi-preconditioned CG (fea_pcg), through the C ABI, on symmetric positive
definite systems assembled by the library (MASS and DIFF terms): the solution agrees with the
oracle's direct solve of the same FP32 matrix, the reported residual is the true one, and the
degenerate cases (zero right-hand side, no iterations, an exact initial guess, a matrix that
is not positive definite) behave as documented."""
import numpy as np
import pytest

import oracle as O
from helpers import GpuRun
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu

SPD = fea.FEA_TERM_MASS | fea.FEA_TERM_DIFF


def spd_system(t, n, q, dt, seed=3):
    mesh = G.structured_mesh(t, n)
    G.perturb_interior(mesh, np.random.default_rng(seed), 0.15 if t != G.HEX27 else 0.0)
    f = G.draw_fields(np.random.default_rng(seed + 1), mesh.coords, q, 50.0, dt=dt)
    run = GpuRun(mesh)
    v, _ = run.assemble(f, fea.FEA_F32_FUSED, terms=SPD)
    return mesh, run, v


def host_residual(rp, ci, vals, x, b):
    import scipy.sparse as sp
    n = rp.size - 1
    A = sp.csr_matrix((vals.astype(np.float64), ci, rp), shape=(n, n))
    return np.linalg.norm(b - A @ x) / np.linalg.norm(b)


@pytest.mark.parametrize("t,n,q,dt", [(G.HEX8, 6, 3, 1e-3), (G.HEX8, 6, 3, 1.0), (G.TET4, 5, 2, 1.0),
                                      (G.HEX27, 3, 2, 1.0), (G.PYR5, 4, 2, 1.0)],
                         ids=["hex8_dt1e-3", "hex8_dt1", "tet4", "hex27", "pyr5"])
def test_pcg_matches_direct_solve(t, n, q, dt):
    import torch
    mesh, run, v = spd_system(t, n, q, dt)
    try:
        rng = np.random.default_rng(11)
        b = rng.standard_normal((q, mesh.n_node)).astype(np.float32)
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros((q, mesh.n_node), device="cuda")
        iters, rel = fea.fea_pcg(run.pattern, v, bd, x, q, 1000, 1e-6)
        torch.cuda.synchronize()
        rp, ci, _ = run.pattern_np()
        vals = v[:, :run.nnz].cpu().numpy()
        xs = x.cpu().numpy().astype(np.float64)
        for k in range(q):
            assert 0 < iters[k] < 1000 and rel[k] <= 1e-6, (k, iters[k], rel[k])
            assert host_residual(rp, ci, vals[k], xs[k], b[k].astype(np.float64)) <= 1e-5
            ref = O.solve(rp, ci, vals[k], b[k])
            assert np.linalg.norm(xs[k] - ref) <= 1e-3 * np.linalg.norm(ref)
    finally:
        run.close()


def test_pcg_degenerate_cases():
    import torch
    mesh, run, v = spd_system(G.HEX8, 4, 2, 1.0)
    try:
        N = mesh.n_node
        zero = torch.zeros((2, N), device="cuda")
        x = torch.zeros((2, N), device="cuda")
        iters, rel = fea.fea_pcg(run.pattern, v, zero, x, 2, 100, 1e-6)  # b = 0, x0 = 0: nothing to do
        assert list(iters) == [0, 0] and float(x.abs().max()) == 0.0
        b = torch.from_numpy(np.random.default_rng(2).standard_normal((2, N)).astype(np.float32)).cuda()
        x = torch.full((2, N), 0.5, device="cuda")
        iters, rel = fea.fea_pcg(run.pattern, v, b, x, 2, 0, 1e-6)  # no iterations: x unchanged
        assert list(iters) == [0, 0] and float((x - 0.5).abs().max()) == 0.0 and (rel > 0).all()
        iters, rel = fea.fea_pcg(run.pattern, v, b, x, 2, 1000, 1e-6)  # then solve from there
        assert (iters > 0).all() and (rel <= 1e-6).all()
        again, rel2 = fea.fea_pcg(run.pattern, v, b, x, 2, 1000, 1e-3)  # already within 1e-3
        assert list(again) == [0, 0]
        with pytest.raises(fea.FeaError) as ei:  # -A is negative definite
            fea.fea_pcg(run.pattern, -v, b, torch.zeros((2, N), device="cuda"), 2, 50, 1e-6)
        assert ei.value.name == "FEA_ERR_ARG"
    finally:
        run.close()
