"""The cancellation check (opts.cancel_check): flagged rows are recomputed in FP64.

Contrived case: an undistorted Hex8 (or prism, or pyramid) mesh, SUPG off, phi_old = x - 1/2 for
one equation; each mesh is mirror-symmetric about x = 1/2.  The
RHS of every node on the plane x = 1/2 is then a sum of element contributions that cancel
(sum |b^e_i| >> |b_i|), so those rows must be flagged; after the FP64 recomputation their
RHS matches the FP64 oracle to FP64 accuracy relative to the magnitude of the contributions,
while every other row is the untouched FP32 result."""
import numpy as np
import pytest

import oracle as O
from helpers import TOL_F32, GpuRun, compare_full
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu

TERMS = fea.FEA_TERM_ALL & ~fea.FEA_TERM_SUPG


def contrived(n=8, t=G.HEX8):
    mesh = G.structured_mesh(t, n)
    rng = np.random.default_rng(3)
    f = G.draw_fields(rng, mesh.coords, 2, 50.0)
    f.phi_old[0] = mesh.coords[:, 0] - 0.5
    return mesh, f.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("t,scatter", [(G.HEX8, fea.FEA_SCATTER_ROWOWNED), (G.HEX8, fea.FEA_SCATTER_GATHER),
                                       (G.HEX8, fea.FEA_SCATTER_ATOMIC), (G.PEN6, fea.FEA_SCATTER_GATHER),
                                       (G.PEN6, fea.FEA_SCATTER_ATOMIC), (G.PYR5, fea.FEA_SCATTER_ATOMIC)],
                         ids=["hex8_rowowned", "hex8_gather", "hex8_atomic", "pen6_gather", "pen6_atomic",
                              "pyr5_atomic"])
def test_cancelling_rows_are_flagged_and_recomputed(t, scatter):
    n = 8
    mesh, f = contrived(n, t)
    run = GpuRun(mesh)
    try:
        v0, r0 = run.assemble(f, fea.FEA_F32_FUSED, terms=TERMS, scatter=scatter)
        with pytest.raises(fea.FeaError):
            fea.fea_cancel_rows(run.pattern, 2)
        v1, r1 = run.assemble(f, fea.FEA_F32_FUSED, terms=TERMS, scatter=scatter, cancel_check=1)
        count = fea.fea_cancel_rows(run.pattern, 2)
        plane = np.isclose(mesh.coords[:, 0], 0.5)
        assert plane.sum() == (n + 1) ** 2
        assert plane.sum() <= count < mesh.n_node // 2

        rp, ci, _ = run.pattern_np()
        _, ref, _, absref = O.assemble(mesh.elem_type, mesh.coords, mesh.conn, rp, ci, f, terms=TERMS, with_abs=True)
        b1, b0 = r1.cpu().numpy().astype(np.float64), r0.cpu().numpy().astype(np.float64)
        err1 = np.abs(b1[0] - ref[0]) / absref[0]
        assert err1[plane].max() <= 1e-12, err1[plane].max()  # FP64 sums (the output rounding of ~0 is ~0)
        # the plain relative error of the recomputed rows, where the exact sum is not zero: FP64
        # sums rounded once to FP32
        flagged_eq1 = plane & (np.abs(ref[1]) > 0)
        plain = np.abs(b1[1] - ref[1])[flagged_eq1] / np.abs(ref[1])[flagged_eq1]
        assert plain.max(initial=0.0) <= 1e-6, plain.max()
        # rows not recomputed are bit for bit the FP32 result (deterministic scatters)
        if scatter != fea.FEA_SCATTER_ATOMIC and count == plane.sum():
            row_of = np.repeat(np.arange(mesh.n_node), np.diff(rp))
            keep = ~plane[row_of]
            assert np.array_equal(v1.cpu().numpy()[:, keep], v0.cpu().numpy()[:, keep])
            assert np.array_equal(b1[:, ~plane], b0[:, ~plane])
        ea, eb = compare_full(run, f, fea.FEA_F32_FUSED, terms=TERMS, values=v1, rhs=r1)
        assert ea <= TOL_F32 and eb <= TOL_F32
    finally:
        run.close()


def test_cancel_check_in_a_step_graph():
    """Flags follow the field: phi_old = x - 1/2 cancels on the plane x = 1/2; the first step's
    update adds the constant -1/6 (amplitude 1/6, wave vector 0, phase -pi/2), so the second
    step's field x - 2/3 cancels on the node plane x = 2/3 instead.  The graph's outputs are
    that second assembly: its x = 2/3 rows must have been flagged and recomputed in FP64 (stale
    flags from the first step would leave them FP32 sums with ~1e-7 error relative to their
    contributions), and the graph must equal the same steps issued one by one."""
    import torch
    n = 6
    mesh, f = contrived(n)
    f32 = f.astype(np.float32)
    run = GpuRun(mesh)
    try:
        q = 2
        prm = np.zeros((2, q, 5), np.float32)
        prm[0, 0] = (1.0 / 6.0, 0.0, 0.0, 0.0, -np.pi / 2)
        d_prm = torch.from_numpy(prm).cuda()
        vel, kd, sr = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f32.velocity, f32.diffusivity,
                                                                                   f32.reaction))
        opts = fea.fea_default_opts(scatter=fea.FEA_SCATTER_ROWOWNED, terms=TERMS, cancel_check=1)
        # eager: assemble, update, assemble, update
        phi_e = torch.from_numpy(np.ascontiguousarray(f32.phi_old)).cuda()
        ve = torch.empty((q, run.nnz), device="cuda")
        re = torch.empty((q, mesh.n_node), device="cuda")
        for s_ in range(2):
            fea.fea_assemble(run.handle, run.pattern, vel, kd, sr, phi_e, f32.dt, q, opts, ve, re)
            fea.fea_update_fields(run.handle, phi_e, q, d_prm[s_])
        fea.fea_sync(run.handle)
        # graph of the same two steps from the same start
        phi_g = torch.from_numpy(np.ascontiguousarray(f32.phi_old)).cuda()
        vg = torch.full((q, run.nnz), float("nan"), device="cuda")
        rg = torch.full((q, mesh.n_node), float("nan"), device="cuda")
        g = fea.fea_graph_capture_steps(run.handle, run.pattern, vel, kd, sr, phi_g, f32.dt, q, opts, vg, rg,
                                        d_prm, 2)
        try:
            phi_g.copy_(torch.from_numpy(np.ascontiguousarray(f32.phi_old)))  # the capture ran one eager call
            torch.cuda.synchronize()
            fea.fea_graph_launch(g)
            fea.fea_sync(run.handle)
        finally:
            fea.fea_graph_destroy(g)
        assert np.array_equal(vg.cpu().numpy(), ve.cpu().numpy())
        assert np.array_equal(rg.cpu().numpy(), re.cpu().numpy())
        assert np.array_equal(phi_g.cpu().numpy(), phi_e.cpu().numpy())
        plane = np.isclose(mesh.coords[:, 0], 2.0 / 3.0)
        assert plane.sum() == (n + 1) ** 2
        assert fea.fea_cancel_rows(run.pattern, q) >= plane.sum()
        # the oracle on the field the second assembly consumed (the second update had amplitude 0)
        wide = G.Fields(f.velocity, f.diffusivity, f.reaction, phi_g.cpu().numpy().astype(np.float64), f.dt)
        rp, ci, _ = run.pattern_np()
        _, ref, _, absref = O.assemble(mesh.elem_type, mesh.coords, mesh.conn, rp, ci, wide, terms=TERMS,
                                       with_abs=True)
        err = np.abs(rg.cpu().numpy()[0].astype(np.float64) - ref[0]) / absref[0]
        assert err[plane].max() <= 1e-12, err[plane].max()
        ea, eb = compare_full(run, wide, fea.FEA_F32_FUSED, terms=TERMS, values=vg, rhs=rg)
        assert ea <= TOL_F32 and eb <= TOL_F32
    finally:
        run.close()


def test_cancel_check_arguments():
    mesh, f = contrived(3)
    run = GpuRun(mesh)
    try:
        for kw in (dict(cancel_check=1, accumulate=1), dict(cancel_check=2)):
            with pytest.raises(fea.FeaError) as e:
                run.assemble(f, fea.FEA_F32_FUSED, **kw)
            assert e.value.code == 1
    finally:
        run.close()
