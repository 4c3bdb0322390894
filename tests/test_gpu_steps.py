"""Time steps on the GPU: the field update and the multi-step CUDA graph, through the C ABI.

A step is "assemble, then update phi_old by the seeded smooth perturbation".  The update is
checked against the oracle's; a graph of steps must give the same bits as the same steps
issued one by one (row-owned and gather scatters are deterministic), and its last assembly
must match the oracle assembled from the oracle's own field after the earlier updates."""
import numpy as np
import pytest

import oracle as O
from helpers import TOL_F32, GpuRun, compare_full
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu


def to_dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_update_fields_matches_oracle():
    import torch
    w = G.make_workload(2, n=9, n_eq=5)
    run = GpuRun(w.mesh)
    try:
        prm = G.step_params(1, 5)[0]
        phi = w.fields.phi_old.astype(np.float32)
        d_phi = to_dev(phi, torch)
        fea.fea_update_fields(run.handle, d_phi, 5, to_dev(prm, torch))
        fea.fea_sync(run.handle)
        want = O.update_fields(w.mesh.coords, phi.astype(np.float64), prm.astype(np.float64))
        got = d_phi.cpu().numpy().astype(np.float64)
        assert np.abs(got - want).max() <= 1e-6
        assert np.abs(got - phi).max() > 1e-3  # it did move
    finally:
        run.close()


@pytest.mark.parametrize("cfg,n,q,scatter", [(2, 6, 4, fea.FEA_SCATTER_ROWOWNED), (1, 5, 2, fea.FEA_SCATTER_GATHER),
                                             (3, 2, 2, fea.FEA_SCATTER_GATHER)],
                         ids=["hex8_rowowned", "tet4_gather", "hex27_gather"])
def test_graph_equals_eager_steps_and_oracle(cfg, n, q, scatter):
    import torch
    steps = 3
    w = G.make_workload(cfg, n=n, n_eq=q)
    f32 = w.fields.astype(np.float32)
    run = GpuRun(w.mesh)
    try:
        prm = G.step_params(steps, q)
        d_prm = to_dev(prm, torch)
        vel, kd, sr = (to_dev(a, torch) for a in (f32.velocity, f32.diffusivity, f32.reaction))
        opts = fea.fea_default_opts(scatter=scatter)

        # eager: assemble, update, three times
        phi_e = to_dev(f32.phi_old, torch)
        val_e = torch.empty((q, run.nnz), device="cuda")
        rhs_e = torch.empty((q, w.mesh.n_node), device="cuda")
        for s in range(steps):
            fea.fea_assemble(run.handle, run.pattern, vel, kd, sr, phi_e, f32.dt, q, opts, val_e, rhs_e)
            fea.fea_update_fields(run.handle, phi_e, q, d_prm[s])
        fea.fea_sync(run.handle)

        # graph of the same steps
        phi_g = to_dev(f32.phi_old, torch)
        val_g = torch.full((q, run.nnz), float("nan"), device="cuda")
        rhs_g = torch.full((q, w.mesh.n_node), float("nan"), device="cuda")
        launches = fea.fea_kernel_launches()
        g = fea.fea_graph_capture_steps(run.handle, run.pattern, vel, kd, sr, phi_g, f32.dt, q, opts, val_g, rhs_g,
                                        d_prm, steps)
        try:
            before = fea.fea_kernel_launches()
            fea.fea_graph_launch(g)
            fea.fea_sync(run.handle)
            assert fea.fea_kernel_launches() - before >= 2 * steps
            assert before - launches >= 1  # the eager warm-up assembly
        finally:
            fea.fea_graph_destroy(g)
        assert np.array_equal(phi_g.cpu().numpy(), phi_e.cpu().numpy())
        assert np.array_equal(val_g.cpu().numpy(), val_e.cpu().numpy())
        assert np.array_equal(rhs_g.cpu().numpy(), rhs_e.cpu().numpy())

        # oracle: the field after each update in FP64; the last assembly used the field after steps-1 updates
        phi = f32.phi_old.astype(np.float64)
        hist = [phi]
        for s in range(steps):
            phi = O.update_fields(w.mesh.coords, phi, prm[s].astype(np.float64))
            hist.append(phi)
        assert np.abs(phi_g.cpu().numpy() - hist[steps]).max() <= 1e-6
        used = G.Fields(f32.velocity.astype(np.float64), f32.diffusivity.astype(np.float64),
                        f32.reaction.astype(np.float64), hist[steps - 1], f32.dt)
        ea, eb = compare_full(run, used, fea.FEA_F32_FUSED, values=val_g, rhs=rhs_g)
        assert ea <= TOL_F32 and eb <= TOL_F32, (ea, eb)
    finally:
        run.close()


def test_graph_bad_arguments():
    import torch
    w = G.make_workload(2, n=3, n_eq=1)
    f32 = w.fields.astype(np.float32)
    run = GpuRun(w.mesh)
    try:
        d = [to_dev(a, torch) for a in (f32.velocity, f32.diffusivity, f32.reaction, f32.phi_old)]
        val = torch.empty((1, run.nnz), device="cuda")
        rhs = torch.empty((1, w.mesh.n_node), device="cuda")
        prm = to_dev(G.step_params(2, 1), torch)
        for opts, steps in ((fea.fea_default_opts(), 0), (fea.fea_default_opts(accumulate=1), 2),
                            (fea.fea_default_opts(precision=fea.FEA_F64_PLAIN), 2)):
            with pytest.raises(fea.FeaError) as e:
                fea.fea_graph_capture_steps(run.handle, run.pattern, *d, f32.dt, 1, opts, val, rhs, prm, steps)
            assert e.value.code == 1
        with pytest.raises(fea.FeaError) as e:
            fea.fea_update_fields(run.handle, d[3], 0, prm)
        assert e.value.code == 1
    finally:
        run.close()
