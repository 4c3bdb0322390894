"""The batched CSR SpMV y_q = A_q x_q (fea_spmv) on assembled matrices, through the C ABI:
against a double-precision CSR product of the same matrices on the host, and the
matrix-free identity b - SpMV(A, phi) = fea_residual(phi) on the GPU."""
import numpy as np
import pytest

from helpers import GpuRun
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg,n,q", [(1, 5, 2), (2, 6, 5), (3, 2, 3)], ids=["tet4", "hex8", "hex27"])
def test_spmv_matches_host_csr_product(cfg, n, q):
    import torch
    w = G.make_workload(cfg, n=n, n_eq=q)
    f32 = w.fields.astype(np.float32).astype(np.float64)
    run = GpuRun(w.mesh)
    try:
        v, b = run.assemble(f32, fea.FEA_F32_FUSED)
        rng = np.random.default_rng(31)
        x = rng.uniform(-1.0, 1.0, size=(q, w.mesh.n_node)).astype(np.float32)
        dx = torch.from_numpy(x).cuda()
        y = torch.full((q, w.mesh.n_node), float("nan"), device="cuda")
        fea.fea_spmv(run.pattern, v, dx, y, q)
        torch.cuda.synchronize()
        rp, ci, _ = run.pattern_np()
        rows = np.repeat(np.arange(w.mesh.n_node), np.diff(rp))
        vv = v.double().cpu().numpy()
        for k in range(q):
            want = np.bincount(rows, weights=vv[k] * x[k].astype(np.float64)[ci], minlength=w.mesh.n_node)
            scale = np.bincount(rows, weights=np.abs(vv[k] * x[k].astype(np.float64)[ci]), minlength=w.mesh.n_node)
            got = y[k].double().cpu().numpy()
            assert (np.abs(got - want) / np.where(scale > 0, scale, 1.0)).max() <= 1e-6
        # accumulate adds
        y2 = y.clone()
        fea.fea_spmv(run.pattern, v, dx, y2, q, accumulate=1)
        torch.cuda.synchronize()
        assert torch.allclose(y2, 2 * y, rtol=1e-6, atol=1e-30)
        # matrix-free identity: b - A phi from the SpMV equals the residual kernel's
        (vel, kd, sr, po), _ = run.upload(f32, fea.FEA_F32_FUSED)
        r = torch.empty((q, w.mesh.n_node), device="cuda")
        fea.fea_residual(run.handle, run.pattern, vel, kd, sr, po, dx, f32.dt, q, fea.fea_default_opts(), r)
        fea.fea_sync(run.handle)
        ax = y.double()
        mag = (b.double().abs() + torch.from_numpy(np.stack([
            np.bincount(rows, weights=np.abs(vv[k] * x[k].astype(np.float64)[ci]), minlength=w.mesh.n_node)
            for k in range(q)])).cuda())
        err = ((r.double() - (b.double() - ax)).abs() / torch.where(mag > 0, mag, torch.ones_like(mag))).max()
        assert float(err) <= 1e-5
    finally:
        run.close()
