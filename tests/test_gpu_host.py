"""The host-array entry point (fea_assemble_host) in its split form: the equations are
assembled in parts, each part's values copied back to the host while the next part computes.

Forced splits (opts.host_parts) on a small mesh are checked whole against the oracle; the
automatic split (values above 256 MB: three parts) on Hex8 64^3 x 21 equations, 622 MB of
values, is checked on sampled rows the oracle computes from their incident elements."""
import numpy as np
import pytest

import oracle as O
from helpers import TOL_F32, GpuRun, compare_full
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("parts", [1, 3, 7])
def test_forced_parts_match_oracle(parts):
    import torch
    w = G.make_workload(2, n=6, n_eq=7)
    run = GpuRun(w.mesh)
    try:
        q = 7
        f = w.fields.astype(np.float32)
        vals = np.full((q, run.nnz), np.nan, np.float32)
        rhs = np.full((q, w.mesh.n_node), np.nan, np.float32)
        fea.fea_assemble_host(run.handle, run.pattern, f.velocity, f.diffusivity, f.reaction, f.phi_old, f.dt, q,
                              fea.fea_default_opts(host_parts=parts), vals, rhs)
        ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=torch.from_numpy(vals),
                              rhs=torch.from_numpy(rhs))
        assert ea <= TOL_F32 and eb <= TOL_F32, (parts, ea, eb)
    finally:
        run.close()


def test_host_parts_argument():
    w = G.make_workload(2, n=3, n_eq=2)
    run = GpuRun(w.mesh)
    try:
        f = w.fields.astype(np.float32)
        vals = np.zeros((2, run.nnz), np.float32)
        rhs = np.zeros((2, w.mesh.n_node), np.float32)
        with pytest.raises(fea.FeaError) as e:
            fea.fea_assemble_host(run.handle, run.pattern, f.velocity, f.diffusivity, f.reaction, f.phi_old, f.dt,
                                  2, fea.fea_default_opts(host_parts=-1), vals, rhs)
        assert e.value.code == 1
    finally:
        run.close()


@pytest.mark.slow
def test_automatic_three_parts_sampled_rows():
    import torch
    w = G.make_workload(2, n=64)
    m = w.mesh
    f32 = w.fields.astype(np.float32)
    q = f32.n_eq
    run = GpuRun(m)
    try:
        assert 4 * q * run.nnz > 256 << 20  # the automatic split applies
        pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
               for a in (f32.velocity, f32.diffusivity, f32.reaction, f32.phi_old)]
        hv = torch.full((q, run.nnz), float("nan")).pin_memory()
        hr = torch.full((q, m.n_node), float("nan")).pin_memory()
        fea.fea_assemble_host(run.handle, run.pattern, *pin, f32.dt, q, fea.fea_default_opts(), hv, hr)
        rp, ci, _ = run.pattern_np()
        rs = O.RowSampler(m.elem_type, m.coords, m.conn, f32.astype(np.float64))
        rng = np.random.default_rng(64)
        rows = np.unique(np.concatenate([[0, m.n_node - 1], rng.integers(0, m.n_node, 40)]))
        values, rhs = hv.numpy(), hr.numpy()
        for r in rows:
            cols, ref, _, refb, absb = rs.row(int(r))
            k0, k1 = rp[r], rp[r + 1]
            assert np.array_equal(ci[k0:k1], cols)
            got = values[:, k0:k1].astype(np.float64)
            ea = np.sqrt(((got - ref) ** 2).sum(axis=1) / (ref ** 2).sum(axis=1)).max()
            eb = (np.abs(rhs[:, r] - refb) / np.where(absb > 0, absb, 1.0)).max()
            assert ea <= TOL_F32 and eb <= TOL_F32, (r, ea, eb)
    finally:
        run.close()
