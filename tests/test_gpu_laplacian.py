"""The Laplacian (the diffusion term alone with k = 1, assembled once per run in Algorithm 1),
through the C ABI, FP64 and FP32, on every element type and on a mixed mesh:
- values within tolerance of the oracle and a zero RHS;
- zero row sums (K 1 = 0);
- symmetry;
- the interior patch test: K phi = 0 at interior nodes for a linear phi, on meshes whose
  quadrature integrates the Laplacian exactly (perturbed Tet4, Hex8 and Pen6; affine Hex27
  and Pyr5)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from helpers import TOL_F32, TOL_F64, GpuRun, compare_full
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu

PRECS = [fea.FEA_F64_PLAIN, fea.FEA_F32_FUSED]
MESHES = [(G.TET4, 4, 0.2), (G.HEX8, 4, 0.15), (G.HEX27, 2, 0.0), (G.PEN6, 4, 0.15), (G.PYR5, 3, 0.0)]
GRAD = np.array([0.7, -0.4, 1.3])


def laplacian_fields(n_node):
    z = np.zeros((1, n_node))
    return G.Fields(np.zeros((3, n_node)), np.ones((1, n_node)), z, z.copy(), 1.0)


def check_operator(rp, ci, v, coords, interior, tol):
    """K 1 = 0, K = K^T and the interior patch test, each relative to the absolute row sums."""
    n = rp.size - 1
    K = sp.csr_matrix((v, ci, rp), shape=(n, n))
    absK = abs(K)
    row_abs = np.asarray(absK.sum(axis=1)).ravel()
    assert (np.abs(K @ np.ones(n)) <= tol * row_abs).all()
    asym = abs(K - K.T).max()
    assert asym <= tol * row_abs.max(), asym
    phi = coords @ GRAD + 0.25
    y = K @ phi
    scale = absK @ np.abs(phi)
    assert (np.abs(y[interior]) <= tol * scale[interior]).all(), np.abs(y[interior] / scale[interior]).max()


@pytest.mark.parametrize("prec", PRECS, ids=["f64", "f32"])
@pytest.mark.parametrize("t,n,frac", MESHES, ids=["tet4", "hex8", "hex27", "pen6", "pyr5"])
def test_laplacian(t, n, frac, prec):
    mesh = G.structured_mesh(t, n)
    if frac > 0:
        G.perturb_interior(mesh, np.random.default_rng(5), frac)
    run = GpuRun(mesh)
    try:
        f = laplacian_fields(mesh.n_node)
        v, r = run.assemble(f, prec, terms=fea.FEA_TERM_DIFF)
        tol = TOL_F64 if prec == fea.FEA_F64_PLAIN else TOL_F32
        ea, eb = compare_full(run, f, prec, terms=fea.FEA_TERM_DIFF, values=v, rhs=r)
        assert ea <= tol and eb <= tol, (ea, eb)
        assert float(r.abs().max()) == 0.0
        rp, ci, _ = run.pattern_np()
        check_operator(rp, ci, v[0, :run.nnz].cpu().numpy().astype(np.float64), mesh.coords,
                       G.interior_mask(mesh), tol)
    finally:
        run.close()


@pytest.mark.parametrize("prec", PRECS, ids=["f64", "f32"])
def test_laplacian_mixed_mesh(prec):
    import torch
    mm = G.mixed_mesh(6)  # affine cells: the pyramids' rational functions are integrated exactly
    h = fea.fea_mesh_create_mixed(mm.coords, mm.blocks)
    p = fea.fea_pattern_build(h)
    try:
        nnz = fea.fea_pattern_get(p)[3]
        dt = torch.float64 if prec == fea.FEA_F64_PLAIN else torch.float32
        np_dt = np.float64 if prec == fea.FEA_F64_PLAIN else np.float32
        f = laplacian_fields(mm.n_node)
        args = [torch.from_numpy(np.ascontiguousarray(a, dtype=np_dt)).cuda()
                for a in (f.velocity, f.diffusivity, f.reaction, f.phi_old)]
        vals = torch.full((1, nnz), float("nan"), dtype=dt, device="cuda")
        rhs = torch.full((1, mm.n_node), float("nan"), dtype=dt, device="cuda")
        fea.fea_assemble(h, p, *args, f.dt, 1, fea.fea_default_opts(precision=prec, terms=fea.FEA_TERM_DIFF),
                         vals, rhs)
        fea.fea_sync(h)
        v = vals.cpu().numpy().astype(np.float64)[0]
        assert float(rhs.abs().max()) == 0.0
        rp, ci, _ = O.pattern_mixed(mm.blocks, mm.n_node, with_pos=False)
        ref, _ = O.assemble_mixed(mm.coords, mm.blocks, rp, ci, f, O.DIFF)
        tol = TOL_F64 if prec == fea.FEA_F64_PLAIN else TOL_F32
        rows = np.repeat(np.arange(mm.n_node), np.diff(rp))
        err = np.sqrt(np.bincount(rows, (v - ref[0]) ** 2, mm.n_node) / np.bincount(rows, ref[0] ** 2, mm.n_node))
        assert err.max() <= tol, err.max()
        interior = np.all((mm.coords > 0.0) & (mm.coords < 1.0), axis=1)
        check_operator(rp, ci, v, mm.coords, interior, tol)
    finally:
        fea.fea_pattern_destroy(p)
        fea.fea_mesh_destroy(h)
