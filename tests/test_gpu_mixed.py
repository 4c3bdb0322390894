"""Prisms (Pen6), pyramids (Pyr5) and meshes that mix element types (Hex8, Pyr5, Pen6 blocks
sharing one node set), through the C ABI, against the FP64 oracle: pattern and position map
bit-exact; values and RHS within 1e-12 (FP64) or 1e-5 (FP32) per row; the matrix-free
residual, the host entry point and the batched SpMV on the mixed mesh; the scatters a mixed
mesh does not offer are refused."""
import numpy as np
import pytest

import oracle as O
from helpers import TOL_F32, TOL_F64, GpuRun, compare_full, row_errors, rhs_errors, widen
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu


def fields_for(coords, q, seed):
    rng = np.random.default_rng(seed)
    return G.draw_fields(rng, coords, q, 50.0)


# ------------------------------------------------------------------ single-type prism and pyramid meshes

@pytest.fixture(scope="module", params=[(G.PEN6, 5, 3), (G.PYR5, 4, 2)], ids=["pen6", "pyr5"])
def single(request):
    t, n, q = request.param
    mesh = G.structured_mesh(t, n)
    G.perturb_interior(mesh, np.random.default_rng(2), 0.15)
    run = GpuRun(mesh)
    yield mesh, fields_for(mesh.coords, q, 3), run
    run.close()


def test_single_type_pattern_bit_exact(single):
    mesh, _, run = single
    rp, ci, pos = run.pattern_np()
    orp, oci, opos = O.pattern(mesh.elem_type, mesh.conn, mesh.n_node)
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci) and np.array_equal(pos, opos)


@pytest.mark.parametrize("prec,scatter", [(fea.FEA_F64_PLAIN, fea.FEA_SCATTER_AUTO),
                                          (fea.FEA_F32_FUSED, fea.FEA_SCATTER_AUTO),
                                          (fea.FEA_F32_FUSED, fea.FEA_SCATTER_ATOMIC),
                                          (fea.FEA_F32_FUSED, fea.FEA_SCATTER_GATHER)],
                         ids=["f64", "f32_auto", "f32_atomic", "f32_gather"])
def test_single_type_parity(single, prec, scatter):
    mesh, f, run = single
    v, r = run.assemble(f, prec, scatter=scatter)
    ea, eb = compare_full(run, f, prec, values=v, rhs=r)
    tol = TOL_F64 if prec == fea.FEA_F64_PLAIN else TOL_F32
    assert ea <= tol and eb <= tol, (ea, eb)


# ------------------------------------------------------------------ mixed meshes

class MixedRun:
    def __init__(self, mm: G.MixedMesh):
        import torch
        self.torch = torch
        self.mm = mm
        self.handle = fea.fea_mesh_create_mixed(mm.coords, mm.blocks)
        self.pattern = fea.fea_pattern_build(self.handle)
        self.nnz = fea.fea_pattern_get(self.pattern)[3]

    def pattern_np(self):
        torch = self.torch
        r, c, p, nnz = fea.fea_pattern_get(self.pattern)
        npos = sum(conn.shape[0] * G.NEN[t] ** 2 for t, conn in self.mm.blocks)
        rowptr = torch.as_tensor(fea._DevView(r, (self.mm.n_node + 1,), "<i8"), device="cuda").cpu().numpy()
        colind = torch.as_tensor(fea._DevView(c, (nnz,), "<i4"), device="cuda").cpu().numpy()
        pos = torch.as_tensor(fea._DevView(p, (npos,), "<i4"), device="cuda").cpu().numpy()
        return rowptr, colind, pos

    def upload(self, f, prec):
        torch = self.torch
        dt = np.float64 if prec == fea.FEA_F64_PLAIN else np.float32
        return [torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
                for a in (f.velocity, f.diffusivity, f.reaction, f.phi_old)]

    def assemble(self, f, prec, scatter=fea.FEA_SCATTER_AUTO):
        torch = self.torch
        dt = torch.float64 if prec == fea.FEA_F64_PLAIN else torch.float32
        q = f.n_eq
        vals = torch.full((q, self.nnz), float("nan"), dtype=dt, device="cuda")
        rhs = torch.full((q, self.mm.n_node), float("nan"), dtype=dt, device="cuda")
        opts = fea.fea_default_opts(precision=prec, scatter=scatter)
        fea.fea_assemble(self.handle, self.pattern, *self.upload(f, prec), f.dt, q, opts, vals, rhs)
        fea.fea_sync(self.handle)
        return vals.cpu().numpy().astype(np.float64), rhs.cpu().numpy().astype(np.float64)

    def close(self):
        fea.fea_pattern_destroy(self.pattern)
        fea.fea_mesh_destroy(self.handle)


@pytest.fixture(scope="module")
def mixed():
    mm = G.mixed_mesh(6)
    G.perturb_interior(mm, np.random.default_rng(6), 0.1)
    run = MixedRun(mm)
    yield mm, fields_for(mm.coords, 3, 7), run
    run.close()


def test_mixed_pattern_bit_exact(mixed):
    mm, _, run = mixed
    rp, ci, pos = run.pattern_np()
    orp, oci, opos = O.pattern_mixed(mm.blocks, mm.n_node)
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci)
    assert np.array_equal(pos, np.concatenate([p.ravel() for p in opos]))


@pytest.mark.parametrize("prec", [fea.FEA_F64_PLAIN, fea.FEA_F32_FUSED], ids=["f64", "f32"])
def test_mixed_parity(mixed, prec):
    mm, f, run = mixed
    v, r = run.assemble(f, prec)
    rp, ci, _ = O.pattern_mixed(mm.blocks, mm.n_node, with_pos=False)
    ref, refb, _, absb = O.assemble_mixed(mm.coords, mm.blocks, rp, ci, widen(f, prec), with_abs=True)
    tol = TOL_F64 if prec == fea.FEA_F64_PLAIN else TOL_F32
    ea, eb = row_errors(rp, v, ref).max(), rhs_errors(r, refb, absb).max()
    assert ea <= tol and eb <= tol, (ea, eb)


def test_mixed_refuses_rowowned_gather_and_cancel_check(mixed):
    mm, f, run = mixed
    for kw in (dict(scatter=fea.FEA_SCATTER_ROWOWNED), dict(scatter=fea.FEA_SCATTER_GATHER), dict(cancel_check=1)):
        torch = run.torch
        vals = torch.empty((f.n_eq, run.nnz), device="cuda")
        rhs = torch.empty((f.n_eq, mm.n_node), device="cuda")
        with pytest.raises(fea.FeaError) as ei:
            fea.fea_assemble(run.handle, run.pattern, *run.upload(f, fea.FEA_F32_FUSED), f.dt, f.n_eq,
                             fea.fea_default_opts(**kw), vals, rhs)
        assert ei.value.name == "FEA_ERR_ARG"


@pytest.mark.parametrize("prec", [fea.FEA_F64_PLAIN, fea.FEA_F32_FUSED], ids=["f64", "f32"])
def test_mixed_residual(mixed, prec):
    mm, f, run = mixed
    torch = run.torch
    q = f.n_eq
    phi = np.random.default_rng(9).uniform(0, 1, (q, mm.n_node))
    wide = widen(f, prec)
    ph = phi if prec == fea.FEA_F64_PLAIN else phi.astype(np.float32).astype(np.float64)
    rp, ci, _ = O.pattern_mixed(mm.blocks, mm.n_node, with_pos=False)
    _, b, absA, absb = O.assemble_mixed(mm.coords, mm.blocks, rp, ci, wide, with_abs=True)
    rows = np.repeat(np.arange(mm.n_node), np.diff(rp))
    dt = torch.float64 if prec == fea.FEA_F64_PLAIN else torch.float32
    r = torch.full((q, mm.n_node), float("nan"), dtype=dt, device="cuda")
    fea.fea_residual(run.handle, run.pattern, *run.upload(f, prec), torch.from_numpy(ph).to(dt).cuda(), f.dt, q,
                     fea.fea_default_opts(precision=prec), r)
    fea.fea_sync(run.handle)
    got = r.cpu().numpy().astype(np.float64)
    tol = TOL_F64 if prec == fea.FEA_F64_PLAIN else TOL_F32
    for k in range(q):
        ref = b[k] - O.apply_mixed(mm.coords, mm.blocks, wide, k, ph[k])
        scale = absb[k] + np.bincount(rows, weights=absA[k] * np.abs(ph[k][ci]), minlength=mm.n_node)
        assert (np.abs(got[k] - ref) / np.where(scale > 0, scale, 1.0)).max() <= tol


def test_mixed_host_entry_point_and_spmv(mixed):
    mm, f, run = mixed
    q = f.n_eq
    v, r = run.assemble(f, fea.FEA_F32_FUSED)
    f32 = f.astype(np.float32)
    hv = np.full((q, run.nnz), np.nan, dtype=np.float32)
    hr = np.full((q, mm.n_node), np.nan, dtype=np.float32)
    fea.fea_assemble_host(run.handle, run.pattern, f32.velocity, f32.diffusivity, f32.reaction, f32.phi_old, f.dt, q,
                          fea.fea_default_opts(), hv, hr)
    rp, ci, _ = run.pattern_np()
    assert row_errors(rp, hv, v).max() <= TOL_F32
    assert np.abs(hr - r).max() <= TOL_F32 * np.abs(r).max()
    torch = run.torch
    x = np.random.default_rng(4).standard_normal((q, mm.n_node)).astype(np.float32)
    y = torch.full((q, mm.n_node), float("nan"), device="cuda")
    vals = torch.from_numpy(v.astype(np.float32)).cuda()
    fea.fea_spmv(run.pattern, vals, torch.from_numpy(x).cuda(), y, q)
    torch.cuda.synchronize()
    ref = np.stack([np.add.reduceat(v[k] * x[k][ci].astype(np.float64), rp[:-1]) for k in range(q)])
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def test_mixed_create_edge_cases():
    """An empty block changes nothing; one block is a single-type mesh; an unknown type, an
    out-of-range node id and an inverted pyramid are refused with their codes."""
    mm = G.mixed_mesh(3)
    run = MixedRun(G.MixedMesh(mm.coords, mm.blocks + [(G.PEN6, np.zeros((0, 6), np.int32))], 3, mm.h))
    rp, ci, pos = run.pattern_np()
    orp, oci, opos = O.pattern_mixed(mm.blocks, mm.n_node)
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci)
    assert np.array_equal(pos, np.concatenate([q.ravel() for q in opos]))
    run.close()
    t, conn = mm.blocks[1]  # the pyramids alone, as one block
    h1 = fea.fea_mesh_create_mixed(mm.coords, [(t, conn)])
    p1 = fea.fea_pattern_build(h1)
    r1, c1, _ = fea.pattern_tensors(p1, mm.n_node, conn.shape[0], G.NEN[t])
    orp, oci, _ = O.pattern(t, conn, mm.n_node, with_pos=False)
    assert np.array_equal(r1.cpu().numpy(), orp) and np.array_equal(c1.cpu().numpy(), oci)
    fea.fea_pattern_destroy(p1)
    fea.fea_mesh_destroy(h1)
    bad = [(7, mm.blocks[0][1])] + mm.blocks[1:]
    with pytest.raises(fea.FeaError) as ei:
        fea.fea_mesh_create_mixed(mm.coords, bad)
    assert ei.value.name == "FEA_ERR_ARG"
    c = mm.blocks[2][1].copy()
    c[0, 0] = mm.n_node
    with pytest.raises(fea.FeaError) as ei:
        fea.fea_mesh_create_mixed(mm.coords, mm.blocks[:2] + [(G.PEN6, c)])
    assert ei.value.name == "FEA_ERR_RANGE"
    c = mm.blocks[1][1].copy()
    c[0, [1, 3]] = c[0, [3, 1]]  # base traversed the other way round: the apex is below it
    with pytest.raises(fea.FeaError) as ei:
        fea.fea_mesh_create_mixed(mm.coords, [mm.blocks[0], (G.PYR5, c), mm.blocks[2]])
    assert ei.value.name == "FEA_ERR_INVERTED"


@pytest.mark.parametrize("terms,accumulate", [(fea.FEA_TERM_ALL, 0), (fea.FEA_TERM_MASS | fea.FEA_TERM_DIFF, 1),
                                              (fea.FEA_TERM_CONV | fea.FEA_TERM_SUPG | fea.FEA_TERM_REAC, 0)],
                         ids=["all", "mass_diff_accumulate", "conv_supg_reac"])
def test_mixed_hex_block_many_equations(terms, accumulate):
    """The Hex8 block of a mixed mesh goes through the batched Hex8 kernel: 13 equations (a
    batch of 39 elements, so the block's 98 end in a batch of 20), a subset of the terms, and the
    accumulate flag (two calls add up to twice the operator); then the residual of the same
    system."""
    mm = G.mixed_mesh(7)
    G.perturb_interior(mm, np.random.default_rng(12), 0.1)
    f = fields_for(mm.coords, 13, 13)
    run = MixedRun(mm)
    torch = run.torch
    try:
        q = f.n_eq
        args = run.upload(f, fea.FEA_F32_FUSED)
        vals = torch.zeros((q, run.nnz), device="cuda")
        rhs = torch.zeros((q, mm.n_node), device="cuda")
        opts = fea.fea_default_opts(terms=terms, accumulate=accumulate)
        for _ in range(2 if accumulate else 1):
            fea.fea_assemble(run.handle, run.pattern, *args, f.dt, q, opts, vals, rhs)
        fea.fea_sync(run.handle)
        scale = 2.0 if accumulate else 1.0
        v = vals.cpu().numpy().astype(np.float64) / scale
        r = rhs.cpu().numpy().astype(np.float64) / scale
        rp, ci, _ = O.pattern_mixed(mm.blocks, mm.n_node, with_pos=False)
        wide = widen(f, fea.FEA_F32_FUSED)
        ref, refb, _, absb = O.assemble_mixed(mm.coords, mm.blocks, rp, ci, wide, terms=terms, with_abs=True)
        ea, eb = row_errors(rp, v, ref).max(), rhs_errors(r, refb, absb).max()
        assert ea <= TOL_F32 and eb <= TOL_F32, (ea, eb)
        if terms != fea.FEA_TERM_ALL:
            return
        phi = np.random.default_rng(14).uniform(0, 1, (q, mm.n_node)).astype(np.float32)
        res = torch.full((q, mm.n_node), float("nan"), device="cuda")
        fea.fea_residual(run.handle, run.pattern, *args, torch.from_numpy(phi).cuda(), f.dt, q,
                         fea.fea_default_opts(), res)
        fea.fea_sync(run.handle)
        got = res.cpu().numpy().astype(np.float64)
        _, b, absA, absb = O.assemble_mixed(mm.coords, mm.blocks, rp, ci, wide, with_abs=True)
        rows = np.repeat(np.arange(mm.n_node), np.diff(rp))
        ph = phi.astype(np.float64)
        for k in range(q):
            ref_r = b[k] - O.apply_mixed(mm.coords, mm.blocks, wide, k, ph[k])
            sc = absb[k] + np.bincount(rows, weights=absA[k] * np.abs(ph[k][ci]), minlength=mm.n_node)
            assert (np.abs(got[k] - ref_r) / np.where(sc > 0, sc, 1.0)).max() <= TOL_F32
    finally:
        run.close()
