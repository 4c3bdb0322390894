"""CUDA path vs the FP64 oracle, through the C ABI, on seeded meshes small enough
for the oracle to assemble completely (several CTAs' worth of elements and a
ragged tail).  Pattern and position map must be bit-identical; values within
1e-12 (FP64 path) or 1e-5 (FP32 path) relative Frobenius norm per row."""
import numpy as np
import pytest

import oracle as O
from helpers import TOL_F32, TOL_F64, GpuRun, compare_full, widen
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu

# (name, config index, cells per axis, equations)
CASES = [
    ("tet4_10", 0, 10, 1),
    ("tet4_perm_9", 1, 9, 2),
    ("hex8_7", 2, 7, 3),
    ("hex27_3", 3, 3, 2),
]


def workload(idx, n, q):
    return G.make_workload(idx, n=n, n_eq=q)


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    name, idx, n, q = request.param
    w = workload(idx, n, q)
    run = GpuRun(w.mesh)
    yield w, run
    run.close()


def test_pattern_bit_exact(case):
    w, run = case
    m = w.mesh
    rp, ci, pos = run.pattern_np()
    orp, oci, opos = O.pattern(m.elem_type, m.conn, m.n_node)
    assert np.array_equal(rp, orp)
    assert np.array_equal(ci, oci)
    assert np.array_equal(pos, opos)


def test_f64_plain_parity(case):
    w, run = case
    v, r = run.assemble(w.fields, fea.FEA_F64_PLAIN)
    ea, eb = compare_full(run, w.fields, fea.FEA_F64_PLAIN, values=v, rhs=r)
    assert ea <= TOL_F64 and eb <= TOL_F64, (ea, eb)


@pytest.mark.parametrize("scatter", [fea.FEA_SCATTER_AUTO, fea.FEA_SCATTER_ATOMIC, fea.FEA_SCATTER_GATHER])
def test_f32_fused_parity(case, scatter):
    w, run = case
    v, r = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=scatter)
    ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=v, rhs=r)
    assert ea <= TOL_F32 and eb <= TOL_F32, (ea, eb)


@pytest.mark.parametrize("terms", [fea.FEA_TERM_MASS, fea.FEA_TERM_CONV, fea.FEA_TERM_DIFF, fea.FEA_TERM_REAC,
                                   fea.FEA_TERM_SUPG])
def test_single_terms(case, terms):
    w, run = case
    for prec, tol in ((fea.FEA_F64_PLAIN, TOL_F64), (fea.FEA_F32_FUSED, TOL_F32)):
        v, r = run.assemble(w.fields, prec, terms=terms)
        ea, eb = compare_full(run, w.fields, prec, terms=terms, values=v, rhs=r)
        assert ea <= tol, (prec, terms, ea)
        if terms in (fea.FEA_TERM_MASS, fea.FEA_TERM_SUPG):
            assert eb <= tol, (prec, terms, eb)


def test_accumulate_adds(case):
    w, run = case
    v1, r1 = run.assemble(w.fields, fea.FEA_F64_PLAIN)
    v2, r2 = run.assemble(w.fields, fea.FEA_F64_PLAIN, accumulate=1, out=(v1.clone(), r1.clone()))
    assert np.allclose(v2.cpu().numpy(), 2 * v1.cpu().numpy(), rtol=1e-13, atol=0)
    assert np.allclose(r2.cpu().numpy(), 2 * r1.cpu().numpy(), rtol=1e-13, atol=0)
    for scatter in (fea.FEA_SCATTER_AUTO, fea.FEA_SCATTER_ATOMIC, fea.FEA_SCATTER_GATHER):
        v1, r1 = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=scatter)
        v2, r2 = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=scatter, accumulate=1,
                              out=(v1.clone(), r1.clone()))
        scale = np.abs(v1.cpu().numpy()).max()
        assert np.abs(v2.cpu().numpy() - 2 * v1.cpu().numpy()).max() <= 1e-6 * scale
        assert np.abs(r2.cpu().numpy() - 2 * r1.cpu().numpy()).max() <= 1e-6 * np.abs(r1.cpu().numpy()).max()


def test_host_entry_point(case):
    w, run = case
    q = w.fields.n_eq
    f = w.fields.astype(np.float32)
    vals = np.zeros((q, run.nnz), np.float32)
    rhs = np.zeros((q, w.mesh.n_node), np.float32)
    opts = fea.fea_default_opts()
    fea.fea_assemble_host(run.handle, run.pattern, f.velocity, f.diffusivity, f.reaction, f.phi_old, f.dt, q, opts,
                          vals, rhs)
    import torch
    ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=torch.from_numpy(vals), rhs=torch.from_numpy(rhs))
    assert ea <= TOL_F32 and eb <= TOL_F32
    # accumulate through the host entry point: the outputs are copied in, added to and copied back
    v2, r2 = vals.copy(), rhs.copy()
    fea.fea_assemble_host(run.handle, run.pattern, f.velocity, f.diffusivity, f.reaction, f.phi_old, f.dt, q,
                          fea.fea_default_opts(accumulate=1), v2, r2)
    assert np.abs(v2 - 2 * vals).max() <= 1e-6 * np.abs(vals).max()
    assert np.abs(r2 - 2 * rhs).max() <= 1e-6 * np.abs(rhs).max()


def test_unused_nodes_and_subset():
    """Ragged mesh: a random subset of elements, so some nodes are in no element (empty rows)."""
    rng = np.random.default_rng(4)
    mesh = G.structured_mesh(G.HEX8, 5)
    G.perturb_interior(mesh, rng, 0.15)
    mesh.conn = mesh.conn[np.sort(rng.permutation(mesh.n_elem)[:37])]
    fields = G.draw_fields(rng, mesh.coords, 2, 50.0)
    run = GpuRun(mesh)
    try:
        rp, ci, pos = run.pattern_np()
        orp, oci, opos = O.pattern(mesh.elem_type, mesh.conn, mesh.n_node)
        assert np.array_equal(rp, orp) and np.array_equal(ci, oci) and np.array_equal(pos, opos)
        assert (np.diff(rp) == 0).any()
        for prec, tol, scatter in ((fea.FEA_F64_PLAIN, TOL_F64, fea.FEA_SCATTER_AUTO),
                                   (fea.FEA_F32_FUSED, TOL_F32, fea.FEA_SCATTER_AUTO),
                                   (fea.FEA_F32_FUSED, TOL_F32, fea.FEA_SCATTER_GATHER)):
            v, r = run.assemble(fields, prec, scatter=scatter)
            ea, eb = compare_full(run, fields, prec, values=v, rhs=r)
            assert ea <= tol and eb <= tol
    finally:
        run.close()


def test_empty_mesh():
    mesh = G.structured_mesh(G.TET4, 2)
    mesh.conn = mesh.conn[:0]
    run = GpuRun(mesh)
    try:
        assert run.nnz == 0
        f = G.draw_fields(np.random.default_rng(0), mesh.coords, 1, 1.0)
        v, r = run.assemble(f, fea.FEA_F32_FUSED)
        assert np.all(r.cpu().numpy() == 0.0)
    finally:
        run.close()


@pytest.mark.parametrize("bad,code", [("range", 2), ("dup", 3), ("inverted", 4)])
def test_bad_mesh_rejected(bad, code):
    mesh = G.structured_mesh(G.HEX8, 3)
    conn = mesh.conn.copy()
    if bad == "range":
        conn[5, 2] = mesh.n_node + 3
    elif bad == "dup":
        conn[5, 2] = conn[5, 3]
    else:
        conn[5, [0, 1]] = conn[5, [1, 0]]
    with pytest.raises(fea.FeaError) as e:
        fea.fea_mesh_create(mesh.coords, conn, G.HEX8)
    assert e.value.code == code


def test_bad_arguments(case):
    w, run = case
    import torch
    (vel, kd, sr, phi), _ = run.upload(w.fields, fea.FEA_F32_FUSED)
    vals = torch.zeros((1, max(run.nnz, 1)), device="cuda")
    rhs = torch.zeros((1, w.mesh.n_node), device="cuda")
    opts = fea.fea_default_opts()
    for args, code in (((0, 1e-3), 1), ((1, 0.0), 1), ((1, -1.0), 1)):
        with pytest.raises(fea.FeaError) as e:
            fea.fea_assemble(run.handle, run.pattern, vel, kd, sr, phi, args[1], args[0], opts, vals, rhs)
        assert e.value.code == code
    for bad in (dict(scatter=7), dict(scatter=fea.FEA_SCATTER_GATHER, precision=fea.FEA_F64_PLAIN)):
        with pytest.raises(fea.FeaError) as e:
            fea.fea_assemble(run.handle, run.pattern, vel, kd, sr, phi, 1e-3, 1, fea.fea_default_opts(**bad), vals,
                             rhs)
        assert e.value.code == 1, bad


@pytest.mark.parametrize("scatter", [fea.FEA_SCATTER_ROWOWNED, fea.FEA_SCATTER_GATHER])
def test_deterministic_scatter_is_bitwise_stable(case, scatter):
    """The deterministic scatters (row-owned where available, gather everywhere) give the
    same bits on every run."""
    w, run = case
    try:
        v1, r1 = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=scatter)
    except fea.FeaError:
        pytest.skip("row-owned scatter not available for this element type")
    v2, r2 = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=scatter)
    assert np.array_equal(v1.cpu().numpy(), v2.cpu().numpy())
    assert np.array_equal(r1.cpu().numpy(), r2.cpu().numpy())
    ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=v1, rhs=r1)
    assert ea <= TOL_F32 and eb <= TOL_F32
