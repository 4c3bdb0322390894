"""The matrix-free residual r = b - A phi (fea_residual), through the C ABI, against the oracle:
b from the oracle's assembly and A phi from its matrix-free element application, both FP64.
Errors are measured against the sizes of the contributions (sum_e |b^e_i| + sum |A_ij| |phi_j|),
because r itself may cancel to near zero."""
import numpy as np
import pytest

import oracle as O
from helpers import TOL_F32, TOL_F64, GpuRun
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu

CASES = [(0, 5, 1), (1, 4, 2), (2, 5, 3), (3, 2, 2)]
IDS = ["tet4", "tet4_perm", "hex8", "hex27"]


def oracle_residual(mesh, fields, phi, terms=O.ALL_TERMS):
    rp, ci, _ = O.pattern(mesh.elem_type, mesh.conn, mesh.n_node, with_pos=False)
    _, b, absA, absb = O.assemble(mesh.elem_type, mesh.coords, mesh.conn, rp, ci, fields, terms=terms, with_abs=True)
    q = fields.n_eq
    r = np.empty_like(b)
    scale = np.empty_like(b)
    rows = np.repeat(np.arange(mesh.n_node), np.diff(rp))
    for k in range(q):
        r[k] = b[k] - O.apply(mesh.elem_type, mesh.coords, mesh.conn, fields, k, phi[k], terms=terms)
        scale[k] = absb[k] + np.bincount(rows, weights=absA[k] * np.abs(phi[k][ci]), minlength=mesh.n_node)
    return r, scale


def gpu_residual(run, fields, phi, precision, terms=fea.FEA_TERM_ALL):
    import torch
    (vel, kd, sr, po), dt = run.upload(fields, precision)
    ph = torch.from_numpy(np.ascontiguousarray(phi)).to(dt).cuda()
    r = torch.full((fields.n_eq, run.mesh.n_node), float("nan"), dtype=dt, device="cuda")
    opts = fea.fea_default_opts(precision=precision, terms=terms)
    fea.fea_residual(run.handle, run.pattern, vel, kd, sr, po, ph, fields.dt, fields.n_eq, opts, r)
    fea.fea_sync(run.handle)
    return r.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_residual_matches_oracle(case):
    cfg, n, q = case
    w = G.make_workload(cfg, n=n, n_eq=q)
    rng = np.random.default_rng(21)
    phi = rng.uniform(0.0, 1.0, size=(q, w.mesh.n_node))
    run = GpuRun(w.mesh)
    try:
        for prec, tol in ((fea.FEA_F64_PLAIN, TOL_F64), (fea.FEA_F32_FUSED, TOL_F32)):
            f = w.fields if prec == fea.FEA_F64_PLAIN else w.fields.astype(np.float32).astype(np.float64)
            ph = phi if prec == fea.FEA_F64_PLAIN else phi.astype(np.float32).astype(np.float64)
            ref, scale = oracle_residual(w.mesh, f, ph)
            got = gpu_residual(run, f, ph, prec)
            err = (np.abs(got - ref) / np.where(scale > 0, scale, 1.0)).max()
            assert err <= tol, (prec, err)
    finally:
        run.close()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_residual_of_a_constant_state_vanishes(case):
    """With s = 0 and phi_old = phi = 1 the discrete operator preserves the constant state:
    A 1 = b, so the residual is zero (to rounding relative to the contributions)."""
    cfg, n, q = case
    w = G.make_workload(cfg, n=n, n_eq=q)
    f = w.fields
    f.reaction[:] = 0.0
    f.phi_old[:] = 1.0
    ones = np.ones((q, w.mesh.n_node))
    _, scale = oracle_residual(w.mesh, f, ones)
    run = GpuRun(w.mesh)
    try:
        for prec, tol in ((fea.FEA_F64_PLAIN, TOL_F64), (fea.FEA_F32_FUSED, TOL_F32)):
            got = gpu_residual(run, f, ones, prec)
            assert (np.abs(got) / np.where(scale > 0, scale, 1.0)).max() <= tol, prec
    finally:
        run.close()


def test_residual_equals_rhs_minus_assembled_matrix_times_phi():
    import torch
    w = G.make_workload(2, n=6, n_eq=3)
    f32 = w.fields.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(22)
    phi = rng.uniform(0.0, 1.0, size=(3, w.mesh.n_node)).astype(np.float32).astype(np.float64)
    run = GpuRun(w.mesh)
    try:
        v, b = run.assemble(f32, fea.FEA_F32_FUSED)
        rp, ci, _ = run.pattern_np()
        vv = v.double().cpu().numpy()
        rows = np.repeat(np.arange(w.mesh.n_node), np.diff(rp))
        ax = np.stack([np.bincount(rows, weights=vv[k] * phi[k][ci], minlength=w.mesh.n_node) for k in range(3)])
        want = b.double().cpu().numpy() - ax
        got = gpu_residual(run, f32, phi, fea.FEA_F32_FUSED)
        _, scale = oracle_residual(w.mesh, f32, phi)
        assert (np.abs(got - want) / scale).max() <= TOL_F32
        # accumulate adds
        import torch as _t
        (vel, kd, sr, po), dt = run.upload(f32, fea.FEA_F32_FUSED)
        r = _t.from_numpy(got.astype(np.float32)).cuda()
        ph = _t.from_numpy(phi.astype(np.float32)).cuda()
        fea.fea_residual(run.handle, run.pattern, vel, kd, sr, po, ph, f32.dt, 3, fea.fea_default_opts(accumulate=1), r)
        fea.fea_sync(run.handle)
        assert (np.abs(r.cpu().numpy() - 2 * got) / scale).max() <= 2 * TOL_F32
    finally:
        run.close()
