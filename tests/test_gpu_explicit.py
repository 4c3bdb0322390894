"""The explicit time step (fea_explicit_step) through the C ABI against the oracle's step.

Sec. 2 advances heat and species with a third-order Runge-Kutta scheme and no solver; the step
here solves M_L dphi/dt = -A phi (convection + diffusion + reaction applied element by element,
row-sum lumped mass) by forward Euler or SSP-RK3.  Every element type and a mesh of several
types, FP64 and FP32, both schemes; and the closed forms on the GPU: constants are preserved
and a linear field under constant velocity moves by -dt u.g."""
import numpy as np
import pytest

import oracle as O
from helpers import GpuRun
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu


def _mesh(t):
    if t in (G.PEN6, G.PYR5):
        mesh = G.structured_mesh(t, 4)
        G.perturb_interior(mesh, np.random.default_rng(5), 0.1)
        return mesh, G.draw_fields(np.random.default_rng(6), mesh.coords, 3, 50.0)
    cfg, n = {G.HEX8: (2, 6), G.TET4: (1, 6), G.HEX27: (3, 3)}[t]
    w = G.make_workload(cfg, n=n, n_eq=3)
    return w.mesh, w.fields


def _gpu_step(run, fields, phi, dt, stages, precision):
    import torch
    (vel, kd, sr, _), tdt = run.upload(fields, precision)
    ph = torch.from_numpy(np.ascontiguousarray(phi)).to(tdt).cuda()
    fea.fea_explicit_step(run.handle, run.pattern, vel, kd, sr, ph, dt, fields.n_eq, stages,
                          fea.fea_default_opts(precision=precision))
    fea.fea_sync(run.handle)
    return ph.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("t", [G.TET4, G.HEX8, G.HEX27, G.PEN6, G.PYR5], ids=["tet4", "hex8", "hex27", "pen6", "pyr5"])
@pytest.mark.parametrize("stages", [1, 3])
def test_explicit_step_matches_oracle(t, stages):
    mesh, fields = _mesh(t)
    run = GpuRun(mesh)
    try:
        dt = 2e-3 * mesh.h  # a fraction of the convective limit h / |u|
        for precision, tol in ((fea.FEA_F64_PLAIN, 1e-12), (fea.FEA_F32_FUSED, 1e-5)):
            f = fields if precision == fea.FEA_F64_PLAIN else fields.astype(np.float32).astype(np.float64)
            phi = f.phi_old
            want = O.explicit_step(t, mesh.coords, mesh.conn, f, phi, dt, stages)
            got = _gpu_step(run, f, phi, dt, stages, precision)
            change = np.abs(want - phi).max()
            assert change > 1e-4 * np.abs(phi).max()  # the step does move the field
            err = np.abs(got - want).max() / np.abs(want).max()
            assert err <= tol, (precision, err)
    finally:
        run.close()


def test_explicit_step_mixed_mesh():
    import torch
    mm = G.mixed_mesh(4)
    G.perturb_interior(mm, np.random.default_rng(7), 0.1)
    f = G.draw_fields(np.random.default_rng(8), mm.coords, 2, 50.0).astype(np.float32).astype(np.float64)
    h = fea.fea_mesh_create_mixed(mm.coords, mm.blocks)
    p = fea.fea_pattern_build(h)
    try:
        dt = 1e-3 / 4
        # one Euler step of the whole mesh: the blocks' operators and lumped masses summed
        ml = sum(O.lumped_mass(t, mm.coords, c) for t, c in mm.blocks)
        ax = np.stack([sum(O.apply(t, mm.coords, c, f, q, f.phi_old[q], O.CONV | O.DIFF | O.REAC)
                           for t, c in mm.blocks) for q in range(2)])
        want = f.phi_old - dt * ax / ml
        dev = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
               for a in (f.velocity, f.diffusivity, f.reaction, f.phi_old)]
        fea.fea_explicit_step(h, p, dev[0], dev[1], dev[2], dev[3], dt, 2, 1, fea.fea_default_opts())
        fea.fea_sync(h)
        got = dev[3].cpu().numpy().astype(np.float64)
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    finally:
        fea.fea_pattern_destroy(p)
        fea.fea_mesh_destroy(h)


@pytest.mark.parametrize("precision,tol", [(fea.FEA_F64_PLAIN, 1e-12), (fea.FEA_F32_FUSED, 2e-6)], ids=["f64", "f32"])
def test_explicit_step_closed_forms(precision, tol):
    mesh = G.structured_mesh(G.HEX8, 5)
    G.perturb_interior(mesh, np.random.default_rng(9), 0.15)
    N = mesh.n_node
    run = GpuRun(mesh)
    try:
        zero = np.zeros((1, N))
        u = G.velocity_field(mesh.coords)
        f = G.Fields(u, np.full((1, N), 0.05), zero, zero, 1.0)
        got = _gpu_step(run, f, np.full((1, N), 0.7), 1e-3, 3, precision)
        assert np.abs(got - 0.7).max() <= tol
        g, u0 = np.array([0.4, -0.3, 0.9]), np.array([0.5, 0.2, -0.1])
        lin = (mesh.coords @ g + 0.25)[None, :]
        fc = G.Fields(np.tile(u0[:, None], (1, N)), zero, zero, zero, 1.0)
        got = _gpu_step(run, fc, lin, 0.01, 3, precision)
        assert np.abs(got - (lin - 0.01 * u0 @ g)).max() <= 10 * tol
    finally:
        run.close()


def test_explicit_step_arguments():
    w = G.make_workload(2, n=2, n_eq=1)
    run = GpuRun(w.mesh)
    try:
        (vel, kd, sr, phi), _ = run.upload(w.fields, fea.FEA_F32_FUSED)
        for stages, terms, dt in ((2, fea.FEA_TERM_ALL, 1e-3), (3, fea.FEA_TERM_MASS | fea.FEA_TERM_SUPG, 1e-3),
                                  (3, fea.FEA_TERM_ALL, 0.0)):
            with pytest.raises(fea.FeaError) as e:
                fea.fea_explicit_step(run.handle, run.pattern, vel, kd, sr, phi, dt, 1, stages,
                                      fea.fea_default_opts(terms=terms))
            assert e.value.code == 1
    finally:
        run.close()
