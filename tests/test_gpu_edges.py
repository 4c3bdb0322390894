"""Degenerate and boundary cases of the method on the GPU, against the oracle: one-element
meshes of every type, tau's vanishing denominator (u = 0, k = 0, s = 0 gives tau = 0),
a single equation and more equations than one shared-memory row window holds comfortably."""
import numpy as np
import pytest

from helpers import TOL_F32, TOL_F64, GpuRun, compare_full
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu

SCATTERS = [fea.FEA_SCATTER_AUTO, fea.FEA_SCATTER_ATOMIC, fea.FEA_SCATTER_GATHER]


def check_all(mesh, fields, scatters=SCATTERS):
    run = GpuRun(mesh)
    try:
        v, r = run.assemble(fields, fea.FEA_F64_PLAIN)
        ea, eb = compare_full(run, fields, fea.FEA_F64_PLAIN, values=v, rhs=r)
        assert ea <= TOL_F64 and eb <= TOL_F64, ("f64", ea, eb)
        for sc in scatters:
            v, r = run.assemble(fields, fea.FEA_F32_FUSED, scatter=sc)
            ea, eb = compare_full(run, fields, fea.FEA_F32_FUSED, values=v, rhs=r)
            assert ea <= TOL_F32 and eb <= TOL_F32, (sc, ea, eb)
    finally:
        run.close()


@pytest.mark.parametrize("t", [G.TET4, G.HEX8, G.HEX27], ids=["tet4", "hex8", "hex27"])
def test_single_element(t):
    rng = np.random.default_rng(9)
    mesh = G.single_element(t, rng, distort=0.1, scale=0.3)
    fields = G.draw_fields(rng, mesh.coords, 3, 50.0)
    check_all(mesh, fields, SCATTERS + ([fea.FEA_SCATTER_ROWOWNED] if t == G.HEX8 else []))


@pytest.mark.parametrize("cfg,n", [(0, 4), (2, 4), (3, 2)], ids=["tet4", "hex8", "hex27"])
def test_tau_denominator_zero(cfg, n):
    """No flow, no diffusion, no reaction: tau's denominator is 0 and tau = 0 everywhere;
    only the mass term and its RHS remain."""
    w = G.make_workload(cfg, n=n, n_eq=2)
    f = w.fields
    f.velocity[:] = 0.0
    f.diffusivity[:] = 0.0
    f.reaction[:] = 0.0
    check_all(w.mesh, f)


@pytest.mark.parametrize("n_eq,groups", [(1, 1), (40, 1), (40, 3)])
def test_rowowned_equation_counts(n_eq, groups):
    w = G.make_workload(2, n=5, n_eq=n_eq)
    run = GpuRun(w.mesh)
    try:
        v, r = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=fea.FEA_SCATTER_ROWOWNED, eq_groups=groups)
        ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=v, rhs=r)
        assert ea <= TOL_F32 and eb <= TOL_F32, (ea, eb)
    finally:
        run.close()
