"""FP64 Jacobians for badly conditioned elements (FP32 path), through the C ABI.

A mesh with one slab of elements 1e4 times thinner than the rest, rotated off the axes so
that the thin direction mixes all three coordinates: in FP32 the cofactor inverse of such a
Jacobian loses about kappa * 6e-8 of relative accuracy.  Gauss points whose condition estimate
exceeds opts.kappa_threshold (default 1e3) get det J and J^-1 in FP64; with the fallback on,
every scatter stays within the FP32 tolerance."""
import numpy as np
import pytest

from helpers import TOL_F32, GpuRun, compare_full
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu


def rotation():
    a, b, c = 0.3, 0.5, 0.7
    rx = np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])
    ry = np.array([[np.cos(b), 0, np.sin(b)], [0, 1, 0], [-np.sin(b), 0, np.cos(b)]])
    rz = np.array([[np.cos(c), -np.sin(c), 0], [np.sin(c), np.cos(c), 0], [0, 0, 1]])
    return rz @ ry @ rx


def rotated_slab(cfg, n, q):
    w = G.make_workload(cfg, n=n, n_eq=q, stretched_slab=True)
    w.mesh.coords = w.mesh.coords @ rotation().T
    return w.mesh, w.fields


def rotated_layer_slab(t, n, q, ratio=1e-4):
    """Elements of type t on an n^3 grid whose middle z layer of cells is `ratio` as thick as the
    others (prisms: triangles in the y-z planes; pyramids: six per cell around its centre;
    tetrahedra: the Kuhn split), rotated off the axes."""
    widths = np.ones(n)
    widths[n // 2] = ratio
    widths /= widths.sum()
    faces = np.concatenate([[0.0], np.cumsum(widths)])
    faces[-1] = 1.0
    mesh = G.structured_mesh(t, n, faces)
    fields = G.draw_fields(np.random.default_rng(12), mesh.coords, q, 50.0)
    mesh.coords = mesh.coords @ rotation().T
    return mesh, fields


def check_fallback(mesh, fields, q, scatter):
    import torch
    run = GpuRun(mesh)
    try:
        errs = {}
        for kappa in (1e3, 1e30):
            (vel, kd, sr, phi), _ = run.upload(fields, fea.FEA_F32_FUSED)
            vals = torch.empty((q, run.nnz), device="cuda")
            rhs = torch.empty((q, mesh.n_node), device="cuda")
            opts = fea.fea_default_opts(scatter=scatter, kappa_threshold=kappa)
            fea.fea_assemble(run.handle, run.pattern, vel, kd, sr, phi, fields.dt, q, opts, vals, rhs)
            fea.fea_sync(run.handle)
            errs[kappa] = compare_full(run, fields, fea.FEA_F32_FUSED, values=vals, rhs=rhs)
        ea, eb = errs[1e3]
        assert ea <= TOL_F32 and eb <= TOL_F32, errs
        # without the fallback the thin elements' FP32 inverse is visibly worse
        assert errs[1e30][0] > ea, errs
    finally:
        run.close()


@pytest.mark.parametrize("cfg,n,q,scatter", [(2, 6, 2, fea.FEA_SCATTER_ROWOWNED), (2, 6, 2, fea.FEA_SCATTER_GATHER),
                                             (3, 3, 2, fea.FEA_SCATTER_ATOMIC), (3, 3, 2, fea.FEA_SCATTER_GATHER)],
                         ids=["hex8_rowowned", "hex8_gather", "hex27_atomic", "hex27_gather"])
def test_kappa_fallback_keeps_fp32_parity(cfg, n, q, scatter):
    mesh, fields = rotated_slab(cfg, n, q)
    check_fallback(mesh, fields, q, scatter)


@pytest.mark.parametrize("t,scatter", [(G.PEN6, fea.FEA_SCATTER_ATOMIC), (G.PEN6, fea.FEA_SCATTER_GATHER),
                                       (G.TET4, fea.FEA_SCATTER_ATOMIC), (G.TET4, fea.FEA_SCATTER_GATHER),
                                       (G.PYR5, fea.FEA_SCATTER_ATOMIC), (G.PYR5, fea.FEA_SCATTER_GATHER)],
                         ids=["pen6_atomic", "pen6_gather", "tet4_atomic", "tet4_gather", "pyr5_atomic",
                              "pyr5_gather"])
def test_kappa_fallback_other_types(t, scatter):
    mesh, fields = rotated_layer_slab(t, 5, 2)
    check_fallback(mesh, fields, 2, scatter)


def test_condition_just_above_threshold_takes_fp64():
    """A Hex8 layer 1/1500 as thick as its neighbours: the Jacobians' 2-norm condition number is
    about 1500, just above the 1e3 threshold, while |J|_F |J^-1|_F / 3 would read about 700.
    The estimate compared is the upper bound |J|_F |J^-1|_F, so these points take FP64 geometry
    and the result meets the FP32 tolerance; the fallback matters here (it is worse without)."""
    mesh, fields = rotated_layer_slab(G.HEX8, 5, 2, ratio=1.0 / 1500.0)
    check_fallback(mesh, fields, 2, fea.FEA_SCATTER_GATHER)
