"""Hex27 with more elements than CTAs: each CTA assembles several elements in turn and fetches
the next element's node data while it contracts the current one.  7^3 = 343 elements over at
most one CTA per SM gives every CTA two or three elements.  5 and 12 equations exercise the
8- and 12-equation register tiles of the kernel; the atomic and gather scatters and the
matrix-free residual are each checked against the FP64 oracle."""
import numpy as np
import pytest

from helpers import TOL_F32, GpuRun, compare_full
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G
from test_gpu_residual import gpu_residual, oracle_residual

pytestmark = pytest.mark.gpu

HEX27 = 3


@pytest.fixture(scope="module", params=[5, 12], ids=["5eq", "12eq"])
def case(request):
    w = G.make_workload(HEX27, n=7, n_eq=request.param)
    run = GpuRun(w.mesh)
    yield w, run
    run.close()


@pytest.mark.parametrize("scatter", [fea.FEA_SCATTER_ATOMIC, fea.FEA_SCATTER_GATHER], ids=["atomic", "gather"])
def test_several_elements_per_cta(case, scatter):
    w, run = case
    assert w.mesh.n_elem > 152
    v, r = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=scatter)
    ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=v, rhs=r)
    assert ea <= TOL_F32 and eb <= TOL_F32, (ea, eb)


def test_residual_several_elements_per_cta(case):
    w, run = case
    q = w.fields.n_eq
    phi = np.random.default_rng(5).uniform(0.0, 1.0, size=(q, w.mesh.n_node)).astype(np.float32).astype(np.float64)
    f = w.fields.astype(np.float32).astype(np.float64)
    ref, scale = oracle_residual(w.mesh, f, phi)
    got = gpu_residual(run, f, phi, fea.FEA_F32_FUSED)
    err = (np.abs(got - ref) / np.where(scale > 0, scale, 1.0)).max()
    assert err <= TOL_F32, err
