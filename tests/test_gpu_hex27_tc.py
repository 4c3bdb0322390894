"""Hex27 element matrices on the tensor cores (tcgen05, BF16 operand parts, FP32 accumulation in
tensor memory), through the C ABI, against the FP64 oracle.

Per element every equation's matrix is one product of its left factor with the right factor
shared by all equations; the rows (equation, node) of all equations are stacked into 128-row
tiles.  1, 5, 11 and 12 equations give one, two and three tiles with ragged last tiles; 7^3 =
343 elements give every CTA several elements in turn (tensor memory, barriers and the two chunk
buffers reused).  The TF32 split (3xTF32) must meet the FP32 tolerance; the BF16 split (bf16x3)
is measured and reported, and must be less accurate than the TF32 one."""
import numpy as np
import pytest

from helpers import TOL_F32, GpuRun, compare_full
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G
from test_gpu_kappa import rotated_slab

pytestmark = pytest.mark.gpu

HEX27 = 3
X3, T3 = fea.FEA_CONTRACT_TC_BF16X3, fea.FEA_CONTRACT_TC_TF32X3


@pytest.fixture(scope="module", params=[1, 5, 11, 12], ids=["1eq", "5eq", "11eq", "12eq"])
def case(request):
    w = G.make_workload(HEX27, n=7, n_eq=request.param)
    run = GpuRun(w.mesh)
    yield w, run
    run.close()


@pytest.mark.parametrize("scatter", [fea.FEA_SCATTER_ATOMIC, fea.FEA_SCATTER_GATHER], ids=["atomic", "gather"])
def test_tensor_core_tf32x3_parity(case, scatter):
    w, run = case
    assert w.mesh.n_elem > 152
    v, r = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=scatter, contraction=T3)
    ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=v, rhs=r)
    print(f"3xtf32 {w.fields.n_eq} eq: max row error A {ea:.3e}, b {eb:.3e}")
    assert ea <= TOL_F32 and eb <= TOL_F32, (ea, eb)


def test_tensor_core_bf16x3_measured(case):
    """The BF16 split keeps about 16 bits of each operand: its row error is measured and must
    exceed the TF32 split's (about 22 bits) while staying near the FP32 tolerance."""
    w, run = case
    v3, r3 = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=fea.FEA_SCATTER_ATOMIC, contraction=X3)
    e3 = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=v3, rhs=r3)
    vt3, rt3 = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=fea.FEA_SCATTER_ATOMIC, contraction=T3)
    et = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=vt3, rhs=rt3)
    vc, rc = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=fea.FEA_SCATTER_ATOMIC,
                          contraction=fea.FEA_CONTRACT_CUDA)
    ec = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=vc, rhs=rc)
    print(f"bf16x3 {w.fields.n_eq} eq: max row error A {e3[0]:.3e} (3xtf32 {et[0]:.3e}, CUDA cores "
          f"{ec[0]:.3e}), b {e3[1]:.3e}")
    assert e3[0] > et[0]
    assert e3[0] <= 1e-3 and e3[1] <= TOL_F32


def test_tensor_core_equals_cuda_cores_closely(case):
    w, run = case
    vc, rc = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=fea.FEA_SCATTER_GATHER,
                          contraction=fea.FEA_CONTRACT_CUDA)
    vt, rt = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=fea.FEA_SCATTER_GATHER, contraction=T3)
    a, b = vc.cpu().numpy().astype(np.float64), vt.cpu().numpy().astype(np.float64)
    assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
    # the RHS is formed on the CUDA cores from the same quantities in both variants
    assert np.abs(rc.cpu().numpy() - rt.cpu().numpy()).max() <= 1e-6 * np.abs(rc.cpu().numpy()).max()


@pytest.mark.parametrize("scatter", [fea.FEA_SCATTER_ATOMIC, fea.FEA_SCATTER_GATHER], ids=["atomic", "gather"])
def test_tensor_core_with_fp64_jacobians(scatter):
    """A rotated 1e-4-thin layer: FP64 geometry feeds the tensor-core products."""
    import torch
    mesh, fields = rotated_slab(HEX27, 3, 2)
    run = GpuRun(mesh)
    try:
        (vel, kd, sr, phi), _ = run.upload(fields, fea.FEA_F32_FUSED)
        vals = torch.empty((2, run.nnz), device="cuda")
        rhs = torch.empty((2, mesh.n_node), device="cuda")
        opts = fea.fea_default_opts(scatter=scatter, contraction=T3)
        fea.fea_assemble(run.handle, run.pattern, vel, kd, sr, phi, fields.dt, 2, opts, vals, rhs)
        fea.fea_sync(run.handle)
        ea, eb = compare_full(run, fields, fea.FEA_F32_FUSED, values=vals, rhs=rhs)
        assert ea <= TOL_F32 and eb <= TOL_F32, (ea, eb)
    finally:
        run.close()


def test_contraction_argument():
    w = G.make_workload(HEX27, n=2, n_eq=1)
    run = GpuRun(w.mesh)
    try:
        with pytest.raises(fea.FeaError) as e:
            run.assemble(w.fields, fea.FEA_F32_FUSED, contraction=7)
        assert e.value.code == 1
    finally:
        run.close()
