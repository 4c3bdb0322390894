"""The autotuned scatter choice and the row-owned equation groups, through the C ABI.

FEA_SCATTER_AUTO times its candidates on the first FP32 call for a pattern and equation
count; the choice is cached (later calls launch only the chosen kernels) and reported by
fea_tuned_strategy.  Equation groups split the row-owned assembly; every split must match
the oracle and give the same bits run to run."""
import numpy as np
import pytest

from helpers import TOL_F32, GpuRun, compare_full
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("groups", [2, 3, 5])
def test_rowowned_equation_groups(groups):
    w = G.make_workload(2, n=7, n_eq=5)
    run = GpuRun(w.mesh)
    try:
        opts = dict(scatter=fea.FEA_SCATTER_ROWOWNED)
        v1, r1 = run.assemble(w.fields, fea.FEA_F32_FUSED, **opts, eq_groups=groups)
        v2, r2 = run.assemble(w.fields, fea.FEA_F32_FUSED, **opts, eq_groups=groups)
        assert np.array_equal(v1.cpu().numpy(), v2.cpu().numpy())
        assert np.array_equal(r1.cpu().numpy(), r2.cpu().numpy())
        ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=v1, rhs=r1)
        assert ea <= TOL_F32 and eb <= TOL_F32, (ea, eb)
    finally:
        run.close()


@pytest.mark.parametrize("cfg,n,q", [(2, 8, 6), (1, 6, 1), (3, 3, 2)], ids=["hex8", "tet4", "hex27"])
def test_autotune_caches_choice(cfg, n, q):
    w = G.make_workload(cfg, n=n, n_eq=q)
    run = GpuRun(w.mesh)
    try:
        with pytest.raises(fea.FeaError) as e:
            fea.fea_tuned_strategy(run.pattern, q)
        assert e.value.code == 9  # FEA_ERR_STATE: not tuned yet
        l0 = fea.fea_kernel_launches()
        v, r = run.assemble(w.fields, fea.FEA_F32_FUSED)  # tunes
        tuning = fea.fea_kernel_launches() - l0
        scatter, groups = fea.fea_tuned_strategy(run.pattern, q)
        assert scatter in (fea.FEA_SCATTER_ATOMIC, fea.FEA_SCATTER_ROWOWNED, fea.FEA_SCATTER_GATHER)
        assert groups >= 1 and (groups == 1 or scatter == fea.FEA_SCATTER_ROWOWNED)
        if cfg != 2:
            assert scatter != fea.FEA_SCATTER_ROWOWNED  # Hex8 only
        ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=v, rhs=r)
        assert ea <= TOL_F32 and eb <= TOL_F32, (ea, eb)
        l1 = fea.fea_kernel_launches()
        v2, r2 = run.assemble(w.fields, fea.FEA_F32_FUSED)  # cached: the chosen kernels only
        again = fea.fea_kernel_launches() - l1
        assert 1 <= again < tuning
        assert again <= 2 * groups
        ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=v2, rhs=r2)
        assert ea <= TOL_F32 and eb <= TOL_F32, (ea, eb)
    finally:
        run.close()


def test_autotune_not_run_when_accumulating():
    """With accumulate = 1 the trials would add into the caller's outputs, so AUTO falls back
    (row-owned where available) without tuning."""
    w = G.make_workload(2, n=5, n_eq=2)
    run = GpuRun(w.mesh)
    try:
        v1, r1 = run.assemble(w.fields, fea.FEA_F32_FUSED, scatter=fea.FEA_SCATTER_ROWOWNED)
        v2, r2 = run.assemble(w.fields, fea.FEA_F32_FUSED, accumulate=1, out=(v1.clone(), r1.clone()))
        with pytest.raises(fea.FeaError):
            fea.fea_tuned_strategy(run.pattern, 2)
        assert np.array_equal(v2.cpu().numpy(), 2 * v1.cpu().numpy())
        assert np.array_equal(r2.cpu().numpy(), 2 * r1.cpu().numpy())
    finally:
        run.close()


def test_tuning_several_equation_counts_keeps_each_choice():
    """Tuning one equation count must not discard the schedules another count uses: after
    tuning 4 and 1 equations, a 4-equation call launches only its chosen kernels again."""
    w4 = G.make_workload(2, n=6, n_eq=4)
    w1 = G.make_workload(2, n=6, n_eq=1)
    run = GpuRun(w4.mesh)
    try:
        run.assemble(w4.fields, fea.FEA_F32_FUSED)
        run.assemble(w1.fields, fea.FEA_F32_FUSED)
        s4, g4 = fea.fea_tuned_strategy(run.pattern, 4)
        l0 = fea.fea_kernel_launches()
        v, r = run.assemble(w4.fields, fea.FEA_F32_FUSED)
        assert fea.fea_kernel_launches() - l0 <= 2 * g4
        assert fea.fea_tuned_strategy(run.pattern, 4) == (s4, g4)
        ea, eb = compare_full(run, w4.fields, fea.FEA_F32_FUSED, values=v, rhs=r)
        assert ea <= TOL_F32 and eb <= TOL_F32
    finally:
        run.close()
