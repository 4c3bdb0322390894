"""The autotuner, through the C ABI.

FEA_SCATTER_AUTO times its candidates (scatter x equation groups x Gauss-point mapping x
elements per CTA x Hex27 contraction) on the first FP32 call for a pattern, equation count
and term mask; the choice is kept (later calls launch only the chosen kernels), reported by
fea_tuned_strategy / fea_tuned_config, and stored in a tuning cache file that a later pattern
of the same GPU, element type, equation count and size class reuses without timing.  Every
candidate the tuner may pick is itself checked against the oracle.  Equation groups split the
row-owned assembly; every split must match the oracle and give the same bits run to run."""
import json
import os

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
        assert again <= 3 * groups
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
        assert fea.fea_kernel_launches() - l0 <= 3 * g4
        assert fea.fea_tuned_strategy(run.pattern, 4) == (s4, g4)
        ea, eb = compare_full(run, w4.fields, fea.FEA_F32_FUSED, values=v, rhs=r)
        assert ea <= TOL_F32 and eb <= TOL_F32
    finally:
        run.close()


def _cand_mesh(t):
    if t == G.PEN6 or t == G.PYR5:
        mesh = G.structured_mesh(t, 4)
        G.perturb_interior(mesh, np.random.default_rng(3), 0.1)
        return mesh, G.draw_fields(np.random.default_rng(4), mesh.coords, 3, 50.0)
    cfg, n = {G.HEX8: (2, 6), G.TET4: (1, 6), G.HEX27: (3, 3)}[t]
    w = G.make_workload(cfg, n=n, n_eq=3)
    return w.mesh, w.fields


@pytest.mark.parametrize("t", [G.HEX8, G.TET4, G.HEX27, G.PEN6, G.PYR5],
                         ids=["hex8", "tet4", "hex27", "pen6", "pyr5"])
def test_every_tuning_candidate_matches_oracle(t):
    """The tuner only picks among configurations that are themselves correct: each candidate,
    set explicitly, matches the oracle."""
    mesh, fields = _cand_mesh(t)
    run = GpuRun(mesh)
    try:
        cands = fea.fea_tune_candidates(run.pattern, 3)
        assert len(cands) >= 2
        kinds = {(c["mapping"], c["elems_per_cta"]) for c in cands}
        assert len(kinds) >= 2  # more than the scatter varies
        for c in cands:
            v, r = run.assemble(fields, fea.FEA_F32_FUSED, scatter=c["scatter"], eq_groups=c["eq_groups"],
                                mapping=c["mapping"], elems_per_cta=c["elems_per_cta"],
                                contraction=c["contraction"])
            ea, eb = compare_full(run, fields, fea.FEA_F32_FUSED, values=v, rhs=r)
            assert ea <= TOL_F32 and eb <= TOL_F32, (c, ea, eb)
        v, r = run.assemble(fields, fea.FEA_F32_FUSED)  # AUTO picks one of them
        got = fea.fea_tuned_config(run.pattern, 3)
        assert any(all(got[k] == c[k] for k in c if k not in ("from_cache", "ms")) for c in cands), got
    finally:
        run.close()


def test_tuning_cache_file_is_reused(tmp_path):
    """A tuned choice is written to the cache file; a new pattern of the same mesh takes it from
    the file without timing (one assembly's launches only) and reports from_cache."""
    path = tmp_path / "tuning.json"
    os.environ["FEA_TUNE_CACHE"] = str(path)
    try:
        w = G.make_workload(2, n=7, n_eq=3)
        run = GpuRun(w.mesh)
        try:
            l0 = fea.fea_kernel_launches()
            run.assemble(w.fields, fea.FEA_F32_FUSED)
            tuning = fea.fea_kernel_launches() - l0
            first = fea.fea_tuned_config(run.pattern, 3)
            assert first["from_cache"] == 0 and first["ms"] > 0
        finally:
            run.close()
        text = path.read_text()
        entries = json.loads(text)
        assert len(entries) == 1
        (key, val), = entries.items()
        assert "|hex8|q3|t31|f32|" in key and val["scatter"] == first["scatter"]
        run = GpuRun(w.mesh)
        try:
            l0 = fea.fea_kernel_launches()
            v, r = run.assemble(w.fields, fea.FEA_F32_FUSED)
            again = fea.fea_kernel_launches() - l0
            second = fea.fea_tuned_config(run.pattern, 3)
            assert second["from_cache"] == 1
            for k in ("scatter", "eq_groups", "mapping", "elems_per_cta", "contraction"):
                assert second[k] == first[k]
            assert again < tuning and again <= 3 * second["eq_groups"]
            ea, eb = compare_full(run, w.fields, fea.FEA_F32_FUSED, values=v, rhs=r)
            assert ea <= TOL_F32 and eb <= TOL_F32
        finally:
            run.close()
    finally:
        os.environ["FEA_TUNE_CACHE"] = "off"


def test_tuning_options_arguments():
    w = G.make_workload(2, n=2, n_eq=1)
    run = GpuRun(w.mesh)
    try:
        for kw in (dict(mapping=4), dict(elems_per_cta=-1), dict(elems_per_cta=1000)):
            with pytest.raises(fea.FeaError) as e:
                run.assemble(w.fields, fea.FEA_F32_FUSED, **kw)
            assert e.value.code == 1
    finally:
        run.close()
