"""Host-side checks that need no GPU: the C-ABI library loads and exports every
symbol include/fea.h declares, argument errors are reported before any device
work, the Fig. 3 packing layout, and the synthetic meshes are valid."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2107_11541_gb300 import build, fea
from paper_2107_11541_gb300 import meshgen as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return fea.lib()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "fea.h")).read()
    return sorted(set(re.findall(r"FEA_API\s+[\w\s\*]+?\b(fea_\w+)\s*\(", text)))


def test_exports_match_header(L):
    syms = header_symbols()
    assert syms == sorted(fea.EXPORTS)
    for s in syms:
        assert hasattr(L, s), s


def test_version_and_defaults(L):
    assert fea.fea_version() >= 10000
    o = fea.fea_default_opts()
    assert (o.precision, o.terms, o.scatter, o.accumulate, o.kappa_threshold) == (1, 31, 0, 0, 1e3)


def test_argument_errors_without_device(L):
    with pytest.raises(fea.FeaError) as e:
        fea.lib()
        fea._check(L.fea_mesh_create(None, 10, None, 0, 1, None, None))
    assert e.value.code == 1
    with pytest.raises(fea.FeaError) as e:
        fea._check(L.fea_mesh_create(None, 10, None, 0, 7, None, None))
    assert e.value.code == 1
    with pytest.raises(fea.FeaError) as e:
        fea.fea_assemble(None, None, None, None, None, None, 1e-3, 1, None, None, None)
    assert e.value.code == 1
    assert "null" in fea.fea_last_error()


def test_pack_plan_fig3(L):
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "fig3_packing.txt")) if l[0] != "#"]
    counts = [int(r[1]) for r in rows]
    vs = int(rows[0][2])
    packs, pads = fea.fea_pack_plan(counts, vs)
    assert packs.tolist() == [int(r[3]) for r in rows]
    assert pads.tolist() == [int(r[4]) for r in rows]
    with pytest.raises(fea.FeaError):
        fea.fea_pack_plan([3], 0)


@pytest.mark.parametrize("t", (G.TET4, G.HEX8, G.HEX27))
def test_generated_meshes_are_valid(t):
    for idx in range(4):
        w = G.make_workload(idx, n=4 if t != G.HEX27 else 2, n_eq=2)
        if w.mesh.elem_type != t:
            continue
        assert O.validate(t, w.mesh.coords, w.mesh.conn) == O.OK
    w = G.make_workload(3, n=4, n_eq=1, stretched_slab=True)
    assert O.validate(G.HEX27, w.mesh.coords, w.mesh.conn) == O.OK
    w = G.make_workload(1, n=5, n_eq=1)
    assert O.validate(G.TET4, w.mesh.coords, w.mesh.conn) == O.OK
    assert sorted(np.unique(w.mesh.conn)) == list(range(w.mesh.n_node))


def test_oracle_all_cores_timing():
    """The all-cores CPU baseline: one spawned process per host core, each assembling its own
    element chunk with the unchanged oracle.  The sub-mesh of all elements is the mesh itself
    (node renumbering keeps ascending ids), and every process reports a positive rate."""
    import bench
    w = G.make_workload(0, n=4)
    m, f = w.mesh, w.fields
    coords, conn, arrays = bench._oracle_submesh(m, f, 0, m.n_elem)
    assert np.array_equal(coords, m.coords) and np.array_equal(conn, m.conn)
    rates, procs, ne = bench.oracle_all_cores(w, 0.05, 2)
    assert procs >= 1 and 0 < ne <= m.n_elem and len(rates) == 2 and min(rates) > 0


def test_mixed_bench_parity_sampler():
    """The mixed-mesh bench compares sampled rows with the oracle's assembly of the incident
    elements: the whole mesh's own FP32-rounded assembly passes, and an error planted in one
    sampled row is reported."""
    import bench
    mm, f = bench.make_mixed("mixed_96_4eq", 6)
    rp, ci, _ = O.pattern_mixed(mm.blocks, mm.n_node, with_pos=False)
    v, b = O.assemble_mixed(mm.coords, mm.blocks, rp, ci, f.astype(np.float32).astype(np.float64))
    v32, b32 = v.astype(np.float32), b.astype(np.float32)
    ok = bench.mixed_parity(mm, f, v32, b32, rp, ci)
    assert ok["pass"] and ok["max_row_err_A"] < 1e-6
    bad = v32.copy()
    bad[0, rp[0]] *= 1.01  # row 0 is always sampled
    assert not bench.mixed_parity(mm, f, bad, b32, rp, ci)["pass"]


def test_roofline_unit_figures():
    """The algorithmic bytes and flops behind the bench's roofline fractions.  Bytes: connectivity,
    coordinates and velocity, per-equation k, s and phi, and the CSR values and RHS written once,
    for the 10^3 Tet4 case in FP64 (0.34 MB) and the Hex8 128^3 x 21 workload in FP32 (5.63 GB), from
    the closed-form node, element and nonzero counts of the structured meshes.  Flops: the
    multiply-adds of the direct form per element and equation, counted term by term here."""
    import bench

    def counted(nen, ng):  # one multiply-add = 2 flops
        madds = 0
        for _g in range(ng):
            madds += nen * nen                                    # rank-1 Galerkin/SUPG product P_a Q_b
            madds += sum(1 for a in range(nen) for b in range(a, nen))  # symmetric diffusion grad N_a . grad N_b
            madds += 6 * nen  # u_g (3), k_g, s_g, phi_g interpolation, each nen long
        return 2 * madds

    for t, ng, want in ((G.TET4, 4, 400), (G.HEX8, 8, 2368), (G.HEX27, 27, 68526), (G.PEN6, 6, 1116),
                        (G.PYR5, 12, 1680)):
        nen = G.NEN[t]
        assert bench.algorithmic_flops_per_elem_eq(nen, ng) == counted(nen, ng) == want
    # Kuhn 10^3: E = 6 n^3, N = (n+1)^3, nnz = N + 2 (edges), edges = 3n(n+1)^2 + 3n^2(n+1) + n^3
    n = 10
    E, N = 6 * n ** 3, (n + 1) ** 3
    nnz = N + 2 * (3 * n * (n + 1) ** 2 + 3 * n ** 2 * (n + 1) + n ** 3)
    assert nnz == 17191
    assert bench.algorithmic_bytes(E, N, nnz, 4, 1, s=8) == 340008
    # Hex8 128^3: nnz = (sum of 1-D row lengths)^3 = (3 * 129 - 2)^3
    n = 128
    E, N, nnz = n ** 3, (n + 1) ** 3, (3 * (n + 1) - 2) ** 3
    assert nnz == 57066625
    assert bench.algorithmic_bytes(E, N, nnz, 8, 21) == 5633513404


def test_reference_arm_line_and_other_ranks():
    """bench.py --impl reference: rank 0 prints one JSON line with the oracle timed on the host
    cores (a shrunken Hex8 case here); any other rank exits 0 without output."""
    import json
    import subprocess
    import sys
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--cells", "4", "--steps", "2",
           "--warmup", "1"]
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == bench_metric() and d["unit"] == "elem*eq/s" and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] == d["e2e"]["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""


def bench_metric():
    import bench
    return bench.METRIC


def test_profiled_traffic_goes_null_when_the_kernels_change(tmp_path, monkeypatch):
    """bench.py reports the DRAM traffic of a committed ncu summary only while the kernel
    sources hash to the digest recorded with it; after any change to them it reports null."""
    import shutil

    import bench
    src = os.path.join(ROOT, "paper_2107_11541_gb300", "csrc")
    csrc = tmp_path / "paper_2107_11541_gb300" / "csrc"
    shutil.copytree(src, csrc)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.kernel_source_digest()
    (tmp_path / "profiles" / "dram_traffic_w.txt").write_text(
        "# a comment: with colons\ntraffic_bytes_per_launch: 1234\nkernel_source_digest: %s\n" % digest)
    assert bench.profiled_traffic("w") == 1234.0
    assert bench.profiled_traffic("absent") is None
    with open(csrc / "fea_api.cu", "a") as f:
        f.write("\n")
    assert bench.kernel_source_digest() != digest and bench.profiled_traffic("w") is None


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without the built CUDA library every call raises; there is no CPU fallback."""
    monkeypatch.setattr(fea, "_lib", None)
    missing = str(tmp_path / "libfea.so")
    with pytest.raises(FileNotFoundError, match="missing"):
        fea.lib(missing)
    monkeypatch.setattr(fea, "LIB_PATH", missing)
    monkeypatch.setattr(fea.lib, "__defaults__", (missing,))
    with pytest.raises(FileNotFoundError):
        fea.fea_version()


def test_bench_closed_form_nnz():
    """The reference arm reports nnz from counting formulas; they give the pattern sizes the
    oracle's own pattern reaches (pinned in the oracle tests), and the oracle's count on small
    grids of every workload's element type."""
    import bench
    import oracle as O
    want = {"tet4_100_perm_1eq": 15_210_901, "hex8_128_21eq": 57_066_625, "hex27_48_11eq": 57_066_625,
            "hex8_256_32eq": 454_756_609}
    for wl, nnz in want.items():
        assert bench.closed_form_nnz(wl) == nnz
    for wl in want:
        m = G.make_mesh(bench.WORKLOADS[wl], n=3)
        rp, _, _ = O.pattern(m.elem_type, m.conn, m.n_node, with_pos=False)
        assert bench.closed_form_nnz(wl, 3) == rp[-1]
