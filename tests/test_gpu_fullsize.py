"""Parity at the full workload sizes, in the launch configuration bench.py times (FP32 fused,
FEA_SCATTER_AUTO: the autotuned scatter), on rows the oracle computes one by one from their
incident elements.  Sampled rows: the first and last node, the corners of the unit cube and
random rows; each row's columns must equal the oracle's (bit-exact) and its values and RHS
must be within the FP32 tolerance.

The pattern itself is checked whole: rowptr, colind and the position map equal the oracle's
bit for bit on the Tet4 100^3, Hex8 128^3 and Hex27 48^3 workloads, and match the CRC-32
checksums of the oracle's pattern (tests/golden/pattern_crc_hex8_256.txt, written by an
oracle-only script) on the Hex8 256^3 workload."""
import os
import zlib

import numpy as np
import pytest

import oracle as O
from helpers import TOL_F32
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pattern_crc_hex8_256.txt")


def device_crc(t, chunk=1 << 26) -> int:
    """CRC-32 of a device tensor's bytes, copied to the host in pieces."""
    flat = t.reshape(-1)
    c = 0
    for i in range(0, flat.numel(), chunk):
        c = zlib.crc32(flat[i:i + chunk].cpu().numpy().view(np.uint8), c)
    return c


def check_pattern(cfg, m, p, nnz):
    rp_t, ci_t, pos_t = fea.pattern_tensors(p, m.n_node, m.n_elem, G.NEN[m.elem_type])
    if cfg == 4:
        want = {}
        for line in open(GOLDEN):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                want[k.strip()] = int(v)
        assert (want["n_node"], want["n_elem"], want["nnz"]) == (m.n_node, m.n_elem, nnz)
        assert device_crc(rp_t) == want["rowptr_int64_crc32"]
        assert device_crc(ci_t) == want["colind_int32_crc32"]
        assert device_crc(pos_t) == want["pos_int32_crc32"]
        return
    orp, oci, opos = O.pattern(m.elem_type, m.conn, m.n_node)
    assert np.array_equal(rp_t.cpu().numpy(), orp)
    assert np.array_equal(ci_t.cpu().numpy(), oci)
    assert np.array_equal(pos_t.cpu().numpy().reshape(opos.shape), opos)


@pytest.mark.parametrize("cfg", [1, 2, 3, 4], ids=["tet4_100_perm_1eq", "hex8_128_21eq", "hex27_48_11eq",
                                                    "hex8_256_32eq"])
def test_full_size_sampled_rows(cfg):
    import torch
    w = G.make_workload(cfg)
    m, f32 = w.mesh, w.fields.astype(np.float32)
    q = f32.n_eq
    stream = torch.cuda.Stream()
    h = fea.fea_mesh_create(m.coords, m.conn, m.elem_type, stream)
    p = fea.fea_pattern_build(h)
    try:
        nnz = fea.fea_pattern_get(p)[3]
        with torch.cuda.stream(stream):
            dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f32.velocity, f32.diffusivity,
                                                                                f32.reaction, f32.phi_old)]
            values = torch.full((q, nnz), float("nan"), device="cuda")
            rhs = torch.full((q, m.n_node), float("nan"), device="cuda")
        torch.cuda.synchronize()
        opts = fea.fea_default_opts()
        for _ in range(2):  # the first call tunes; the second runs the chosen scatter
            fea.fea_assemble(h, p, *dev, f32.dt, q, opts, values, rhs)
        fea.fea_sync(h)
        scatter, groups = fea.fea_tuned_strategy(p, q)
        check_pattern(cfg, m, p, nnz)
        rp_t, ci_t, _ = fea.pattern_tensors(p, m.n_node, 0, G.NEN[m.elem_type])
        rp = rp_t.cpu().numpy()
        assert rp[-1] == nnz
        rs = O.RowSampler(m.elem_type, m.coords, m.conn, f32.astype(np.float64))
        rng = np.random.default_rng(100 + cfg)
        corners = np.flatnonzero(np.all(np.isclose(m.coords, 0.0) | np.isclose(m.coords, 1.0), axis=1))
        rows = np.unique(np.concatenate([[0, m.n_node - 1], corners, rng.integers(0, m.n_node, 56)]))
        worst = [0.0, 0.0]
        for r in rows:
            cols, ref, _, refb, absb = rs.row(int(r))
            k0, k1 = rp[r], rp[r + 1]
            assert np.array_equal(ci_t[k0:k1].cpu().numpy(), cols), r
            got = values[:, k0:k1].double().cpu().numpy()
            ea = np.sqrt(((got - ref) ** 2).sum(axis=1) / (ref ** 2).sum(axis=1)).max()
            gb = rhs[:, r].double().cpu().numpy()
            eb = (np.abs(gb - refb) / np.where(absb > 0, absb, 1.0)).max()
            worst = [max(worst[0], ea), max(worst[1], eb)]
        assert worst[0] <= TOL_F32 and worst[1] <= TOL_F32, (worst, scatter, groups)
    finally:
        fea.fea_pattern_destroy(p)
        fea.fea_mesh_destroy(h)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
