"""The allocation-free row-pointer entry point, for callers that cannot let a library
allocate device memory (their device memory all belongs to their own pool or arena).

fea_csr_rowptr_noalloc must give the same row pointers as fea_pattern_build, call after
call: its scratch is a fixed device array shared by all calls, so two calls in a row are
checked, on meshes whose rows span several scan tiles and end in a ragged tile.  This file
is collected last so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

pytestmark = pytest.mark.gpu


def pattern_rowptr(mesh):
    import torch
    h = fea.fea_mesh_create(mesh.coords, mesh.conn, mesh.elem_type)
    p = fea.fea_pattern_build(h)
    rowptr, _, _ = fea.pattern_tensors(p, mesh.n_node, mesh.n_elem, G.NEN[mesh.elem_type])
    fea.fea_pattern_destroy(p)
    fea.fea_mesh_destroy(h)
    torch.cuda.synchronize()
    return rowptr


def test_noalloc_rowptr_matches_pattern_build_twice():
    import torch
    meshes = [G.make_workload(2, n=20, n_eq=1).mesh,   # 9,261 rows: 5 scan tiles, ragged tail
              G.make_workload(1, n=14, n_eq=1).mesh]   # permuted tets, 3,375 rows
    for mesh in meshes:
        want = pattern_rowptr(mesh)
        counts = (want[1:] - want[:-1]).to(torch.int32).contiguous()
        n = counts.numel()
        for _ in range(2):  # two calls in a row share (and reuse) the fixed scratch
            got = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
            fea.fea_csr_rowptr_noalloc(counts, n, got)
            torch.cuda.synchronize()
            assert torch.equal(got, want)


def test_noalloc_rowptr_edges():
    import torch
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    fea.fea_csr_rowptr_noalloc(torch.zeros(1, dtype=torch.int32, device="cuda"), 0, out)
    torch.cuda.synchronize()
    assert out.item() == 0
    with pytest.raises(fea.FeaError) as e:
        fea.fea_csr_rowptr_noalloc(torch.zeros(1, dtype=torch.int32, device="cuda"), 33_554_433, out)
    assert e.value.code == 5  # FEA_ERR_TOO_LARGE, refused before any device work
    rng = np.random.default_rng(3)
    counts = torch.from_numpy(rng.integers(0, 40, size=70_001).astype(np.int32)).cuda()
    got = torch.empty(70_002, dtype=torch.int64, device="cuda")
    fea.fea_csr_rowptr_noalloc(counts, counts.numel(), got)
    torch.cuda.synchronize()
    want = np.concatenate([[0], np.cumsum(counts.cpu().numpy().astype(np.int64))])
    assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("n", [5_000_001, 33_554_432], ids=["5M_rows", "max_rows"])
def test_noalloc_rowptr_many_tiles(n):
    """More than 2048 scan tiles (the tile-offset pass then carries over several rounds), up to
    exactly the largest accepted size, against numpy's cumulative sum, twice in a row."""
    import torch
    rng = np.random.default_rng(n)
    host = rng.integers(0, 130, size=n).astype(np.int32)
    counts = torch.from_numpy(host).cuda()
    want = np.concatenate([[0], np.cumsum(host.astype(np.int64))])
    for _ in range(2):
        got = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
        fea.fea_csr_rowptr_noalloc(counts, n, got)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), want)
