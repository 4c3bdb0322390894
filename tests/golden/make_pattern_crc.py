#!/usr/bin/env python3
"""Writes ``pattern_crc_hex8_256.txt``: CRC-32 checksums of the CSR pattern of the Hex8 256^3
workload (16,777,216 elements, 16,974,593 nodes) as the FP64 oracle builds it (Sec. 4.2: the
CSR rows and, per element, the position of each element-matrix entry in them).

The pattern depends on the connectivity only, which the seeded mesh generator fixes, so the
checksums hold on any machine.  The GPU test compares the library's rowptr, colind and
position map against them; this script calls nothing but the oracle and the generator.

    python tests/golden/make_pattern_crc.py      (several minutes and ~10 GB of host memory)
"""
import os
import sys
import time
import zlib

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2107_11541_gb300 import meshgen as G  # noqa: E402

OUT = os.path.join(HERE, "pattern_crc_hex8_256.txt")


def crc(a: np.ndarray) -> int:
    """CRC-32 of the array's little-endian bytes, in 256 MB pieces."""
    b = np.ascontiguousarray(a).view(np.uint8).ravel()
    c = 0
    for i in range(0, b.size, 1 << 28):
        c = zlib.crc32(b[i:i + (1 << 28)], c)
    return c


def main():
    t0 = time.time()
    mesh = G.make_mesh(4)
    rowptr, colind, pos = O.pattern(mesh.elem_type, mesh.conn, mesh.n_node)
    lines = [
        "# CRC-32 (zlib) of the little-endian bytes of the oracle's pattern of the Hex8 256^3 workload",
        "# written by tests/golden/make_pattern_crc.py (oracle only); Sec. 4.2 CSR storage",
        f"n_node: {mesh.n_node}",
        f"n_elem: {mesh.n_elem}",
        f"nnz: {int(rowptr[-1])}",
        f"rowptr_int64_crc32: {crc(rowptr.astype('<i8'))}",
        f"colind_int32_crc32: {crc(colind.astype('<i4'))}",
        f"pos_int32_crc32: {crc(pos.astype('<i4'))}",
    ]
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines), f"\n({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
