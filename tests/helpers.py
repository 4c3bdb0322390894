"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and
compare it with the FP64 oracle row by row."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2107_11541_gb300 import fea
from paper_2107_11541_gb300 import meshgen as G

TOL_F64 = 1e-12  # per-row relative Frobenius error, FP64 path
TOL_F32 = 1e-5   # per-row relative Frobenius error, FP32 path


def torch_mod():
    import torch
    return torch


class GpuRun:
    """Mesh + pattern on the device, fields uploaded in the path's precision."""

    def __init__(self, mesh: G.Mesh, stream=None):
        torch = torch_mod()
        self.mesh = mesh
        self.handle = fea.fea_mesh_create(mesh.coords, mesh.conn, mesh.elem_type, stream)
        self.pattern = fea.fea_pattern_build(self.handle)
        self.nnz = fea.fea_pattern_get(self.pattern)[3]
        self.torch = torch

    def pattern_np(self):
        r, c, p = fea.pattern_tensors(self.pattern, self.mesh.n_node, self.mesh.n_elem, G.NEN[self.mesh.elem_type])
        return r.cpu().numpy(), c.cpu().numpy(), p.cpu().numpy()

    def upload(self, fields: G.Fields, precision: int):
        torch = self.torch
        dt = torch.float64 if precision == fea.FEA_F64_PLAIN else torch.float32
        np_dt = np.float64 if precision == fea.FEA_F64_PLAIN else np.float32
        dev = [torch.from_numpy(np.ascontiguousarray(a, dtype=np_dt)).cuda()
               for a in (fields.velocity, fields.diffusivity, fields.reaction, fields.phi_old)]
        return dev, dt

    def assemble(self, fields: G.Fields, precision: int, terms=fea.FEA_TERM_ALL, scatter=fea.FEA_SCATTER_AUTO,
                 accumulate=0, out=None, eq_groups=0, cancel_check=0, contraction=fea.FEA_CONTRACT_AUTO,
                 mapping=fea.FEA_MAP_AUTO, elems_per_cta=0):
        torch = self.torch
        (vel, kd, sr, phi), dt = self.upload(fields, precision)
        q = fields.n_eq
        if out is None:
            values = torch.full((q, max(self.nnz, 1)), float("nan"), dtype=dt, device="cuda")
            rhs = torch.full((q, self.mesh.n_node), float("nan"), dtype=dt, device="cuda")
        else:
            values, rhs = out
        opts = fea.fea_default_opts(precision=precision, terms=terms, scatter=scatter, accumulate=accumulate,
                                    eq_groups=eq_groups, cancel_check=cancel_check, contraction=contraction,
                                    mapping=mapping, elems_per_cta=elems_per_cta)
        fea.fea_assemble(self.handle, self.pattern, vel, kd, sr, phi, fields.dt, q, opts, values, rhs)
        fea.fea_sync(self.handle)
        return values, rhs

    def close(self):
        fea.fea_pattern_destroy(self.pattern)
        fea.fea_mesh_destroy(self.handle)


def widen(fields: G.Fields, precision: int) -> G.Fields:
    """The arrays the GPU path consumed, widened to FP64 for the oracle."""
    if precision == fea.FEA_F32_FUSED:
        return fields.astype(np.float32).astype(np.float64)
    return fields


def row_errors(rowptr, vals, ref, absref=None):
    """Per-row relative Frobenius error ||A_i - A*_i|| / ||A*_i|| for every equation."""
    vals = np.asarray(vals, np.float64)
    full = np.diff(rowptr) > 0
    d2 = np.zeros((ref.shape[0], rowptr.size - 1))
    r2 = np.ones((ref.shape[0], rowptr.size - 1))
    if full.any():  # reduceat over the starts of the non-empty rows only
        d2[:, full] = np.add.reduceat((vals - ref) ** 2, rowptr[:-1][full], axis=1)
        r2[:, full] = np.add.reduceat(ref ** 2, rowptr[:-1][full], axis=1)
    return np.sqrt(d2 / r2)


def rhs_errors(rhs, ref, absref):
    rhs = np.asarray(rhs, np.float64)
    den = np.where(absref > 0, absref, 1.0)
    return np.abs(rhs - ref) / den


def compare_full(run: GpuRun, fields: G.Fields, precision: int, terms=fea.FEA_TERM_ALL, values=None, rhs=None):
    """Oracle on the whole mesh vs the GPU output; returns (max row error A, max error b)."""
    m = run.mesh
    rp, ci, pos = run.pattern_np()
    wide = widen(fields, precision)
    ref, refb, absA, absb = O.assemble(m.elem_type, m.coords, m.conn, rp, ci, wide, terms, with_abs=True)
    ea = row_errors(rp, values[:, :run.nnz].cpu().numpy(), ref)
    eb = rhs_errors(rhs.cpu().numpy(), refb, absb)
    return float(ea.max(initial=0.0)), float(eb.max(initial=0.0))
