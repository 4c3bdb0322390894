"""FP64 CPU oracle for CDR finite-element assembly (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library path never calls it.

The arithmetic lives in ``fea_oracle.c`` (plain C, double precision, compiled
with ``-ffp-contract=off`` so x86 and Arm give the same bits); this module only
marshals numpy arrays.  ``build()`` compiles it with gcc into ``oracle/_build``.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

TET4, HEX8, HEX27, PEN6, PYR5 = 0, 1, 2, 3, 4
MASS, CONV, DIFF, REAC, SUPG = 1, 2, 4, 8, 16
ALL_TERMS = 31
OK, ERR_ARG, ERR_RANGE, ERR_DUP, ERR_INVERTED, ERR_CAP = 0, 1, 2, 3, 4, 5
NEN = {TET4: 4, HEX8: 8, HEX27: 27, PEN6: 6, PYR5: 5}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fea_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libfea_oracle.so")
# a second build with the planted mistakes compiled in (-DOR_MUTATION), loaded only by
# ``mutation()``; the oracle proper has none of them
_MUT_PATH = os.path.join(_HERE, "_build", "libfea_oracle_mut.so")
_lib = None
_mut_lib = None
_lock = threading.Lock()

_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_L = C.c_int64
_I = C.c_int
_D = C.c_double


def _compile(path: str, extra, force: bool) -> str:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FP contraction)."""
    return _compile(_LIB_PATH, [], force)


def build_mutant(force: bool = False) -> str:
    """Compile the test-only build that carries the planted mistakes (``mutation()``)."""
    return _compile(_MUT_PATH, ["-DOR_MUTATION"], force)


def _declare(L):
    L.or_shape.argtypes = [_I, _d, _d, _d]
    L.or_quadrature.argtypes = [_I, _d, _d]
    L.or_element.argtypes = [_I, _d, _d, _d, _d, _d, _D, _I, _d, _d]
    L.or_validate.argtypes = [_I, _d, _L, _i32, _L]
    L.or_incidence.argtypes = [_I, _i32, _L, _L, _i64, _i64]
    L.or_pattern_rowptr.argtypes = [_I, _i32, _L, _L, _i64, _i64, _i64]
    L.or_pattern_rowptr.restype = C.c_int64
    L.or_pattern_colind.argtypes = [_I, _i32, _L, _i64, _i64, _i64, _i32]
    L.or_posmap.argtypes = [_I, _i32, _L, _i64, _i32, _i32]
    L.or_assemble.argtypes = [_I, _d, _L, _i32, _L, _L, _i64, _i32, _L, _d, _d, _d, _d, _D, _I, _I,
                              _d, _d, C.c_void_p, C.c_void_p]
    L.or_row.argtypes = [_I, _d, _L, _i32, _i64, _i64, _L, _d, _d, _d, _d, _D, _I, _I, _L, _i32, _d, _d,
                         _d, _d]
    L.or_row.restype = C.c_int64
    L.or_apply.argtypes = [_I, _d, _L, _i32, _L, _d, _d, _d, _d, _D, _I, _I, _d, _d]
    L.or_update_fields.argtypes = [_d, _L, _I, _d, _d]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
    return _lib


def _f(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _c(conn) -> np.ndarray:
    return np.ascontiguousarray(conn, dtype=np.int32)


@contextlib.contextmanager
def mutation(m: int):
    """Temporarily route every call to the test-only build with deliberate mistake ``m``
    switched on (tests of the pins)."""
    global _lib, _mut_lib
    with _lock:
        if _mut_lib is None:
            _mut_lib = _declare(C.CDLL(build_mutant()))
            _mut_lib.or_set_mutation.argtypes = [_I]
    good = lib()
    _mut_lib.or_set_mutation(int(m))
    _lib = _mut_lib
    try:
        yield
    finally:
        _mut_lib.or_set_mutation(0)
        _lib = good


def quadrature(elem_type: int):
    xi = np.zeros(27 * 3)
    w = np.zeros(27)
    ng = lib().or_quadrature(elem_type, xi, w)
    return xi[: 3 * ng].reshape(ng, 3).copy(), w[:ng].copy()


def shape(elem_type: int, xi):
    N = np.zeros(27)
    dN = np.zeros(27 * 3)
    nen = lib().or_shape(elem_type, _f(xi), N, dN)
    return N[:nen].copy(), dN[: 3 * nen].reshape(nen, 3).copy()


def element(elem_type, xe, ue, ke, se, phie, dt, terms=ALL_TERMS):
    nen = NEN[elem_type]
    Ae = np.zeros(nen * nen)
    be = np.zeros(nen)
    st = lib().or_element(elem_type, _f(xe).ravel(), _f(ue).ravel(), _f(ke), _f(se), _f(phie), float(dt),
                          int(terms), Ae, be)
    if st:
        raise ValueError(f"oracle element error {st}")
    return Ae.reshape(nen, nen), be


def validate(elem_type, coords, conn) -> int:
    conn = _c(conn)
    return int(lib().or_validate(elem_type, _f(coords).ravel(), coords.shape[0], conn.ravel(), conn.shape[0]))


def incidence(elem_type, conn, n_node):
    conn = _c(conn)
    inc_ptr = np.zeros(n_node + 1, dtype=np.int64)
    inc_elem = np.zeros(conn.size, dtype=np.int64)
    st = lib().or_incidence(elem_type, conn.ravel(), conn.shape[0], n_node, inc_ptr, inc_elem)
    if st:
        raise ValueError(f"oracle incidence error {st}")
    return inc_ptr, inc_elem


def pattern(elem_type, conn, n_node, with_pos=True):
    """CSR pattern: rowptr (int64[N+1]), colind (int32[nnz]) and pos (int32[E,nen,nen])."""
    conn = _c(conn)
    inc_ptr, inc_elem = incidence(elem_type, conn, n_node)
    rowptr = np.zeros(n_node + 1, dtype=np.int64)
    nnz = lib().or_pattern_rowptr(elem_type, conn.ravel(), conn.shape[0], n_node, inc_ptr, inc_elem, rowptr)
    if nnz < 0:
        raise ValueError("oracle pattern error")
    colind = np.zeros(nnz, dtype=np.int32)
    st = lib().or_pattern_colind(elem_type, conn.ravel(), n_node, inc_ptr, inc_elem, rowptr, colind)
    if st:
        raise ValueError(f"oracle colind error {st}")
    pos = None
    if with_pos:
        nen = NEN[elem_type]
        pos = np.zeros((conn.shape[0], nen, nen), dtype=np.int32)
        st = lib().or_posmap(elem_type, conn.ravel(), conn.shape[0], rowptr, colind, pos.ravel())
        if st:
            raise ValueError(f"oracle posmap error {st}")
    return rowptr, colind, pos


def assemble(elem_type, coords, conn, rowptr, colind, fields, terms=ALL_TERMS, e_range=None, with_abs=False):
    """values (n_eq, nnz), rhs (n_eq, N) and, if asked, abs-sum denominators."""
    conn = _c(conn)
    n_node = coords.shape[0]
    nnz = colind.shape[0]
    n_eq = fields.diffusivity.shape[0]
    values = np.zeros((n_eq, nnz))
    rhs = np.zeros((n_eq, n_node))
    absA = np.zeros((n_eq, nnz)) if with_abs else None
    absb = np.zeros((n_eq, n_node)) if with_abs else None
    e0, e1 = (0, conn.shape[0]) if e_range is None else e_range
    st = lib().or_assemble(elem_type, _f(coords).ravel(), n_node, conn.ravel(), e0, e1,
                           np.ascontiguousarray(rowptr, dtype=np.int64), _c(colind), nnz,
                           _f(fields.velocity).ravel(), _f(fields.diffusivity).ravel(),
                           _f(fields.reaction).ravel(), _f(fields.phi_old).ravel(), float(fields.dt), n_eq,
                           int(terms), values.ravel(), rhs.ravel(),
                           absA.ctypes.data if with_abs else None, absb.ctypes.data if with_abs else None)
    if st:
        raise ValueError(f"oracle assemble error {st}")
    if with_abs:
        return values, rhs, absA, absb
    return values, rhs


def pattern_mixed(blocks, n_node, with_pos=True):
    """CSR pattern of a mesh made of element blocks [(elem_type, conn), ...] of different types,
    from its definition (Sec. 4.2: the CSR matrix the element contributions go to): row i holds
    column j iff some element of any block contains both nodes, columns ascending.  pos is one
    int32 array [E_b, nen_b, nen_b] per block."""
    keys = []
    for t, conn in blocks:
        c = _c(conn).astype(np.int64)
        nen = NEN[t]
        keys.append((np.repeat(c, nen, axis=1) * n_node + np.tile(c, (1, nen))).ravel())
    key = np.unique(np.concatenate(keys)) if keys else np.zeros(0, np.int64)
    rows, cols = key // n_node, key % n_node
    rowptr = np.zeros(n_node + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n_node), out=rowptr[1:])
    colind = cols.astype(np.int32)
    pos = None
    if with_pos:
        pos = []
        for t, conn in blocks:
            c = _c(conn).astype(np.int64)
            nen = NEN[t]
            k = c[:, :, None] * n_node + c[:, None, :]
            pos.append(np.searchsorted(key, k).astype(np.int32).reshape(c.shape[0], nen, nen))
    return rowptr, colind, pos


def assemble_mixed(coords, blocks, rowptr, colind, fields, terms=ALL_TERMS, with_abs=False):
    """Assembly of a mesh of element blocks: the sum of every block's element contributions."""
    outs = [assemble(t, coords, conn, rowptr, colind, fields, terms, with_abs=with_abs) for t, conn in blocks]
    return tuple(sum(o[i] for o in outs) for i in range(len(outs[0])))


def apply_mixed(coords, blocks, fields, q, x, terms=ALL_TERMS):
    """Matrix-free A x of a mesh of element blocks, summed over the blocks."""
    return sum(apply(t, coords, conn, fields, q, x, terms) for t, conn in blocks)


class RowSampler:
    """Computes single rows of every equation from the elements incident to them."""

    def __init__(self, elem_type, coords, conn, fields, terms=ALL_TERMS):
        self.t = elem_type
        self.coords = _f(coords).ravel()
        self.n_node = coords.shape[0]
        self.conn = _c(conn).ravel()
        self.inc_ptr, self.inc_elem = incidence(elem_type, _c(conn), self.n_node)
        self.f = (_f(fields.velocity).ravel(), _f(fields.diffusivity).ravel(), _f(fields.reaction).ravel(),
                  _f(fields.phi_old).ravel())
        self.dt = float(fields.dt)
        self.n_eq = fields.diffusivity.shape[0]
        self.terms = int(terms)
        self.cap = int(np.max(np.diff(self.inc_ptr))) * NEN[elem_type] + 1

    def row(self, r):
        cap, q = self.cap, self.n_eq
        cols = np.zeros(cap, dtype=np.int32)
        vals = np.zeros(q * cap)
        absv = np.zeros(q * cap)
        rhs = np.zeros(q)
        absr = np.zeros(q)
        nc = lib().or_row(self.t, self.coords, self.n_node, self.conn, self.inc_ptr, self.inc_elem, int(r),
                          *self.f, self.dt, q, self.terms, cap, cols, vals, absv, rhs, absr)
        if nc < 0:
            raise ValueError(f"oracle row error {-nc}")
        vals = vals.reshape(q, cap)[:, :nc].copy()
        absv = absv.reshape(q, cap)[:, :nc].copy()
        return cols[:nc].copy(), vals, absv, rhs, absr


def apply(elem_type, coords, conn, fields, q, x, terms=ALL_TERMS):
    conn = _c(conn)
    y = np.zeros(coords.shape[0])
    st = lib().or_apply(elem_type, _f(coords).ravel(), coords.shape[0], conn.ravel(), conn.shape[0],
                        _f(fields.velocity).ravel(), _f(fields.diffusivity).ravel(), _f(fields.reaction).ravel(),
                        _f(fields.phi_old).ravel(), float(fields.dt), int(q), int(terms), _f(x), y)
    if st:
        raise ValueError(f"oracle apply error {st}")
    return y


def solve(rowptr, colind, values, b):
    """The exact solution x = A^-1 b of one assembled system (the result the preconditioned CG
    of Sec. 2, Alg. 1 converges to), by a sparse direct solve in FP64."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    n = rowptr.size - 1
    A = sp.csr_matrix((np.asarray(values, np.float64), np.asarray(colind), np.asarray(rowptr)), shape=(n, n))
    return spla.spsolve(A.tocsc(), np.asarray(b, np.float64))


def update_fields(coords, phi, params):
    """One step's field update: returns phi + A sin(k . x + psi) per equation (FP64).
    phi is (n_eq, N); params is (n_eq, 5) = A, kx, ky, kz, psi."""
    out = np.array(phi, dtype=np.float64, copy=True, order="C")
    p = _f(params).reshape(-1, 5)
    if p.shape[0] != out.shape[0]:
        raise ValueError("params must have one row per equation")
    st = lib().or_update_fields(_f(coords).ravel(), out.shape[1], out.shape[0], p.ravel(), out.ravel())
    if st:
        raise ValueError(f"oracle update error {st}")
    return out


class _Coefficients:
    """Nodal arrays of one call (the attributes the element routines read)."""

    def __init__(self, velocity, diffusivity, reaction, phi_old, dt):
        self.velocity, self.diffusivity, self.reaction, self.phi_old, self.dt = (
            velocity, diffusivity, reaction, phi_old, dt)


def lumped_mass(elem_type, coords, conn):
    """Row sums of the consistent mass matrix, M_L[i] = sum_j M_ij = int N_i dV (the lumped mass of
    the explicit stepping of Sec. 2), as the mass operator applied to the vector of ones."""
    n = coords.shape[0]
    z = np.zeros((1, n))
    c = _Coefficients(np.zeros((3, n)), z, z, z, 1.0)
    return apply(elem_type, coords, conn, c, 0, np.ones(n), terms=MASS)


def explicit_step(elem_type, coords, conn, fields, phi, dt, stages=3, terms=CONV | DIFF | REAC):
    """One explicit time step of M_L dphi/dt = -A phi for every equation (Sec. 2: heat and species
    advance by RK3 without an algebraic solver), A the operator of the chosen terms (convection,
    diffusion, reaction; SUPG and the mass are not among them) applied matrix-free, M_L the lumped
    mass.  stages = 1: forward Euler; stages = 3: the three-stage strong-stability-preserving
    Runge-Kutta scheme
        phi1 = phi + dt L(phi),  phi2 = 3/4 phi + 1/4 (phi1 + dt L(phi1)),
        phi_new = 1/3 phi + 2/3 (phi2 + dt L(phi2)),   L(x) = -M_L^-1 A x.
    phi is (n_eq, N); returns the new (n_eq, N) field in FP64."""
    phi = np.asarray(phi, dtype=np.float64)
    ml = lumped_mass(elem_type, coords, conn)

    def L(x):
        return np.stack([-apply(elem_type, coords, conn, fields, q, x[q], terms) for q in range(x.shape[0])]) / ml

    if stages == 1:
        return phi + dt * L(phi)
    if stages != 3:
        raise ValueError("stages must be 1 or 3")
    p1 = phi + dt * L(phi)
    p2 = 0.75 * phi + 0.25 * (p1 + dt * L(p1))
    return phi / 3.0 + 2.0 / 3.0 * (p2 + dt * L(p2))
