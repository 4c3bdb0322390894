"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each check reaches its expected value by a route that does not go through the
oracle's own formulas: exact polynomial integration, closed forms of linear and
box elements, conservation and consistency invariants, the patch test against
face integrals of the boundary flux, brute-force dense assembly, and closed-form
pattern counts.  ``test_pins_catch_planted_mistakes`` plants plausible errors in
the oracle and checks that every one of them fails at least one pin.
"""
import functools
import math

import numpy as np
import pytest
import scipy.sparse as sp
from numpy.polynomial import polynomial as P

import oracle as O
from paper_2107_11541_gb300 import meshgen as G

TYPES = (O.TET4, O.HEX8, O.HEX27, O.PEN6, O.PYR5)
REF_VOLUME = {O.TET4: 1.0 / 6.0, O.HEX8: 8.0, O.HEX27: 8.0, O.PEN6: 1.0, O.PYR5: 4.0 / 3.0}


def ref_nodes(t):
    """Reference coordinates of the nodes in the documented local order (the pyramid's apex
    a hair below z = 1, where its rational functions are singular)."""
    if t == O.TET4:
        return np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    if t == O.PEN6:
        return np.array([[0, 0, -1], [1, 0, -1], [0, 1, -1], [0, 0, 1], [1, 0, 1], [0, 1, 1]], float)
    if t == O.PYR5:
        return np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0], [0, 0, 1 - 1e-15]], float)
    q = 2 if t == O.HEX8 else 3
    pts = np.linspace(-1, 1, q)
    return np.array([[pts[i], pts[j], pts[k]] for k in range(q) for j in range(q) for i in range(q)])


# ------------------------------------------------------------------ reference element pins

def check_quadrature(t):
    xi, w = O.quadrature(t)
    assert np.isclose(w.sum(), REF_VOLUME[t], rtol=0, atol=1e-14)
    if t == O.TET4:  # exact for total degree <= 2: int x^a y^b z^c = a! b! c! / (a+b+c+3)!
        for a in range(3):
            for b in range(3 - a):
                for c in range(3 - a - b):
                    exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                    got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
                    assert abs(got - exact) < 1e-15
    elif t == O.PEN6:  # triangle degree 2 x line degree 3: int x^a y^b = a! b! / (a+b+2)!, int z^c = 2/(c+1)
        for a in range(3):
            for b in range(3 - a):
                for c in range(4):
                    tri = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
                    exact = tri * (2.0 / (c + 1) if c % 2 == 0 else 0.0)
                    got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
                    assert abs(got - exact) < 1e-14
    elif t == O.PYR5:  # int over |x|,|y| <= 1-z: I_a I_b c! (a+b+2)! / (a+b+c+3)!, I_a = 2/(a+1) (a even)
        for a, b, c in ((a, b, c) for a in range(4) for b in range(4) for c in range(4) if a + b + c <= 3):
            ia = 2.0 / (a + 1) if a % 2 == 0 else 0.0
            ib = 2.0 / (b + 1) if b % 2 == 0 else 0.0
            exact = ia * ib * math.factorial(c) * math.factorial(a + b + 2) / math.factorial(a + b + c + 3)
            got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
            assert abs(got - exact) < 1e-14
    else:  # Gauss-Legendre with n points per axis is exact to degree 2n-1 per axis
        deg = 3 if t == O.HEX8 else 5
        for a in range(deg + 1):
            for b in range(deg + 1):
                for c in range(deg + 1):
                    one = [2.0 / (k + 1) if k % 2 == 0 else 0.0 for k in (a, b, c)]
                    got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
                    assert abs(got - np.prod(one)) < 1e-13


def check_shape_functions(t, rng):
    nodes = ref_nodes(t)
    for b, x in enumerate(nodes):  # Kronecker property at the nodes
        N, _ = O.shape(t, x)
        assert np.allclose(N, np.eye(len(nodes))[b], atol=1e-14)
    for _ in range(5):
        if t == O.TET4:
            x = rng.uniform(0, 0.3, 3)
        elif t == O.PEN6:
            x = np.array([rng.uniform(0, 0.45), rng.uniform(0, 0.45), rng.uniform(-1, 1)])
        elif t == O.PYR5:
            z = rng.uniform(0, 0.8)
            x = np.array([rng.uniform(-0.9, 0.9) * (1 - z), rng.uniform(-0.9, 0.9) * (1 - z), z])
        else:
            x = rng.uniform(-1, 1, 3)
        N, dN = O.shape(t, x)
        assert abs(N.sum() - 1.0) < 1e-14  # partition of unity
        assert np.allclose(dN.sum(axis=0), 0.0, atol=1e-13)
        eps = 1e-6
        for j in range(3):  # derivative against central differences
            e = np.zeros(3)
            e[j] = eps
            fd = (O.shape(t, x + e)[0] - O.shape(t, x - e)[0]) / (2 * eps)
            assert np.allclose(dN[:, j], fd, atol=1e-8)


@pytest.mark.parametrize("t", TYPES)
def test_quadrature(t):
    check_quadrature(t)


@pytest.mark.parametrize("t", TYPES)
def test_shape_functions(t):
    check_shape_functions(t, np.random.default_rng(1))


# ------------------------------------------------------------------ closed-form element matrices

def lagrange_1d(nodes):
    """Lagrange basis polynomials on the given nodes (numpy polynomial coefficients)."""
    basis = []
    for i, xi in enumerate(nodes):
        c = np.array([1.0])
        for m, xm in enumerate(nodes):
            if m != i:
                c = P.polymul(c, np.array([-xm, 1.0]) / (xi - xm))
        basis.append(c)
    return basis


def matrices_1d(H, order):
    """Exact 1-D mass, stiffness and convection (int l_a l_b') matrices on [0, H]."""
    nodes = np.linspace(0.0, H, order + 1)
    L = lagrange_1d(nodes)
    dL = [P.polyder(c) for c in L]

    def integ(c):
        ci = P.polyint(c)
        return P.polyval(H, ci) - P.polyval(0.0, ci)

    q = order + 1
    M = np.array([[integ(P.polymul(L[a], L[b])) for b in range(q)] for a in range(q)])
    K = np.array([[integ(P.polymul(dL[a], dL[b])) for b in range(q)] for a in range(q)])
    Cv = np.array([[integ(P.polymul(L[a], dL[b])) for b in range(q)] for a in range(q)])
    return M, K, Cv


def box_element(t, H):
    q = 2 if t == O.HEX8 else 3
    pts = [np.linspace(0, H[d], q) for d in range(3)]
    return np.array([[pts[0][i], pts[1][j], pts[2][k]] for k in range(q) for j in range(q) for i in range(q)])


def element_terms(t, xe, ue, k, s, phi, dt, terms):
    nen = xe.shape[0]
    return O.element(t, xe, ue, np.full(nen, k), np.full(nen, s), phi, dt, terms)


def check_box_closed_forms(t):
    H = (0.7, 1.3, 0.45)  # distinct sides catch axis mix-ups
    order = 1 if t == O.HEX8 else 2
    xe = box_element(t, H)
    nen = xe.shape[0]
    u = np.array([0.3, -0.8, 0.55])
    ue = np.tile(u, (nen, 1))
    phi = np.linspace(0.1, 0.9, nen)
    m = [matrices_1d(H[d], order) for d in range(3)]
    Mx, My, Mz = m[0][0], m[1][0], m[2][0]
    M = np.kron(Mz, np.kron(My, Mx))
    K = (np.kron(Mz, np.kron(My, m[0][1])) + np.kron(Mz, np.kron(m[1][1], Mx)) + np.kron(m[2][1], np.kron(My, Mx)))
    Cv = (u[0] * np.kron(Mz, np.kron(My, m[0][2])) + u[1] * np.kron(Mz, np.kron(m[1][2], Mx)) +
          u[2] * np.kron(m[2][2], np.kron(My, Mx)))
    scale = np.abs(M).max()
    A, b = element_terms(t, xe, ue, 0.0, 0.0, phi, 1.0, O.MASS)
    assert np.allclose(A, M, rtol=0, atol=1e-13 * scale)
    assert np.allclose(b, M @ phi, rtol=0, atol=1e-13 * scale)
    A, _ = element_terms(t, xe, ue, 0.37, 0.0, phi, 1.0, O.DIFF)
    assert np.allclose(A, 0.37 * K, rtol=0, atol=1e-12 * np.abs(K).max())
    A, _ = element_terms(t, xe, ue, 0.0, 0.0, phi, 1.0, O.CONV)
    assert np.allclose(A, Cv, rtol=0, atol=1e-12 * np.abs(Cv).max())
    A, _ = element_terms(t, xe, ue, 0.0, 4.2, phi, 1.0, O.REAC)
    assert np.allclose(A, 4.2 * M, rtol=0, atol=1e-12 * 4.2 * scale)
    A, _ = element_terms(t, xe, ue, 0.0, 0.0, phi, 0.25, O.MASS)
    assert np.allclose(A, M / 0.25, rtol=0, atol=1e-12 * scale / 0.25)


def check_prism_closed_forms():
    """A right prism (legs a, b of the triangle in the x-y plane, length c along z): the mass and
    stiffness matrices are Kronecker products of the linear triangle's and the linear line's
    (node i + 3k: vertex i of the triangle at end k), which the 3 x 2 rule integrates exactly."""
    a, b, c = 0.8, 0.5, 1.3
    tri = np.array([[0, 0], [a, 0], [0, b]], float)
    xe = np.array([[x, y, z] for z in (0.0, c) for x, y in tri])
    area = a * b / 2
    Mt = area / 12 * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]])
    g = np.array([[-1 / a, -1 / b], [1 / a, 0], [0, 1 / b]])  # gradients of the triangle's barycentrics
    Kt = area * g @ g.T
    Ml = c / 6 * np.array([[2, 1], [1, 2]])
    Kl = 1 / c * np.array([[1, -1], [-1, 1]])
    M = np.kron(Ml, Mt)
    K = np.kron(Ml, Kt) + np.kron(Kl, Mt)
    ue = np.zeros((6, 3))
    phi = np.linspace(0.2, 0.7, 6)
    A, bb = element_terms(O.PEN6, xe, ue, 0.0, 0.0, phi, 1.0, O.MASS)
    assert np.allclose(A, M, rtol=0, atol=1e-14 * np.abs(M).max())
    assert np.allclose(bb, M @ phi, rtol=0, atol=1e-14 * np.abs(M).max())
    A, _ = element_terms(O.PEN6, xe, ue, 0.6, 0.0, phi, 1.0, O.DIFF)
    assert np.allclose(A, 0.6 * K, rtol=0, atol=1e-13 * np.abs(K).max())


@functools.lru_cache(maxsize=1)
def pyramid_reference_integrals():
    """Exact mass and stiffness integrals of the reference pyramid's functions, by sympy in the
    collapsed coordinates x = r (1 - z), y = t (1 - z) (dx dy dz = (1 - z)^2 dr dt dz), where the
    functions and their derivatives are polynomials."""
    import sympy as spy
    r, t, z = spy.symbols("r t z")
    sx, sy = [-1, 1, 1, -1], [-1, -1, 1, 1]
    N, dx, dy, dz = [], [], [], []
    for a in range(4):  # base corner a, in collapsed form (1 - z)(1 + sx r)(1 + sy t) / 4
        N.append((1 - z) * (1 + sx[a] * r) * (1 + sy[a] * t) / 4)
        dx.append((sx[a] + sx[a] * sy[a] * t) / 4)
        dy.append((sy[a] + sx[a] * sy[a] * r) / 4)
        dz.append((-1 + sx[a] * sy[a] * r * t) / 4)
    N.append(z)
    dx.append(spy.Integer(0))
    dy.append(spy.Integer(0))
    dz.append(spy.Integer(1))

    def integral(f):
        return float(spy.integrate(f * (1 - z) ** 2, (r, -1, 1), (t, -1, 1), (z, 0, 1)))
    M = np.array([[integral(N[i] * N[j]) for j in range(5)] for i in range(5)])
    Kxy = np.array([[integral(dx[i] * dx[j] + dy[i] * dy[j]) for j in range(5)] for i in range(5)])
    Kz = np.array([[integral(dz[i] * dz[j]) for j in range(5)] for i in range(5)])
    return M, Kxy, Kz


def check_pyramid_closed_forms():
    """An affine pyramid (base [-s, s]^2 at z = 0, apex at height H): mass = s^2 H M_ref and
    stiffness = H K_xy,ref + (s^2 / H) K_z,ref, from the exact reference integrals."""
    s_, H = 0.6, 0.9
    xe = np.array([[-s_, -s_, 0], [s_, -s_, 0], [s_, s_, 0], [-s_, s_, 0], [0, 0, H]], float)
    Mr, Kxy, Kz = pyramid_reference_integrals()
    M = s_ * s_ * H * Mr
    K = H * Kxy + s_ * s_ / H * Kz
    ue = np.zeros((5, 3))
    phi = np.linspace(0.1, 0.5, 5)
    A, bb = element_terms(O.PYR5, xe, ue, 0.0, 0.0, phi, 1.0, O.MASS)
    assert np.allclose(A, M, rtol=0, atol=1e-14 * np.abs(M).max())
    assert np.allclose(bb, M @ phi, rtol=0, atol=1e-14 * np.abs(M).max())
    A, _ = element_terms(O.PYR5, xe, ue, 0.45, 0.0, phi, 1.0, O.DIFF)
    assert np.allclose(A, 0.45 * K, rtol=0, atol=1e-13 * np.abs(K).max())


def lagrange_1d_from_roots(q):
    """The 1-D Lagrange bases on q equispaced nodes of [-1, 1] (q = 2 or 3), built from their
    roots, with their derivatives."""
    nodes = np.linspace(-1.0, 1.0, q)
    basis = []
    for i in range(q):
        others = np.delete(nodes, i)
        p = np.poly1d(others, r=True) / np.prod(nodes[i] - others)
        basis.append((p, p.deriv()))
    return nodes, basis


def gl01(n):
    """n-point Gauss-Legendre rule on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1.0) / 2.0, w / 2.0


def high_order_points(t):
    """Points of a high-order rule on the reference element, as (weight, N, grad_xi N): tensor
    Gauss-Legendre for the hexahedra; the tetrahedron, the prism's triangle and the pyramid
    integrated in collapsed (Duffy) coordinates, where the integrands of affine elements are
    polynomials.  The shape functions are written here from their definitions (tensor-product
    Lagrange bases; barycentrics; triangle x line; the pyramid's functions in collapsed form)."""
    pts = []
    g5, w5 = np.polynomial.legendre.leggauss(5)
    r6, w6 = gl01(6)
    if t in (O.HEX8, O.HEX27):
        q = 2 if t == O.HEX8 else 3
        _, basis = lagrange_1d_from_roots(q)
        idx = [(i, j, k) for k in range(q) for j in range(q) for i in range(q)]
        for a1, w1 in zip(g5, w5):
            for a2, w2 in zip(g5, w5):
                for a3, w3 in zip(g5, w5):
                    xi = (a1, a2, a3)
                    v = [[basis[i][d == 0](xi[0]) * basis[j][d == 1](xi[1]) * basis[k][d == 2](xi[2])
                          for i, j, k in idx] for d in (-1, 0, 1, 2)]
                    pts.append((w1 * w2 * w3, np.array(v[0]), np.array(v[1:]).T))
    elif t == O.TET4:  # xi = a, eta = b (1 - a), zeta = c (1 - a)(1 - b)
        dN = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
        for a, wa in zip(r6, w6):
            for b, wb in zip(r6, w6):
                for c, wc in zip(r6, w6):
                    x, y, z = a, b * (1 - a), c * (1 - a) * (1 - b)
                    pts.append((wa * wb * wc * (1 - a) ** 2 * (1 - b), np.array([1 - x - y - z, x, y, z]), dN))
    elif t == O.PEN6:  # triangle (xi, eta) = (a, b (1 - a)) times zeta in [-1, 1]
        for a, wa in zip(r6, w6):
            for b, wb in zip(r6, w6):
                x, y = a, b * (1 - a)
                L = np.array([1 - x - y, x, y])
                dL = np.array([[-1, -1], [1, 0], [0, 1]], float)
                for z, wz in zip(g5, w5):
                    lo, hi = (1 - z) / 2, (1 + z) / 2
                    N = np.concatenate([L * lo, L * hi])
                    dN = np.vstack([np.column_stack([dL * lo, -L / 2]), np.column_stack([dL * hi, L / 2])])
                    pts.append((wa * wb * wz * (1 - a), N, dN))
    else:  # pyramid: x = r (1 - z), y = s (1 - z), dV = (1 - z)^2 dr ds dz
        sx, sy = np.array([-1, 1, 1, -1.0]), np.array([-1, -1, 1, 1.0])
        for r, wr in zip(g5, w5):
            for s_, ws in zip(g5, w5):
                for z, wz in zip(r6, w6):
                    N = np.append((1 - z) * (1 + sx * r) * (1 + sy * s_) / 4, z)
                    dN = np.vstack([np.column_stack([(sx + sx * sy * s_) / 4, (sy + sx * sy * r) / 4,
                                                     (-1 + sx * sy * r * s_) / 4]), [0.0, 0.0, 1.0]])
                    pts.append((wr * ws * wz * (1 - z) ** 2, N, dN))
    return pts


def exact_ref_nodes(t):
    nodes = ref_nodes(t)
    if t == O.PYR5:
        nodes[4, 2] = 1.0
    return nodes


def check_affine_high_order(t, seed=4):
    """An affine, sheared element x = F xi + c with constant u, k and s: every term of the
    operator is then a polynomial (in collapsed coordinates for the tetrahedron, the prism's
    triangle and the pyramid) that the element's own rule integrates exactly, so the oracle's
    matrix and RHS must equal the same integrand under a rule of much higher order.  F is not
    symmetric, unlike a box's Jacobian, so F^-T and F^-1 differ."""
    rng = np.random.default_rng(seed)
    order = 2 if t == O.HEX27 else 1
    F = np.eye(3) * 0.6 + rng.uniform(-0.15, 0.15, (3, 3))
    assert np.linalg.det(F) > 0.1
    c = rng.uniform(-1, 1, 3)
    xe = exact_ref_nodes(t) @ F.T + c
    nen = xe.shape[0]
    u = np.array([0.7, -0.35, 0.5])
    kd, sr, dt = 0.08, 3.0, 0.05
    phi = rng.uniform(0, 1, nen)
    det = np.linalg.det(F)
    Ginv = np.linalg.inv(F).T
    pts = high_order_points(t)
    assert abs(sum(w for w, _, _ in pts) - REF_VOLUME[t]) < 1e-13
    h = (REF_VOLUME[t] * det) ** (1.0 / 3.0) / order
    tau = 1.0 / (4.0 * kd / h ** 2 + 2.0 * np.linalg.norm(u) / h + sr)
    A = np.zeros((nen, nen))
    b = np.zeros(nen)
    for w, N, dN in pts:
        grad = dN @ Ginv.T  # row a: F^-T grad_xi N_a
        ua = grad @ u
        dV = w * det
        A += dV * (np.outer(N, N) / dt + np.outer(N, ua) + kd * grad @ grad.T + sr * np.outer(N, N)
                   + tau * np.outer(ua, N / dt + ua + sr * N))
        b += dV * (N + tau * ua) * (N @ phi) / dt
    Ao, bo = element_terms(t, xe, np.tile(u, (nen, 1)), kd, sr, phi, dt, O.ALL_TERMS)
    assert np.abs(Ao - A).max() <= 1e-12 * np.abs(A).max()
    assert np.abs(bo - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("t", TYPES)
def test_affine_element_matches_high_order_rule(t):
    check_affine_high_order(t)


def test_prism_closed_forms():
    check_prism_closed_forms()


def test_pyramid_closed_forms():
    pytest.importorskip("sympy")
    check_pyramid_closed_forms()


def random_tet(rng):
    while True:
        x = rng.uniform(-1, 1, (4, 3))
        if np.linalg.det(np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]])) > 0.2:
            return x


def check_tet_closed_forms(rng):
    xe = random_tet(rng)
    V = np.linalg.det(np.stack([xe[1] - xe[0], xe[2] - xe[0], xe[3] - xe[0]])) / 6.0
    # barycentric gradients: rows 1..3 of inv([[1, x_a]]^T)
    T4 = np.hstack([np.ones((4, 1)), xe])
    grad = np.linalg.inv(T4)[1:, :].T  # (4, 3): grad lambda_a
    M = V / 20.0 * (np.ones((4, 4)) + np.eye(4))
    K = V * grad @ grad.T
    u = np.array([0.4, -0.2, 0.9])
    ue = np.tile(u, (4, 1))
    Cv = (V / 4.0) * np.tile(grad @ u, (4, 1))  # row a, column b: (V/4) u . grad lambda_b
    phi = np.array([0.2, 0.5, 0.1, 0.9])
    A, b = element_terms(O.TET4, xe, ue, 0.0, 0.0, phi, 1.0, O.MASS)
    assert np.allclose(A, M, atol=1e-14) and np.allclose(b, M @ phi, atol=1e-14)
    A, _ = element_terms(O.TET4, xe, ue, 0.9, 0.0, phi, 1.0, O.DIFF)
    assert np.allclose(A, 0.9 * K, atol=1e-13)
    A, _ = element_terms(O.TET4, xe, ue, 0.0, 0.0, phi, 1.0, O.CONV)
    assert np.allclose(A, Cv, atol=1e-13)
    A, _ = element_terms(O.TET4, xe, ue, 0.0, 3.0, phi, 1.0, O.REAC)
    assert np.allclose(A, 3.0 * M, atol=1e-13)


@pytest.mark.parametrize("t", (O.HEX8, O.HEX27))
def test_box_closed_forms(t):
    check_box_closed_forms(t)


def test_tet_closed_forms():
    rng = np.random.default_rng(7)
    for _ in range(5):
        check_tet_closed_forms(rng)


# ------------------------------------------------------------------ assembled-operator invariants

def small_mesh(t, n, frac, seed=3):
    mesh = G.structured_mesh(t, n)
    rng = np.random.default_rng(seed)
    G.perturb_interior(mesh, rng, frac)
    return mesh


def const_fields(n_node, coords, k=0.0, s=0.0, phi=None, u=None, dt=1.0):
    vel = np.zeros((3, n_node)) if u is None else (np.tile(np.asarray(u, float)[:, None], (1, n_node))
                                                   if np.ndim(u) == 1 else u)
    ph = np.zeros(n_node) if phi is None else phi
    return G.Fields(vel, np.full((1, n_node), k), np.full((1, n_node), s), ph[None, :].copy(), dt)


def csr(mesh, fields, terms):
    rp, ci, _ = O.pattern(mesh.elem_type, mesh.conn, mesh.n_node, with_pos=False)
    vals, rhs = O.assemble(mesh.elem_type, mesh.coords, mesh.conn, rp, ci, fields, terms)
    A = sp.csr_matrix((vals[0], ci, rp), shape=(mesh.n_node, mesh.n_node))
    return A, rhs[0]


INV_MESH = {O.TET4: (3, 0.2), O.HEX8: (3, 0.15), O.HEX27: (2, 0.1), O.PEN6: (3, 0.15), O.PYR5: (3, 0.15)}


def check_invariants(t):
    n, frac = INV_MESH[t]
    mesh = small_mesh(t, n, frac)
    N = mesh.n_node
    rng = np.random.default_rng(11)
    one = np.ones(N)
    uvar = G.velocity_field(mesh.coords)
    kvar = G.Fields(uvar, rng.uniform(0.01, 0.1, (1, N)), rng.uniform(0, 5, (1, N)), rng.uniform(0, 1, (1, N)), 1e-3)
    # diffusion and convection annihilate constants
    A, _ = csr(mesh, kvar, O.DIFF)
    assert np.abs(A @ one).max() < 1e-12 * abs(A).max()
    A, _ = csr(mesh, kvar, O.CONV)
    assert np.abs(A @ one).max() < 1e-12 * abs(A).max()
    # mass matrix entries sum to the volume of the unit cube
    M, _ = csr(mesh, const_fields(N, mesh.coords), O.MASS)
    assert abs(M.sum() - 1.0) < 1e-12
    # symmetry of mass, diffusion, reaction
    for terms in (O.MASS, O.DIFF, O.REAC):
        A, _ = csr(mesh, kvar, terms)
        assert abs(A - A.T).max() < 1e-13 * abs(A).max()
    # constant state is preserved: s = 0, phi_old = 1 -> A 1 = b
    f = G.Fields(uvar, kvar.diffusivity, np.zeros((1, N)), np.ones((1, N)), 1e-3)
    A, b = csr(mesh, f, O.ALL_TERMS)
    assert np.abs(A @ one - b).max() < 1e-11 * np.abs(b).max()
    # SUPG sees a zero residual: constant s, phi = c, phi_old = c (1 + s dt)
    s0, c0, dt = 3.5, 0.7, 1e-3
    f = G.Fields(uvar, kvar.diffusivity, np.full((1, N), s0), np.full((1, N), c0 * (1 + s0 * dt)), dt)
    A, b = csr(mesh, f, O.SUPG)
    assert np.abs(A @ (c0 * one) - b).max() < 1e-11 * np.abs(b).max()
    # SUPG zero residual for a linear field advected by a constant velocity
    g, u0 = np.array([0.3, -1.1, 0.6]), np.array([0.8, 0.2, -0.5])
    phi = mesh.coords @ g + 0.4
    f = const_fields(N, mesh.coords, k=0.02, s=0.0, phi=phi + dt * (u0 @ g), u=u0, dt=dt)
    A, b = csr(mesh, f, O.SUPG)
    assert np.abs(A @ phi - b).max() < 1e-10 * np.abs(b).max()
    # zero velocity switches SUPG off
    f0 = G.Fields(np.zeros((3, N)), kvar.diffusivity, kvar.reaction, kvar.phi_old, kvar.dt)
    A, b = csr(mesh, f0, O.ALL_TERMS)
    A2, b2 = csr(mesh, f0, O.ALL_TERMS & ~O.SUPG)
    assert abs(A - A2).max() == 0.0 and np.abs(b - b2).max() == 0.0
    # the convection term goes with the velocity linearly and the SUPG-free operator is the sum of its terms
    At, bt = csr(mesh, kvar, O.ALL_TERMS & ~O.SUPG)
    parts = [csr(mesh, kvar, tm) for tm in (O.MASS, O.CONV, O.DIFF, O.REAC)]
    assert abs(At - sum(p[0] for p in parts)).max() < 1e-12 * abs(At).max()
    assert np.abs(bt - parts[0][1]).max() < 1e-13 * np.abs(bt).max()


def check_scaling_translation(t):
    n, frac = INV_MESH[t]
    mesh = small_mesh(t, n, frac)
    N = mesh.n_node
    rng = np.random.default_rng(5)
    f = G.Fields(np.tile(np.array([[0.5], [0.1], [-0.3]]), (1, N)), rng.uniform(0.01, 0.1, (1, N)),
                 rng.uniform(0, 5, (1, N)), rng.uniform(0, 1, (1, N)), 1e-2)
    lam = 2.5
    big = G.Mesh(t, mesh.coords * lam, mesh.conn, mesh.n_cells, mesh.h * lam)
    for terms, power in ((O.MASS, 3), (O.REAC, 3), (O.CONV, 2), (O.DIFF, 1)):
        A, _ = csr(mesh, f, terms)
        B, _ = csr(big, f, terms)
        assert abs(B - lam ** power * A).max() < 1e-12 * abs(B).max()
    moved = G.Mesh(t, mesh.coords + np.array([3.0, -7.0, 11.0]), mesh.conn, mesh.n_cells, mesh.h)
    A, b = csr(mesh, f, O.ALL_TERMS)
    B, c = csr(moved, f, O.ALL_TERMS)
    assert abs(A - B).max() < 1e-10 * abs(A).max() and np.abs(b - c).max() < 1e-10 * np.abs(b).max()


@pytest.mark.parametrize("t", TYPES)
def test_invariants(t):
    check_invariants(t)


@pytest.mark.parametrize("t", TYPES)
def test_scaling_translation(t):
    check_scaling_translation(t)


# ------------------------------------------------------------------ patch test

# local faces: triangles as 3 nodes, quads as 2 x 2 arrays (tensor layout of the face's bilinear basis)
LOCAL_FACES = {
    O.TET4: [[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]],
    O.PEN6: [[0, 1, 2], [3, 4, 5], [[0, 1], [3, 4]], [[1, 2], [4, 5]], [[2, 0], [5, 3]]],
    O.PYR5: [[[0, 1], [3, 2]], [0, 1, 4], [1, 2, 4], [2, 3, 4], [3, 0, 4]],
}


def on_cube_boundary(x):
    return any(np.all(np.abs(x[:, d] - v) < 1e-12) for d in range(3) for v in (0.0, 1.0))


def boundary_faces_of(t, conn, coords):
    """Node arrays of the faces of elements of type t that lie on the boundary of the unit cube."""
    out = []
    if t in LOCAL_FACES:
        for e in conn:
            for f in LOCAL_FACES[t]:
                nodes = e[np.asarray(f)]
                if on_cube_boundary(coords[nodes.ravel()]):
                    out.append(nodes)
        return out
    q = 2 if t == O.HEX8 else 3
    for e in conn:
        loc = e.reshape(q, q, q)  # [k][j][i]
        for sl in (loc[0], loc[-1], loc[:, 0, :], loc[:, -1, :], loc[:, :, 0], loc[:, :, -1]):
            if on_cube_boundary(coords[sl.ravel()]):
                out.append(sl)
    return out


def boundary_faces(mesh):
    return boundary_faces_of(mesh.elem_type, mesh.conn, mesh.coords)


def boundary_flux_faces(faces, coords, n_node, kval, g):
    """f_i = int_dOmega N_i k g.n over planar boundary faces of the unit cube: a linear triangle
    gives each vertex a third of its area; a flat rectangle with the tensor basis of 2 or 3
    nodes per side takes the trapezoid or Simpson weights, which integrate it exactly."""
    f = np.zeros(n_node)
    for face in faces:
        arr = np.asarray(face)
        nodes = arr.ravel()
        x = coords[nodes]
        d = [d for d in range(3) if np.all(np.abs(x[:, d] - x[0, d]) < 1e-12)][0]
        n = np.zeros(3)
        n[d] = 1.0 if x[0, d] > 0.5 else -1.0
        if arr.ndim == 1:
            area = 0.5 * np.linalg.norm(np.cross(x[1] - x[0], x[2] - x[0]))
            w = np.full(3, area / 3.0)
        else:
            q = arr.shape[0]
            ext = [np.ptp(x[:, dd]) for dd in range(3) if dd != d]
            area = ext[0] * ext[1]
            w1 = np.array([0.5, 0.5]) if q == 2 else np.array([1.0, 4.0, 1.0]) / 6.0
            w = (np.outer(w1, w1) * area).ravel()
        f[nodes] += kval * (g @ n) * w
    return f


def boundary_flux(mesh, kval, g):
    return boundary_flux_faces(boundary_faces(mesh), mesh.coords, mesh.n_node, kval, g)


PATCH = [(O.TET4, 0.2), (O.HEX8, 0.15), (O.HEX27, 0.0), (O.PEN6, 0.15), (O.PYR5, 0.0)]


@pytest.mark.parametrize("t,frac", PATCH)
def test_patch_test(t, frac):
    check_patch(t, frac)


def check_patch(t, frac):
    n = 3 if t != O.HEX27 else 2
    mesh = small_mesh(t, n, frac)
    N = mesh.n_node
    g = np.array([0.7, -0.4, 1.3])
    phi = mesh.coords @ g + 0.25
    kval = 0.3
    f = const_fields(N, mesh.coords, k=kval)
    K, _ = csr(mesh, f, O.DIFF)
    got = K @ phi
    want = boundary_flux(mesh, kval, g)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


# ------------------------------------------------------------------ matrix-free, brute force, pattern

def check_matfree(t):
    n, frac = INV_MESH[t]
    mesh = small_mesh(t, n, frac)
    N = mesh.n_node
    rng = np.random.default_rng(9)
    f = G.Fields(G.velocity_field(mesh.coords), rng.uniform(0.01, 0.1, (1, N)), rng.uniform(0, 5, (1, N)),
                 rng.uniform(0, 1, (1, N)), 1e-3)
    A, _ = csr(mesh, f, O.ALL_TERMS)
    x = rng.standard_normal(N)
    y = O.apply(t, mesh.coords, mesh.conn, f, 0, x)
    assert np.abs(A @ x - y).max() < 1e-12 * np.abs(y).max()


def dense_bruteforce(mesh, f, terms):
    t, N = mesh.elem_type, mesh.n_node
    A = np.zeros((N, N))
    b = np.zeros(N)
    for e in mesh.conn:
        Ae, be = O.element(t, mesh.coords[e], f.velocity[:, e].T, f.diffusivity[0, e], f.reaction[0, e],
                           f.phi_old[0, e], f.dt, terms)
        for a in range(len(e)):
            b[e[a]] += be[a]
            for bb in range(len(e)):
                A[e[a], e[bb]] += Ae[a, bb]
    return A, b


def check_bruteforce(t):
    rng = np.random.default_rng(21)
    for n_el in (1, 2, 5, 8):
        mesh = G.structured_mesh(t, 2)
        mesh.conn = mesh.conn[rng.permutation(mesh.n_elem)[:n_el]]
        G.perturb_interior(mesh, rng, 0.1)
        N = mesh.n_node
        f = G.Fields(G.velocity_field(mesh.coords), rng.uniform(0.01, 0.1, (1, N)), rng.uniform(0, 5, (1, N)),
                     rng.uniform(0, 1, (1, N)), 1e-3)
        A, b = csr(mesh, f, O.ALL_TERMS)
        D, db = dense_bruteforce(mesh, f, O.ALL_TERMS)
        assert np.abs(A.toarray() - D).max() < 1e-12 * np.abs(D).max()
        assert np.abs(b - db).max() < 1e-12 * np.abs(db).max()
        # pattern = nonzero structure of (node-element incidence)(its transpose), diagonal of used nodes included
        inc = np.zeros((N, len(mesh.conn)))
        for i, e in enumerate(mesh.conn):
            inc[e, i] = 1.0
        S = (inc @ inc.T) > 0
        rp, ci, pos = O.pattern(t, mesh.conn, N)
        P_ = np.zeros((N, N), bool)
        for r in range(N):
            P_[r, ci[rp[r]:rp[r + 1]]] = True
            assert np.all(np.diff(ci[rp[r]:rp[r + 1]]) > 0)
        assert np.array_equal(S, P_)
        for e in range(len(mesh.conn)):
            for a in range(mesh.conn.shape[1]):
                for bb in range(mesh.conn.shape[1]):
                    k = pos[e, a, bb]
                    assert rp[mesh.conn[e, a]] <= k < rp[mesh.conn[e, a] + 1]
                    assert ci[k] == mesh.conn[e, bb]


def kuhn_nnz(n):
    m = n + 1
    edges = 3 * n * m * m + 3 * n * n * m + n ** 3  # axis edges + face diagonals + body diagonals
    return m ** 3 + 2 * edges


def tensor_nnz(n, order):
    m = order * n + 1
    rows = np.zeros(m, int)
    for c in range(n):  # 1-D pattern: nodes of one cell are all coupled
        idx = np.arange(order * c, order * c + order + 1)
        for i in idx:
            rows[i] = 0
    couple = np.zeros((m, m), bool)
    for c in range(n):
        idx = np.arange(order * c, order * c + order + 1)
        couple[np.ix_(idx, idx)] = True
    return int(couple.sum(axis=1).sum()) ** 3


def check_pattern_counts():
    for n in (2, 4, 10):
        m = G.structured_mesh(O.TET4, n)
        rp, ci, _ = O.pattern(O.TET4, m.conn, m.n_node, with_pos=False)
        assert rp[-1] == kuhn_nnz(n)
        inner = (n // 2) * (1 + (n + 1) + (n + 1) ** 2)
        assert rp[inner + 1] - rp[inner] == 15
    assert kuhn_nnz(10) == 17191 and kuhn_nnz(100) == 15210901
    for t, order, n, interior in ((O.HEX8, 1, 4, [27]), (O.HEX27, 2, 2, [125, 75, 45, 27])):
        m = G.structured_mesh(t, n)
        rp, ci, _ = O.pattern(t, m.conn, m.n_node, with_pos=False)
        assert rp[-1] == tensor_nnz(n, order)
        M = order * n + 1
        rows = np.diff(rp)
        if t == O.HEX8:
            assert rows[2 + 2 * M + 2 * M * M] == 27
        else:  # vertex (2,2,2), edge (1,2,2), face (1,1,2), centre (1,1,1) of the 2x2x2 grid of elements
            for (i, j, k), want in zip(((2, 2, 2), (1, 2, 2), (1, 1, 2), (1, 1, 1)), interior):
                assert rows[i + j * M + k * M * M] == want
    assert tensor_nnz(128, 1) == 57066625 and tensor_nnz(48, 2) == 57066625 and tensor_nnz(256, 1) == 454756609


@pytest.mark.parametrize("t", TYPES)
def test_matfree_equals_spmv(t):
    check_matfree(t)


@pytest.mark.parametrize("t", TYPES)
def test_bruteforce_small_meshes(t):
    check_bruteforce(t)


def test_pattern_counts():
    check_pattern_counts()


def test_validation_codes():
    m = G.structured_mesh(O.TET4, 2)
    assert O.validate(O.TET4, m.coords, m.conn) == O.OK
    bad = m.conn.copy()
    bad[3, 1] = m.n_node
    assert O.validate(O.TET4, m.coords, bad) == O.ERR_RANGE
    bad = m.conn.copy()
    bad[3, 1] = bad[3, 2]
    assert O.validate(O.TET4, m.coords, bad) == O.ERR_DUP
    bad = m.conn.copy()
    bad[3, [1, 2]] = bad[3, [2, 1]]
    assert O.validate(O.TET4, m.coords, bad) == O.ERR_INVERTED
    h = G.structured_mesh(O.HEX8, 2)
    bad = h.conn.copy()
    bad[0, [0, 1]] = bad[0, [1, 0]]
    assert O.validate(O.HEX8, h.coords, bad) == O.ERR_INVERTED


# ------------------------------------------------------------------ mixed element types

def check_mixed():
    """A mesh of Hex8, Pyr5 and Pen6 blocks: its pattern is the incidence product over all
    blocks; the mass matrix sums to the cube's volume; diffusion and convection annihilate
    constants; the constant state is preserved; the patch test holds against the boundary
    flux of all blocks' faces; matrix-free equals SpMV."""
    mm = G.mixed_mesh(3)
    G.perturb_interior(mm, np.random.default_rng(4), 0.1)
    N = mm.n_node
    rp, ci, pos = O.pattern_mixed(mm.blocks, N)
    inc = np.zeros((N, mm.n_elem))
    e0 = 0
    for t, conn in mm.blocks:
        for i, e in enumerate(conn):
            inc[e, e0 + i] = 1.0
        e0 += conn.shape[0]
    S = (inc @ inc.T) > 0
    P_ = np.zeros((N, N), bool)
    for r in range(N):
        P_[r, ci[rp[r]:rp[r + 1]]] = True
    assert np.array_equal(S, P_)
    for (t, conn), pb in zip(mm.blocks, pos):
        assert np.array_equal(ci[pb], np.broadcast_to(conn[:, None, :], pb.shape))
    rng = np.random.default_rng(8)
    f = G.Fields(G.velocity_field(mm.coords), rng.uniform(0.01, 0.1, (1, N)), rng.uniform(0, 5, (1, N)),
                 rng.uniform(0, 1, (1, N)), 1e-3)

    def mat(fields, terms):
        v, b = O.assemble_mixed(mm.coords, mm.blocks, rp, ci, fields, terms)
        return sp.csr_matrix((v[0], ci, rp), shape=(N, N)), b[0]

    one = np.ones(N)
    M, _ = mat(f, O.MASS)
    assert abs(M.sum() / (1.0 / f.dt) - 1.0) < 1e-12
    for terms in (O.DIFF, O.CONV):
        A, _ = mat(f, terms)
        assert np.abs(A @ one).max() < 1e-12 * abs(A).max()
    fc = G.Fields(f.velocity, f.diffusivity, np.zeros((1, N)), np.ones((1, N)), f.dt)
    A, b = mat(fc, O.ALL_TERMS)
    assert np.abs(A @ one - b).max() < 1e-11 * np.abs(b).max()
    x = rng.standard_normal(N)
    A, _ = mat(f, O.ALL_TERMS)
    y = O.apply_mixed(mm.coords, mm.blocks, f, 0, x)
    assert np.abs(A @ x - y).max() < 1e-12 * np.abs(y).max()
    # patch test on the unperturbed mesh (the pyramids' rational functions are integrated exactly there)
    flat = G.mixed_mesh(3)
    rpf, cif, _ = O.pattern_mixed(flat.blocks, flat.n_node, with_pos=False)
    g, kval = np.array([0.7, -0.4, 1.3]), 0.3
    ff = const_fields(flat.n_node, flat.coords, k=kval)
    v, _ = O.assemble_mixed(flat.coords, flat.blocks, rpf, cif, ff, O.DIFF)
    K = sp.csr_matrix((v[0], cif, rpf), shape=(flat.n_node, flat.n_node))
    faces = [fc_ for t, conn in flat.blocks for fc_ in boundary_faces_of(t, conn, flat.coords)]
    want = boundary_flux_faces(faces, flat.coords, flat.n_node, kval, g)
    assert np.abs(K @ (flat.coords @ g + 0.25) - want).max() < 1e-12 * np.abs(want).max()


def test_mixed_element_types():
    check_mixed()


def test_solve_recovers_a_chosen_solution():
    """The direct solve on an assembled mass + diffusion system (symmetric positive definite)
    returns the vector the right-hand side was made from, and the residual of a random
    right-hand side's solution vanishes to rounding."""
    mesh = small_mesh(O.HEX8, 3, 0.15)
    N = mesh.n_node
    rng = np.random.default_rng(17)
    f = G.Fields(np.zeros((3, N)), rng.uniform(0.01, 0.1, (1, N)), np.zeros((1, N)), np.zeros((1, N)), 1.0)
    rp, ci, _ = O.pattern(O.HEX8, mesh.conn, N, with_pos=False)
    v, _ = O.assemble(O.HEX8, mesh.coords, mesh.conn, rp, ci, f, O.MASS | O.DIFF)
    A = sp.csr_matrix((v[0], ci, rp), shape=(N, N))
    assert abs(A - A.T).max() < 1e-15 * abs(A).max() and np.linalg.eigvalsh(A.toarray()).min() > 0
    x_true = rng.standard_normal(N)
    x = O.solve(rp, ci, v[0], A @ x_true)
    assert np.abs(x - x_true).max() < 1e-10 * np.abs(x_true).max()
    bb = rng.standard_normal(N)
    assert np.abs(A @ O.solve(rp, ci, v[0], bb) - bb).max() < 1e-12 * np.abs(bb).max()


# ------------------------------------------------------------------ planted mistakes

# ------------------------------------------------------------------ sampled rows and abs-sum denominators

def _fields_two_eq(rng, mesh, signed_phi=False):
    N = mesh.n_node
    lo = -1.0 if signed_phi else 0.0
    return G.Fields(G.velocity_field(mesh.coords), rng.uniform(0.01, 0.1, (2, N)), rng.uniform(0, 5, (2, N)),
                    rng.uniform(lo, 1, (2, N)), 1e-3)


def check_row_sampler(t):
    """RowSampler (the oracle's row-by-row path, ``or_row``: its own column list, local-index
    search and accumulation) gives every row of the whole-mesh assembly ``or_assemble`` (itself
    pinned by the checks above): the same columns, values, abs-sum denominators, RHS entry and
    RHS denominator, for two equations.  Node and element ids are permuted, so neither the local
    index of a row's node nor the order of its incident elements is the natural one (Sec. 4.2:
    the CSR rows both paths build)."""
    n, frac = INV_MESH[t]
    mesh = small_mesh(t, n, frac, seed=17)
    rng = np.random.default_rng(23)
    G.permute_nodes(mesh, rng.permutation(mesh.n_node).astype(np.int64))
    G.permute_elements(mesh, rng.permutation(mesh.n_elem).astype(np.int64))
    f = _fields_two_eq(rng, mesh, signed_phi=True)
    rp, ci, _ = O.pattern(t, mesh.conn, mesh.n_node, with_pos=False)
    vals, rhs, absA, absb = O.assemble(t, mesh.coords, mesh.conn, rp, ci, f, with_abs=True)
    rs = O.RowSampler(t, mesh.coords, mesh.conn, f)
    for r in range(mesh.n_node):
        cols, v, av, b, ab = rs.row(r)
        k0, k1 = rp[r], rp[r + 1]
        assert np.array_equal(cols, ci[k0:k1])
        for got, want in ((v, vals[:, k0:k1]), (av, absA[:, k0:k1]), (b, rhs[:, r]), (ab, absb[:, r])):
            assert np.abs(got - want).max() <= 1e-15 * np.abs(want).max()


def check_row_sampler_mixed():
    """On a mesh of Hex8, Pyr5 and Pen6 blocks, the rows RowSampler gives for each block, added
    into the union pattern, are the rows of the whole-mesh assembly of all blocks."""
    mm = G.mixed_mesh(3)
    G.perturb_interior(mm, np.random.default_rng(31), 0.1)
    N = mm.n_node
    rng = np.random.default_rng(32)
    f = G.Fields(G.velocity_field(mm.coords), rng.uniform(0.01, 0.1, (2, N)), rng.uniform(0, 5, (2, N)),
                 rng.uniform(-1, 1, (2, N)), 1e-3)
    rp, ci, _ = O.pattern_mixed(mm.blocks, N, with_pos=False)
    vals, rhs, absA, absb = O.assemble_mixed(mm.coords, mm.blocks, rp, ci, f, with_abs=True)
    samplers = [O.RowSampler(t, mm.coords, conn, f) for t, conn in mm.blocks]
    for r in range(N):
        k0, k1 = rp[r], rp[r + 1]
        v = np.zeros((2, k1 - k0))
        av = np.zeros_like(v)
        b = np.zeros(2)
        ab = np.zeros(2)
        for rs in samplers:
            cols, bv, bav, bb, bab = rs.row(r)
            idx = np.searchsorted(ci[k0:k1], cols)
            assert np.array_equal(ci[k0:k1][idx], cols)
            v[:, idx] += bv
            av[:, idx] += bav
            b += bb
            ab += bab
        for got, want in ((v, vals[:, k0:k1]), (av, absA[:, k0:k1]), (b, rhs[:, r]), (ab, absb[:, r])):
            assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


def check_abs_sums(t):
    """The abs-sum denominators of the parity tolerances: absA_ij = sum_e |A^e_ij| (the element
    matrices scattered densely by numpy, in magnitude), and absA >= |A|, absb >= |b| everywhere."""
    n, frac = INV_MESH[t]
    mesh = small_mesh(t, n, frac, seed=19)
    rng = np.random.default_rng(29)
    f = _fields_two_eq(rng, mesh, signed_phi=True)
    N = mesh.n_node
    rp, ci, _ = O.pattern(t, mesh.conn, N, with_pos=False)
    vals, rhs, absA, absb = O.assemble(t, mesh.coords, mesh.conn, rp, ci, f, with_abs=True)
    assert np.all(absA >= np.abs(vals)) and np.all(absb >= np.abs(rhs))
    assert np.any(absb > 1.5 * np.abs(rhs))  # signed fields: some RHS entries do cancel
    for q in range(2):
        dense = np.zeros((N, N))
        for e in mesh.conn:
            Ae, _ = O.element(t, mesh.coords[e], f.velocity[:, e].T, f.diffusivity[q, e], f.reaction[q, e],
                              f.phi_old[q, e], f.dt)
            dense[np.ix_(e, e)] += np.abs(Ae)
        got = sp.csr_matrix((absA[q], ci, rp), shape=(N, N)).toarray()
        assert np.abs(got - dense).max() <= 1e-13 * dense.max()


TET_BARY_A, TET_BARY_B = 0.5854101966249685, 0.1381966011250105


def check_abs_rhs_by_hand():
    """absb on two tetrahedra, summed by hand: for every element, Gauss point and node, the
    magnitudes of the Galerkin summand dV N_a phi_g/dt and of the SUPG summand
    dV tau (u_g.grad N_a) phi_g/dt.  The P1 gradients come from inverting the 4 x 4 matrix of
    barycentric coordinates, the points are the (a, b, b, b) barycentric points with dV = V/4,
    tau = 1/(4k/h^2 + 2|u|/h + s) with h = V^(1/3).  phi changes sign inside each element, so
    the summands of one node do have both signs (the sum of magnitudes exceeds |b|)."""
    coords = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1.2]], float)
    conn = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], np.int32)
    # the second tet: make it positively oriented
    x = coords[conn[1]]
    if np.dot(np.cross(x[1] - x[0], x[2] - x[0]), x[3] - x[0]) < 0:
        conn[1] = conn[1][[0, 2, 1, 3]]
    N = coords.shape[0]
    vel = np.array([[0.3, -0.2, 0.5, 0.1, 0.4], [0.1, 0.6, -0.3, 0.2, 0.0], [0.2, 0.2, 0.2, -0.5, 0.3]])
    k = np.array([[0.02, 0.05, 0.03, 0.04, 0.01]])
    s = np.array([[1.0, 2.0, 0.5, 3.0, 1.5]])
    phi = np.array([[1.0, -0.8, 0.6, -1.1, 0.9]])
    dt = 1e-2
    f = G.Fields(vel, k, s, phi, dt)
    rp, ci, _ = O.pattern(O.TET4, conn, N, with_pos=False)
    _, rhs, _, absb = O.assemble(O.TET4, coords, conn, rp, ci, f, with_abs=True)
    want_b = np.zeros(N)
    want_abs = np.zeros(N)
    signs = set()
    for e in conn:
        X = coords[e]
        M = np.hstack([np.ones((4, 1)), X])
        V = abs(np.linalg.det(M)) / 6.0
        grad = np.linalg.inv(M)[1:, :].T          # row a = grad of barycentric coordinate a
        h = V ** (1.0 / 3.0)
        for g in range(4):
            lam = np.full(4, TET_BARY_B)
            lam[g] = TET_BARY_A
            ug = vel[:, e] @ lam
            kg, sg, pg = k[0, e] @ lam, s[0, e] @ lam, phi[0, e] @ lam
            tau = 1.0 / (4 * kg / h ** 2 + 2 * np.linalg.norm(ug) / h + sg)
            dV = V / 4.0
            for a in range(4):
                gal = dV * lam[a] * pg / dt
                supg = dV * tau * (ug @ grad[a]) * pg / dt
                want_b[e[a]] += gal + supg
                want_abs[e[a]] += abs(gal) + abs(supg)
                signs.add((int(e[a]), np.sign(gal)))
    assert any((n, 1.0) in signs and (n, -1.0) in signs for n in range(N))
    assert np.any(want_abs > 1.2 * np.abs(want_b))
    assert np.allclose(rhs[0], want_b, rtol=1e-13, atol=0)
    assert np.allclose(absb[0], want_abs, rtol=1e-13, atol=0)


@pytest.mark.parametrize("t", TYPES)
def test_row_sampler_equals_assembly(t):
    check_row_sampler(t)


def test_row_sampler_mixed_mesh():
    check_row_sampler_mixed()


@pytest.mark.parametrize("t", TYPES)
def test_abs_sum_denominators(t):
    check_abs_sums(t)


def test_abs_rhs_summed_by_hand():
    check_abs_rhs_by_hand()


# ------------------------------------------------------------------ explicit time stepping

def check_explicit_step(t):
    """The explicit step against closed forms (Sec. 2: RK3 without a solver; lumped mass):
    - the lumped mass sums to the volume of the unit cube;
    - a constant field with u, k arbitrary and s = 0 stays constant (C 1 = K 1 = 0);
    - pure reaction s0 on a constant field c: the lumped system is dphi/dt = -s0 phi at every node,
      so one step gives c (1 - z) (Euler) or c (1 - z + z^2/2 - z^3/6) (RK3), z = s0 dt;
    - a linear field g.x + c under constant u, with k = s = 0: the Galerkin convection of a
      linear field is (u.g) int N_i, so every node moves by -dt u.g exactly, for both schemes."""
    n, frac = INV_MESH[t]
    mesh = small_mesh(t, n, frac, seed=41)
    N = mesh.n_node
    ml = O.lumped_mass(t, mesh.coords, mesh.conn)
    assert abs(ml.sum() - 1.0) < 1e-13 and np.all(ml > 0)
    rng = np.random.default_rng(43)
    u = G.velocity_field(mesh.coords)
    zero = np.zeros((1, N))
    f = G.Fields(u, rng.uniform(0.01, 0.1, (1, N)), zero, zero, 1e-3)
    const = np.full((1, N), 0.7)
    for st in (1, 3):
        out = O.explicit_step(t, mesh.coords, mesh.conn, f, const, 2e-3, st)
        assert np.abs(out - 0.7).max() < 1e-13
    s0, dt, c = 3.0, 0.05, 1.3
    fr = G.Fields(np.zeros((3, N)), zero, np.full((1, N), s0), zero, 1.0)
    z = s0 * dt
    e1 = O.explicit_step(t, mesh.coords, mesh.conn, fr, np.full((1, N), c), dt, 1)
    e3 = O.explicit_step(t, mesh.coords, mesh.conn, fr, np.full((1, N), c), dt, 3)
    assert np.abs(e1 - c * (1 - z)).max() < 1e-13
    assert np.abs(e3 - c * (1 - z + z * z / 2 - z ** 3 / 6)).max() < 1e-13
    g, u0 = np.array([0.4, -0.3, 0.9]), np.array([0.5, 0.2, -0.1])
    lin = (mesh.coords @ g + 0.25)[None, :]
    fc = G.Fields(np.tile(u0[:, None], (1, N)), zero, zero, zero, 1.0)
    for st in (1, 3):
        out = O.explicit_step(t, mesh.coords, mesh.conn, fc, lin, 0.01, st)
        assert np.abs(out - (lin - 0.01 * u0 @ g)).max() < 1e-13


@pytest.mark.parametrize("t", TYPES)
def test_explicit_step_closed_forms(t):
    check_explicit_step(t)


def all_pins():
    rng = np.random.default_rng(1)
    pins = []
    for t in TYPES:
        pins += [lambda t=t: check_quadrature(t), lambda t=t: check_shape_functions(t, rng),
                 lambda t=t: check_invariants(t), lambda t=t: check_matfree(t),
                 lambda t=t: check_scaling_translation(t)]
    pins += [lambda: check_box_closed_forms(O.HEX8), lambda: check_box_closed_forms(O.HEX27),
             lambda: check_tet_closed_forms(np.random.default_rng(7)), check_pattern_counts,
             lambda: check_bruteforce(O.HEX8), check_mixed, check_prism_closed_forms,
             *[lambda t=t: check_affine_high_order(t) for t in TYPES],
             *[lambda t=t: check_row_sampler(t) for t in TYPES], check_row_sampler_mixed,
             *[lambda t=t: check_abs_sums(t) for t in TYPES], check_abs_rhs_by_hand,
             *[lambda t=t: check_explicit_step(t) for t in TYPES]]
    try:
        import sympy  # noqa: F401  (the pyramid's exact integrals)
        pins.append(check_pyramid_closed_forms)
    except ImportError:
        pass
    pins += [lambda t=t, fr=fr: check_patch(t, fr) for t, fr in PATCH]
    return pins


def test_field_update_closed_forms():
    """The per-step perturbation at points where sin has a known value: zero amplitude
    leaves phi unchanged; k = 0 adds A sin(psi) everywhere; on the plane k . x + psi = pi
    the update vanishes, and a quarter period further it adds exactly A."""
    rng = np.random.default_rng(5)
    coords = rng.random((40, 3))
    phi = rng.random((3, 40))
    p = np.array([[0.0, 3.0, -1.0, 2.0, 0.7],      # A = 0
                  [0.25, 0.0, 0.0, 0.0, np.pi / 6],  # k = 0: + A/2
                  [0.5, 2.0, 0.0, 0.0, 0.0]])       # sin(2x)
    out = O.update_fields(coords, phi, p)
    assert np.array_equal(out[0], phi[0])
    assert np.allclose(out[1], phi[1] + 0.125, rtol=0, atol=1e-15)
    # nodes on x = pi/2 (2x = pi) and x = pi/4 (2x = pi/2)
    c2 = np.array([[np.pi / 2, 0.3, 0.9], [np.pi / 4, 0.1, 0.2]])
    o2 = O.update_fields(c2, np.zeros((3, 2)), p)
    assert abs(o2[2, 0]) < 1e-15 and abs(o2[2, 1] - 0.5) < 1e-15
    # linear in A; steps compose additively
    half = p.copy()
    half[:, 0] *= 0.5
    twice = O.update_fields(coords, O.update_fields(coords, phi, half), half)
    assert np.allclose(twice, out, rtol=0, atol=1e-14)


MUTATIONS = {
    1: "diffusion term dropped",
    2: "convection sign flipped",
    3: "convection operands transposed",
    4: "physical gradient uses J^-1 instead of J^-T",
    5: "wrong tetrahedron quadrature weight",
    6: "SUPG part of the RHS dropped",
    7: "reaction term dropped from the SUPG residual",
    8: "diagonal missing from the pattern",
    9: "element matrix scattered transposed",
    10: "mass term uses N_a N_a",
    11: "quadratic 1-D nodes in the wrong order",
    12: "pyramid rule without the collapse factor (1 - zeta)^2",
    13: "prism triangle functions permuted, derivatives not",
    14: "sampled row uses the wrong local index of its node",
    15: "sampled row skips an incident element",
    16: "RHS denominator sums the Galerkin summands with their signs",
    17: "matrix denominator sums the element entries with their signs",
}


@pytest.mark.parametrize("m", sorted(MUTATIONS))
def test_pins_catch_planted_mistakes(m):
    failed = 0
    with O.mutation(m):
        for pin in all_pins():
            try:
                pin()
            except (AssertionError, ValueError):
                failed += 1
    assert failed > 0, f"no pin caught mutation {m}: {MUTATIONS[m]}"
