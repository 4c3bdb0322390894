/*
 * fea_oracle.c -- plain FP64 CPU oracle for finite-element assembly of
 * convection-diffusion-reaction (CDR) transport equations into CSR.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code, header,
 * table or constant with the CUDA library: every shape function, quadrature
 * point and element term is written out here again, from its definition, in
 * double precision, with no blocking, fusion or reordering.
 *
 * What it follows (arXiv 2107.11541):
 *   - Sec. 4.2, Listing 1: element-by-element assembly, outer loop over
 *     elements, inner loop over Gauss points and node pairs, Ae(a,b) +=
 *     Jac(g) N(a,g) N(b,g).  Jac(g) is read as w_g * det J_g.
 *   - Sec. 4.2: the global matrix is stored in CSR.
 *   - Sec. 2 and Sec. 4.2: the meshes are unstructured and mix element kinds
 *     (tetrahedra, prisms, pyramids, hexahedra).  Element types here: Tet4,
 *     Hex8, Hex27, Pen6 (linear prism: triangle x line) and Pyr5 (linear
 *     pyramid with rational base functions, integrated on a collapsed cube).
 *     The paper gives no shape functions or rules; these are textbook ones.
 *     A mesh of several types is a list of single-type blocks (the Python
 *     wrapper sums their contributions into one CSR pattern).
 *   - Sec. 2: heat and species transport equations assembled every step.
 *     The paper does not write these equations; the operator used is the
 *     backward-Euler Galerkin + SUPG discretisation of
 *        d(phi)/dt + u.grad(phi) - div(k grad(phi)) + s phi = 0
 *     (readings listed in the design notes).
 *
 * Element matrix (per Gauss point g, dV = w_g det J_g), evaluated term by term:
 *   MASS : dV N_a N_b / dt
 *   CONV : dV N_a (u_g . grad N_b)
 *   DIFF : dV k_g grad N_a . grad N_b
 *   REAC : dV s_g N_a N_b
 *   SUPG : dV tau_g (u_g . grad N_a) (N_b/dt + u_g . grad N_b + s_g N_b)
 * RHS:   MASS part dV N_a phi_g / dt, SUPG part dV tau_g (u_g.grad N_a) phi_g / dt.
 * tau_g = 1 / (4 k_g / h^2 + 2 |u_g| / h + s_g)  (0 when the denominator is 0),
 * h = V_e^(1/3) / p with V_e = sum_g dV and p the polynomial order.
 * Parity unpinned: the constants of tau (4, 2) and the element length h are not
 * fixed by the paper; only their use inside the SUPG term is pinned (by the
 * constant-state and zero-residual checks).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_TET4 = 0, OR_HEX8 = 1, OR_HEX27 = 2, OR_PEN6 = 3, OR_PYR5 = 4 };
enum { OR_MASS = 1, OR_CONV = 2, OR_DIFF = 4, OR_REAC = 8, OR_SUPG = 16, OR_ALL = 31 };
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_RANGE = 2, OR_ERR_DUP = 3, OR_ERR_INVERTED = 4, OR_ERR_CAP = 5 };

#define MAXN 27

/* Deliberate mistakes, for the tests that show the pins catch plausible errors.
 * They exist only in a second, test-only build compiled with -DOR_MUTATION; in the
 * oracle itself MUT(k) is the constant 0 and every planted branch compiles away. */
#ifdef OR_MUTATION
static int g_mutation = 0;
#define MUT(k) (g_mutation == (k))
void or_set_mutation(int m) { g_mutation = m; }
int or_get_mutation(void) { return g_mutation; }
#else
#define MUT(k) 0
#endif

/* ---------------------------------------------------------------- reference elements */

/* 1-D Lagrange basis on the equispaced nodes of [-1, 1] (order 1: -1, 1;
 * order 2: -1, 0, 1), by the product formula, and its derivative. */
static void lagrange1d(int order, int i, double t, double* val, double* der) {
  double nodes[3];
  int q = order + 1;
  for (int m = 0; m < q; ++m) nodes[m] = -1.0 + 2.0 * m / order;
  if (MUT(11) && order == 2) { double s = nodes[1]; nodes[1] = nodes[2]; nodes[2] = s; }
  double v = 1.0;
  for (int m = 0; m < q; ++m)
    if (m != i) v *= (t - nodes[m]) / (nodes[i] - nodes[m]);
  double d = 0.0;
  for (int l = 0; l < q; ++l) {
    if (l == i) continue;
    double term = 1.0 / (nodes[i] - nodes[l]);
    for (int m = 0; m < q; ++m)
      if (m != i && m != l) term *= (t - nodes[m]) / (nodes[i] - nodes[m]);
    d += term;
  }
  *val = v;
  *der = d;
}

int or_nen(int type) {
  return type == OR_TET4 ? 4 : type == OR_HEX8 ? 8 : type == OR_HEX27 ? 27 : type == OR_PEN6 ? 6 : type == OR_PYR5 ? 5 : 0;
}
int or_order(int type) { return type == OR_HEX27 ? 2 : 1; }

/* Shape functions N[a] and reference derivatives dN[a][j] = dN_a/dxi_j at xi. */
int or_shape(int type, const double* xi, double* N, double* dN) {
  if (type == OR_TET4) {
    N[0] = 1.0 - xi[0] - xi[1] - xi[2];
    N[1] = xi[0];
    N[2] = xi[1];
    N[3] = xi[2];
    for (int a = 0; a < 4; ++a)
      for (int j = 0; j < 3; ++j) dN[a * 3 + j] = (a == 0) ? -1.0 : (a - 1 == j ? 1.0 : 0.0);
    return 4;
  }
  if (type == OR_PEN6) {
    /* prism: linear triangle in (xi, eta) times linear in zeta on [-1, 1]; node i + 3k is
     * triangle vertex i ((0,0), (1,0), (0,1)) on the face zeta = -1 (k = 0) or +1 (k = 1) */
    double L[3] = {1.0 - xi[0] - xi[1], xi[0], xi[1]};
    if (MUT(13)) { double t = L[0]; L[0] = L[1]; L[1] = t; }
    const double dLx[3] = {-1.0, 1.0, 0.0}, dLy[3] = {-1.0, 0.0, 1.0};
    const double l[2] = {0.5 * (1.0 - xi[2]), 0.5 * (1.0 + xi[2])}, dl[2] = {-0.5, 0.5};
    for (int k = 0; k < 2; ++k)
      for (int i = 0; i < 3; ++i) {
        int a = i + 3 * k;
        N[a] = L[i] * l[k];
        dN[a * 3 + 0] = dLx[i] * l[k];
        dN[a * 3 + 1] = dLy[i] * l[k];
        dN[a * 3 + 2] = L[i] * dl[k];
      }
    return 6;
  }
  if (type == OR_PYR5) {
    /* pyramid: square base [-1,1]^2 at zeta = 0 with corners (xi_a, eta_a) = (-1,-1), (1,-1),
     * (1,1), (-1,1), apex (0,0,1).  Base functions (1/4) [(1 - zeta) + xi_a xi + eta_a eta +
     * xi_a eta_a xi eta / (1 - zeta)], apex function zeta (rational, defined for zeta < 1). */
    const double sx[4] = {-1.0, 1.0, 1.0, -1.0}, sy[4] = {-1.0, -1.0, 1.0, 1.0};
    const double x = xi[0], y = xi[1], z = xi[2], c = 1.0 - z;
    for (int a = 0; a < 4; ++a) {
      N[a] = 0.25 * (c + sx[a] * x + sy[a] * y + sx[a] * sy[a] * x * y / c);
      dN[a * 3 + 0] = 0.25 * (sx[a] + sx[a] * sy[a] * y / c);
      dN[a * 3 + 1] = 0.25 * (sy[a] + sx[a] * sy[a] * x / c);
      dN[a * 3 + 2] = 0.25 * (-1.0 + sx[a] * sy[a] * x * y / (c * c));
    }
    N[4] = z;
    dN[12] = 0.0;
    dN[13] = 0.0;
    dN[14] = 1.0;
    return 5;
  }
  if (type != OR_HEX8 && type != OR_HEX27) return 0;
  int order = or_order(type), q = order + 1;
  double l[3][3], dl[3][3];
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < q; ++i) lagrange1d(order, i, xi[d], &l[d][i], &dl[d][i]);
  int a = 0;
  for (int k = 0; k < q; ++k)
    for (int j = 0; j < q; ++j)
      for (int i = 0; i < q; ++i, ++a) {
        N[a] = l[0][i] * l[1][j] * l[2][k];
        dN[a * 3 + 0] = dl[0][i] * l[1][j] * l[2][k];
        dN[a * 3 + 1] = l[0][i] * dl[1][j] * l[2][k];
        dN[a * 3 + 2] = l[0][i] * l[1][j] * dl[2][k];
      }
  return a;
}

/* Quadrature: Tet4 4-point rule (barycentric (a,b,b,b) permutations, point g has
 * weight a on vertex g, weights 1/24); Hex8 2x2x2 and Hex27 3x3x3 Gauss-Legendre,
 * points ordered lexicographically with x fastest. */
int or_quadrature(int type, double* xi, double* w) {
  if (type == OR_TET4) {
    const double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;
    for (int g = 0; g < 4; ++g) {
      double lam[4] = {b, b, b, b};
      lam[g] = a;
      xi[g * 3 + 0] = lam[1];
      xi[g * 3 + 1] = lam[2];
      xi[g * 3 + 2] = lam[3];
      w[g] = (MUT(5)) ? 1.0 / 6.0 : 1.0 / 24.0;
    }
    return 4;
  }
  if (type == OR_PEN6) {
    /* triangle rule of degree 2 (points (1/6,1/6), (2/3,1/6), (1/6,2/3), weight 1/6 each)
     * times 2-point Gauss-Legendre in zeta; point t + 3k */
    const double tp[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
    const double zp[2] = {-1.0 / sqrt(3.0), 1.0 / sqrt(3.0)};
    for (int k = 0; k < 2; ++k)
      for (int t = 0; t < 3; ++t) {
        int g = t + 3 * k;
        xi[g * 3 + 0] = tp[t][0];
        xi[g * 3 + 1] = tp[t][1];
        xi[g * 3 + 2] = zp[k];
        w[g] = 1.0 / 6.0;
      }
    return 6;
  }
  if (type == OR_PYR5) {
    /* collapsed cube: xi = r (1 - zeta), eta = s (1 - zeta), dxi deta dzeta = (1 - zeta)^2 dr ds
     * dzeta; 2-point Gauss-Legendre in r and s, 3-point Gauss-Legendre in zeta mapped to [0, 1];
     * point i + 2j + 4k (r fastest) */
    const double rp[2] = {-1.0 / sqrt(3.0), 1.0 / sqrt(3.0)};
    const double zt[3] = {-sqrt(0.6), 0.0, sqrt(0.6)}, zw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i) {
          int g = i + 2 * j + 4 * k;
          double z = 0.5 * (1.0 + zt[k]), c = 1.0 - z;
          xi[g * 3 + 0] = rp[i] * c;
          xi[g * 3 + 1] = rp[j] * c;
          xi[g * 3 + 2] = z;
          w[g] = 0.5 * zw[k] * (MUT(12) ? 1.0 : c * c);
        }
    return 12;
  }
  double p[3], pw[3];
  int q;
  if (type == OR_HEX8) {
    q = 2;
    p[0] = -1.0 / sqrt(3.0); p[1] = 1.0 / sqrt(3.0);
    pw[0] = pw[1] = 1.0;
  } else if (type == OR_HEX27) {
    q = 3;
    p[0] = -sqrt(0.6); p[1] = 0.0; p[2] = sqrt(0.6);
    pw[0] = 5.0 / 9.0; pw[1] = 8.0 / 9.0; pw[2] = 5.0 / 9.0;
  } else {
    return 0;
  }
  int g = 0;
  for (int k = 0; k < q; ++k)
    for (int j = 0; j < q; ++j)
      for (int i = 0; i < q; ++i, ++g) {
        xi[g * 3 + 0] = p[i];
        xi[g * 3 + 1] = p[j];
        xi[g * 3 + 2] = p[k];
        w[g] = pw[i] * pw[j] * pw[k];
      }
  return g;
}

/* Reference corner points used by the orientation check (the pyramid's base corners only:
 * its rational functions are singular at the apex). */
static int corner_points(int type, double* xi) {
  if (type == OR_TET4) {
    const double c[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    memcpy(xi, c, sizeof(c));
    return 4;
  }
  if (type == OR_PEN6) {
    const double c[6][3] = {{0, 0, -1}, {1, 0, -1}, {0, 1, -1}, {0, 0, 1}, {1, 0, 1}, {0, 1, 1}};
    memcpy(xi, c, sizeof(c));
    return 6;
  }
  if (type == OR_PYR5) {
    const double c[4][3] = {{-1, -1, 0}, {1, -1, 0}, {1, 1, 0}, {-1, 1, 0}};
    memcpy(xi, c, sizeof(c));
    return 4;
  }
  int n = 0;
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < 2; ++j)
      for (int i = 0; i < 2; ++i, ++n) {
        xi[n * 3 + 0] = i ? 1.0 : -1.0;
        xi[n * 3 + 1] = j ? 1.0 : -1.0;
        xi[n * 3 + 2] = k ? 1.0 : -1.0;
      }
  return 8;
}

/* ---------------------------------------------------------------- geometry */

/* J_ij = sum_a x_{a,i} dN_a/dxi_j at one point; returns det J. */
static double jacobian(int nen, const double* xe, const double* dN, double J[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int a = 0; a < nen; ++a) s += xe[a * 3 + i] * dN[a * 3 + j];
      J[i][j] = s;
    }
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* Inverse by the adjugate. */
static void inverse3(double J[3][3], double det, double Ji[3][3]) {
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
}

/* ---------------------------------------------------------------- element matrix */

/* Element matrix Ae[a*nen+b] and RHS be[a] of one equation from gathered nodal
 * data: xe[a*3+i] coordinates, ue[a*3+i] velocity, ke/se/phie nodal diffusivity,
 * reaction and previous-step values.  Only the terms in `terms` are added. */
static int element_impl(int type, const double* xe, const double* ue, const double* ke, const double* se,
                        const double* phie, double dt, int terms, double* Ae, double* be, double* babs);

int or_element(int type, const double* xe, const double* ue, const double* ke, const double* se,
               const double* phie, double dt, int terms, double* Ae, double* be) {
  return element_impl(type, xe, ue, ke, se, phie, dt, terms, Ae, be, NULL);
}

/* As or_element; babs[a] (if not NULL) receives sum_g |dV (N_a + tau u.grad N_a) phi_g / dt| over the
 * included RHS terms: the magnitude of the summands of b_a, which bounds its rounding error. */
static int element_impl(int type, const double* xe, const double* ue, const double* ke, const double* se,
                        const double* phie, double dt, int terms, double* Ae, double* be, double* babs) {
  int nen = or_nen(type);
  if (!nen || dt <= 0.0) return OR_ERR_ARG;
  double xq[MAXN * 3], wq[MAXN];
  int ng = or_quadrature(type, xq, wq);
  double N[MAXN][MAXN], dNr[MAXN][MAXN * 3];
  for (int g = 0; g < ng; ++g) or_shape(type, &xq[g * 3], N[g], dNr[g]);

  double gradN[MAXN][MAXN][3], dV[MAXN];
  double V = 0.0;
  for (int g = 0; g < ng; ++g) {
    double J[3][3], Ji[3][3];
    double det = jacobian(nen, xe, dNr[g], J);
    if (!(det > 0.0)) return OR_ERR_INVERTED;
    inverse3(J, det, Ji);
    for (int a = 0; a < nen; ++a)
      for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j)
          s += (MUT(4) ? Ji[i][j] : Ji[j][i]) * dNr[g][a * 3 + j];
        gradN[g][a][i] = s;
      }
    dV[g] = wq[g] * det;
    V += dV[g];
  }
  double h = cbrt(V) / or_order(type);

  for (int i = 0; i < nen * nen; ++i) Ae[i] = 0.0;
  for (int a = 0; a < nen; ++a) be[a] = 0.0;
  if (babs)
    for (int a = 0; a < nen; ++a) babs[a] = 0.0;

  for (int g = 0; g < ng; ++g) {
    const double* Ng = N[g];
    double ug[3] = {0, 0, 0}, kg = 0.0, sg = 0.0, pg = 0.0;
    for (int a = 0; a < nen; ++a) {
      for (int i = 0; i < 3; ++i) ug[i] += Ng[a] * ue[a * 3 + i];
      kg += Ng[a] * ke[a];
      sg += Ng[a] * se[a];
      pg += Ng[a] * phie[a];
    }
    double ua[MAXN];
    for (int a = 0; a < nen; ++a)
      ua[a] = ug[0] * gradN[g][a][0] + ug[1] * gradN[g][a][1] + ug[2] * gradN[g][a][2];
    double unorm = sqrt(ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2]);
    double den = 4.0 * kg / (h * h) + 2.0 * unorm / h + sg;
    double tau = den > 0.0 ? 1.0 / den : 0.0;
    double w = dV[g];

    if (terms & OR_MASS)
      for (int a = 0; a < nen; ++a)
        for (int b = 0; b < nen; ++b)
          Ae[a * nen + b] += w * Ng[a] * (MUT(10) ? Ng[a] : Ng[b]) / dt;
    if (terms & OR_CONV)
      for (int a = 0; a < nen; ++a)
        for (int b = 0; b < nen; ++b) {
          double c = (MUT(3)) ? Ng[b] * ua[a] : Ng[a] * ua[b];
          Ae[a * nen + b] += (MUT(2) ? -w : w) * c;
        }
    if ((terms & OR_DIFF) && !MUT(1))
      for (int a = 0; a < nen; ++a)
        for (int b = 0; b < nen; ++b)
          Ae[a * nen + b] += w * kg *
                             (gradN[g][a][0] * gradN[g][b][0] + gradN[g][a][1] * gradN[g][b][1] +
                              gradN[g][a][2] * gradN[g][b][2]);
    if (terms & OR_REAC)
      for (int a = 0; a < nen; ++a)
        for (int b = 0; b < nen; ++b) Ae[a * nen + b] += w * sg * Ng[a] * Ng[b];
    if (terms & OR_SUPG)
      for (int a = 0; a < nen; ++a)
        for (int b = 0; b < nen; ++b) {
          double resid = Ng[b] / dt + ua[b] + (MUT(7) ? 0.0 : sg * Ng[b]);
          Ae[a * nen + b] += w * tau * ua[a] * resid;
        }
    if (terms & OR_MASS)
      for (int a = 0; a < nen; ++a) be[a] += w * Ng[a] * pg / dt;
    if ((terms & OR_SUPG) && !MUT(6))
      for (int a = 0; a < nen; ++a) be[a] += w * tau * ua[a] * pg / dt;
    if (babs)
      for (int a = 0; a < nen; ++a) {
        if (terms & OR_MASS) babs[a] += MUT(16) ? w * Ng[a] * pg / dt : fabs(w * Ng[a] * pg / dt);
        if (terms & OR_SUPG) babs[a] += fabs(w * tau * ua[a] * pg / dt);
      }
  }
  return OR_OK;
}

/* Gather one element's nodal data (coords AoS [N][3], velocity SoA [3][N],
 * per-equation fields [n_eq][N]) for equation q. */
static void gather(int nen, const int32_t* ce, const double* coords, int64_t n_node, const double* vel,
                   const double* kd, const double* sr, const double* phi, int q, double* xe, double* ue,
                   double* ke, double* se, double* pe) {
  for (int a = 0; a < nen; ++a) {
    int64_t n = ce[a];
    for (int i = 0; i < 3; ++i) {
      xe[a * 3 + i] = coords[n * 3 + i];
      ue[a * 3 + i] = vel[(int64_t)i * n_node + n];
    }
    ke[a] = kd[(int64_t)q * n_node + n];
    se[a] = sr[(int64_t)q * n_node + n];
    pe[a] = phi[(int64_t)q * n_node + n];
  }
}

/* ---------------------------------------------------------------- validation */

/* Node ids in range, no node repeated inside an element, det J > 0 at every
 * Gauss point and every corner point of every element. */
int or_validate(int type, const double* coords, int64_t n_node, const int32_t* conn, int64_t n_elem) {
  int nen = or_nen(type);
  if (!nen || n_node <= 0 || n_elem < 0) return OR_ERR_ARG;
  for (int64_t e = 0; e < n_elem; ++e)
    for (int a = 0; a < nen; ++a) {
      int32_t n = conn[e * nen + a];
      if (n < 0 || n >= n_node) return OR_ERR_RANGE;
    }
  for (int64_t e = 0; e < n_elem; ++e)
    for (int a = 0; a < nen; ++a)
      for (int b = a + 1; b < nen; ++b)
        if (conn[e * nen + a] == conn[e * nen + b]) return OR_ERR_DUP;
  double xq[MAXN * 3], wq[MAXN], xc[8 * 3];
  int ng = or_quadrature(type, xq, wq);
  int nc = corner_points(type, xc);
  for (int64_t e = 0; e < n_elem; ++e) {
    double xe[MAXN * 3];
    for (int a = 0; a < nen; ++a)
      for (int i = 0; i < 3; ++i) xe[a * 3 + i] = coords[(int64_t)conn[e * nen + a] * 3 + i];
    for (int p = 0; p < ng + nc; ++p) {
      double N[MAXN], dN[MAXN * 3], J[3][3];
      or_shape(type, p < ng ? &xq[p * 3] : &xc[(p - ng) * 3], N, dN);
      if (!(jacobian(nen, xe, dN, J) > 0.0)) return OR_ERR_INVERTED;
    }
  }
  return OR_OK;
}

/* ---------------------------------------------------------------- CSR pattern */

static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

/* Node -> element incidence in CSR form: inc_ptr[n_node+1], inc_elem[nen*n_elem]. */
int or_incidence(int type, const int32_t* conn, int64_t n_elem, int64_t n_node, int64_t* inc_ptr,
                 int64_t* inc_elem) {
  int nen = or_nen(type);
  if (!nen) return OR_ERR_ARG;
  for (int64_t n = 0; n <= n_node; ++n) inc_ptr[n] = 0;
  for (int64_t e = 0; e < n_elem; ++e)
    for (int a = 0; a < nen; ++a) inc_ptr[conn[e * nen + a] + 1]++;
  for (int64_t n = 0; n < n_node; ++n) inc_ptr[n + 1] += inc_ptr[n];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_node);
  if (!fill) return OR_ERR_ARG;
  for (int64_t n = 0; n < n_node; ++n) fill[n] = inc_ptr[n];
  for (int64_t e = 0; e < n_elem; ++e)
    for (int a = 0; a < nen; ++a) inc_elem[fill[conn[e * nen + a]]++] = e;
  free(fill);
  return OR_OK;
}

/* Sorted, unique columns of row `r`: every node that shares an element with r
 * (r itself included).  Writes up to cap columns; returns the count or -1. */
static int64_t row_columns(int nen, const int32_t* conn, const int64_t* inc_ptr, const int64_t* inc_elem,
                           int64_t r, int32_t* buf, int64_t cap) {
  int64_t c = 0;
  for (int64_t t = inc_ptr[r]; t < inc_ptr[r + 1]; ++t) {
    int64_t e = inc_elem[t];
    for (int b = 0; b < nen; ++b) {
      if (c >= cap) return -1;
      buf[c++] = conn[e * nen + b];
    }
  }
  qsort(buf, (size_t)c, sizeof(int32_t), cmp_i32);
  int64_t u = 0;
  for (int64_t i = 0; i < c; ++i)
    if (i == 0 || buf[i] != buf[u - 1]) buf[u++] = buf[i];
  if (MUT(8)) { /* drop the diagonal */
    int64_t v = 0;
    for (int64_t i = 0; i < u; ++i)
      if (buf[i] != r) buf[v++] = buf[i];
    u = v;
  }
  return u;
}

/* rowptr[n_node+1] of the pattern; returns nnz (or -1). */
int64_t or_pattern_rowptr(int type, const int32_t* conn, int64_t n_elem, int64_t n_node, const int64_t* inc_ptr,
                          const int64_t* inc_elem, int64_t* rowptr) {
  int nen = or_nen(type);
  int64_t maxdeg = 0;
  for (int64_t n = 0; n < n_node; ++n)
    if (inc_ptr[n + 1] - inc_ptr[n] > maxdeg) maxdeg = inc_ptr[n + 1] - inc_ptr[n];
  int64_t cap = maxdeg * nen + 1;
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  if (!buf) return -1;
  rowptr[0] = 0;
  for (int64_t r = 0; r < n_node; ++r) {
    int64_t c = row_columns(nen, conn, inc_ptr, inc_elem, r, buf, cap);
    if (c < 0) { free(buf); return -1; }
    rowptr[r + 1] = rowptr[r] + c;
  }
  free(buf);
  (void)n_elem;
  return rowptr[n_node];
}

int or_pattern_colind(int type, const int32_t* conn, int64_t n_node, const int64_t* inc_ptr,
                      const int64_t* inc_elem, const int64_t* rowptr, int32_t* colind) {
  int nen = or_nen(type);
  int64_t maxdeg = 0;
  for (int64_t n = 0; n < n_node; ++n)
    if (inc_ptr[n + 1] - inc_ptr[n] > maxdeg) maxdeg = inc_ptr[n + 1] - inc_ptr[n];
  int64_t cap = maxdeg * nen + 1;
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  if (!buf) return OR_ERR_ARG;
  for (int64_t r = 0; r < n_node; ++r) {
    int64_t c = row_columns(nen, conn, inc_ptr, inc_elem, r, buf, cap);
    if (c != rowptr[r + 1] - rowptr[r]) { free(buf); return OR_ERR_ARG; }
    memcpy(colind + rowptr[r], buf, sizeof(int32_t) * (size_t)c);
  }
  free(buf);
  return OR_OK;
}

/* pos[e][a][b] = the k in row conn[e][a] with colind[k] == conn[e][b] (linear scan). */
int or_posmap(int type, const int32_t* conn, int64_t n_elem, const int64_t* rowptr, const int32_t* colind,
              int32_t* pos) {
  int nen = or_nen(type);
  for (int64_t e = 0; e < n_elem; ++e)
    for (int a = 0; a < nen; ++a)
      for (int b = 0; b < nen; ++b) {
        int32_t r = conn[e * nen + a], c = conn[e * nen + b];
        int64_t k = rowptr[r];
        while (k < rowptr[r + 1] && colind[k] != c) ++k;
        if (k == rowptr[r + 1]) return OR_ERR_ARG;
        pos[(e * nen + a) * nen + b] = (int32_t)k;
      }
  return OR_OK;
}

/* ---------------------------------------------------------------- assembly */

/* Column position of node c in row r (linear scan). */
static int64_t find_col(const int64_t* rowptr, const int32_t* colind, int32_t r, int32_t c) {
  for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k)
    if (colind[k] == c) return k;
  return -1;
}

/* Assemble elements [e_begin, e_end) of all n_eq equations into values[n_eq][nnz]
 * and rhs[n_eq][n_node] (added to what is there), plus optional abs-sum
 * denominators absA[n_eq][nnz] = sum_e |A^e_ij| and absb[n_eq][n_node] = the sum over elements and
 * Gauss points of the magnitudes of the summands of b_i (cancellation inside one element counts too).
 * Element loop outermost, plain `+=` in element order (Sec. 4.2). */
int or_assemble(int type, const double* coords, int64_t n_node, const int32_t* conn, int64_t e_begin,
                int64_t e_end, const int64_t* rowptr, const int32_t* colind, int64_t nnz, const double* vel,
                const double* kd, const double* sr, const double* phi, double dt, int n_eq, int terms,
                double* values, double* rhs, double* absA, double* absb) {
  int nen = or_nen(type);
  if (!nen || n_eq <= 0) return OR_ERR_ARG;
  double xe[MAXN * 3], ue[MAXN * 3], ke[MAXN], se[MAXN], pe[MAXN], Ae[MAXN * MAXN], be[MAXN], bab[MAXN];
  for (int64_t e = e_begin; e < e_end; ++e) {
    const int32_t* ce = conn + e * nen;
    for (int q = 0; q < n_eq; ++q) {
      gather(nen, ce, coords, n_node, vel, kd, sr, phi, q, xe, ue, ke, se, pe);
      int st = element_impl(type, xe, ue, ke, se, pe, dt, terms, Ae, be, bab);
      if (st) return st;
      for (int a = 0; a < nen; ++a) {
        for (int b = 0; b < nen; ++b) {
          int32_t r = ce[a], c = ce[b];
          if (MUT(9)) { r = ce[b]; c = ce[a]; }
          int64_t k = find_col(rowptr, colind, r, c);
          if (k < 0) return OR_ERR_ARG;
          values[(int64_t)q * nnz + k] += Ae[a * nen + b];
          if (absA) absA[(int64_t)q * nnz + k] += MUT(17) ? Ae[a * nen + b] : fabs(Ae[a * nen + b]);
        }
        rhs[(int64_t)q * n_node + ce[a]] += be[a];
        if (absb) absb[(int64_t)q * n_node + ce[a]] += bab[a];
      }
    }
  }
  return OR_OK;
}

/* One full row r of every equation, from the elements incident to r only
 * (for sampled checks of meshes too large to assemble on the CPU).
 * cols[cap] receives the sorted columns, vals[n_eq][cap] the values,
 * absv[n_eq][cap] the abs-sum denominators, rhs[n_eq] and absr[n_eq] the
 * RHS entry and its denominator.  Returns the number of columns, or -err. */
int64_t or_row(int type, const double* coords, int64_t n_node, const int32_t* conn, const int64_t* inc_ptr,
               const int64_t* inc_elem, int64_t r, const double* vel, const double* kd, const double* sr,
               const double* phi, double dt, int n_eq, int terms, int64_t cap, int32_t* cols, double* vals,
               double* absv, double* rhs, double* absr) {
  int nen = or_nen(type);
  if (!nen || r < 0 || r >= n_node) return -OR_ERR_ARG;
  int64_t nc = row_columns(nen, conn, inc_ptr, inc_elem, r, cols, cap);
  if (nc < 0) return -OR_ERR_CAP;
  for (int q = 0; q < n_eq; ++q) {
    for (int64_t k = 0; k < nc; ++k) { vals[q * cap + k] = 0.0; absv[q * cap + k] = 0.0; }
    rhs[q] = 0.0;
    absr[q] = 0.0;
  }
  double xe[MAXN * 3], ue[MAXN * 3], ke[MAXN], se[MAXN], pe[MAXN], Ae[MAXN * MAXN], be[MAXN], bab[MAXN];
  for (int64_t t = inc_ptr[r]; t < inc_ptr[r + 1] - (MUT(15) ? 1 : 0); ++t) {
    int64_t e = inc_elem[t];
    const int32_t* ce = conn + e * nen;
    int a = 0;
    while (ce[a] != r) ++a;
    if (MUT(14)) a = (a + 1) % nen;
    for (int q = 0; q < n_eq; ++q) {
      gather(nen, ce, coords, n_node, vel, kd, sr, phi, q, xe, ue, ke, se, pe);
      int st = element_impl(type, xe, ue, ke, se, pe, dt, terms, Ae, be, bab);
      if (st) return -st;
      for (int b = 0; b < nen; ++b) {
        int64_t k = 0;
        while (k < nc && cols[k] != ce[b]) ++k;
        if (k == nc) return -OR_ERR_ARG;
        vals[q * cap + k] += Ae[a * nen + b];
        absv[q * cap + k] += fabs(Ae[a * nen + b]);
      }
      rhs[q] += be[a];
      absr[q] += bab[a];
    }
  }
  return nc;
}

/* Matrix-free application y += sum_e P_e^T A^e P_e x for equation q. */
int or_apply(int type, const double* coords, int64_t n_node, const int32_t* conn, int64_t n_elem,
             const double* vel, const double* kd, const double* sr, const double* phi, double dt, int q,
             int terms, const double* x, double* y) {
  int nen = or_nen(type);
  if (!nen) return OR_ERR_ARG;
  double xe[MAXN * 3], ue[MAXN * 3], ke[MAXN], se[MAXN], pe[MAXN], Ae[MAXN * MAXN], be[MAXN];
  for (int64_t e = 0; e < n_elem; ++e) {
    const int32_t* ce = conn + e * nen;
    gather(nen, ce, coords, n_node, vel, kd, sr, phi, q, xe, ue, ke, se, pe);
    int st = or_element(type, xe, ue, ke, se, pe, dt, terms, Ae, be);
    if (st) return st;
    for (int a = 0; a < nen; ++a) {
      double s = 0.0;
      for (int b = 0; b < nen; ++b) s += Ae[a * nen + b] * x[ce[b]];
      y[ce[a]] += s;
    }
  }
  return OR_OK;
}

/* Field update of one time step (the stepping reading of Sec. 2: fields change between
 * assemblies): phi[q][n] += A_q sin(kx_q x_n + ky_q y_n + kz_q z_n + psi_q), params
 * [n_eq][5] = A, kx, ky, kz, psi.  The definition written out, in double precision. */
int or_update_fields(const double* coords, int64_t n_node, int n_eq, const double* params, double* phi) {
  if (n_node < 0 || n_eq < 0) return OR_ERR_ARG;
  for (int q = 0; q < n_eq; ++q) {
    const double* p = params + 5 * q;
    for (int64_t n = 0; n < n_node; ++n) {
      const double* x = coords + 3 * n;
      phi[q * n_node + n] += p[0] * sin(p[1] * x[0] + p[2] * x[1] + p[3] * x[2] + p[4]);
    }
  }
  return OR_OK;
}
