/*
 * Dense FP64 Galerkin oracle for the boundary-integral Poisson-Boltzmann system.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call this file;
 * only the test suite, the smoke check and the CPU-baseline leg of the benchmark use it.
 * It shares no code, header or table with the CUDA library.
 *
 * What it computes (all in double precision, plain loops, no blocking or reordering):
 *   - the kernels K1..K4 of Eq_K1/Eq_K2 (Section 2.2) written out as the paper defines them:
 *     differences of the Coulomb kernel G0 = 1/(4 pi r), the screened kernel
 *     Gk = exp(-kappa r)/(4 pi r) and their first and mixed second normal derivatives;
 *   - the Galerkin entries of eq_linsysEntry (Section 2.3) with piecewise-constant basis
 *     functions, signs taken from the variational form eqbim_5/eqbim_6:
 *        A11 = diag(1/2 (1+eps) A_i) - [I2],  A12 = -[I1],
 *        A21 = -[I4],                         A22 = diag(1/2 (1+1/eps) A_i) - [I3];
 *   - I_m(i,j) = int_{tau_i} int_{tau_j} K_m(x,y) dS_y dS_x by the one-point (centroid) rule
 *     for pairs of triangles that share no vertex, and by the Sauter-Schwab singularity
 *     removing transformation to the 4-cube with tensor Gauss-Legendre quadrature for
 *     identical, edge-adjacent and vertex-adjacent pairs (Section 2.3, the paragraph after
 *     the right-hand side definition);
 *   - the right-hand side b1, b2 (source_terms, Section 2.2) by the centroid rule;
 *   - the per-element energy weights of eqsolengdis (Section 2.3);
 *   - optionally (Section 3.1, Table 2) a regular rule of order 2-4 in place of the centroid
 *     for regular pairs, the right-hand side and the energy (orc_rule).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ---------- Gauss-Legendre rule on [0,1]: Newton iteration on P_n (textbook method) ---------- */
int orc_gauss_legendre01(int n, double* x, double* w)
{
    if (n < 1 || n > 64) return -1;
    for (int i = 0; i < n; ++i) {
        /* initial guess: Chebyshev-like approximation of the i-th root of P_n on [-1,1] */
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? z : p1;
            double pnm1 = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pnm1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged root */
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? z : p1;
            double pnm1 = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pnm1) / (z * z - 1.0);
        }
        double wz = 2.0 / ((1.0 - z * z) * dp * dp);
        /* map [-1,1] -> [0,1] */
        x[i] = 0.5 * (1.0 - z);
        w[i] = 0.5 * wz;
    }
    return 0;
}

/* ---------- kernels of Eq_K1 / Eq_K2, as the paper writes them ---------- */
typedef struct {
    double eps;   /* eps = eps2/eps1 */
    double kappa; /* inverse Debye length */
} orc_phys;

/* Regular quadrature rule on the reference triangle {0 <= e2 <= e1 <= 1} (Section 3.1,
 * Table 2: orders 1-4): n points (e1[a], e2[a]) with weights w[a] summing to 1/2; on an element
 * with corners P0, P1, P2 the point is P0 + e1 (P1 - P0) + e2 (P2 - P1) and the weight is
 * multiplied by the map's Jacobian 2A. n == 1 is the centroid rule (e1, e2) = (2/3, 1/3),
 * w = 1/2, evaluated as the plain centroid with weight A. */
typedef struct {
    int n;
    const double* e1;
    const double* e2;
    const double* w;
} orc_rule;

static void orc_rule_point(const double* u, const double* v, const double* w, double e1, double e2, double* x)
{
    for (int k = 0; k < 3; ++k) x[k] = u[k] + e1 * (v[k] - u[k]) + e2 * (w[k] - v[k]);
}

/* The six terms the kernels are made of, at x (normal nx) and y (normal ny):
 * Q[0] = G0 - Gk, Q[1] = d2Gk/dnx dny - d2G0/dnx dny, Q[2] = dG0/dny, Q[3] = dGk/dny,
 * Q[4] = dG0/dnx, Q[5] = dGk/dnx; and, for the pins of the singular quadrature only,
 * Q[6] = G0 and Q[7] = Gk on their own. */
static void orc_kernel_terms(const double* x, const double* nx, const double* y, const double* ny,
                             const orc_phys* ph, double* Q)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r = sqrt(r2);
    double kr = ph->kappa * r;
    double e = exp(-kr);
    double fpi = 4.0 * ORC_PI;
    double G0 = 1.0 / (fpi * r);
    double Gk = e / (fpi * r);
    double g0p = -1.0 / (fpi * r2);
    double gkp = -(1.0 + kr) * e / (fpi * r2);
    double g0pp = 2.0 / (fpi * r2 * r);
    double gkpp = (2.0 + 2.0 * kr + kr * kr) * e / (fpi * r2 * r);
    double nxd = nx[0] * d[0] + nx[1] * d[1] + nx[2] * d[2];
    double nyd = ny[0] * d[0] + ny[1] * d[1] + ny[2] * d[2];
    double nxny = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
    double d2G0 = -((g0pp - g0p / r) * nxd * nyd / r2 + (g0p / r) * nxny);
    double d2Gk = -((gkpp - gkp / r) * nxd * nyd / r2 + (gkp / r) * nxny);
    Q[0] = G0 - Gk;
    Q[1] = d2Gk - d2G0;
    Q[2] = -g0p * nyd / r;
    Q[3] = -gkp * nyd / r;
    Q[4] = g0p * nxd / r;
    Q[5] = gkp * nxd / r;
    Q[6] = G0;
    Q[7] = Gk;
}

/* Kout[0..3] = K1..K4 at target x (normal nx) and source y (normal ny). */
static void orc_kernels(const double* x, const double* nx, const double* y, const double* ny,
                        const orc_phys* ph, double* Kout)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r = sqrt(r2);
    double kr = ph->kappa * r;
    double e = exp(-kr);
    double fpi = 4.0 * ORC_PI;
    /* g(r) and its radial derivatives for G0 and Gk */
    double G0 = 1.0 / (fpi * r);
    double Gk = e / (fpi * r);
    double g0p = -1.0 / (fpi * r2);
    double gkp = -(1.0 + kr) * e / (fpi * r2);
    double g0pp = 2.0 / (fpi * r2 * r);
    double gkpp = (2.0 + 2.0 * kr + kr * kr) * e / (fpi * r2 * r);
    double nxd = nx[0] * d[0] + nx[1] * d[1] + nx[2] * d[2];
    double nyd = ny[0] * d[0] + ny[1] * d[1] + ny[2] * d[2];
    double nxny = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
    /* d/dnu_x G = g'(r) (nx.d)/r ; d/dnu_y G = -g'(r) (ny.d)/r */
    double dG0x = g0p * nxd / r, dGkx = gkp * nxd / r;
    double dG0y = -g0p * nyd / r, dGky = -gkp * nyd / r;
    /* d2/(dnu_x dnu_y) G = -[(g'' - g'/r)(nx.d)(ny.d)/r^2 + (g'/r)(nx.ny)] */
    double d2G0 = -((g0pp - g0p / r) * nxd * nyd / r2 + (g0p / r) * nxny);
    double d2Gk = -((gkpp - gkp / r) * nxd * nyd / r2 + (gkp / r) * nxny);
    Kout[0] = G0 - Gk;
    Kout[1] = ph->eps * dGky - dG0y;
    Kout[2] = dG0x - dGkx / ph->eps;
    Kout[3] = d2Gk - d2G0;
}

/* exported for the tests: K1..K4 at one point pair */
void orc_kernel_point(const double* x, const double* nx, const double* y, const double* ny,
                      double eps, double kappa, double* Kout)
{
    orc_phys ph = {eps, kappa};
    orc_kernels(x, nx, y, ny, &ph, Kout);
}

/* ---------- geometry (Section 2.3, eqparameter): centroid, area, unit normal ---------- */
static void orc_tri(const double* V, const int32_t* T, int i, double* u, double* v, double* w)
{
    for (int k = 0; k < 3; ++k) {
        u[k] = V[3 * T[3 * i + 0] + k];
        v[k] = V[3 * T[3 * i + 1] + k];
        w[k] = V[3 * T[3 * i + 2] + k];
    }
}

/* centroid c, area A, unit normal n = (v-u)x(w-u)/|..| (outward for counter-clockwise
 * vertex order seen from outside) */
static void orc_geom(const double* u, const double* v, const double* w, double* c, double* A,
                     double* n)
{
    double a[3] = {v[0] - u[0], v[1] - u[1], v[2] - u[2]};
    double b[3] = {w[0] - u[0], w[1] - u[1], w[2] - u[2]};
    double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    *A = 0.5 * len;
    for (int k = 0; k < 3; ++k) {
        n[k] = cr[k] / len;
        c[k] = (u[k] + v[k] + w[k]) / 3.0;
    }
}

void orc_geometry(const double* V, const int32_t* T, int nt, double* cent, double* area,
                  double* normal)
{
    for (int i = 0; i < nt; ++i) {
        double u[3], v[3], w[3];
        orc_tri(V, T, i, u, v, w);
        orc_geom(u, v, w, cent + 3 * i, area + i, normal + 3 * i);
    }
}

/* ---------- Sauter-Schwab sub-maps of tau x tau onto the 4-cube ----------
 * tau = {0 <= e2 <= e1 <= 1} is the paper's reference triangle (eqreftri). For a point
 * (xi, h1, h2, h3) of [0,1]^4 each case returns k sub-maps (xhat, yhat, jacobian weight):
 *   case 3 identical triangles, case 2 a common edge mapped to the reference edge
 *   (0,0)-(1,0) of both triangles, case 1 a common vertex mapped to (0,0) of both.
 * The sum over sub-maps of the integral over the cube equals the integral over tau x tau. */
int orc_ss_points(int kase, double xi, double h1, double h2, double h3, double* xh, double* yh,
                  double* jac)
{
    if (kase == 3) {
        double w = xi * xi * xi * h1 * h1 * h2;
        double a[6][4] = {
            {1.0, 1.0 - h1 + h1 * h2, 1.0 - h1 * h2 * h3, 1.0 - h1},
            {1.0 - h1 * h2 * h3, 1.0 - h1, 1.0, 1.0 - h1 + h1 * h2},
            {1.0, h1 * (1.0 - h2 + h2 * h3), 1.0 - h1 * h2, h1 * (1.0 - h2)},
            {1.0 - h1 * h2, h1 * (1.0 - h2), 1.0, h1 * (1.0 - h2 + h2 * h3)},
            {1.0 - h1 * h2 * h3, h1 * (1.0 - h2 * h3), 1.0, h1 * (1.0 - h2)},
            {1.0, h1 * (1.0 - h2), 1.0 - h1 * h2 * h3, h1 * (1.0 - h2 * h3)},
        };
        for (int s = 0; s < 6; ++s) {
            xh[2 * s] = xi * a[s][0];
            xh[2 * s + 1] = xi * a[s][1];
            yh[2 * s] = xi * a[s][2];
            yh[2 * s + 1] = xi * a[s][3];
            jac[s] = w;
        }
        return 6;
    }
    if (kase == 2) {
        double w1 = xi * xi * xi * h1 * h1;
        double w2 = w1 * h2;
        double a[5][4] = {
            {1.0, h1 * h3, 1.0 - h1 * h2, h1 * (1.0 - h2)},
            {1.0, h1, 1.0 - h1 * h2 * h3, h1 * h2 * (1.0 - h3)},
            {1.0 - h1 * h2, h1 * (1.0 - h2), 1.0, h1 * h2 * h3},
            {1.0 - h1 * h2 * h3, h1 * h2 * (1.0 - h3), 1.0, h1},
            {1.0 - h1 * h2 * h3, h1 * (1.0 - h2 * h3), 1.0, h1 * h2},
        };
        for (int s = 0; s < 5; ++s) {
            xh[2 * s] = xi * a[s][0];
            xh[2 * s + 1] = xi * a[s][1];
            yh[2 * s] = xi * a[s][2];
            yh[2 * s + 1] = xi * a[s][3];
            jac[s] = (s == 0) ? w1 : w2;
        }
        return 5;
    }
    if (kase == 1) {
        double w = xi * xi * xi * h2;
        xh[0] = xi;           xh[1] = xi * h1;
        yh[0] = xi * h2;      yh[1] = xi * h2 * h3;
        xh[2] = xi * h2;      xh[3] = xi * h2 * h1;
        yh[2] = xi;           yh[3] = xi * h3;
        jac[0] = w;
        jac[1] = w;
        return 2;
    }
    return 0;
}

/* number of vertex indices shared by triangles i and j (3 when i == j) */
static int orc_shared(const int32_t* T, int i, int j)
{
    if (i == j) return 3;
    int s = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (T[3 * i + a] == T[3 * j + b]) ++s;
    return s;
}

/* Reorder the vertices of triangles i and j so that the shared ones come first, in the same
 * order in both (the layout the sub-maps above expect). */
static void orc_reorder(const int32_t* T, int i, int j, int shared, int32_t* ti, int32_t* tj)
{
    for (int k = 0; k < 3; ++k) {
        ti[k] = T[3 * i + k];
        tj[k] = T[3 * j + k];
    }
    if (shared == 3) return;
    int si[3], sj[3], ns = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (T[3 * i + a] == T[3 * j + b]) {
                si[ns] = a;
                sj[ns] = b;
                ++ns;
            }
    int oi[3], oj[3], p = 0, q = 0;
    for (int s = 0; s < ns; ++s) {
        oi[p++] = T[3 * i + si[s]];
        oj[q++] = T[3 * j + sj[s]];
    }
    for (int a = 0; a < 3; ++a) {
        int used = 0;
        for (int s = 0; s < ns; ++s) used |= (si[s] == a);
        if (!used) oi[p++] = T[3 * i + a];
    }
    for (int b = 0; b < 3; ++b) {
        int used = 0;
        for (int s = 0; s < ns; ++s) used |= (sj[s] == b);
        if (!used) oj[q++] = T[3 * j + b];
    }
    for (int k = 0; k < 3; ++k) {
        ti[k] = oi[k];
        tj[k] = oj[k];
    }
}

/* ---------- Galerkin pair integrals I_m(i,j), m = 1..4 ---------- */
#define ORC_NTERMS 8

/* Sauter-Schwab integrals over tau_first x tau_second of the eight terms of
 * orc_kernel_terms, x on the first triangle (normal na), y on the second (normal nb).
 * One quadrature serves both orderings of a touching pair: the rule is always laid out from
 * the triangle with the smaller index (its shared vertices first, in its order). */
static void orc_ss_terms(const double* V, const int32_t* T, int first, int second, int shared,
                         const double* na, const double* nb, double Afirst, double Asecond,
                         const orc_phys* ph, const double* gx, const double* gw, int qs,
                         double* acc)
{
    int32_t ti[3], tj[3];
    orc_reorder(T, first, second, shared, ti, tj);
    double P[3][3], Q[3][3];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
            P[a][k] = V[3 * ti[a] + k];
            Q[a][k] = V[3 * tj[a] + k];
        }
    /* The reference triangle {0 <= e2 <= e1 <= 1} has corners (0,0), (1,0), (1,1); the affine
     * map sending them to P0, P1, P2 is P0 + e1 (P1 - P0) + e2 (P2 - P1). (eqparameter prints
     * P2 - P0 in the last term, which sends (1,1) to P1 + P2 - P0, outside the element.) */
    for (int m = 0; m < ORC_NTERMS; ++m) acc[m] = 0.0;
    for (int a = 0; a < qs; ++a)
        for (int b = 0; b < qs; ++b)
            for (int c = 0; c < qs; ++c)
                for (int d = 0; d < qs; ++d) {
                    double wq = gw[a] * gw[b] * gw[c] * gw[d];
                    double xh[12], yh[12], jac[6];
                    int ns = orc_ss_points(shared, gx[a], gx[b], gx[c], gx[d], xh, yh, jac);
                    for (int s = 0; s < ns; ++s) {
                        double x[3], y[3], Qt[ORC_NTERMS];
                        for (int k = 0; k < 3; ++k) {
                            x[k] = P[0][k] + xh[2 * s] * (P[1][k] - P[0][k]) +
                                   xh[2 * s + 1] * (P[2][k] - P[1][k]);
                            y[k] = Q[0][k] + yh[2 * s] * (Q[1][k] - Q[0][k]) +
                                   yh[2 * s + 1] * (Q[2][k] - Q[1][k]);
                        }
                        orc_kernel_terms(x, na, y, nb, ph, Qt);
                        for (int m = 0; m < ORC_NTERMS; ++m) acc[m] += wq * jac[s] * Qt[m];
                    }
                }
    /* Jacobian of each affine element map is 2 A */
    for (int m = 0; m < ORC_NTERMS; ++m) acc[m] *= (2.0 * Afirst) * (2.0 * Asecond);
}

static void orc_pair(const double* V, const int32_t* T, int i, int j, const orc_phys* ph,
                     const double* gx, const double* gw, int qs, const orc_rule* qr, double* I)
{
    double ci[3], cj[3], ni[3], nj[3], Ai, Aj;
    {
        double u[3], v[3], w[3];
        orc_tri(V, T, i, u, v, w);
        orc_geom(u, v, w, ci, &Ai, ni);
        orc_tri(V, T, j, u, v, w);
        orc_geom(u, v, w, cj, &Aj, nj);
    }
    int shared = orc_shared(T, i, j);
    if (shared == 0 && qr->n == 1) {
        /* one-point Gauss (centroid) rule for regular pairs */
        double K[4];
        orc_kernels(ci, ni, cj, nj, ph, K);
        for (int m = 0; m < 4; ++m) I[m] = Ai * Aj * K[m];
        return;
    }
    if (shared == 0) {
        /* the rule's points on both elements, every pair of them */
        double ui[3], vi[3], wi[3], uj[3], vj[3], wj[3];
        orc_tri(V, T, i, ui, vi, wi);
        orc_tri(V, T, j, uj, vj, wj);
        double acc[4] = {0, 0, 0, 0};
        for (int a = 0; a < qr->n; ++a) {
            double x[3];
            orc_rule_point(ui, vi, wi, qr->e1[a], qr->e2[a], x);
            for (int b = 0; b < qr->n; ++b) {
                double y[3], K[4];
                orc_rule_point(uj, vj, wj, qr->e1[b], qr->e2[b], y);
                orc_kernels(x, ni, y, nj, ph, K);
                for (int m = 0; m < 4; ++m) acc[m] += qr->w[a] * qr->w[b] * K[m];
            }
        }
        for (int m = 0; m < 4; ++m) I[m] = (2.0 * Ai) * (2.0 * Aj) * acc[m];
        return;
    }
    /* the integrals of (j, i) follow from those of (i, j) by exchanging the roles of the two
     * normals */
    int first = i < j ? i : j, second = i < j ? j : i;
    double na[3], nb[3];
    for (int k = 0; k < 3; ++k) {
        na[k] = (first == i) ? ni[k] : nj[k];
        nb[k] = (first == i) ? nj[k] : ni[k];
    }
    double acc[ORC_NTERMS];
    orc_ss_terms(V, T, first, second, shared, na, nb, first == i ? Ai : Aj, first == i ? Aj : Ai,
                 ph, gx, gw, qs, acc);
    double eps = ph->eps;
    I[0] = acc[0];
    I[3] = acc[1];
    if (first == i) {
        /* target = first triangle: K2 = eps dGk/dny - dG0/dny, K3 = dG0/dnx - dGk/dnx / eps */
        I[1] = eps * acc[3] - acc[2];
        I[2] = acc[4] - acc[5] / eps;
    } else {
        /* target = second triangle: its source normal derivative is the first's dn_x */
        I[1] = eps * acc[5] - acc[4];
        I[2] = acc[2] - acc[3] / eps;
    }
}

/* exported for the pins of the singular quadrature: the eight Sauter-Schwab term integrals
 * (orc_kernel_terms order) of the touching pair (min(i,j), max(i,j)), x on the triangle with
 * the smaller index. Returns the number of shared vertices, or -1 for a bad order / a pair
 * that shares no vertex. */
int orc_pair_terms(const double* V, const int32_t* T, int i, int j, double kappa, int qs,
                   double* out)
{
    double gx[64], gw[64];
    if (orc_gauss_legendre01(qs, gx, gw)) return -1;
    int shared = orc_shared(T, i, j);
    if (shared == 0) return -1;
    orc_phys ph = {1.0, kappa};
    int first = i < j ? i : j, second = i < j ? j : i;
    double c[3], na[3], nb[3], Aa, Ab, u[3], v[3], w[3];
    orc_tri(V, T, first, u, v, w);
    orc_geom(u, v, w, c, &Aa, na);
    orc_tri(V, T, second, u, v, w);
    orc_geom(u, v, w, c, &Ab, nb);
    orc_ss_terms(V, T, first, second, shared, na, nb, Aa, Ab, &ph, gx, gw, qs, out);
    return shared;
}

/* exported: the four integrals for one ordered pair (target i, source j) */
int orc_pair_integrals(const double* V, const int32_t* T, int i, int j, double eps, double kappa,
                       int qs, int nq, const double* qe1, const double* qe2, const double* qw, double* I)
{
    double gx[64], gw[64];
    if (orc_gauss_legendre01(qs, gx, gw)) return -1;
    orc_phys ph = {eps, kappa};
    orc_rule qr = {nq, qe1, qe2, qw};
    orc_pair(V, T, i, j, &ph, gx, gw, qs, &qr, I);
    return 0;
}

/* exported: the dense 2N x 2N matrix of def:linsys, row-major, unknowns [phi ; dphi/dn] */
int orc_assemble(const double* V, const int32_t* T, int nt, double eps, double kappa, int qs,
                 int nq, const double* qe1, const double* qe2, const double* qw, double* A)
{
    double gx[64], gw[64];
    if (orc_gauss_legendre01(qs, gx, gw)) return -1;
    orc_phys ph = {eps, kappa};
    orc_rule qr = {nq, qe1, qe2, qw};
    long n2 = 2L * nt;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < nt; ++i) {
        double c[3], n[3], Ai;
        {
            double u[3], v[3], w[3];
            orc_tri(V, T, i, u, v, w);
            orc_geom(u, v, w, c, &Ai, n);
        }
        for (int j = 0; j < nt; ++j) {
            double I[4];
            orc_pair(V, T, i, j, &ph, gx, gw, qs, &qr, I);
            A[(long)i * n2 + j] = -I[1];
            A[(long)i * n2 + nt + j] = -I[0];
            A[(long)(nt + i) * n2 + j] = -I[3];
            A[(long)(nt + i) * n2 + nt + j] = -I[2];
        }
        A[(long)i * n2 + i] += 0.5 * (1.0 + eps) * Ai;
        A[(long)(nt + i) * n2 + nt + i] += 0.5 * (1.0 + 1.0 / eps) * Ai;
    }
    return 0;
}

/* exported: rows of A x for selected elements. For element e = elems[k] it writes
 * y[2k] = (A x)_e (the phi row) and y[2k+1] = (A x)_{N+e} (the dphi/dn row). */
int orc_rows_matvec(const double* V, const int32_t* T, int nt, double eps, double kappa, int qs,
                    int nq, const double* qe1, const double* qe2, const double* qw, int nrows,
                    const int32_t* elems, const double* x, double* y)
{
    double gx[64], gw[64];
    if (orc_gauss_legendre01(qs, gx, gw)) return -1;
    orc_phys ph = {eps, kappa};
    orc_rule qr = {nq, qe1, qe2, qw};
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nrows; ++k) {
        int i = elems[k];
        double c[3], n[3], Ai;
        {
            double u[3], v[3], w[3];
            orc_tri(V, T, i, u, v, w);
            orc_geom(u, v, w, c, &Ai, n);
        }
        double y1 = 0.5 * (1.0 + eps) * Ai * x[i];
        double y2 = 0.5 * (1.0 + 1.0 / eps) * Ai * x[nt + i];
        for (int j = 0; j < nt; ++j) {
            double I[4];
            orc_pair(V, T, i, j, &ph, gx, gw, qs, &qr, I);
            y1 -= I[0] * x[nt + j] + I[1] * x[j];
            y2 -= I[2] * x[nt + j] + I[3] * x[j];
        }
        y[2 * k] = y1;
        y[2 * k + 1] = y2;
    }
    return 0;
}

/* exported: right-hand side b = [b1; b2] (source_terms) by the centroid rule */
/* S1 and S2 of source_terms at x (normal n), before the 1/eps1 factor */
static void orc_sources(const double* x, const double* n, const double* qpos, const double* q, int nc,
                        double* s1, double* s2)
{
    *s1 = 0.0;
    *s2 = 0.0;
    for (int k = 0; k < nc; ++k) {
        double d[3] = {x[0] - qpos[3 * k], x[1] - qpos[3 * k + 1], x[2] - qpos[3 * k + 2]};
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double r = sqrt(r2);
        double nd = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
        *s1 += q[k] / (4.0 * ORC_PI * r);
        /* d G0/d nu_x = g0'(r) (n.d)/r = -(n.d)/(4 pi r^3) */
        *s2 += q[k] * (-nd / (4.0 * ORC_PI * r2 * r));
    }
}

void orc_rhs(const double* V, const int32_t* T, int nt, const double* qpos, const double* q,
             int nc, double eps1, int nq, const double* qe1, const double* qe2, const double* qw,
             double* b)
{
    for (int i = 0; i < nt; ++i) {
        double c[3], n[3], Ai;
        double u[3], v[3], w[3];
        orc_tri(V, T, i, u, v, w);
        orc_geom(u, v, w, c, &Ai, n);
        double s1 = 0.0, s2 = 0.0;
        if (nq == 1) {
            orc_sources(c, n, qpos, q, nc, &s1, &s2);
            s1 *= Ai;
            s2 *= Ai;
        } else {
            for (int a = 0; a < nq; ++a) {
                double x[3], t1, t2;
                orc_rule_point(u, v, w, qe1[a], qe2[a], x);
                orc_sources(x, n, qpos, q, nc, &t1, &t2);
                s1 += 2.0 * Ai * qw[a] * t1;
                s2 += 2.0 * Ai * qw[a] * t2;
            }
        }
        b[i] = s1 / eps1;
        b[nt + i] = s2 / eps1;
    }
}

/* exported: solvation energy of eqsolengdis in kcal/mol for the solution x = [phi; dphi/dn]:
 * E = 1/2 sum_n q_n sum_i A_i [K1(x_n, c_i) dphi_i + K2(x_n, c_i) phi_i], converted from
 * e_c/(4 pi Angstrom) by the factor 4 pi 332.0716 (Section 3). */
double orc_energy(const double* V, const int32_t* T, int nt, const double* qpos, const double* q,
                  int nc, double eps, double kappa, int nq, const double* qe1, const double* qe2,
                  const double* qw, const double* x)
{
    orc_phys ph = {eps, kappa};
    double zero[3] = {0.0, 0.0, 0.0};
    double E = 0.0;
    for (int k = 0; k < nc; ++k) {
        double sk = 0.0;
        for (int i = 0; i < nt; ++i) {
            double c[3], n[3], Ai, K[4];
            double u[3], v[3], w[3];
            orc_tri(V, T, i, u, v, w);
            orc_geom(u, v, w, c, &Ai, n);
            if (nq == 1) {
                orc_kernels(qpos + 3 * k, zero, c, n, &ph, K);
                sk += Ai * (K[0] * x[nt + i] + K[1] * x[i]);
            } else {
                for (int a = 0; a < nq; ++a) {
                    double y[3];
                    orc_rule_point(u, v, w, qe1[a], qe2[a], y);
                    orc_kernels(qpos + 3 * k, zero, y, n, &ph, K);
                    sk += 2.0 * Ai * qw[a] * (K[0] * x[nt + i] + K[1] * x[i]);
                }
            }
        }
        E += q[k] * sk;
    }
    return 0.5 * E * 4.0 * ORC_PI * 332.0716;
}

/* ---------- piecewise-linear Galerkin: continuous hat functions (S^1_h, Section 2.3) ----------
 * The unknowns live at the vertices: x = [phi_1..phi_nv ; dphi_1..dphi_nv]. On an element with
 * corners P0, P1, P2 the point P0 + e1 (P1 - P0) + e2 (P2 - P1) carries the three linear
 * functions of eqlinearfcn, 1 - e1, e1 - e2 and e2, which are the barycentric weights of P0,
 * P1 and P2; the hat function of vertex v (eqglinearcfcn) is, on every element containing v,
 * the one of them that is 1 at v. The entries become
 *    I_m(a, b) = sum over elements tau containing a, sigma containing b of
 *                int_tau int_sigma psi_a(x) K_m(x, y) psi_b(y) dS_y dS_x,
 * and the identity term of the variational form the mass matrix
 *    M(a, b) = int psi_a psi_b = sum_tau A_tau (1 + [a == b]) / 12 over tau containing both. */
static void orc_lambda(double e1, double e2, double* lam)
{
    lam[0] = 1.0 - e1;
    lam[1] = e1 - e2;
    lam[2] = e2;
}

/* position of vertex id v in triangle i (uploaded order) */
static int orc_corner(const int32_t* T, int i, int32_t v)
{
    for (int a = 0; a < 3; ++a)
        if (T[3 * i + a] == v) return a;
    return -1;
}

/* Sauter-Schwab integrals of the eight kernel terms weighted by the linear functions of both
 * triangles: acc[m][a][b], a a corner of `first` and b a corner of `second`, both in the
 * reordered (shared corners first) layout whose vertex ids come back in ti, tj. */
static void orc_p1_ss_terms(const double* V, const int32_t* T, int first, int second, int shared,
                            const double* na, const double* nb, double Afirst, double Asecond,
                            const orc_phys* ph, const double* gx, const double* gw, int qs,
                            double acc[ORC_NTERMS][3][3], int32_t* ti, int32_t* tj)
{
    orc_reorder(T, first, second, shared, ti, tj);
    double P[3][3], Q[3][3];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
            P[a][k] = V[3 * ti[a] + k];
            Q[a][k] = V[3 * tj[a] + k];
        }
    memset(acc, 0, sizeof(double) * ORC_NTERMS * 9);
    for (int a = 0; a < qs; ++a)
        for (int b = 0; b < qs; ++b)
            for (int c = 0; c < qs; ++c)
                for (int d = 0; d < qs; ++d) {
                    double wq = gw[a] * gw[b] * gw[c] * gw[d];
                    double xh[12], yh[12], jac[6];
                    int ns = orc_ss_points(shared, gx[a], gx[b], gx[c], gx[d], xh, yh, jac);
                    for (int s = 0; s < ns; ++s) {
                        double x[3], y[3], Qt[ORC_NTERMS], lx[3], ly[3];
                        for (int k = 0; k < 3; ++k) {
                            x[k] = P[0][k] + xh[2 * s] * (P[1][k] - P[0][k]) +
                                   xh[2 * s + 1] * (P[2][k] - P[1][k]);
                            y[k] = Q[0][k] + yh[2 * s] * (Q[1][k] - Q[0][k]) +
                                   yh[2 * s + 1] * (Q[2][k] - Q[1][k]);
                        }
                        orc_lambda(xh[2 * s], xh[2 * s + 1], lx);
                        orc_lambda(yh[2 * s], yh[2 * s + 1], ly);
                        orc_kernel_terms(x, na, y, nb, ph, Qt);
                        for (int m = 0; m < ORC_NTERMS; ++m)
                            for (int p = 0; p < 3; ++p)
                                for (int r = 0; r < 3; ++r)
                                    acc[m][p][r] += wq * jac[s] * lx[p] * ly[r] * Qt[m];
                    }
                }
    for (int m = 0; m < ORC_NTERMS; ++m)
        for (int p = 0; p < 3; ++p)
            for (int r = 0; r < 3; ++r) acc[m][p][r] *= (2.0 * Afirst) * (2.0 * Asecond);
}

/* I[m][a][b] = int_{tau_i} int_{tau_j} lambda_a(x) K_m(x, y) lambda_b(y), m = 1..4, a and b the
 * corners of i and j in uploaded order. Regular pairs by the rule qr (the centroid rule, where
 * every linear function is 1/3, for qr->n == 1); touching pairs by Sauter-Schwab. */
static void orc_p1_pair(const double* V, const int32_t* T, int i, int j, const orc_phys* ph,
                        const double* gx, const double* gw, int qs, const orc_rule* qr, double I[4][3][3])
{
    double ci[3], cj[3], ni[3], nj[3], Ai, Aj;
    double ui[3], vi[3], wi[3], uj[3], vj[3], wj[3];
    orc_tri(V, T, i, ui, vi, wi);
    orc_geom(ui, vi, wi, ci, &Ai, ni);
    orc_tri(V, T, j, uj, vj, wj);
    orc_geom(uj, vj, wj, cj, &Aj, nj);
    int shared = orc_shared(T, i, j);
    if (shared == 0) {
        memset(I, 0, sizeof(double) * 36);
        if (qr->n == 1) {
            double K[4];
            orc_kernels(ci, ni, cj, nj, ph, K);
            for (int m = 0; m < 4; ++m)
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) I[m][a][b] = Ai * Aj * K[m] / 9.0;
            return;
        }
        for (int p = 0; p < qr->n; ++p) {
            double x[3], lx[3];
            orc_rule_point(ui, vi, wi, qr->e1[p], qr->e2[p], x);
            orc_lambda(qr->e1[p], qr->e2[p], lx);
            for (int r = 0; r < qr->n; ++r) {
                double y[3], ly[3], K[4];
                orc_rule_point(uj, vj, wj, qr->e1[r], qr->e2[r], y);
                orc_lambda(qr->e1[r], qr->e2[r], ly);
                orc_kernels(x, ni, y, nj, ph, K);
                double wgt = (2.0 * Ai) * (2.0 * Aj) * qr->w[p] * qr->w[r];
                for (int m = 0; m < 4; ++m)
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) I[m][a][b] += wgt * lx[a] * ly[b] * K[m];
            }
        }
        return;
    }
    int first = i < j ? i : j, second = i < j ? j : i;
    double na[3], nb[3];
    for (int k = 0; k < 3; ++k) {
        na[k] = (first == i) ? ni[k] : nj[k];
        nb[k] = (first == i) ? nj[k] : ni[k];
    }
    double acc[ORC_NTERMS][3][3];
    int32_t ta[3], tb[3];
    orc_p1_ss_terms(V, T, first, second, shared, na, nb, first == i ? Ai : Aj, first == i ? Aj : Ai,
                    ph, gx, gw, qs, acc, ta, tb);
    double eps = ph->eps;
    /* acc is laid out [first corner][second corner]; the result [target corner][source corner] */
    for (int p = 0; p < 3; ++p)
        for (int r = 0; r < 3; ++r) {
            int a, b;
            double t[ORC_NTERMS];
            if (first == i) {
                a = orc_corner(T, i, ta[p]);
                b = orc_corner(T, j, tb[r]);
            } else {
                a = orc_corner(T, i, tb[r]);
                b = orc_corner(T, j, ta[p]);
            }
            for (int m = 0; m < ORC_NTERMS; ++m) t[m] = acc[m][p][r];
            I[0][a][b] = t[0];
            I[3][a][b] = t[1];
            if (first == i) {
                I[1][a][b] = eps * t[3] - t[2];
                I[2][a][b] = t[4] - t[5] / eps;
            } else {
                I[1][a][b] = eps * t[5] - t[4];
                I[2][a][b] = t[2] - t[3] / eps;
            }
        }
}

/* exported: the 4 x 3 x 3 weighted integrals of the ordered pair (target i, source j), corners
 * in uploaded order */
int orc_p1_pair_integrals(const double* V, const int32_t* T, int i, int j, double eps, double kappa,
                          int qs, int nq, const double* qe1, const double* qe2, const double* qw,
                          double* out)
{
    double gx[64], gw[64];
    if (orc_gauss_legendre01(qs, gx, gw)) return -1;
    orc_phys ph = {eps, kappa};
    orc_rule qr = {nq, qe1, qe2, qw};
    double I[4][3][3];
    orc_p1_pair(V, T, i, j, &ph, gx, gw, qs, &qr, I);
    memcpy(out, I, sizeof(I));
    return 0;
}

/* exported, for the pins: the eight Sauter-Schwab term integrals of a touching pair weighted by
 * the linear functions, out[m][a][b] with a a corner of min(i, j) and b a corner of max(i, j),
 * both in uploaded order. Returns the number of shared vertices (-1: no touching pair). */
int orc_p1_pair_terms(const double* V, const int32_t* T, int i, int j, double kappa, int qs, double* out)
{
    double gx[64], gw[64];
    if (orc_gauss_legendre01(qs, gx, gw)) return -1;
    int shared = orc_shared(T, i, j);
    if (shared == 0) return -1;
    orc_phys ph = {1.0, kappa};
    int first = i < j ? i : j, second = i < j ? j : i;
    double c[3], na[3], nb[3], Aa, Ab, u[3], v[3], w[3];
    orc_tri(V, T, first, u, v, w);
    orc_geom(u, v, w, c, &Aa, na);
    orc_tri(V, T, second, u, v, w);
    orc_geom(u, v, w, c, &Ab, nb);
    double acc[ORC_NTERMS][3][3];
    int32_t ta[3], tb[3];
    orc_p1_ss_terms(V, T, first, second, shared, na, nb, Aa, Ab, &ph, gx, gw, qs, acc, ta, tb);
    for (int p = 0; p < 3; ++p)
        for (int r = 0; r < 3; ++r) {
            int a = orc_corner(T, first, ta[p]), b = orc_corner(T, second, tb[r]);
            for (int m = 0; m < ORC_NTERMS; ++m) out[(m * 3 + a) * 3 + b] = acc[m][p][r];
        }
    return shared;
}

/* exported: y = A x for the piecewise-linear system, x and y of length 2 nv,
 *    y1_a = 1/2 (1 + eps) sum_b M(a,b) phi_b - sum_b [I1(a,b) dphi_b + I2(a,b) phi_b]
 *    y2_a = 1/2 (1 + 1/eps) sum_b M(a,b) dphi_b - sum_b [I3(a,b) dphi_b + I4(a,b) phi_b].
 * Every element's three test rows are summed first (in parallel over elements), then added to
 * their vertices in element order. */
int orc_p1_matvec(const double* V, const int32_t* T, int nt, int nv, double eps, double kappa, int qs,
                  int nq, const double* qe1, const double* qe2, const double* qw, const double* x,
                  double* y)
{
    double gx[64], gw[64];
    if (orc_gauss_legendre01(qs, gx, gw)) return -1;
    orc_phys ph = {eps, kappa};
    orc_rule qr = {nq, qe1, qe2, qw};
    double* yl = (double*)calloc((size_t)6 * nt, sizeof(double));
    if (!yl) return -2;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < nt; ++i) {
        double c[3], n[3], Ai, u[3], v[3], w[3];
        orc_tri(V, T, i, u, v, w);
        orc_geom(u, v, w, c, &Ai, n);
        double y1[3] = {0, 0, 0}, y2[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double M = Ai * (a == b ? 2.0 : 1.0) / 12.0;
                y1[a] += 0.5 * (1.0 + eps) * M * x[T[3 * i + b]];
                y2[a] += 0.5 * (1.0 + 1.0 / eps) * M * x[nv + T[3 * i + b]];
            }
        for (int j = 0; j < nt; ++j) {
            double I[4][3][3];
            orc_p1_pair(V, T, i, j, &ph, gx, gw, qs, &qr, I);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double ph_b = x[T[3 * j + b]], dph_b = x[nv + T[3 * j + b]];
                    y1[a] -= I[0][a][b] * dph_b + I[1][a][b] * ph_b;
                    y2[a] -= I[2][a][b] * dph_b + I[3][a][b] * ph_b;
                }
        }
        for (int a = 0; a < 3; ++a) {
            yl[6 * i + a] = y1[a];
            yl[6 * i + 3 + a] = y2[a];
        }
    }
    for (int k = 0; k < 2 * nv; ++k) y[k] = 0.0;
    for (int i = 0; i < nt; ++i)
        for (int a = 0; a < 3; ++a) {
            y[T[3 * i + a]] += yl[6 * i + a];
            y[nv + T[3 * i + a]] += yl[6 * i + 3 + a];
        }
    free(yl);
    return 0;
}

/* exported: the dense 2 nv x 2 nv piecewise-linear matrix (row-major), same layout as the
 * product above. Serial: small meshes only. */
int orc_p1_assemble(const double* V, const int32_t* T, int nt, int nv, double eps, double kappa, int qs,
                    int nq, const double* qe1, const double* qe2, const double* qw, double* A)
{
    double gx[64], gw[64];
    if (orc_gauss_legendre01(qs, gx, gw)) return -1;
    orc_phys ph = {eps, kappa};
    orc_rule qr = {nq, qe1, qe2, qw};
    long n2 = 2L * nv;
    memset(A, 0, sizeof(double) * n2 * n2);
    for (int i = 0; i < nt; ++i) {
        double c[3], n[3], Ai, u[3], v[3], w[3];
        orc_tri(V, T, i, u, v, w);
        orc_geom(u, v, w, c, &Ai, n);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                long ra = T[3 * i + a], cb = T[3 * i + b];
                double M = Ai * (a == b ? 2.0 : 1.0) / 12.0;
                A[ra * n2 + cb] += 0.5 * (1.0 + eps) * M;
                A[(nv + ra) * n2 + nv + cb] += 0.5 * (1.0 + 1.0 / eps) * M;
            }
        for (int j = 0; j < nt; ++j) {
            double I[4][3][3];
            orc_p1_pair(V, T, i, j, &ph, gx, gw, qs, &qr, I);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    long ra = T[3 * i + a], cb = T[3 * j + b];
                    A[ra * n2 + cb] -= I[1][a][b];
                    A[ra * n2 + nv + cb] -= I[0][a][b];
                    A[(nv + ra) * n2 + cb] -= I[3][a][b];
                    A[(nv + ra) * n2 + nv + cb] -= I[2][a][b];
                }
        }
    }
    return 0;
}

/* exported: piecewise-linear right-hand side, b_a = int psi_a S(x) / eps1 for both source terms
 * of source_terms, by the rule (the centroid rule weighs every corner by 1/3) */
void orc_p1_rhs(const double* V, const int32_t* T, int nt, int nv, const double* qpos, const double* q,
                int nc, double eps1, int nq, const double* qe1, const double* qe2, const double* qw,
                double* b)
{
    for (int k = 0; k < 2 * nv; ++k) b[k] = 0.0;
    for (int i = 0; i < nt; ++i) {
        double c[3], n[3], Ai, u[3], v[3], w[3];
        orc_tri(V, T, i, u, v, w);
        orc_geom(u, v, w, c, &Ai, n);
        for (int p = 0; p < nq; ++p) {
            double x[3], lam[3], t1, t2, wgt;
            if (nq == 1) {
                for (int k = 0; k < 3; ++k) x[k] = c[k];
                lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
                wgt = Ai;
            } else {
                orc_rule_point(u, v, w, qe1[p], qe2[p], x);
                orc_lambda(qe1[p], qe2[p], lam);
                wgt = 2.0 * Ai * qw[p];
            }
            orc_sources(x, n, qpos, q, nc, &t1, &t2);
            for (int a = 0; a < 3; ++a) {
                b[T[3 * i + a]] += wgt * lam[a] * t1 / eps1;
                b[nv + T[3 * i + a]] += wgt * lam[a] * t2 / eps1;
            }
        }
    }
}

/* exported: the energy of eqsolengdis for a piecewise-linear solution (the densities at each
 * rule point interpolated from the element's corners), kcal/mol as orc_energy */
double orc_p1_energy(const double* V, const int32_t* T, int nt, int nv, const double* qpos, const double* q,
                     int nc, double eps, double kappa, int nq, const double* qe1, const double* qe2,
                     const double* qw, const double* x)
{
    orc_phys ph = {eps, kappa};
    double zero[3] = {0.0, 0.0, 0.0};
    double E = 0.0;
    for (int k = 0; k < nc; ++k) {
        double sk = 0.0;
        for (int i = 0; i < nt; ++i) {
            double c[3], n[3], Ai, u[3], v[3], w[3];
            orc_tri(V, T, i, u, v, w);
            orc_geom(u, v, w, c, &Ai, n);
            for (int p = 0; p < nq; ++p) {
                double y[3], lam[3], K[4], wgt;
                if (nq == 1) {
                    for (int d = 0; d < 3; ++d) y[d] = c[d];
                    lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
                    wgt = Ai;
                } else {
                    orc_rule_point(u, v, w, qe1[p], qe2[p], y);
                    orc_lambda(qe1[p], qe2[p], lam);
                    wgt = 2.0 * Ai * qw[p];
                }
                double phv = 0.0, dphv = 0.0;
                for (int a = 0; a < 3; ++a) {
                    phv += lam[a] * x[T[3 * i + a]];
                    dphv += lam[a] * x[nv + T[3 * i + a]];
                }
                orc_kernels(qpos + 3 * k, zero, y, n, &ph, K);
                sk += wgt * (K[0] * dphv + K[1] * phv);
            }
        }
        E += q[k] * sk;
    }
    return 0.5 * E * 4.0 * ORC_PI * 332.0716;
}
