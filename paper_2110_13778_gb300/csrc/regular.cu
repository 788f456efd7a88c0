// Regular quadrature of order q = 2..4 (Section 3.1, Table 2) in place of the one-point
// (centroid) rule for non-touching pairs, the right-hand side and the energy.
//
// The rule on the reference triangle {0 <= e2 <= e1 <= 1} is the collapsed product of a Gauss
// rule for the weight e1 in e1 (the Jacobian of e2 = e1 s) and a Gauss-Legendre rule in s:
// q^2 points, exact for polynomials of total degree 2q - 1, and for q = 1 the centroid with
// weight 1/2. On an element with corners u, v, w (as uploaded) the point is
// u + e1 (v - u) + e2 (w - v) and the weight 2 A w_a.
//
// Every element is expanded into its q^2 points (tree order, element-major), so the far field
// (P2M and LtP), the right-hand side and the energy run the one-point kernels unchanged on the
// points, followed by a sum over each element's points. The near field evaluates all q^2 x q^2
// point pairs of every non-identical pair in the neighbouring leaves, and the stored
// Sauter-Schwab corrections of touching pairs become exact minus the order-q rule.
#include <math.h>

#include <vector>

#include "kernels.cuh"
#include "pb_internal.cuh"

#define QMAX2 16  // points of the order-4 rule

__constant__ double c_qe1[QMAX2], c_qe2[QMAX2], c_qw[QMAX2];

// Gauss rule of a measure with monic recurrence coefficients a_k (k < n), b_k (1 <= k < n) and
// total mass mu0, nodes in [lo, hi]: each node by bisection on the Sturm count of the Jacobi
// matrix (number of negative pivots of J - tI = eigenvalues below t), each weight from the
// Christoffel function 1 / sum_{k<n} p_k(t)^2 of the orthonormal polynomials.
static void gauss_sturm(int n, const double* a, const double* b, double mu0, double lo, double hi, double* x,
                        double* w)
{
    auto below = [&](double t) {
        int cnt = 0;
        double d = 1.0;
        for (int k = 0; k < n; ++k) {
            d = (a[k] - t) - (k ? b[k] / d : 0.0);
            if (d == 0.0) d = -1e-300;
            cnt += d < 0.0;
        }
        return cnt;
    };
    for (int i = 0; i < n; ++i) {
        double l = lo, h = hi;
        for (int it = 0; it < 200 && h - l > 1e-17; ++it) {
            const double m = 0.5 * (l + h);
            if (m == l || m == h) break;
            if (below(m) > i) h = m; else l = m;
        }
        const double t = 0.5 * (l + h);
        double pm = 0.0, p = 1.0 / sqrt(mu0), s = p * p;
        for (int k = 0; k + 1 < n; ++k) {
            const double pn = ((t - a[k]) * p - (k ? sqrt(b[k]) : 0.0) * pm) / sqrt(b[k + 1]);
            pm = p;
            p = pn;
            s += p * p;
        }
        x[i] = t;
        w[i] = 1.0 / s;
    }
}

// order-q rule on the reference triangle: e1, e2, w of q^2 points (weights sum to 1/2)
void pb_triangle_rule(int q, double* e1, double* e2, double* w)
{
    if (q == 1) {
        e1[0] = 2.0 / 3.0;
        e2[0] = 1.0 / 3.0;
        w[0] = 0.5;
        return;
    }
    double a[8], b[8], t[8], wt[8], s[8], ws[8];
    // weight t on [0, 1]: a_k = (1 + 1/((2k+1)(2k+3))) / 2, b_k = k (k+1) / (4 (2k+1)^2), mass 1/2
    for (int k = 0; k < q; ++k) {
        a[k] = 0.5 * (1.0 + 1.0 / ((2.0 * k + 1.0) * (2.0 * k + 3.0)));
        b[k] = k ? k * (k + 1.0) / (4.0 * (2.0 * k + 1.0) * (2.0 * k + 1.0)) : 0.0;
    }
    gauss_sturm(q, a, b, 0.5, 0.0, 1.0, t, wt);
    // weight 1 on [0, 1]: a_k = 1/2, b_k = k^2 / (4 (4k^2 - 1)), mass 1
    for (int k = 0; k < q; ++k) {
        a[k] = 0.5;
        b[k] = k ? k * (double)k / (4.0 * (4.0 * k * k - 1.0)) : 0.0;
    }
    gauss_sturm(q, a, b, 1.0, 0.0, 1.0, s, ws);
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
            e1[i * q + j] = t[i];
            e2[i * q + j] = t[i] * s[j];
            w[i * q + j] = wt[i] * ws[j];
        }
}

// the points of every sorted element: (x, y, z, 2 A w_a) and the element's normal
__global__ void k_points(int nt, int q2, const int* __restrict__ stris, const double* __restrict__ V,
                         const double4_32a* __restrict__ ep, const double4_32a* __restrict__ en,
                         double4_32a* __restrict__ pp, double4_32a* __restrict__ pn)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)nt * q2) return;
    const int k = (int)(p / q2), a = (int)(p % q2);
    const double* u = V + 3 * stris[3 * k];
    const double* v = V + 3 * stris[3 * k + 1];
    const double* w = V + 3 * stris[3 * k + 2];
    const double e1 = c_qe1[a], e2 = c_qe2[a];
    double4_32a r;
    r.x = u[0] + e1 * (v[0] - u[0]) + e2 * (w[0] - v[0]);
    r.y = u[1] + e1 * (v[1] - u[1]) + e2 * (w[1] - v[1]);
    r.z = u[2] + e1 * (v[2] - u[2]) + e2 * (w[2] - v[2]);
    r.w = 2.0 * ep[k].w * c_qw[a];
    pp[p] = r;
    pn[p] = en[k];
}

__global__ void k_scale_begin(int n, int q2, const int* __restrict__ begin, int* __restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c <= n) out[c] = begin[c] * q2;
}

// xq = the element values at each of their points (both halves)
__global__ void k_to_points(int nt, int q2, const double* __restrict__ xs, double* __restrict__ xq)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long np = (long long)nt * q2;
    if (p >= np) return;
    const int k = (int)(p / q2);
    xq[p] = xs[k];
    xq[np + p] = xs[nt + k];
}

// ys = the sum over each element's points (both halves); add != 0 adds to ys
__global__ void k_from_points(int nt, int q2, const double* __restrict__ yq, double* __restrict__ ys, int add)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const long long np = (long long)nt * q2;
    double s1 = 0.0, s2 = 0.0;
    for (int a = 0; a < q2; ++a) {
        s1 += yq[(long long)k * q2 + a];
        s2 += yq[np + (long long)k * q2 + a];
    }
    ys[k] = add ? ys[k] + s1 : s1;
    ys[nt + k] = add ? ys[nt + k] + s2 : s2;
}

// order-q rule of the pair (k, j): sum_a sum_b W_a W_b K_m(x_a, y_b) in precision R
template <class R>
__device__ __forceinline__ void qrule_pair(int q2, const double4_32a* __restrict__ pp, int k, int j, const double4_32a& nk,
                                           const double4_32a& nj, R eps, R ieps, R kappa, R* I)
{
    R acc[4] = {0, 0, 0, 0};
    for (int a = 0; a < q2; ++a) {
        const double4_32a x = pp[(long long)k * q2 + a];
        for (int b = 0; b < q2; ++b) {
            const double4_32a y = pp[(long long)j * q2 + b];
            R K[4];
            pb_kernels<R>((R)(x.x - y.x), (R)(x.y - y.y), (R)(x.z - y.z), (R)nk.x, (R)nk.y, (R)nk.z, (R)nj.x,
                          (R)nj.y, (R)nj.z, eps, ieps, kappa, K);
            const R ww = (R)(x.w * y.w);
            for (int m = 0; m < 4; ++m) acc[m] += ww * K[m];
        }
    }
    for (int m = 0; m < 4; ++m) I[m] = acc[m];
}

// Near field of order q with the mass terms: one block per leaf, one warp per target element,
// the lanes over the source elements of the leaf's neighbour list (identical pair excluded;
// the touching pairs' corrections are added afterwards). Writes ys.
template <class R>
__global__ void __launch_bounds__(128) k_near_q(int nt, int q2, const int* __restrict__ begin,
                                                const int* __restrict__ noff, const int* __restrict__ nidx,
                                                const double4_32a* __restrict__ ep, const double4_32a* __restrict__ en,
                                                const double4_32a* __restrict__ pp, const double* __restrict__ xs,
                                                double eps, double kappa, double* __restrict__ ys)
{
    const int c = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const R epsr = (R)eps, ieps = (R)(1.0 / eps), kap = (R)kappa;
    for (int k = begin[c] + warp; k < begin[c + 1]; k += 4) {
        const double4_32a nk = en[k];
        double y1 = 0.0, y2 = 0.0;
        for (int t = noff[c]; t < noff[c + 1]; ++t) {
            const int c2 = nidx[t];
            for (int j = begin[c2] + lane; j < begin[c2 + 1]; j += 32) {
                if (j == k) continue;
                R I[4];
                qrule_pair<R>(q2, pp, k, j, nk, en[j], epsr, ieps, kap, I);
                const double ph = xs[j], dph = xs[nt + j];
                y1 += (double)I[0] * dph + (double)I[1] * ph;
                y2 += (double)I[2] * dph + (double)I[3] * ph;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            y1 += __shfl_xor_sync(0xffffffffu, y1, o);
            y2 += __shfl_xor_sync(0xffffffffu, y2, o);
        }
        if (lane == 0) {
            const double A = ep[k].w;
            ys[k] = 0.5 * (1.0 + eps) * A * xs[k] - y1;
            ys[nt + k] = 0.5 * (1.0 + 1.0 / eps) * A * xs[nt + k] - y2;
        }
    }
}

// corrections of touching pairs: exact - one-point (as the singular pass stored them) becomes
// exact - order-q rule (FP64)
__global__ void k_corr_q(int nt, int q2, const int* __restrict__ toff, const int* __restrict__ tj,
                         const double4_32a* __restrict__ ep, const double4_32a* __restrict__ en,
                         const double4_32a* __restrict__ pp, double eps, double kappa, double* __restrict__ corr)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const double4_32a pk = ep[k], nk = en[k];
    for (int t = toff[k]; t < toff[k + 1]; ++t) {
        const int j = tj[t];
        if (j == k) continue;
        const double4_32a pj = ep[j], nj = en[j];
        double one[4], I[4];
        pb_kernels<double>(pk.x - pj.x, pk.y - pj.y, pk.z - pj.z, nk.x, nk.y, nk.z, nj.x, nj.y, nj.z, eps, 1.0 / eps,
                           kappa, one);
        qrule_pair<double>(q2, pp, k, j, nk, nj, eps, 1.0 / eps, kappa, I);
        for (int m = 0; m < 4; ++m) corr[4LL * t + m] += pk.w * pj.w * one[m] - I[m];
    }
}

// build: the points, the leaf ranges in points and the corrections (after the singular pass)
int pb_regular_setup(pb_ctx* c)
{
    const int q = c->prm.qr > 1 ? c->prm.qr : 1;  // 0 and 1: the centroid rule
    const int q2 = q * q;
    c->q2 = q2;
    if (q2 == 1) return PB_OK;
    double e1[QMAX2], e2[QMAX2], w[QMAX2];
    pb_triangle_rule(q, e1, e2, w);
    PB_CUDA(c, cudaMemcpyToSymbol(c_qe1, e1, sizeof(double) * q2));
    PB_CUDA(c, cudaMemcpyToSymbol(c_qe2, e2, sizeof(double) * q2));
    PB_CUDA(c, cudaMemcpyToSymbol(c_qw, w, sizeof(double) * q2));
    const long long np = (long long)c->nt * q2;
    const PbLevel& lv = c->lev[c->L];
    c->pts_p = (double4_32a*)pb_alloc(c, sizeof(double4_32a) * np);
    c->pts_n = (double4_32a*)pb_alloc(c, sizeof(double4_32a) * np);
    c->begin_q = (int*)pb_alloc(c, sizeof(int) * (lv.ncl + 1));
    c->xq = (double*)pb_alloc(c, sizeof(double) * 2 * np);
    c->yq = (double*)pb_alloc(c, sizeof(double) * 2 * np);
    if (!c->pts_p || !c->pts_n || !c->begin_q || !c->xq || !c->yq)
        return pb_fail(c, PB_ERR_NOMEM, "regular rule: out of memory");
    k_points<<<(unsigned)((np + 255) / 256), 256, 0, c->st>>>(c->nt, q2, c->stris, c->verts, c->e64p, c->e64n,
                                                             c->pts_p, c->pts_n);
    PB_LAUNCH(c);
    k_scale_begin<<<(lv.ncl + 256) / 256, 256, 0, c->st>>>(lv.ncl, q2, lv.begin, c->begin_q);
    PB_LAUNCH(c);
    return PB_OK;
}

int pb_regular_corrections(pb_ctx* c)
{
    if (c->q2 <= 1) return PB_OK;
    const double eps = c->prm.eps_out / c->prm.eps_in;
    k_corr_q<<<(c->nt + 127) / 128, 128, 0, c->st>>>(c->nt, c->q2, c->touch_off, c->touch_j, c->e64p, c->e64n,
                                                     c->pts_p, eps, c->prm.kappa, c->corr);
    PB_LAUNCH(c);
    return PB_OK;
}

int pb_near_q_apply(pb_ctx* c, const double* xs, double* ys)
{
    if (pb_near_points_ok(c)) return pb_near_points_elem(c, xs, ys);
    const PbLevel& lv = c->lev[c->L];
    const double eps = c->prm.eps_out / c->prm.eps_in;
    if (c->prm.precision == PB_MIXED)
        k_near_q<float><<<lv.ncl, 128, 0, c->st>>>(c->nt, c->q2, lv.begin, lv.near_off, lv.near_idx, c->e64p, c->e64n,
                                                  c->pts_p, xs, eps, c->prm.kappa, ys);
    else
        k_near_q<double><<<lv.ncl, 128, 0, c->st>>>(c->nt, c->q2, lv.begin, lv.near_off, lv.near_idx, c->e64p,
                                                   c->e64n, c->pts_p, xs, eps, c->prm.kappa, ys);
    PB_LAUNCH(c);
    return PB_OK;
}

int pb_to_points(pb_ctx* c, const double* xs, double* xq, cudaStream_t st)
{
    if (c->prm.basis == PB_BASIS_LINEAR) return pb_p1_to_points(c, xs, xq, st);
    const long long np = (long long)c->nt * c->q2;
    k_to_points<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(c->nt, c->q2, xs, xq);
    PB_LAUNCH(c);
    return PB_OK;
}

int pb_from_points(pb_ctx* c, const double* yq, double* ys, int add, cudaStream_t st)
{
    if (c->prm.basis == PB_BASIS_LINEAR) return pb_p1_from_points(c, yq, ys, add, st);
    k_from_points<<<(c->nt + 255) / 256, 256, 0, st>>>(c->nt, c->q2, yq, ys, add);
    PB_LAUNCH(c);
    return PB_OK;
}
