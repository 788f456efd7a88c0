// Touching element pairs and their Galerkin integrals by the Sauter-Schwab singularity
// removing transformation (Section 2.3, the paragraph after the right-hand side: identical,
// edge-adjacent and vertex-adjacent triangles mapped to the 4-cube, tensor Gauss-Legendre).
//
// For every ordered pair (i, j) of triangles sharing at least one vertex the kernel stores
//   corr_m(i, j) = I_m(i, j) - [i != j] A_i A_j K_m(c_i, c_j),   m = 1..4,
// the exact (FP64, qs^4-point) integral minus the one-point rule that the near-field kernel
// applies to every non-identical pair. Adding corr to the near-field product therefore gives
// the Galerkin entries of eq_linsysEntry for touching pairs.

#include <math.h>

#include <vector>

#include "ff.cuh"
#include "kernels.cuh"
#include "pb_internal.cuh"

#define PB_MAXCAND 128  // candidates gathered from the three vertex stars of one triangle

__constant__ double c_gx[8], c_gw[8];

// Gauss-Legendre rule on [0,1] as in Golub and Welsch (Math. Comp. 23, 1969): the nodes are
// the eigenvalues of the symmetric tridiagonal Jacobi matrix of the Legendre polynomials
// (zero diagonal, off-diagonal b_k = k / sqrt(4k^2 - 1)), each found here by bisection on its
// Sturm count (the number of negative pivots of J - xI); the weights follow from the
// Christoffel function w = 1 / sum_{k<n} q_k(x)^2 of the orthonormal polynomials q_k.
static void gauss01(int n, double* x, double* w)
{
    auto b = [](int k) { return k / sqrt(4.0 * k * k - 1.0); };
    auto below = [&](double t) {  // eigenvalues of J smaller than t
        int cnt = 0;
        double d = 1.0;
        for (int k = 0; k < n; ++k) {
            double off = k ? b(k) : 0.0;
            d = -t - (k ? off * off / d : 0.0);
            if (d == 0.0) d = -1e-300;
            cnt += d < 0.0;
        }
        return cnt;
    };
    for (int i = 0; i < n; ++i) {
        double lo = -1.0, hi = 1.0;  // all nodes lie in (-1, 1)
        for (int it = 0; it < 200 && hi - lo > 1e-17; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (below(mid) > i) hi = mid; else lo = mid;
        }
        double t = 0.5 * (lo + hi);
        double qm = 0.0, q = 1.0 / sqrt(2.0), sum = q * q;
        for (int k = 0; k + 1 < n; ++k) {
            double qn = (t * q - (k ? b(k) : 0.0) * qm) / b(k + 1);
            qm = q;
            q = qn;
            sum += q * q;
        }
        x[i] = 0.5 * (1.0 + t);
        w[i] = 0.5 / sum;
    }
}

// ---------- vertex stars ----------
__global__ void k_vcount(int nt, const int* __restrict__ stris, int* __restrict__ vcnt)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nt)
        for (int a = 0; a < 3; ++a) atomicAdd(&vcnt[stris[3 * k + a]], 1);
}

__global__ void k_vfill(int nt, const int* __restrict__ stris, const int* __restrict__ voff,
                        int* __restrict__ vfill, int* __restrict__ vlist)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nt)
        for (int a = 0; a < 3; ++a) {
            int v = stris[3 * k + a];
            vlist[voff[v] + atomicAdd(&vfill[v], 1)] = k;
        }
}

// Touching triangles of k: the union of its three vertex stars (k itself included), sorted.
// PASS 0 counts, PASS 1 writes. Sets *bad if a star union exceeds PB_MAXCAND.
template <int PASS>
__global__ void k_touch(int nt, const int* __restrict__ stris, const int* __restrict__ voff,
                        const int* __restrict__ vlist, int* __restrict__ cnt,
                        const int* __restrict__ off, int* __restrict__ tj, int* __restrict__ bad)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    int cand[PB_MAXCAND];
    int n = 0;
    for (int a = 0; a < 3; ++a) {
        int v = stris[3 * k + a];
        for (int t = voff[v]; t < voff[v + 1]; ++t) {
            int j = vlist[t];
            bool seen = false;
            for (int q = 0; q < n; ++q) seen |= (cand[q] == j);
            if (!seen) {
                if (n == PB_MAXCAND) {
                    atomicExch(bad, 1);
                    if (!PASS) cnt[k] = 0;
                    return;
                }
                cand[n++] = j;
            }
        }
    }
    if (!PASS) {
        cnt[k] = n;
        return;
    }
    // insertion sort for a deterministic order
    for (int a = 1; a < n; ++a) {
        int v = cand[a], b = a - 1;
        while (b >= 0 && cand[b] > v) {
            cand[b + 1] = cand[b];
            --b;
        }
        cand[b + 1] = v;
    }
    for (int q = 0; q < n; ++q) tj[off[k] + q] = cand[q];
}

__global__ void k_touch_classes(int nt, const int* __restrict__ toff, const int* __restrict__ tj,
                                const int* __restrict__ stris, unsigned long long* __restrict__ cls)
{
    // per-warp sums first, then one atomic per warp and class (not one per thread)
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned n[4] = {0, 0, 0, 0};
    if (k < nt)
        for (int t = toff[k]; t < toff[k + 1]; ++t) {
            int j = tj[t], s = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) s += stris[3 * k + a] == stris[3 * j + b];
            n[s > 3 ? 3 : s]++;
        }
    for (int q = 1; q < 4; ++q) {
        const unsigned w = __reduce_add_sync(0xffffffffu, n[q]);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&cls[q], (unsigned long long)w);
    }
}

// ---------- Sauter-Schwab sub-maps (reference triangle {0 <= e2 <= e1 <= 1}) ----------
// Each writes xhat, yhat and the Jacobian weight of sub-map s at cube point (xi, h1, h2, h3).
__host__ __device__ __forceinline__ int ss_map(int shared, int s, double xi, double h1, double h2, double h3,
                                      double* xh, double* yh)
{
    double x0, x1, y0, y1, w;
    double xi3 = xi * xi * xi;
    if (shared == 3) {
        w = xi3 * h1 * h1 * h2;
        switch (s) {
            case 0: x0 = 1; x1 = 1 - h1 + h1 * h2; y0 = 1 - h1 * h2 * h3; y1 = 1 - h1; break;
            case 1: x0 = 1 - h1 * h2 * h3; x1 = 1 - h1; y0 = 1; y1 = 1 - h1 + h1 * h2; break;
            case 2: x0 = 1; x1 = h1 * (1 - h2 + h2 * h3); y0 = 1 - h1 * h2; y1 = h1 * (1 - h2); break;
            case 3: x0 = 1 - h1 * h2; x1 = h1 * (1 - h2); y0 = 1; y1 = h1 * (1 - h2 + h2 * h3); break;
            case 4: x0 = 1 - h1 * h2 * h3; x1 = h1 * (1 - h2 * h3); y0 = 1; y1 = h1 * (1 - h2); break;
            default: x0 = 1; x1 = h1 * (1 - h2); y0 = 1 - h1 * h2 * h3; y1 = h1 * (1 - h2 * h3); break;
        }
    } else if (shared == 2) {
        w = xi3 * h1 * h1 * (s == 0 ? 1.0 : h2);
        switch (s) {
            case 0: x0 = 1; x1 = h1 * h3; y0 = 1 - h1 * h2; y1 = h1 * (1 - h2); break;
            case 1: x0 = 1; x1 = h1; y0 = 1 - h1 * h2 * h3; y1 = h1 * h2 * (1 - h3); break;
            case 2: x0 = 1 - h1 * h2; x1 = h1 * (1 - h2); y0 = 1; y1 = h1 * h2 * h3; break;
            case 3: x0 = 1 - h1 * h2 * h3; x1 = h1 * h2 * (1 - h3); y0 = 1; y1 = h1; break;
            default: x0 = 1 - h1 * h2 * h3; x1 = h1 * (1 - h2 * h3); y0 = 1; y1 = h1 * h2; break;
        }
    } else {
        w = xi3 * h2;
        if (s == 0) {
            x0 = 1; x1 = h1; y0 = h2; y1 = h2 * h3;
        } else {
            x0 = h2; x1 = h2 * h1; y0 = 1; y1 = h3;
        }
    }
    xh[0] = xi * x0;
    xh[1] = xi * x1;
    yh[0] = xi * y0;
    yh[1] = xi * y1;
    return 0 * (int)w;  // unused
}

__host__ __device__ __forceinline__ double ss_weight(int shared, int s, double xi, double h1, double h2)
{
    double xi3 = xi * xi * xi;
    if (shared == 3) return xi3 * h1 * h1 * h2;
    if (shared == 2) return xi3 * h1 * h1 * (s == 0 ? 1.0 : h2);
    return xi3 * h2;
}

// One warp per touching pair (target k, source j). Lanes split the qs^4 cube points.
__global__ void __launch_bounds__(256) k_singular(long long npairs, int nt, const int* __restrict__ toff,
                                                  const int* __restrict__ tj, const int* __restrict__ stris,
                                                  const int* __restrict__ order, const double* __restrict__ V,
                                                  const double4_32a* __restrict__ ep,
                                                  const double4_32a* __restrict__ en, int qs, double eps,
                                                  double kappa, double* __restrict__ corr)
{
    long long pair = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (pair >= npairs) return;
    // target k: largest k with toff[k] <= pair
    int lo = 0, hi = nt;
    while (hi - lo > 1) {
        int m = (lo + hi) / 2;
        if (toff[m] <= pair) lo = m;
        else hi = m;
    }
    int k = lo, j = tj[pair];
    // One quadrature serves both orderings: it is laid out from the triangle with the smaller
    // element index (shared vertices first, in that triangle's order); that warp writes the
    // corrections of (k, j) and (j, k).
    if (order[k] > order[j]) return;
    int ti[3] = {stris[3 * k], stris[3 * k + 1], stris[3 * k + 2]};
    int tjv[3] = {stris[3 * j], stris[3 * j + 1], stris[3 * j + 2]};
    // shared vertices first, in the same order for both triangles
    int oi[3], oj[3], ns = 0;
    if (k == j) {
        ns = 3;
        for (int a = 0; a < 3; ++a) oi[a] = oj[a] = ti[a];
    } else {
        int usedi[3] = {0, 0, 0}, usedj[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (ti[a] == tjv[b]) {
                    oi[ns] = ti[a];
                    oj[ns] = tjv[b];
                    usedi[a] = usedj[b] = 1;
                    ++ns;
                }
        int p = ns, q = ns;
        for (int a = 0; a < 3; ++a)
            if (!usedi[a]) oi[p++] = ti[a];
        for (int b = 0; b < 3; ++b)
            if (!usedj[b]) oj[q++] = tjv[b];
    }
    double P[3][3], Q[3][3];
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) {
            P[a][d] = V[3 * oi[a] + d];
            Q[a][d] = V[3 * oj[a] + d];
        }
    double4_32a pi = ep[k], pj = ep[j], ni = en[k], nj = en[j];
    // Identical flat triangle: (x - y) is tangent, so the normal-derivative parts vanish and
    // K1, K4 depend on |x - y| only; the six sub-maps pair up under xhat <-> yhat (1-2, 3-4,
    // 5-6), so sub-maps 1, 3, 5 are evaluated with weight 2.
    const bool ident = ns == 3;
    const int nsub = ident ? 3 : (ns == 2 ? 5 : 2);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    int npts = qs * qs * qs * qs;
    double inv_eps = 1.0 / eps;
    double eP[2][3], eQ[2][3], d0[3];
    for (int e = 0; e < 3; ++e) {
        eP[0][e] = P[1][e] - P[0][e];
        eP[1][e] = P[2][e] - P[1][e];
        eQ[0][e] = Q[1][e] - Q[0][e];
        eQ[1][e] = Q[2][e] - Q[1][e];
        d0[e] = P[0][e] - Q[0][e];
    }
    for (int t = lane; t < npts; t += 32) {
        int a = t % qs, b = (t / qs) % qs, cc = (t / (qs * qs)) % qs, d = t / (qs * qs * qs);
        double xi = c_gx[a], h1 = c_gx[b], h2 = c_gx[cc], h3 = c_gx[d];
        double wq = c_gw[a] * c_gw[b] * c_gw[cc] * c_gw[d];
        for (int s = 0; s < nsub; ++s) {
            const int sm = ident ? 2 * s : s;
            double xh[2], yh[2];
            ss_map(ns, sm, xi, h1, h2, h3, xh, yh);
            double w = wq * ss_weight(ns, sm, xi, h1, h2) * (ident ? 2.0 : 1.0);
            double dv[3];
            for (int e = 0; e < 3; ++e)
                dv[e] = d0[e] + xh[0] * eP[0][e] + xh[1] * eP[1][e] - yh[0] * eQ[0][e] - yh[1] * eQ[1][e];
            double Pt[6];
            pb_kernel_parts<double>(dv[0], dv[1], dv[2], ni.x, ni.y, ni.z, nj.x, nj.y, nj.z, kappa, Pt);
            if (ident) {
                acc[0] += w * Pt[0];
                acc[1] += w * Pt[1];
            } else {
                for (int m = 0; m < 6; ++m) acc[m] += w * Pt[m];
            }
        }
    }
    for (int m = 0; m < 6; ++m)
        for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
    if (lane == 0) {
        double jac = (2.0 * pi.w) * (2.0 * pj.w);
        for (int m = 0; m < 6; ++m) acc[m] *= jac;
        // (k, j): target k, source j
        double Ikj[4] = {acc[0], eps * acc[3] - acc[2], -acc[4] + acc[5] * inv_eps, acc[1]};
        double reg[4] = {0, 0, 0, 0};
        if (k != j)
            pb_kernels<double>(pi.x - pj.x, pi.y - pj.y, pi.z - pj.z, ni.x, ni.y, ni.z, nj.x, nj.y, nj.z, eps,
                               inv_eps, kappa, reg);
        for (int m = 0; m < 4; ++m) corr[4 * pair + m] = Ikj[m] - pi.w * pj.w * reg[m];
        if (k != j) {
            // (j, k): the same integrals with the roles of the normals exchanged
            double Ijk[4] = {acc[0], acc[4] - eps * acc[5], acc[2] - acc[3] * inv_eps, acc[1]};
            pb_kernels<double>(pj.x - pi.x, pj.y - pi.y, pj.z - pi.z, nj.x, nj.y, nj.z, ni.x, ni.y, ni.z, eps,
                               inv_eps, kappa, reg);
            int q = toff[j];
            while (q < toff[j + 1] && tj[q] != k) ++q;
            if (q < toff[j + 1])
                for (int m = 0; m < 4; ++m) corr[4 * (long long)q + m] = Ijk[m] - pi.w * pj.w * reg[m];
        }
    }
}

// ---------- piecewise-linear basis (continuous hat functions, Section 2.3) ----------
// The same Sauter-Schwab quadrature weighted by the linear functions of both triangles: at the
// reference point (e1, e2) of a triangle laid out as P0 + e1 (P1 - P0) + e2 (P2 - P1) they are
// 1 - e1, e1 - e2 and e2 (eqlinearfcn), the weights of P0, P1 and P2. One warp per unordered
// touching pair, laid out from the triangle with the smaller element index as above; all six
// kernel parts and all sub-maps (the identical pair's x <-> y pairing of sub-maps does not
// carry over to the weighted integrand). The warp writes the 3 x 3 blocks of (k, j) and
// (j, k), corner indices in uploaded corner order: corr1[36 t + 9 m + 3 a + b] for kernel K_m,
// target corner a, source corner b; and adds every entry whose two corners are the same vertex
// into diag[4 v + m] (FP64 atomics: the exact diagonal of the vertex system).
__global__ void __launch_bounds__(256) k_singular_p1(long long npairs, int nt, const int* __restrict__ toff,
                                                     const int* __restrict__ tj, const int* __restrict__ stris,
                                                     const int* __restrict__ order, const double* __restrict__ V,
                                                     const double4_32a* __restrict__ ep,
                                                     const double4_32a* __restrict__ en, int qs, double eps,
                                                     double kappa, double* __restrict__ corr1,
                                                     double* __restrict__ diag)
{
    long long pair = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (pair >= npairs) return;
    int lo = 0, hi = nt;
    while (hi - lo > 1) {
        int m = (lo + hi) / 2;
        if (toff[m] <= pair) lo = m;
        else hi = m;
    }
    int k = lo, j = tj[pair];
    if (order[k] > order[j]) return;
    int ti[3] = {stris[3 * k], stris[3 * k + 1], stris[3 * k + 2]};
    int tjv[3] = {stris[3 * j], stris[3 * j + 1], stris[3 * j + 2]};
    // shared vertices first (in k's corner order), then the others; ci / cj: the corner index
    // of each laid-out position
    int ci[3], cj[3], ns = 0;
    if (k == j) {
        ns = 3;
        for (int a = 0; a < 3; ++a) ci[a] = cj[a] = a;
    } else {
        int usedi[3] = {0, 0, 0}, usedj[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (ti[a] == tjv[b]) {
                    ci[ns] = a;
                    cj[ns] = b;
                    usedi[a] = usedj[b] = 1;
                    ++ns;
                }
        int p = ns, q = ns;
        for (int a = 0; a < 3; ++a)
            if (!usedi[a]) ci[p++] = a;
        for (int b = 0; b < 3; ++b)
            if (!usedj[b]) cj[q++] = b;
    }
    double P[3][3], Q[3][3];
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) {
            P[a][d] = V[3 * ti[ci[a]] + d];
            Q[a][d] = V[3 * tjv[cj[a]] + d];
        }
    const double4_32a pi = ep[k], pj = ep[j], ni = en[k], nj = en[j];
    const int nsub = ns == 3 ? 6 : (ns == 2 ? 5 : 2);
    double acc[6][9];
    for (int m = 0; m < 6; ++m)
        for (int e = 0; e < 9; ++e) acc[m][e] = 0.0;
    const int npts = qs * qs * qs * qs;
    double eP[2][3], eQ[2][3], d0[3];
    for (int e = 0; e < 3; ++e) {
        eP[0][e] = P[1][e] - P[0][e];
        eP[1][e] = P[2][e] - P[1][e];
        eQ[0][e] = Q[1][e] - Q[0][e];
        eQ[1][e] = Q[2][e] - Q[1][e];
        d0[e] = P[0][e] - Q[0][e];
    }
    for (int t = lane; t < npts; t += 32) {
        int a = t % qs, b = (t / qs) % qs, cc = (t / (qs * qs)) % qs, d = t / (qs * qs * qs);
        double xi = c_gx[a], h1 = c_gx[b], h2 = c_gx[cc], h3 = c_gx[d];
        double wq = c_gw[a] * c_gw[b] * c_gw[cc] * c_gw[d];
        for (int sm = 0; sm < nsub; ++sm) {
            double xh[2], yh[2];
            ss_map(ns, sm, xi, h1, h2, h3, xh, yh);
            const double w = wq * ss_weight(ns, sm, xi, h1, h2);
            double dv[3];
            for (int e = 0; e < 3; ++e)
                dv[e] = d0[e] + xh[0] * eP[0][e] + xh[1] * eP[1][e] - yh[0] * eQ[0][e] - yh[1] * eQ[1][e];
            double Pt[6];
            pb_kernel_parts<double>(dv[0], dv[1], dv[2], ni.x, ni.y, ni.z, nj.x, nj.y, nj.z, kappa, Pt);
            const double lx[3] = {1.0 - xh[0], xh[0] - xh[1], xh[1]};
            const double ly[3] = {1.0 - yh[0], yh[0] - yh[1], yh[1]};
            for (int p = 0; p < 3; ++p)
                for (int r = 0; r < 3; ++r) {
                    const double wl = w * lx[p] * ly[r];
                    for (int m = 0; m < 6; ++m) acc[m][3 * p + r] += wl * Pt[m];
                }
        }
    }
    for (int m = 0; m < 6; ++m)
        for (int e = 0; e < 9; ++e)
            for (int o = 16; o > 0; o >>= 1) acc[m][e] += __shfl_xor_sync(0xffffffffu, acc[m][e], o);
    // lanes 0..8: one laid-out position pair (p, r) each
    if (lane < 9) {
        const int p = lane / 3, r = lane % 3;
        const double jac = (2.0 * pi.w) * (2.0 * pj.w);
        double A6[6];
        for (int m = 0; m < 6; ++m) A6[m] = acc[m][lane] * jac;
        const double inv_eps = 1.0 / eps;
        const int a = ci[p], b = cj[r];
        const bool same = ti[a] == tjv[b];
        // (k, j): target k (corner a), source j (corner b)
        const double Ikj[4] = {A6[0], eps * A6[3] - A6[2], -A6[4] + A6[5] * inv_eps, A6[1]};
        for (int m = 0; m < 4; ++m) {
            corr1[36 * pair + 9 * m + 3 * a + b] = Ikj[m];
            if (same) atomicAdd(&diag[4LL * ti[a] + m], Ikj[m]);
        }
        if (k != j) {
            // (j, k): target j (corner b), source k (corner a), the normals' roles exchanged
            const double Ijk[4] = {A6[0], A6[4] - eps * A6[5], A6[2] - A6[3] * inv_eps, A6[1]};
            int q = toff[j];
            while (q < toff[j + 1] && tj[q] != k) ++q;
            if (q < toff[j + 1])
                for (int m = 0; m < 4; ++m) {
                    corr1[36LL * q + 9 * m + 3 * b + a] = Ijk[m];
                    if (same) atomicAdd(&diag[4LL * ti[a] + m], Ijk[m]);
                }
        }
    }
}

// ---------- the same integrals in float-float arithmetic (mixed precision) ----------
// Every step of k_singular, carried out in float-float (ff.cuh) on the FP32 pipe: ~1e-13
// relative instead of FP64's ~1e-16, at a fraction of the FP64 pipe's time. The cube points
// of each Sauter-Schwab class come from a table built on the host in FP64, holding for each
// point the coefficients of x - y in the pair's edge vectors (so that x - y never forms as the
// difference of two absolute positions) and the quadrature weight. Per element, the three edge
// vectors, the unit normal, the centroid and the area are held as float-float records.

// g = e^-t - 1 + t and E = g - t in float-float. Below t = 0.5 from the Taylor series of
// g / t^2 = sum_k (-t)^k / (k + 2)!, the terms k >= 5 (at most 6.2e-6 of the sum) in FP32;
// above it from the FP64 exponential (touching pairs reach t = 0.5 only at kappa r = 0.5).
__device__ __forceinline__ void ff_screen(ff t, ff& E, ff& g)
{
    if (t.h < 0.5f) {
        const float mt = -t.h;
        float tail = (float)(1.0 / 1307674368000.0);  // 1/15!
        tail = fmaf(tail, mt, (float)(1.0 / 87178291200.0));
        tail = fmaf(tail, mt, (float)(1.0 / 6227020800.0));
        tail = fmaf(tail, mt, (float)(1.0 / 479001600.0));
        tail = fmaf(tail, mt, (float)(1.0 / 39916800.0));
        tail = fmaf(tail, mt, (float)(1.0 / 3628800.0));
        tail = fmaf(tail, mt, (float)(1.0 / 362880.0));
        tail = fmaf(tail, mt, (float)(1.0 / 40320.0));
        tail = fmaf(tail, mt, (float)(1.0 / 5040.0));  // k = 5: 1/7!
        const ff nt = ff_neg(t);
        constexpr double c4 = 1.0 / 720.0, c3 = 1.0 / 120.0, c2 = 1.0 / 24.0, c1 = 1.0 / 6.0;
        ff u = ff_add(ff_mul_f(nt, tail), ff{(float)c4, (float)(c4 - (double)(float)c4)});
        u = ff_add(ff_mul(nt, u), ff{(float)c3, (float)(c3 - (double)(float)c3)});
        u = ff_add(ff_mul(nt, u), ff{(float)c2, (float)(c2 - (double)(float)c2)});
        u = ff_add(ff_mul(nt, u), ff{(float)c1, (float)(c1 - (double)(float)c1)});
        u = ff_add_f(ff_mul(nt, u), 0.5f);
        g = ff_mul(u, ff_sqr(t));
        E = ff_sub(g, t);
    } else {
        const double td = ff_to(t);
        const double Ed = expm1(-td);
        E = ff_from(Ed);
        g = ff_from(Ed + td);
    }
}

// The six parts of pb_kernel_parts from r^2 and the normal projections n_x.d and n_y.d.
// PARTS = 2 computes P[0], P[1] only (identical triangles, where both projections vanish).
template <int PARTS>
__device__ __forceinline__ void ff_parts(ff r2, ff nxd, ff nyd, ff nxny, ff kap, ff* P)
{
    constexpr double i4pi = 0.07957747154594767;
    const ff I4PI = {(float)i4pi, (float)(i4pi - (double)(float)i4pi)};
    ff rinv = ff_rsqrt(r2);
    ff r = ff_mul(r2, rinv);
    ff t = ff_mul(kap, r);
    ff E, g;
    ff_screen(t, E, g);
    ff tE = ff_mul(t, E);
    ff c1 = ff_neg(ff_add(g, tE));
    ff rinv2 = ff_sqr(rinv);
    ff ri3 = ff_mul(ff_mul(rinv, I4PI), rinv2);
    P[0] = ff_neg(ff_mul(ff_mul(E, rinv), I4PI));
    if (PARTS == 2) {
        P[1] = ff_neg(ff_mul(ri3, ff_mul(c1, nxny)));
        return;
    }
    // c3 = -3 g - t^2 - t E (3 + t)
    ff c3 = ff_neg(ff_add(ff_add(ff_mul_f(g, 3.0f), ff_sqr(t)), ff_mul(tE, ff_add_f(t, 3.0f))));
    P[1] = ff_mul(ri3, ff_sub(ff_mul(ff_mul(c3, ff_mul(nxd, nyd)), rinv2), ff_mul(c1, nxny)));
    ff e1 = ff_add_f(ff_neg(c1), 1.0f);
    P[2] = ff_mul(nyd, ri3);
    P[3] = ff_mul(P[2], e1);
    P[4] = ff_mul(nxd, ri3);
    P[5] = ff_mul(P[4], e1);
}

// The parts of ff_parts, weighted by a quadrature weight w that carries the 1 / (4 pi), added
// into acc[0 .. PARTS): w is folded into 1 / r once (w / r, w / r^3), so each part costs one
// product fewer than forming it and then weighting it.
template <int PARTS>
__device__ __forceinline__ void ff_parts_w(ff w, ff r2, ff nxd, ff nyd, ff nxny, ff kap, ff* acc)
{
    ff rinv = ff_rsqrt(r2);
    ff r = ff_mul(r2, rinv);
    ff t = ff_mul(kap, r);
    ff E, g;
    ff_screen(t, E, g);
    ff tE = ff_mul(t, E);
    ff c1 = ff_neg(ff_add(g, tE));
    ff rinv2 = ff_sqr(rinv);
    const ff wri = ff_mul(w, rinv);       // w / (4 pi r)
    const ff wri3 = ff_mul(wri, rinv2);   // w / (4 pi r^3)
    acc[0] = ff_sub(acc[0], ff_mul(E, wri));
    if (PARTS == 2) {
        acc[1] = ff_sub(acc[1], ff_mul(wri3, ff_mul(c1, nxny)));
        return;
    }
    // c3 = -3 g - t^2 - t E (3 + t)
    ff c3 = ff_neg(ff_add(ff_add(ff_mul_f(g, 3.0f), ff_sqr(t)), ff_mul(tE, ff_add_f(t, 3.0f))));
    acc[1] = ff_add(acc[1], ff_mul(wri3, ff_sub(ff_mul(ff_mul(c3, ff_mul(nxd, nyd)), rinv2), ff_mul(c1, nxny))));
    ff e1 = ff_add_f(ff_neg(c1), 1.0f);
    const ff p2 = ff_mul(nyd, wri3), p4 = ff_mul(nxd, wri3);
    acc[2] = ff_add(acc[2], p2);
    acc[3] = ff_add(acc[3], ff_mul(p2, e1));
    acc[4] = ff_add(acc[4], p4);
    acc[5] = ff_add(acc[5], ff_mul(p4, e1));
}

__device__ __forceinline__ ff ff_dot3(const ff* a, const ff* b)
{
    return ff_add(ff_add(ff_mul(a[0], b[0]), ff_mul(a[1], b[1])), ff_mul(a[2], b[2]));
}

// Per sorted element: slots 0-8 the edge vectors e_a = v_{a+1} - v_a (a = 0, 1, 2, vertices in
// stris order), 9-11 the unit normal, 12-14 the centroid, 15 the area.
#define FF_ESLOTS 16
__global__ void k_elem_ff(int nt, const int* __restrict__ stris, const double* __restrict__ V,
                          const double4_32a* __restrict__ ep, const double4_32a* __restrict__ en,
                          float2* __restrict__ out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    float2* o = out + (size_t)k * FF_ESLOTS;
    for (int a = 0; a < 3; ++a) {
        const int u = stris[3 * k + a], w = stris[3 * k + (a + 1) % 3];
        for (int c = 0; c < 3; ++c) {
            ff e = ff_from(V[3 * w + c] - V[3 * u + c]);
            o[3 * a + c] = make_float2(e.h, e.l);
        }
    }
    const double4_32a p = ep[k], n = en[k];
    const double nv[3] = {n.x, n.y, n.z}, pv[4] = {p.x, p.y, p.z, p.w};
    for (int c = 0; c < 3; ++c) {
        ff a = ff_from(nv[c]);
        o[9 + c] = make_float2(a.h, a.l);
    }
    for (int c = 0; c < 4; ++c) {
        ff a = ff_from(pv[c]);
        o[12 + c] = make_float2(a.h, a.l);
    }
}

__device__ __forceinline__ ff ld_ff(const float2* p)
{
    float2 v = __ldg(p);
    return {v.x, v.y};
}

// edge vector from local vertex a to local vertex b of an element (b = a + 1 or a - 1 mod 3)
__device__ __forceinline__ void ff_edge(const float2* rec, int a, int b, ff* e)
{
    const bool fwd = b == (a + 1) % 3;
    const int slot = 3 * (fwd ? a : b);
    for (int c = 0; c < 3; ++c) {
        ff v = ld_ff(rec + slot + c);
        e[c] = fwd ? v : ff_neg(v);
    }
}

// Table of cube points per class (0: one shared vertex, 1: shared edge, 2: identical), each
// record the float-float coefficients (a0, a1, b0, b1) of x - y = a0 eP0 + a1 eP1 - b0 eQ0 -
// b1 eQ1 and the weight w (Gauss weights x Jacobian x symmetry factor x 1 / (4 pi)). For a shared edge
// eQ0 = eP0 is merged into a0; for identical triangles eQ = eP is merged into a0, a1.
struct SsTable {
    std::vector<float2> rec;  // [5][n]: a0, a1, b0, b1, w
    int off[3], cnt[3], n;
};

static void ss_table(int qs, SsTable& T)
{
    double gx[8], gw[8];
    gauss01(qs, gx, gw);
    const int q4 = qs * qs * qs * qs;
    const int nsub[3] = {2, 5, 3};
    std::vector<double> f[5];
    int n = 0;
    for (int cls = 0; cls < 3; ++cls) {
        const int ns = cls + 1;
        T.off[cls] = n;
        T.cnt[cls] = nsub[cls] * q4;
        for (int s = 0; s < nsub[cls]; ++s) {
            const int sm = ns == 3 ? 2 * s : s;
            for (int t = 0; t < q4; ++t) {
                int a = t % qs, b = (t / qs) % qs, c = (t / (qs * qs)) % qs, d = t / (qs * qs * qs);
                double xh[2], yh[2];
                ss_map(ns, sm, gx[a], gx[b], gx[c], gx[d], xh, yh);
                double w = gw[a] * gw[b] * gw[c] * gw[d] * ss_weight(ns, sm, gx[a], gx[b], gx[c]) *
                           (ns == 3 ? 2.0 : 1.0);
                double co[4];
                if (ns == 3) {
                    co[0] = xh[0] - yh[0];
                    co[1] = xh[1] - yh[1];
                    co[2] = co[3] = 0.0;
                } else if (ns == 2) {
                    co[0] = xh[0] - yh[0];
                    co[1] = xh[1];
                    co[2] = 0.0;
                    co[3] = yh[1];
                } else {
                    co[0] = xh[0];
                    co[1] = xh[1];
                    co[2] = yh[0];
                    co[3] = yh[1];
                }
                for (int m = 0; m < 4; ++m) f[m].push_back(co[m]);
                f[4].push_back(w * 0.07957747154594767);  // the weight carries the 1 / (4 pi)
                ++n;
            }
        }
    }
    T.n = n;
    T.rec.resize(5 * (size_t)n);
    for (int m = 0; m < 5; ++m)
        for (int i = 0; i < n; ++i) {
            ff v = ff_from(f[m][i]);
            T.rec[(size_t)m * n + i] = make_float2(v.h, v.l);
        }
}

// The cube points of one pair's class (lane, lane + stride, ...), one body per class: CLS = 0,
// a shared vertex (all four coefficients); 1, a shared edge (b0 = 0: eQ0 = eP0 is merged into
// a0); 2, identical triangles, where x - y lies in the triangle's own plane (only a0, a1 are
// nonzero) and both normal projections vanish, so only parts 0 and 1 of the kernel remain.
// Pairs are grouped by class, so the warps that run each body are uniform.
template <int CLS>
__device__ __forceinline__ void ss_points_ff(int lane, const float2* __restrict__ tab, int tn, int off, int cnt,
                                             const ff (*eP)[3], const ff (*eQ)[3], const ff* proj, ff nxny, ff kap,
                                             ff* acc, int stride)
{
    for (int i = off + lane; i < off + cnt; i += stride) {
        const ff a0 = ld_ff(tab + i), a1 = ld_ff(tab + tn + i), w = ld_ff(tab + 4 * tn + i);
        ff d[3];
        if (CLS == 2) {
            for (int c = 0; c < 3; ++c) d[c] = ff_add(ff_mul(a0, eP[0][c]), ff_mul(a1, eP[1][c]));
            const ff r2 = ff_add(ff_add(ff_sqr(d[0]), ff_sqr(d[1])), ff_sqr(d[2]));
            ff_parts_w<2>(w, r2, ff{0.f, 0.f}, ff{0.f, 0.f}, nxny, kap, acc);
        } else {
            const ff b0 = CLS == 1 ? ff{0.f, 0.f} : ld_ff(tab + 2 * tn + i), b1 = ld_ff(tab + 3 * tn + i);
            for (int c = 0; c < 3; ++c) {
                d[c] = ff_add(ff_mul(a0, eP[0][c]), ff_mul(a1, eP[1][c]));
                d[c] = ff_sub(d[c], CLS == 1 ? ff_mul(b1, eQ[1][c]) : ff_add(ff_mul(b0, eQ[0][c]), ff_mul(b1, eQ[1][c])));
            }
            const ff r2 = ff_add(ff_add(ff_sqr(d[0]), ff_sqr(d[1])), ff_sqr(d[2]));
            // n_x.(x - y) and n_y.(x - y): a triangle's own edges are orthogonal to its normal;
            // proj = {n_x.eQ0, n_x.eQ1, n_y.eP0, n_y.eP1}
            const ff nxd = ff_neg(CLS == 1 ? ff_mul(b1, proj[1]) : ff_add(ff_mul(b0, proj[0]), ff_mul(b1, proj[1])));
            const ff nyd = ff_add(ff_mul(a0, proj[2]), ff_mul(a1, proj[3]));
            ff_parts_w<6>(w, r2, nxd, nyd, nxny, kap, acc);
        }
    }
}

// Unordered touching pairs: the ordered pairs (k, j) with order[k] <= order[j] (the quadrature is
// laid out from the triangle of smaller element index), as (k, ordered-pair index), grouped
// by class: shared edge first (405 cube points at q_s = 3), then identical triangles (243),
// then a shared vertex (162), so that the 32 pairs of a warp share one trip count and the
// longest pairs start first. cnt[g nt + k]: pairs of group g whose first triangle is k.
__device__ __forceinline__ int canon_group(const int* __restrict__ stris, int k, int j)
{
    if (k == j) return 1;
    int ns = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) ns += stris[3 * k + a] == stris[3 * j + b];
    return ns == 2 ? 0 : 2;
}

template <int PASS>
__global__ void k_canon(int nt, const int* __restrict__ toff, const int* __restrict__ tj,
                        const int* __restrict__ order, const int* __restrict__ stris, int* __restrict__ cnt,
                        const int* __restrict__ coff, int* __restrict__ ck, int* __restrict__ cp, int cap)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    int n[3] = {0, 0, 0};
    if (PASS)
        for (int g = 0; g < 3; ++g) n[g] = coff[g * nt + k];
    for (int t = toff[k]; t < toff[k + 1]; ++t) {
        const int j = tj[t];
        if (order[k] <= order[j]) {
            const int g = canon_group(stris, k, j);
            if (PASS && n[g] < cap) {  // cap: the pairs allocated (a mismatch fails the build)
                ck[n[g]] = k;
                cp[n[g]] = t;
            }
            ++n[g];
        }
    }
    if (!PASS)
        for (int g = 0; g < 3; ++g) cnt[g * nt + k] = n[g];
}

// SS_LPP threads per unordered touching pair (1: one thread per pair). Pairs are grouped by
// class, so the pairs of a warp share one trip count and read the same (or neighbouring) table
// entries together. With one thread per pair no per-pair work is repeated across lanes, no
// cross-lane reduction is needed and no lane idles in a last, partial round of points (the
// warp-per-pair form of this kernel left 10 % of its point slots idle and repeated the pair's
// setup on 32 lanes). Both ordered entries, (k, j) and (j, k), come from the same sums and the
// same one-point evaluation (under the exchange d -> -d, n_x <-> n_y the parts 0 and 1 are
// unchanged and parts 2..5 map to -4, -5, -2, -3).
#define SS_LPP 1
__global__ void __launch_bounds__(128) k_singular_ff1(int ncanon, const int* __restrict__ ncanon_dev,
                                                      const int* __restrict__ ck, const int* __restrict__ cp,
                                                      const int* __restrict__ toff, const int* __restrict__ tj,
                                                      const int* __restrict__ stris, const float2* __restrict__ erec,
                                                      const float2* __restrict__ tab, int tn, int3 toffs, int3 tcnts,
                                                      ff kap, ff epsf, ff iepsf, double* __restrict__ corr)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = tid / SS_LPP, sub = tid % SS_LPP;
    // (all SS_LPP threads of a pair leave together: the shuffles below stay within live groups)
    if (w >= ncanon || w >= *ncanon_dev) return;  // allocated pairs, and those the scan found
    const int k = ck[w];
    const long long pair = cp[w];
    const int j = tj[pair];
    // local vertex indices (0..2) of both triangles, shared vertices first in k's order
    int oi[3], oj[3], ns = 0;
    if (k == j) {
        ns = 3;
        for (int a = 0; a < 3; ++a) oi[a] = oj[a] = a;
    } else {
        int usedi[3] = {0, 0, 0}, usedj[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (stris[3 * k + a] == stris[3 * j + b]) {
                    oi[ns] = a;
                    oj[ns] = b;
                    usedi[a] = usedj[b] = 1;
                    ++ns;
                }
        int p = ns, q = ns;
        for (int a = 0; a < 3; ++a)
            if (!usedi[a]) oi[p++] = a;
        for (int b = 0; b < 3; ++b)
            if (!usedj[b]) oj[q++] = b;
    }
    const float2* rk = erec + (size_t)k * FF_ESLOTS;
    const float2* rj = erec + (size_t)j * FF_ESLOTS;
    ff eP[2][3], eQ[2][3], ni[3], nj[3];
    ff_edge(rk, oi[0], oi[1], eP[0]);
    ff_edge(rk, oi[1], oi[2], eP[1]);
    ff_edge(rj, oj[0], oj[1], eQ[0]);
    ff_edge(rj, oj[1], oj[2], eQ[1]);
    for (int c = 0; c < 3; ++c) {
        ni[c] = ld_ff(rk + 9 + c);
        nj[c] = ld_ff(rj + 9 + c);
    }
    const ff nxny = ff_dot3(ni, nj);
    ff acc[6];
    for (int m = 0; m < 6; ++m) acc[m] = ff{0.f, 0.f};
    const ff z = {0.f, 0.f};
    ff proj[4] = {z, z, z, z};
    if (ns < 3) {
        proj[0] = ff_dot3(ni, eQ[0]);
        proj[1] = ff_dot3(ni, eQ[1]);
        proj[2] = ff_dot3(nj, eP[0]);
        proj[3] = ff_dot3(nj, eP[1]);
    }
    const int off = ns == 3 ? toffs.z : ns == 2 ? toffs.y : toffs.x;
    const int cnt = ns == 3 ? tcnts.z : ns == 2 ? tcnts.y : tcnts.x;
    if (ns == 3) ss_points_ff<2>(sub, tab, tn, off, cnt, eP, eQ, proj, nxny, kap, acc, SS_LPP);
    else if (ns == 2) ss_points_ff<1>(sub, tab, tn, off, cnt, eP, eQ, proj, nxny, kap, acc, SS_LPP);
    else ss_points_ff<0>(sub, tab, tn, off, cnt, eP, eQ, proj, nxny, kap, acc, SS_LPP);
    // the pair's own SS_LPP lanes, all alive (a pair's lanes leave together)
    const unsigned gmask = ((1u << SS_LPP) - 1u) << ((threadIdx.x & 31) & ~(SS_LPP - 1));
    for (int m = 0; m < 6; ++m)
        for (int o = 1; o < SS_LPP; o <<= 1) {
            ff v = {__shfl_xor_sync(gmask, acc[m].h, o), __shfl_xor_sync(gmask, acc[m].l, o)};
            acc[m] = ff_add(acc[m], v);
        }
    if (sub > 1) return;
    const ff Ak = ld_ff(rk + 15), Aj = ld_ff(rj + 15);
    const ff AA = ff_mul(Ak, Aj);
    const ff jac = ff_mul_f(AA, 4.0f);
    for (int m = 0; m < 6; ++m) acc[m] = ff_mul(acc[m], jac);
    // exact integrals of (k, j) and, with the normals exchanged, of (j, k)
    ff I[2][4];
    I[0][0] = I[1][0] = acc[0];
    I[0][3] = I[1][3] = acc[1];
    I[0][1] = ff_sub(ff_mul(epsf, acc[3]), acc[2]);
    I[0][2] = ff_sub(ff_mul(acc[5], iepsf), acc[4]);
    I[1][1] = ff_sub(acc[4], ff_mul(epsf, acc[5]));
    I[1][2] = ff_sub(acc[2], ff_mul(acc[3], iepsf));
    long long qr = pair;  // position of (j, k) in j's list
    if (k != j) {
        // one-point rule at the centroids for (k, j): d = c_k - c_j, n_x = n_k, n_y = n_j
        ff d[3];
        for (int c = 0; c < 3; ++c) d[c] = ff_sub(ld_ff(rk + 12 + c), ld_ff(rj + 12 + c));
        ff P[6];
        ff_parts<6>(ff_dot3(d, d), ff_dot3(ni, d), ff_dot3(nj, d), nxny, kap, P);
        const ff reg[2][4] = {{P[0], ff_sub(ff_mul(epsf, P[3]), P[2]), ff_sub(ff_mul(P[5], iepsf), P[4]), P[1]},
                              {P[0], ff_sub(P[4], ff_mul(epsf, P[5])), ff_sub(P[2], ff_mul(P[3], iepsf)), P[1]}};
        for (int o = 0; o < 2; ++o)
            for (int m = 0; m < 4; ++m) I[o][m] = ff_sub(I[o][m], ff_mul(AA, reg[o][m]));
        qr = toff[j];
        while (qr < toff[j + 1] && tj[qr] != k) ++qr;
    }
    if (sub == 0) {
        double2* o0 = (double2*)(corr + 4 * pair);
        o0[0] = make_double2(ff_to(I[0][0]), ff_to(I[0][1]));
        o0[1] = make_double2(ff_to(I[0][2]), ff_to(I[0][3]));
    }
    if (sub == (SS_LPP > 1 ? 1 : 0) && k != j && qr < toff[j + 1]) {
        double2* o1 = (double2*)(corr + 4 * qr);
        o1[0] = make_double2(ff_to(I[1][0]), ff_to(I[1][1]));
        o1[1] = make_double2(ff_to(I[1][2]), ff_to(I[1][3]));
    }
}

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

int pb_touching_and_singular(pb_ctx* c)
{
    const int nt = c->nt, nv = c->nv, B = 256;
    int* vcnt = (int*)pb_alloc(c, sizeof(int) * (nv + 1));
    int* voff = (int*)pb_alloc(c, sizeof(int) * (nv + 1));
    int* vfill = (int*)pb_alloc(c, sizeof(int) * (nv + 1));
    int* vlist = (int*)pb_alloc(c, sizeof(int) * 3 * nt);
    int* tcnt = (int*)pb_alloc(c, sizeof(int) * (nt + 1));
    int* bad = (int*)pb_alloc(c, sizeof(int));
    c->touch_off = (int*)pb_alloc(c, sizeof(int) * (nt + 1));
    if (!vcnt || !voff || !vfill || !vlist || !tcnt || !bad || !c->touch_off)
        return pb_fail(c, PB_ERR_NOMEM, "touching: out of memory");
    k_vcount<<<nblk(nt, B), B, 0, c->st>>>(nt, c->stris, vcnt);
    PB_LAUNCH(c);
    if (int rc = pb_scan_exclusive(c, vcnt, voff, nv)) return rc;
    k_vfill<<<nblk(nt, B), B, 0, c->st>>>(nt, c->stris, voff, vfill, vlist);
    PB_LAUNCH(c);
    k_touch<0><<<nblk(nt, 128), 128, 0, c->st>>>(nt, c->stris, voff, vlist, tcnt, nullptr, nullptr, bad);
    PB_LAUNCH(c);
    if (int rc = pb_scan_exclusive(c, tcnt, c->touch_off, nt)) return rc;
    int hb = 0, htot = 0;
    PB_CUDA(c, cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaMemcpyAsync(&htot, c->touch_off + nt, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    if (hb) return pb_fail(c, PB_ERR_MESH, "a triangle touches more than %d others", PB_MAXCAND);
    c->ntouch = htot;
    c->touch_j = (int*)pb_alloc(c, sizeof(int) * (htot + 1));
    c->corr = (double*)pb_alloc(c, sizeof(double) * 4 * (htot + 1));
    if (!c->touch_j || !c->corr) return pb_fail(c, PB_ERR_NOMEM, "touching: out of memory");
    k_touch<1><<<nblk(nt, 128), 128, 0, c->st>>>(nt, c->stris, voff, vlist, nullptr, c->touch_off, c->touch_j, bad);
    PB_LAUNCH(c);
    {
        // ordered touching pairs by number of shared vertices (for the work counts of reports;
        // left on the device until they are asked for)
        unsigned long long* cls = (unsigned long long*)pb_alloc(c, sizeof(unsigned long long) * 4);
        if (!cls) return pb_fail(c, PB_ERR_NOMEM, "touching: out of memory");
        k_touch_classes<<<nblk(nt, 128), 128, 0, c->st>>>(nt, c->touch_off, c->touch_j, c->stris, cls);
        PB_LAUNCH(c);
        c->touch_class_dev = cls;  // read back by pb_get_tree_stats
    }
    // Gauss-Legendre rule of the 4-cube
    double gx[8] = {0}, gw[8] = {0};
    gauss01(c->prm.qs, gx, gw);
    // (upload sources live in the context until the next build: no synchronisation needed)
    c->h_up_d.assign(gx, gx + 8);
    c->h_up_d.insert(c->h_up_d.end(), gw, gw + 8);
    PB_CUDA(c, cudaMemcpyToSymbolAsync(c_gx, c->h_up_d.data(), sizeof(gx), 0, cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyToSymbolAsync(c_gw, c->h_up_d.data() + 8, sizeof(gw), 0, cudaMemcpyHostToDevice, c->st));
    double eps = c->prm.eps_out / c->prm.eps_in;
    if (c->prm.basis == PB_BASIS_LINEAR) {
        // the vertex system's blocks (FP64); the order-q rule part is taken off afterwards
        c->p1_corr = (double*)pb_alloc(c, sizeof(double) * 36 * (size_t)(htot + 1));
        c->p1_diag = (double*)pb_alloc(c, sizeof(double) * 4 * (size_t)(c->nv + 1));
        if (!c->p1_corr || !c->p1_diag) return pb_fail(c, PB_ERR_NOMEM, "singular: out of memory");
        k_singular_p1<<<nblk(htot, 8), 256, 0, c->st>>>(htot, nt, c->touch_off, c->touch_j, c->stris, c->order,
                                                        c->verts, c->e64p, c->e64n, c->prm.qs, eps, c->prm.kappa,
                                                        c->p1_corr, c->p1_diag);
        PB_LAUNCH(c);
        return PB_OK;
    }
    const int mode = c->prm.singular ? c->prm.singular : (c->prm.precision == PB_MIXED ? PB_SINGULAR_FF : PB_SINGULAR_FP64);
    if (mode == PB_SINGULAR_FP64) {
        k_singular<<<nblk(htot, 8), 256, 0, c->st>>>(htot, nt, c->touch_off, c->touch_j, c->stris, c->order, c->verts,
                                                     c->e64p, c->e64n, c->prm.qs, eps, c->prm.kappa, c->corr);
        PB_LAUNCH(c);
        return PB_OK;
    }
    SsTable T;
    ss_table(c->prm.qs, T);
    float2* tab = (float2*)pb_alloc(c, sizeof(float2) * T.rec.size());
    float2* erec = (float2*)pb_alloc(c, sizeof(float2) * FF_ESLOTS * (size_t)nt);
    if (!tab || !erec) return pb_fail(c, PB_ERR_NOMEM, "singular: out of memory");
    c->h_up_f2.swap(T.rec);
    PB_CUDA(c, cudaMemcpyAsync(tab, c->h_up_f2.data(), sizeof(float2) * c->h_up_f2.size(), cudaMemcpyHostToDevice,
                               c->st));
    k_elem_ff<<<nblk(nt, B), B, 0, c->st>>>(nt, c->stris, c->verts, c->e64p, c->e64n, erec);
    PB_LAUNCH(c);
    // unordered pairs
    // (three groups of nt counts: shared edge, identical, shared vertex)
    int* ccnt = (int*)pb_alloc(c, sizeof(int) * (3 * nt + 1));
    int* coff = (int*)pb_alloc(c, sizeof(int) * (3 * nt + 1));
    if (!ccnt || !coff) return pb_fail(c, PB_ERR_NOMEM, "singular: out of memory");
    k_canon<0><<<nblk(nt, B), B, 0, c->st>>>(nt, c->touch_off, c->touch_j, c->order, c->stris, ccnt, nullptr, nullptr,
                                             nullptr, 0);
    PB_LAUNCH(c);
    if (int rc = pb_scan_exclusive(c, ccnt, coff, 3 * nt)) return rc;
    // Touching is symmetric and every triangle touches itself, so the unordered pairs number
    // (ordered pairs + nt) / 2; the kernel takes the count from the scan (coff[3 nt]) and the
    // build checks the two agree when it synchronises at its end.
    const int ncanon = (int)((htot + (long long)nt) / 2);
    c->canon_check = coff + 3 * nt;
    c->canon_expect = ncanon;
    int* ck = (int*)pb_alloc(c, sizeof(int) * (ncanon + 1));
    int* cp = (int*)pb_alloc(c, sizeof(int) * (ncanon + 1));
    if (!ck || !cp) return pb_fail(c, PB_ERR_NOMEM, "singular: out of memory");
    k_canon<1><<<nblk(nt, B), B, 0, c->st>>>(nt, c->touch_off, c->touch_j, c->order, c->stris, nullptr, coff, ck, cp,
                                             ncanon);
    PB_LAUNCH(c);
    k_singular_ff1<<<nblk((long long)ncanon * SS_LPP, 128), 128, 0, c->st>>>(ncanon, coff + 3 * nt, ck, cp, c->touch_off, c->touch_j, c->stris, erec, tab,
                                                    T.n, make_int3(T.off[0], T.off[1], T.off[2]),
                                                    make_int3(T.cnt[0], T.cnt[1], T.cnt[2]), ff_from(c->prm.kappa),
                                                    ff_from(eps), ff_from(1.0 / eps), c->corr);
    PB_LAUNCH(c);
    // (the singular pass is left running)
    return PB_OK;
}
