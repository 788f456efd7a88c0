// Touching element pairs and their Galerkin integrals by the Sauter-Schwab singularity
// removing transformation (Section 2.3, the paragraph after the right-hand side: identical,
// edge-adjacent and vertex-adjacent triangles mapped to the 4-cube, tensor Gauss-Legendre).
//
// For every ordered pair (i, j) of triangles sharing at least one vertex the kernel stores
//   corr_m(i, j) = I_m(i, j) - [i != j] A_i A_j K_m(c_i, c_j),   m = 1..4,
// the exact (FP64, qs^4-point) integral minus the one-point rule that the near-field kernel
// applies to every non-identical pair. Adding corr to the near-field product therefore gives
// the Galerkin entries of eq_linsysEntry for touching pairs.
#include <cub/cub.cuh>

#include <math.h>

#include <vector>

#include "kernels.cuh"
#include "pb_internal.cuh"

#define PB_MAXCAND 128  // candidates gathered from the three vertex stars of one triangle

__constant__ double c_gx[8], c_gw[8];

// Gauss-Legendre nodes on [0,1] by Newton's method on the Legendre recurrence
static void gauss01(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(PB_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = n == 1 ? z : p1, pm = n == 1 ? 1.0 : p0;
            double dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) {
                p0 = 1.0;
                p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                pn = n == 1 ? z : p1;
                pm = n == 1 ? 1.0 : p0;
                dp = n * (z * pn - pm) / (z * z - 1.0);
                w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/(..) on [-1,1], halved for [0,1]
                x[i] = 0.5 * (1.0 - z);
                break;
            }
        }
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
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    unsigned long long n[4] = {0, 0, 0, 0};
    for (int t = toff[k]; t < toff[k + 1]; ++t) {
        int j = tj[t], s = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) s += stris[3 * k + a] == stris[3 * j + b];
        n[s > 3 ? 3 : s]++;
    }
    for (int q = 1; q < 4; ++q)
        if (n[q]) atomicAdd(&cls[q], n[q]);
}

// ---------- Sauter-Schwab sub-maps (reference triangle {0 <= e2 <= e1 <= 1}) ----------
// Each writes xhat, yhat and the Jacobian weight of sub-map s at cube point (xi, h1, h2, h3).
__device__ __forceinline__ int ss_map(int shared, int s, double xi, double h1, double h2, double h3,
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

__device__ __forceinline__ double ss_weight(int shared, int s, double xi, double h1, double h2)
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
    size_t tmp = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tmp, vcnt, voff, nv + 1, c->st);
    void* t = nullptr;
    PB_CUDA(c, cudaMallocAsync(&t, tmp, c->st));
    cub::DeviceScan::ExclusiveSum(t, tmp, vcnt, voff, nv + 1, c->st);
    PB_LAUNCH(c);
    k_vfill<<<nblk(nt, B), B, 0, c->st>>>(nt, c->stris, voff, vfill, vlist);
    PB_LAUNCH(c);
    k_touch<0><<<nblk(nt, 128), 128, 0, c->st>>>(nt, c->stris, voff, vlist, tcnt, nullptr, nullptr, bad);
    PB_LAUNCH(c);
    size_t tmp2 = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tmp2, tcnt, c->touch_off, nt + 1, c->st);
    if (tmp2 > tmp) {
        PB_CUDA(c, cudaFreeAsync(t, c->st));
        PB_CUDA(c, cudaMallocAsync(&t, tmp2, c->st));
        tmp = tmp2;
    }
    cub::DeviceScan::ExclusiveSum(t, tmp, tcnt, c->touch_off, nt + 1, c->st);
    PB_LAUNCH(c);
    PB_CUDA(c, cudaFreeAsync(t, c->st));
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
        // ordered touching pairs by number of shared vertices (for the work counts of reports)
        unsigned long long* cls = (unsigned long long*)pb_alloc(c, sizeof(unsigned long long) * 4);
        if (!cls) return pb_fail(c, PB_ERR_NOMEM, "touching: out of memory");
        k_touch_classes<<<nblk(nt, 128), 128, 0, c->st>>>(nt, c->touch_off, c->touch_j, c->stris, cls);
        PB_LAUNCH(c);
        unsigned long long h[4];
        PB_CUDA(c, cudaMemcpyAsync(h, cls, sizeof(h), cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
        for (int q = 0; q < 4; ++q) c->touch_class[q] = (long long)h[q];
    }
    // Gauss-Legendre rule of the 4-cube
    double gx[8] = {0}, gw[8] = {0};
    gauss01(c->prm.qs, gx, gw);
    PB_CUDA(c, cudaMemcpyToSymbolAsync(c_gx, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyToSymbolAsync(c_gw, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, c->st));
    double eps = c->prm.eps_out / c->prm.eps_in;
    k_singular<<<nblk(htot, 8), 256, 0, c->st>>>(htot, nt, c->touch_off, c->touch_j, c->stris, c->order, c->verts, c->e64p,
                                                 c->e64n, c->prm.qs, eps, c->prm.kappa, c->corr);
    PB_LAUNCH(c);
    return PB_OK;
}
