// Piecewise-linear Galerkin: continuous hat functions (S^1_h of Section 2.3, eqlinearfcn and
// eqglinearcfcn). The unknowns live at the vertices, x = [phi_v ; dphi_v] (2 nv values, the
// uploaded vertex order), and the system is
//    y1_a = 1/2 (1 + eps) sum_b M(a,b) phi_b - sum_b [I1(a,b) dphi_b + I2(a,b) phi_b]
//    y2_a = 1/2 (1 + 1/eps) sum_b M(a,b) dphi_b - sum_b [I3(a,b) dphi_b + I4(a,b) phi_b]
// with I_m(a,b) the kernel integrals weighted by the hat functions of a and b and M the mass
// matrix int psi_a psi_b (A (1 + [a == b]) / 12 per element).
//
// The product reuses the regular rule's points (order q >= 2): the densities at each point are
// interpolated from the element's corners (weights 1 - e1, e1 - e2, e2 at the point
// u + e1 (v - u) + e2 (w - v), the linear functions of eqlinearfcn); the far field runs on the
// points unchanged; the near field evaluates every point pair of non-identical neighbouring
// elements into per-point potentials; the test integrals weigh each point by the linear
// function of the corner; touching pairs (identical included) get stored 3 x 3 blocks of exact
// (Sauter-Schwab) minus order-q rule; everything is summed per element corner, then per vertex
// over the vertex's corners in a fixed order.
#include <algorithm>

#include "kernels.cuh"
#include "pb_internal.cuh"

#define P1_QMAX2 16

__constant__ double c_lam[3 * P1_QMAX2];  // c_lam[3 a + i]: linear function of corner i at rule point a

static inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// ---------- vertex lists ----------
__global__ void k_p1_vcount(int n3, const int* __restrict__ stris, int* __restrict__ vcnt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n3) atomicAdd(&vcnt[stris[e]], 1);
}

__global__ void k_p1_vkeys(int n3, const int* __restrict__ stris, unsigned* __restrict__ keys, int* __restrict__ vals)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n3) {
        keys[e] = (unsigned)stris[e];
        vals[e] = e;
    }
}

// ---------- points ----------
// xq[p] (both halves, stride np) = the element's corner values weighted at point p = k q2 + a
__global__ void k_p1_to_points(int nt, int q2, const int* __restrict__ stris, const double* __restrict__ x, int nv,
                               double* __restrict__ xq)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long np = (long long)nt * q2;
    if (p >= np) return;
    const int k = (int)(p / q2), a = (int)(p % q2);
    double s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < 3; ++i) {
        const int v = stris[3 * k + i];
        s1 += c_lam[3 * a + i] * x[v];
        s2 += c_lam[3 * a + i] * x[nv + v];
    }
    xq[p] = s1;
    xq[np + p] = s2;
}

// y[v] (both halves) = sum over the vertex's corners (k, i) of sum_a lam_i(a) yq[k q2 + a]
__global__ void k_p1_from_points(int nv, const int* __restrict__ voff, const int* __restrict__ vlist, int q2,
                                 long long np, const double* __restrict__ yq, double* __restrict__ y, int add)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double s1 = 0.0, s2 = 0.0;
    for (int t = voff[v]; t < voff[v + 1]; ++t) {
        const int e = vlist[t], k = e / 3, i = e % 3;
        for (int a = 0; a < q2; ++a) {
            s1 += c_lam[3 * a + i] * yq[(long long)k * q2 + a];
            s2 += c_lam[3 * a + i] * yq[np + (long long)k * q2 + a];
        }
    }
    y[v] = add ? y[v] + s1 : s1;
    y[nv + v] = add ? y[nv + v] + s2 : s2;
}

// ---------- set-up ----------
// take the order-q rule off the stored exact blocks of every non-identical touching pair
// (the near field evaluates those pairs with the rule); one warp per ordered pair, FP64
__global__ void __launch_bounds__(256) k_p1_rule(long long npairs, int nt, const int* __restrict__ toff,
                                                 const int* __restrict__ tj, int q2, const double4_32a* __restrict__ pp,
                                                 const double4_32a* __restrict__ en, double eps, double kappa,
                                                 double* __restrict__ corr1)
{
    const long long pair = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (pair >= npairs) return;
    int lo = 0, hi = nt;
    while (hi - lo > 1) {
        const int m = (lo + hi) / 2;
        if (toff[m] <= pair) lo = m;
        else hi = m;
    }
    const int k = lo, j = tj[pair];
    if (j == k) return;
    const double4_32a nk = en[k], nj = en[j];
    double acc[36];
    for (int e = 0; e < 36; ++e) acc[e] = 0.0;
    for (int t = lane; t < q2 * q2; t += 32) {
        const int a = t / q2, b = t % q2;
        const double4_32a x = pp[(long long)k * q2 + a], y = pp[(long long)j * q2 + b];
        double K[4];
        pb_kernels<double>(x.x - y.x, x.y - y.y, x.z - y.z, nk.x, nk.y, nk.z, nj.x, nj.y, nj.z, eps, 1.0 / eps, kappa,
                           K);
        const double w = x.w * y.w;
        for (int i = 0; i < 3; ++i)
            for (int bb = 0; bb < 3; ++bb) {
                const double wl = w * c_lam[3 * a + i] * c_lam[3 * b + bb];
                for (int m = 0; m < 4; ++m) acc[9 * m + 3 * i + bb] += wl * K[m];
            }
    }
    for (int e = 0; e < 36; ++e)
        for (int o = 16; o > 0; o >>= 1) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
    for (int e = lane; e < 36; e += 32) corr1[36 * pair + e] -= acc[e];
}

// 2 x 2 inverse per vertex of the system's diagonal block (exact entries):
//   [ 1/2 (1 + eps) M_vv - I2_vv   -I1_vv                     ]
//   [ -I4_vv                       1/2 (1 + 1/eps) M_vv - I3_vv ],   M_vv = sum A / 6
__global__ void k_p1_pinv(int nv, const int* __restrict__ voff, const int* __restrict__ vlist,
                          const double4_32a* __restrict__ ep, const double* __restrict__ diag, double eps,
                          double* __restrict__ pinv)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double M = 0.0;
    for (int t = voff[v]; t < voff[v + 1]; ++t) M += ep[vlist[t] / 3].w / 6.0;
    const double I1 = diag[4 * v], I2 = diag[4 * v + 1], I3 = diag[4 * v + 2], I4 = diag[4 * v + 3];
    const double d11 = 0.5 * (1.0 + eps) * M - I2, d12 = -I1, d21 = -I4, d22 = 0.5 * (1.0 + 1.0 / eps) * M - I3;
    const double det = d11 * d22 - d12 * d21;
    const bool ok = det != 0.0 && isfinite(det);  // a vertex of no element: identity
    pinv[4 * v] = ok ? d22 / det : 1.0;
    pinv[4 * v + 1] = ok ? -d12 / det : 0.0;
    pinv[4 * v + 2] = ok ? -d21 / det : 0.0;
    pinv[4 * v + 3] = ok ? d11 / det : 1.0;
}

__global__ void k_p1_precond(int nv, const double* __restrict__ pinv, const double* __restrict__ r,
                             double* __restrict__ z)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const double r1 = r[v], r2 = r[nv + v];
    z[v] = pinv[4 * v] * r1 + pinv[4 * v + 1] * r2;
    z[nv + v] = pinv[4 * v + 2] * r1 + pinv[4 * v + 3] * r2;
}

// ---------- near field ----------
// One block per leaf, one warp per target element k, the lanes over the source elements of the
// leaf's neighbour list (k itself excluded: its block is stored whole with the touching pairs).
// For every target point a: sum_j sum_b W_b [K1 dphi_b + K2 phi_b] (first half) and
// [K3 dphi_b + K4 phi_b] (second), the kernels in precision R, each source element's sum over
// its points in R and added in FP64. (Under mixed precision with 4 or 16 points per element the
// pair-tile kernel of the near field computes the same sums instead.)
template <class R, int Q2>
__global__ void __launch_bounds__(128) k_near_p1(int nt, const int* __restrict__ begin, const int* __restrict__ noff,
                                                 const int* __restrict__ nidx, const double4_32a* __restrict__ pp,
                                                 const double4_32a* __restrict__ en, const double* __restrict__ xq,
                                                 double eps, double kappa, double* __restrict__ yqn)
{
    const int c = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long np = (long long)nt * Q2;
    const R epsr = (R)eps, ieps = (R)(1.0 / eps), kap = (R)kappa;
    for (int k = begin[c] + warp; k < begin[c + 1]; k += 4) {
        const double4_32a nk = en[k];
        double y1[Q2], y2[Q2];
#pragma unroll
        for (int a = 0; a < Q2; ++a) y1[a] = y2[a] = 0.0;
        for (int t = noff[c]; t < noff[c + 1]; ++t) {
            const int c2 = nidx[t];
            for (int j = begin[c2] + lane; j < begin[c2 + 1]; j += 32) {
                if (j == k) continue;
                const double4_32a nj = en[j];
#pragma unroll
                for (int a = 0; a < Q2; ++a) {
                    const double4_32a x = pp[(long long)k * Q2 + a];
                    R s1 = 0, s2 = 0;
                    for (int b = 0; b < Q2; ++b) {
                        const double4_32a y = pp[(long long)j * Q2 + b];
                        const R ph = (R)xq[(long long)j * Q2 + b], dph = (R)xq[np + (long long)j * Q2 + b];
                        R K[4];
                        pb_kernels<R>((R)(x.x - y.x), (R)(x.y - y.y), (R)(x.z - y.z), (R)nk.x, (R)nk.y, (R)nk.z,
                                      (R)nj.x, (R)nj.y, (R)nj.z, epsr, ieps, kap, K);
                        const R wb = (R)y.w;
                        s1 += wb * (K[0] * dph + K[1] * ph);
                        s2 += wb * (K[2] * dph + K[3] * ph);
                    }
                    y1[a] += (double)s1;
                    y2[a] += (double)s2;
                }
            }
        }
#pragma unroll
        for (int a = 0; a < Q2; ++a)
            for (int o = 16; o > 0; o >>= 1) {
                y1[a] += __shfl_xor_sync(0xffffffffu, y1[a], o);
                y2[a] += __shfl_xor_sync(0xffffffffu, y2[a], o);
            }
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < Q2; ++a) {
                yqn[(long long)k * Q2 + a] = y1[a];
                yqn[np + (long long)k * Q2 + a] = y2[a];
            }
        }
    }
}

// per element corner (k, i), both halves: the near field's point sums weighed by -W_a and the
// corner's linear function, the mass terms and the touching pairs' stored blocks
__global__ void k_p1_local(int nt, int q2, const double* __restrict__ yqn, const double4_32a* __restrict__ pp,
                           const double4_32a* __restrict__ ep,
                           const int* __restrict__ stris, const double* __restrict__ x, int nv,
                           const int* __restrict__ toff, const int* __restrict__ tj,
                           const double* __restrict__ corr1, double eps, double* __restrict__ yl)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const long long np = (long long)nt * q2;
    double y1[3] = {0, 0, 0}, y2[3] = {0, 0, 0};
    for (int a = 0; a < q2; ++a) {
        const double W = pp[(long long)k * q2 + a].w;
        const double u1 = -W * yqn[(long long)k * q2 + a], u2 = -W * yqn[np + (long long)k * q2 + a];
        for (int i = 0; i < 3; ++i) {
            y1[i] += c_lam[3 * a + i] * u1;
            y2[i] += c_lam[3 * a + i] * u2;
        }
    }
    const double A = ep[k].w;
    int vk[3];
    for (int b = 0; b < 3; ++b) vk[b] = stris[3 * k + b];
    for (int i = 0; i < 3; ++i)
        for (int b = 0; b < 3; ++b) {
            const double M = A * (i == b ? 2.0 : 1.0) / 12.0;
            y1[i] += 0.5 * (1.0 + eps) * M * x[vk[b]];
            y2[i] += 0.5 * (1.0 + 1.0 / eps) * M * x[nv + vk[b]];
        }
    for (int t = toff[k]; t < toff[k + 1]; ++t) {
        const int j = tj[t];
        const double* C = corr1 + 36LL * t;
        for (int b = 0; b < 3; ++b) {
            const int v = stris[3 * j + b];
            const double ph = x[v], dph = x[nv + v];
            for (int i = 0; i < 3; ++i) {
                y1[i] -= C[3 * i + b] * dph + C[9 + 3 * i + b] * ph;
                y2[i] -= C[18 + 3 * i + b] * dph + C[27 + 3 * i + b] * ph;
            }
        }
    }
    for (int i = 0; i < 3; ++i) {
        yl[6LL * k + i] = y1[i];
        yl[6LL * k + 3 + i] = y2[i];
    }
}

// y[v] = sum over the vertex's corners of the corner rows + the far field's vertex rows
__global__ void k_p1_gather(int nv, const int* __restrict__ voff, const int* __restrict__ vlist,
                            const double* __restrict__ yl, const double* __restrict__ yfar, double* __restrict__ y)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double s1 = yfar[v], s2 = yfar[nv + v];
    for (int t = voff[v]; t < voff[v + 1]; ++t) {
        const int e = vlist[t], k = e / 3, i = e % 3;
        s1 += yl[6LL * k + i];
        s2 += yl[6LL * k + 3 + i];
    }
    y[v] = s1;
    y[nv + v] = s2;
}

// ---------- host side ----------
int pb_p1_to_points(pb_ctx* c, const double* x, double* xq, cudaStream_t st)
{
    const long long np = (long long)c->nt * c->q2;
    k_p1_to_points<<<nblk(np, 256), 256, 0, st>>>(c->nt, c->q2, c->stris, x, c->nv, xq);
    PB_LAUNCH(c);
    return PB_OK;
}

int pb_p1_from_points(pb_ctx* c, const double* yq, double* y, int add, cudaStream_t st)
{
    const long long np = (long long)c->nt * c->q2;
    k_p1_from_points<<<nblk(c->nv, 256), 256, 0, st>>>(c->nv, c->p1_voff, c->p1_vlist, c->q2, np, yq, y, add);
    PB_LAUNCH(c);
    return PB_OK;
}

// after the singular pass (which stored the exact blocks and the exact vertex diagonal)
int pb_p1_setup(pb_ctx* c)
{
    if (c->prm.basis != PB_BASIS_LINEAR) return PB_OK;
    const int nt = c->nt, nv = c->nv, q2 = c->q2;
    const int q = c->prm.qr;
    double e1[P1_QMAX2], e2[P1_QMAX2], w[P1_QMAX2], lam[3 * P1_QMAX2];
    pb_triangle_rule(q, e1, e2, w);
    for (int a = 0; a < q2; ++a) {
        lam[3 * a] = 1.0 - e1[a];
        lam[3 * a + 1] = e1[a] - e2[a];
        lam[3 * a + 2] = e2[a];
    }
    PB_CUDA(c, cudaMemcpyToSymbol(c_lam, lam, sizeof(double) * 3 * q2));
    // the vertex lists: corners 3 k + i sorted by vertex (ties in corner order), offsets by a scan
    const int n3 = 3 * nt;
    int* vcnt = (int*)pb_alloc(c, sizeof(int) * ((size_t)nv + 1));
    unsigned *keys = (unsigned*)pb_alloc(c, sizeof(unsigned) * n3), *skeys = (unsigned*)pb_alloc(c, sizeof(unsigned) * n3);
    int* vals = (int*)pb_alloc(c, sizeof(int) * n3);
    c->p1_voff = (int*)pb_alloc(c, sizeof(int) * ((size_t)nv + 1));
    c->p1_vlist = (int*)pb_alloc(c, sizeof(int) * n3);
    c->p1_pinv = (double*)pb_alloc(c, sizeof(double) * 4 * ((size_t)nv + 1));
    c->p1_yqn = (double*)pb_alloc(c, sizeof(double) * 2 * (size_t)nt * q2);
    c->p1_yl = (double*)pb_alloc(c, sizeof(double) * 6 * (size_t)nt);
    if (!vcnt || !keys || !skeys || !vals || !c->p1_voff || !c->p1_vlist || !c->p1_pinv || !c->p1_yqn || !c->p1_yl)
        return pb_fail(c, PB_ERR_NOMEM, "piecewise-linear set-up: out of memory");
    k_p1_vcount<<<nblk(n3, 256), 256, 0, c->st>>>(n3, c->stris, vcnt);
    PB_LAUNCH(c);
    int rc;
    if ((rc = pb_scan_exclusive(c, vcnt, c->p1_voff, nv))) return rc;
    k_p1_vkeys<<<nblk(n3, 256), 256, 0, c->st>>>(n3, c->stris, keys, vals);
    PB_LAUNCH(c);
    int bits = 1;
    while (bits < 31 && (1LL << bits) < nv) ++bits;
    if ((rc = pb_radix_sort_pairs(c, keys, vals, skeys, c->p1_vlist, n3, bits))) return rc;
    // the order-q rule off the touching pairs' exact blocks, then the preconditioner's inverses
    const double eps = c->prm.eps_out / c->prm.eps_in;
    if (c->ntouch > 0) {
        k_p1_rule<<<nblk(c->ntouch, 8), 256, 0, c->st>>>(c->ntouch, nt, c->touch_off, c->touch_j, q2, c->pts_p,
                                                         c->e64n, eps, c->prm.kappa, c->p1_corr);
        PB_LAUNCH(c);
    }
    k_p1_pinv<<<nblk(nv, 256), 256, 0, c->st>>>(nv, c->p1_voff, c->p1_vlist, c->e64p, c->p1_diag, eps, c->p1_pinv);
    PB_LAUNCH(c);
    return PB_OK;
}

template <class R, int Q2>
static void near_p1_launch(pb_ctx* c, const double* xq, double eps)
{
    const PbLevel& lv = c->lev[c->L];
    k_near_p1<R, Q2><<<lv.ncl, 128, 0, c->st>>>(c->nt, lv.begin, lv.near_off, lv.near_idx, c->pts_p, c->e64n, xq, eps,
                                                c->prm.kappa, c->p1_yqn);
}

// y = A x (vertex vectors of 2 nv). The far field (second stream) and the near field share the
// point densities xq, computed first; the far field ends in per-vertex rows (yfar).
int pb_p1_matvec(pb_ctx* c, const double* x, double* y)
{
    int rc;
    if ((rc = pb_matvec_reserve(c, 1))) return rc;
    const double eps = c->prm.eps_out / c->prm.eps_in;
    if ((rc = pb_p1_to_points(c, x, c->xq, c->st))) return rc;
    PB_CUDA(c, cudaEventRecord(c->ev_fork, c->st));
    PB_CUDA(c, cudaStreamWaitEvent(c->st2, c->ev_fork, 0));
    if ((rc = pb_far_apply(c, nullptr, c->yfar, 1, c->st2))) return rc;
    PB_CUDA(c, cudaEventRecord(c->ev_join, c->st2));
    pb_tic(c, PB_T_NEAR);
    const bool mixed = c->prm.precision == PB_MIXED;
    if (pb_near_points_ok(c)) {
        if ((rc = pb_near_points_apply(c, nullptr, c->xq, c->p1_yqn))) return rc;
    } else switch (c->q2) {
        case 4: mixed ? near_p1_launch<float, 4>(c, c->xq, eps) : near_p1_launch<double, 4>(c, c->xq, eps); break;
        case 9: mixed ? near_p1_launch<float, 9>(c, c->xq, eps) : near_p1_launch<double, 9>(c, c->xq, eps); break;
        case 16: mixed ? near_p1_launch<float, 16>(c, c->xq, eps) : near_p1_launch<double, 16>(c, c->xq, eps); break;
        default: return pb_fail(c, PB_ERR_ARG, "piecewise-linear basis: rule of %d points", c->q2);
    }
    if (!pb_near_points_ok(c)) PB_LAUNCH(c);
    pb_toc(c, PB_T_NEAR);
    pb_tic(c, PB_T_CORR);
    k_p1_local<<<nblk(c->nt, 128), 128, 0, c->st>>>(c->nt, c->q2, c->p1_yqn, c->pts_p, c->e64p, c->stris, x, c->nv,
                                                    c->touch_off,
                                                    c->touch_j, c->p1_corr, eps, c->p1_yl);
    PB_LAUNCH(c);
    PB_CUDA(c, cudaStreamWaitEvent(c->st, c->ev_join, 0));
    k_p1_gather<<<nblk(c->nv, 256), 256, 0, c->st>>>(c->nv, c->p1_voff, c->p1_vlist, c->p1_yl, c->yfar, y);
    PB_LAUNCH(c);
    pb_toc(c, PB_T_CORR);
    return PB_OK;
}

int pb_p1_precond(pb_ctx* c, const double* r, double* z)
{
    pb_tic(c, PB_T_PRECOND);
    if (c->prm.precond == PB_PRECOND_NONE) {
        PB_CUDA(c, cudaMemcpyAsync(z, r, sizeof(double) * 2 * (size_t)c->nv, cudaMemcpyDeviceToDevice, c->st));
    } else {
        k_p1_precond<<<nblk(c->nv, 256), 256, 0, c->st>>>(c->nv, c->p1_pinv, r, z);
        PB_LAUNCH(c);
    }
    pb_toc(c, PB_T_PRECOND);
    return PB_OK;
}
