// Right-hand side (source_terms), solvation energy (eqsolengdis) and restarted GMRES with
// right preconditioning (Section 2.3 last paragraph; Section 2.6). All vectors are in tree
// order. Arnoldi orthogonalisation (classical Gram-Schmidt applied twice), Givens rotations,
// the triangular solve and the update run in FP64 kernels; the host only reads one residual
// estimate per iteration to decide whether to continue.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "f32x2.cuh"
#include "kernels.cuh"
#include "pb_internal.cuh"

#define KB 256

// ---------- right-hand side: b1 = A S1(c), b2 = A S2(c) ----------
// FP64: every pair in double precision. Mixed: pair terms in FP32 with hi + lo coordinates
// (separations keep FP32 relative accuracy), each tile of charges summed in FP32 and added
// into FP64 accumulators.
template <class R>
struct RhsCharge {
    R x, y, z, q;
};

// Each thread takes two target elements (k and k + blockDim.x of the block's pair of slices),
// so that every staged charge (its hi and lo coordinates and charge: two broadcast
// shared-memory reads) serves two pair evaluations.
template <class R>
__global__ void __launch_bounds__(KB) k_rhs(int nt, int nc, const double4_32a* __restrict__ ep,
                                            const double4_32a* __restrict__ en, const double* __restrict__ qpos,
                                            const double* __restrict__ q, double eps1, double* __restrict__ b)
{
    __shared__ RhsCharge<R> shq[KB], slo[KB];
    const int k0 = blockIdx.x * 2 * KB + threadIdx.x;
    R ph[2][3], pl[2][3], nr[2][3];
    double w[2];
    bool act[2];
    for (int u = 0; u < 2; ++u) {
        const int k = k0 + u * KB;
        act[u] = k < nt;
        double4_32a p = make_double4_32a(0, 0, 0, 0), n = p;
        if (act[u]) {
            p = ep[k];
            n = en[k];
        }
        const double pc[3] = {p.x, p.y, p.z}, nc3[3] = {n.x, n.y, n.z};
        for (int a = 0; a < 3; ++a) {
            ph[u][a] = (R)pc[a];
            pl[u][a] = (R)(pc[a] - (double)ph[u][a]);
            nr[u][a] = (R)nc3[a];
        }
        w[u] = p.w;
    }
    double s1[2] = {0.0, 0.0}, s2[2] = {0.0, 0.0};
    const double i4pi = 0.07957747154594767;
    for (int t0 = 0; t0 < nc; t0 += KB) {
        __syncthreads();
        if (t0 + threadIdx.x < nc) {
            const int t = t0 + threadIdx.x;
            const double v[3] = {qpos[3 * t], qpos[3 * t + 1], qpos[3 * t + 2]};
            const R h[3] = {(R)v[0], (R)v[1], (R)v[2]};
            shq[threadIdx.x] = {h[0], h[1], h[2], (R)q[t]};
            slo[threadIdx.x] = {(R)(v[0] - (double)h[0]), (R)(v[1] - (double)h[1]), (R)(v[2] - (double)h[2]), R(0)};
        }
        __syncthreads();
        const int m = min(KB, nc - t0);
        R a1[2] = {0, 0}, a2[2] = {0, 0};
        for (int t = 0; t < m; ++t) {
            const RhsCharge<R> ch = shq[t], cl = slo[t];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const R dx = (ph[u][0] - ch.x) + (pl[u][0] - cl.x);
                const R dy = (ph[u][1] - ch.y) + (pl[u][1] - cl.y);
                const R dz = (ph[u][2] - ch.z) + (pl[u][2] - cl.z);
                const R r2 = dx * dx + dy * dy + dz * dz;
                const R ri = PbKer<R>::rsqrt_(r2);
                const R nd = nr[u][0] * dx + nr[u][1] * dy + nr[u][2] * dz;
                const R qr = ch.q * ri;
                a1[u] += qr;
                a2[u] -= qr * nd * ri * ri;  // dG0/dn_x = -(n.d)/(4 pi r^3)
            }
        }
        for (int u = 0; u < 2; ++u) {
            s1[u] += (double)a1[u];
            s2[u] += (double)a2[u];
        }
    }
    for (int u = 0; u < 2; ++u) {
        const int k = k0 + u * KB;
        if (act[u]) {
            b[k] = w[u] * s1[u] * i4pi / eps1;
            b[nt + k] = w[u] * s2[u] * i4pi / eps1;
        }
    }
}

// The mixed-precision form on packed FP32 pairs: the two target elements of a thread are the
// two halves of every f32x2 operation, and each staged charge is stored duplicated in both
// halves (x, x, y, y), (z, z, q, q) and (x_lo, x_lo, y_lo, y_lo), (z_lo, z_lo, 0, 0), so one
// instruction does the work of both pair evaluations; only the reciprocal square root runs per
// half.
__global__ void __launch_bounds__(KB, 4) k_rhs_x2(int nt, int nc, const double4_32a* __restrict__ ep,
                                               const double4_32a* __restrict__ en, const double* __restrict__ qpos,
                                               const double* __restrict__ q, double eps1, double* __restrict__ b)
{
    __shared__ float4 sq[4][KB];
    const int k0 = blockIdx.x * 2 * KB + threadIdx.x;
    float ph[2][3], pl[2][3], nr[2][3];
    double w[2];
    bool act[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int k = k0 + u * KB;
        act[u] = k < nt;
        double4_32a p = make_double4_32a(0, 0, 0, 0), n = p;
        if (act[u]) {
            p = ep[k];
            n = en[k];
        }
        const double pc[3] = {p.x, p.y, p.z}, nc3[3] = {n.x, n.y, n.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ph[u][a] = (float)pc[a];
            pl[u][a] = (float)(pc[a] - (double)ph[u][a]);
            nr[u][a] = (float)nc3[a];
        }
        w[u] = p.w;
    }
    const f2x px = x2_pack(ph[0][0], ph[1][0]), py = x2_pack(ph[0][1], ph[1][1]), pz = x2_pack(ph[0][2], ph[1][2]);
    const f2x lx = x2_pack(pl[0][0], pl[1][0]), ly = x2_pack(pl[0][1], pl[1][1]), lz = x2_pack(pl[0][2], pl[1][2]);
    const f2x nx = x2_pack(nr[0][0], nr[1][0]), ny = x2_pack(nr[0][1], nr[1][1]), nz = x2_pack(nr[0][2], nr[1][2]);
    double s1[2] = {0.0, 0.0}, s2[2] = {0.0, 0.0};
    const double i4pi = 0.07957747154594767;
    for (int t0 = 0; t0 < nc; t0 += KB) {
        __syncthreads();
        if (t0 + threadIdx.x < nc) {
            const int t = t0 + threadIdx.x;
            const double v[3] = {qpos[3 * t], qpos[3 * t + 1], qpos[3 * t + 2]};
            const float h[3] = {(float)v[0], (float)v[1], (float)v[2]};
            const float l[3] = {(float)(v[0] - (double)h[0]), (float)(v[1] - (double)h[1]), (float)(v[2] - (double)h[2])};
            const float qq = (float)q[t];
            sq[0][threadIdx.x] = make_float4(h[0], h[0], h[1], h[1]);
            sq[1][threadIdx.x] = make_float4(h[2], h[2], qq, qq);
            sq[2][threadIdx.x] = make_float4(l[0], l[0], l[1], l[1]);
            sq[3][threadIdx.x] = make_float4(l[2], l[2], 0.f, 0.f);
        }
        __syncthreads();
        const int m = min(KB, nc - t0);
        f2x a1 = x2_dup(0.f), a2 = x2_dup(0.f);
        for (int t = 0; t < m; ++t) {
            const float4 g0 = sq[0][t], g1 = sq[1][t], g2 = sq[2][t], g3 = sq[3][t];
            const f2x dx = x2_add(x2_sub(px, x2_pack(g0.x, g0.y)), x2_sub(lx, x2_pack(g2.x, g2.y)));
            const f2x dy = x2_add(x2_sub(py, x2_pack(g0.z, g0.w)), x2_sub(ly, x2_pack(g2.z, g2.w)));
            const f2x dz = x2_add(x2_sub(pz, x2_pack(g1.x, g1.y)), x2_sub(lz, x2_pack(g3.x, g3.y)));
            const f2x r2 = x2_fma(dz, dz, x2_fma(dy, dy, x2_mul(dx, dx)));
            float ra, rb;
            x2_unpack(r2, ra, rb);
            const f2x ri = x2_pack(rsqrtf(ra), rsqrtf(rb));
            const f2x nd = x2_fma(nz, dz, x2_fma(ny, dy, x2_mul(nx, dx)));
            const f2x qr = x2_mul(x2_pack(g1.z, g1.w), ri);
            a1 = x2_add(a1, qr);
            a2 = x2_sub(a2, x2_mul(x2_mul(qr, nd), x2_mul(ri, ri)));  // dG0/dn_x = -(n.d)/(4 pi r^3)
        }
        float u0, u1;
        x2_unpack(a1, u0, u1);
        s1[0] += (double)u0;
        s1[1] += (double)u1;
        x2_unpack(a2, u0, u1);
        s2[0] += (double)u0;
        s2[1] += (double)u1;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int k = k0 + u * KB;
        if (act[u]) {
            b[k] = w[u] * s1[u] * i4pi / eps1;
            b[nt + k] = w[u] * s2[u] * i4pi / eps1;
        }
    }
}

int pb_rhs_sorted(pb_ctx* c, double* bs)
{
    // with a regular rule of order > 1 the kernel runs on the points, summed per element after
    const int nt = c->nt * c->q2;
    const double4_32a* ep = c->q2 > 1 ? c->pts_p : c->e64p;
    const double4_32a* en = c->q2 > 1 ? c->pts_n : c->e64n;
    double* out = c->q2 > 1 ? c->yq : bs;
    pb_tic(c, PB_T_RHS);
    if (c->prm.precision == PB_MIXED)
        k_rhs_x2<<<(nt + 2 * KB - 1) / (2 * KB), KB, 0, c->st>>>(nt, c->nc, ep, en, c->qpos, c->q, c->prm.eps_in, out);
    else
        k_rhs<double><<<(nt + 2 * KB - 1) / (2 * KB), KB, 0, c->st>>>(nt, c->nc, ep, en, c->qpos, c->q, c->prm.eps_in,
                                                                      out);
    PB_LAUNCH(c);
    if (c->q2 > 1) {
        int rc = pb_from_points(c, c->yq, bs, 0, c->st);
        if (rc) return rc;
    }
    pb_toc(c, PB_T_RHS);
    return PB_OK;
}

// ---------- energy: 1/2 sum_n q_n sum_i A_i [K1(x_n, c_i) dphi_i + K2(x_n, c_i) phi_i] ----------
// Only K1 and K2 are needed (the charge side carries no normal). FP64: every pair in double
// precision. Mixed: pair terms in FP32 with hi + lo coordinates on both sides, each tile of
// charges summed in FP32 and added into FP64.
template <class R>
__device__ __forceinline__ void energy_k12(R dx, R dy, R dz, R nx, R ny, R nz, R e, R kp, R& K1, R& K2)
{
    const R i4pi = R(0.07957747154594767);
    const R r2 = dx * dx + dy * dy + dz * dz;
    const R rinv = PbKer<R>::rsqrt_(r2);
    const R t = kp * (r2 * rinv);
    R E, g;
    pb_screen<R>(t, E, g);
    const R e1 = R(1) + g + t * E;  // e^-t (1 + t)
    const R ri = rinv * i4pi;
    K1 = -E * ri;
    K2 = (nx * dx + ny * dy + nz * dz) * ri * rinv * rinv * (e * e1 - R(1));
}

template <class R>
__global__ void k_energy(int nt, int nc, const double4_32a* __restrict__ ep, const double4_32a* __restrict__ en,
                         const double* __restrict__ qpos, const double* __restrict__ q, double eps, double kappa,
                         const double* __restrict__ xs, double* __restrict__ part)
{
    __shared__ R sh[KB][3], sl[KB][3], sq[KB];
    __shared__ double red[KB];
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    double4_32a p = make_double4_32a(0, 0, 0, 0), n = p;
    double ph = 0, dph = 0;
    if (k < nt) {
        p = ep[k];
        n = en[k];
        ph = xs[k];
        dph = xs[nt + k];
    }
    const R eh[3] = {(R)p.x, (R)p.y, (R)p.z};
    const R el[3] = {(R)(p.x - (double)eh[0]), (R)(p.y - (double)eh[1]), (R)(p.z - (double)eh[2])};
    const R nx = (R)n.x, ny = (R)n.y, nz = (R)n.z, rph = (R)ph, rdph = (R)dph;
    double acc = 0.0;
    const R e = (R)eps, kp = (R)kappa;
    for (int t0 = 0; t0 < nc; t0 += KB) {
        __syncthreads();
        if (t0 + threadIdx.x < nc) {
            int t = t0 + threadIdx.x;
            for (int a = 0; a < 3; ++a) {
                const double v = qpos[3 * t + a];
                const R hv = (R)v;
                sh[threadIdx.x][a] = hv;
                sl[threadIdx.x][a] = (R)(v - (double)hv);
            }
            sq[threadIdx.x] = (R)q[t];
        }
        __syncthreads();
        int m = min(KB, nc - t0);
        if (k < nt) {
            R s = 0;
            for (int t = 0; t < m; ++t) {
                // d = x_n - c_i
                const R dx = (sh[t][0] - eh[0]) + (sl[t][0] - el[0]);
                const R dy = (sh[t][1] - eh[1]) + (sl[t][1] - el[1]);
                const R dz = (sh[t][2] - eh[2]) + (sl[t][2] - el[2]);
                R K1, K2;
                energy_k12<R>(dx, dy, dz, nx, ny, nz, e, kp, K1, K2);
                s += sq[t] * (K1 * rdph + K2 * rph);
            }
            acc += (double)s;
        }
    }
    red[threadIdx.x] = acc * p.w;
    __syncthreads();
    for (int h = KB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// ---------- several charge states at once (same positions, charges Q[r nc + t]) ----------
// The pair geometry is evaluated once for up to 16 states; each state adds its own weighted
// sums (right-hand side: two FMAs per state; energy: the state's solution values too).
template <class R, int NR>
__global__ void k_rhs_m(int nt, int nc, const double4_32a* __restrict__ ep, const double4_32a* __restrict__ en,
                        const double* __restrict__ qpos, const double* __restrict__ Q, double eps1,
                        double* __restrict__ B, int nr)
{
    __shared__ R sh[KB][3], sl[KB][3], sq[NR][KB];
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    double4_32a p = make_double4_32a(0, 0, 0, 0), n = p;
    if (k < nt) {
        p = ep[k];
        n = en[k];
    }
    const R ph[3] = {(R)p.x, (R)p.y, (R)p.z};
    const R pl[3] = {(R)(p.x - (double)ph[0]), (R)(p.y - (double)ph[1]), (R)(p.z - (double)ph[2])};
    const R nx = (R)n.x, ny = (R)n.y, nz = (R)n.z;
    double s1[NR], s2[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) s1[r] = s2[r] = 0.0;
    const double i4pi = 0.07957747154594767;
    for (int t0 = 0; t0 < nc; t0 += KB) {
        __syncthreads();
        if (t0 + threadIdx.x < nc) {
            int t = t0 + threadIdx.x;
            for (int a = 0; a < 3; ++a) {
                double v = qpos[3 * t + a];
                R hv = (R)v;
                sh[threadIdx.x][a] = hv;
                sl[threadIdx.x][a] = (R)(v - (double)hv);
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) sq[r][threadIdx.x] = r < nr ? (R)Q[(size_t)r * nc + t] : R(0);
        }
        __syncthreads();
        int m = min(KB, nc - t0);
        if (k < nt) {
            R a1[NR], a2[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) a1[r] = a2[r] = 0;
            for (int t = 0; t < m; ++t) {
                R dx = (ph[0] - sh[t][0]) + (pl[0] - sl[t][0]);
                R dy = (ph[1] - sh[t][1]) + (pl[1] - sl[t][1]);
                R dz = (ph[2] - sh[t][2]) + (pl[2] - sl[t][2]);
                R r2 = dx * dx + dy * dy + dz * dz;
                R ri = PbKer<R>::rsqrt_(r2);
                R g2 = -(nx * dx + ny * dy + nz * dz) * ri * ri * ri;  // dG0/dn_x up to 1/(4 pi)
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    a1[r] += sq[r][t] * ri;
                    a2[r] += sq[r][t] * g2;
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                s1[r] += (double)a1[r];
                s2[r] += (double)a2[r];
            }
        }
    }
    if (k < nt)
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r < nr) {
                B[2LL * nt * r + k] = p.w * s1[r] * i4pi / eps1;
                B[2LL * nt * r + nt + k] = p.w * s2[r] * i4pi / eps1;
            }
}

template <class R, int NR>
__global__ void k_energy_m(int nt, int nc, const double4_32a* __restrict__ ep, const double4_32a* __restrict__ en,
                           const double* __restrict__ qpos, const double* __restrict__ Q, double eps, double kappa,
                           const double* __restrict__ X, double* __restrict__ part, int nr)
{
    __shared__ R sh[KB][3], sl[KB][3], sq[NR][KB];
    __shared__ double red[KB / 32][NR];
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    double4_32a p = make_double4_32a(0, 0, 0, 0), n = p;
    R rph[NR], rdph[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) rph[r] = rdph[r] = 0;
    if (k < nt) {
        p = ep[k];
        n = en[k];
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r < nr) {
                rph[r] = (R)X[2LL * nt * r + k];
                rdph[r] = (R)X[2LL * nt * r + nt + k];
            }
    }
    const R eh[3] = {(R)p.x, (R)p.y, (R)p.z};
    const R el[3] = {(R)(p.x - (double)eh[0]), (R)(p.y - (double)eh[1]), (R)(p.z - (double)eh[2])};
    const R nx = (R)n.x, ny = (R)n.y, nz = (R)n.z;
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0;
    const R e = (R)eps, kp = (R)kappa;
    for (int t0 = 0; t0 < nc; t0 += KB) {
        __syncthreads();
        if (t0 + threadIdx.x < nc) {
            int t = t0 + threadIdx.x;
            for (int a = 0; a < 3; ++a) {
                const double v = qpos[3 * t + a];
                const R hv = (R)v;
                sh[threadIdx.x][a] = hv;
                sl[threadIdx.x][a] = (R)(v - (double)hv);
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) sq[r][threadIdx.x] = r < nr ? (R)Q[(size_t)r * nc + t] : R(0);
        }
        __syncthreads();
        int m = min(KB, nc - t0);
        if (k < nt) {
            R s[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) s[r] = 0;
            for (int t = 0; t < m; ++t) {
                const R dx = (sh[t][0] - eh[0]) + (sl[t][0] - el[0]);
                const R dy = (sh[t][1] - eh[1]) + (sl[t][1] - el[1]);
                const R dz = (sh[t][2] - eh[2]) + (sl[t][2] - el[2]);
                R K1, K2;
                energy_k12<R>(dx, dy, dz, nx, ny, nz, e, kp, K1, K2);
#pragma unroll
                for (int r = 0; r < NR; ++r) s[r] += sq[r][t] * (K1 * rdph[r] + K2 * rph[r]);
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += (double)s[r];
        }
    }
    // block sums per state: warp shuffles, then the block's warps
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        double v = acc[r] * p.w;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[w][r] = v;
    }
    __syncthreads();
    if (threadIdx.x < NR && threadIdx.x < nr) {
        double v = 0.0;
        for (int q = 0; q < KB / 32; ++q) v += red[q][threadIdx.x];
        part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_sum(int n, const double* __restrict__ part, double* __restrict__ out, double scale)
{
    __shared__ double red[KB];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += KB) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = KB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * scale;
}

int pb_energy_sorted(pb_ctx* c, const double* xs, double* E)
{
    // with a regular rule of order > 1 the kernel runs on the points (densities copied to them)
    int nt = c->nt * c->q2, nb = (nt + KB - 1) / KB;
    if (!c->scratch) {
        c->scratch = (double*)pb_alloc(c, sizeof(double) * ((size_t)nb + 8));
        if (!c->scratch) return pb_fail(c, PB_ERR_NOMEM, "energy: out of memory");
    }
    double eps = c->prm.eps_out / c->prm.eps_in;
    const double4_32a* ep = c->q2 > 1 ? c->pts_p : c->e64p;
    const double4_32a* en = c->q2 > 1 ? c->pts_n : c->e64n;
    if (c->q2 > 1) {
        int rc = pb_to_points(c, xs, c->xq, c->st);
        if (rc) return rc;
        xs = c->xq;
    }
    pb_tic(c, PB_T_ENERGY);
    if (c->prm.precision == PB_MIXED)
        k_energy<float><<<nb, KB, 0, c->st>>>(nt, c->nc, ep, en, c->qpos, c->q, eps, c->prm.kappa, xs, c->scratch);
    else
        k_energy<double><<<nb, KB, 0, c->st>>>(nt, c->nc, ep, en, c->qpos, c->q, eps, c->prm.kappa, xs, c->scratch);
    PB_LAUNCH(c);
    k_sum<<<1, KB, 0, c->st>>>(nb, c->scratch, c->scratch + nb, 0.5 * 4.0 * PB_PI * 332.0716);
    PB_LAUNCH(c);
    pb_toc(c, PB_T_ENERGY);
    PB_CUDA(c, cudaMemcpyAsync(c->hscal, c->scratch + nb, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    *E = c->hscal[0];
    return PB_OK;
}

// right-hand sides of nr <= 16 charge states (device charges Q, nr x nc) into B (nr x 2N)
int pb_rhs_states_sorted(pb_ctx* c, const double* Q, double* B, int nr)
{
    const int nt = c->nt;
    pb_tic(c, PB_T_RHS);
    if (c->prm.precision == PB_MIXED)
        k_rhs_m<float, 16><<<(nt + KB - 1) / KB, KB, 0, c->st>>>(nt, c->nc, c->e64p, c->e64n, c->qpos, Q,
                                                                 c->prm.eps_in, B, nr);
    else
        k_rhs_m<double, 16><<<(nt + KB - 1) / KB, KB, 0, c->st>>>(nt, c->nc, c->e64p, c->e64n, c->qpos, Q,
                                                                  c->prm.eps_in, B, nr);
    PB_LAUNCH(c);
    pb_toc(c, PB_T_RHS);
    return PB_OK;
}

// energy scratch: nb partials for each of 16 states, then 16 results
int pb_energy_reserve(pb_ctx* c)
{
    const int nb = (c->nt + KB - 1) / KB;
    if (!c->escratch) {
        c->escratch = (double*)pb_alloc(c, sizeof(double) * ((size_t)nb * 16 + 16));
        if (!c->escratch) return pb_fail(c, PB_ERR_NOMEM, "energy: out of memory");
    }
    return PB_OK;
}

// energies of nr <= 16 states (charges Q, solutions X, nr x 2N) into Edev[0..nr) (device);
// queued only (pb_energy_reserve first)
int pb_energy_states_queue(pb_ctx* c, const double* Q, const double* X, int nr, double* Edev)
{
    const int nt = c->nt, nb = (nt + KB - 1) / KB;
    double* part = c->escratch;
    const double eps = c->prm.eps_out / c->prm.eps_in;
    pb_tic(c, PB_T_ENERGY);
    if (c->prm.precision == PB_MIXED)
        k_energy_m<float, 16><<<nb, KB, 0, c->st>>>(nt, c->nc, c->e64p, c->e64n, c->qpos, Q, eps, c->prm.kappa, X,
                                                     part, nr);
    else
        k_energy_m<double, 16><<<nb, KB, 0, c->st>>>(nt, c->nc, c->e64p, c->e64n, c->qpos, Q, eps, c->prm.kappa, X,
                                                      part, nr);
    PB_LAUNCH(c);
    for (int r = 0; r < nr; ++r) {
        k_sum<<<1, KB, 0, c->st>>>(nb, part + (size_t)r * nb, Edev + r, 0.5 * 4.0 * PB_PI * 332.0716);
        PB_LAUNCH(c);
    }
    pb_toc(c, PB_T_ENERGY);
    return PB_OK;
}

// energies of nr <= 16 states (charges Q, solutions X, nr x 2N) into E[0..nr) (host); synchronises
int pb_energy_states_sorted(pb_ctx* c, const double* Q, const double* X, int nr, double* E)
{
    int rc;
    if ((rc = pb_energy_reserve(c))) return rc;
    const int nb = (c->nt + KB - 1) / KB;
    double* Ed = c->escratch + (size_t)nb * 16;
    if ((rc = pb_energy_states_queue(c, Q, X, nr, Ed))) return rc;
    std::vector<double> h(nr);
    PB_CUDA(c, cudaMemcpyAsync(h.data(), Ed, sizeof(double) * nr, cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    for (int r = 0; r < nr; ++r) E[r] = h[r];
    return PB_OK;
}

// ---------- GMRES building blocks ----------
#define DOT_BLOCKS 304  // 2 x 152 SMs

// part[col * DOT_BLOCKS + blk] = partial of <V[col], w> (or of <w, w> when V == nullptr)
__global__ void k_multidot(long long n, const double* __restrict__ V, const double* __restrict__ w,
                           double* __restrict__ part)
{
    __shared__ double red[KB];
    const int col = blockIdx.y;
    const double* v = V ? V + (size_t)col * n : w;
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) s += v[i] * w[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = KB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)col * gridDim.x + blockIdx.x] = red[0];
}

// out[col] (+)= sum of partials of column col
__global__ void k_finish(int nparts, const double* __restrict__ part, double* __restrict__ out, int accumulate)
{
    __shared__ double red[KB];
    const int col = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += KB) s += part[(size_t)col * nparts + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = KB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[col] = accumulate ? out[col] + red[0] : red[0];
}

// w -= V[:, 0..ncol) h
__global__ void k_orth_update(long long n, int ncol, const double* __restrict__ V, const double* __restrict__ h,
                              double* __restrict__ w)
{
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        double s = 0.0;
        for (int c = 0; c < ncol; ++c) s += V[(size_t)c * n + i] * h[c];
        w[i] -= s;
    }
}

// dst = src * (1 / *nrm) (nrm read from device)
__global__ void k_scale(long long n, const double* __restrict__ src, const double* __restrict__ nrm, double* __restrict__ dst)
{
    double f = 1.0 / sqrt(*nrm);
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) dst[i] = src[i] * f;
}

// Scale a nonzero start x (w = A x) by a = <w, b> / <w, w>, the factor that minimises
// ||b - a A x||; a start with no positive finite factor (a useless or non-finite guess)
// becomes exactly zero, so GMRES falls back to the zero start. d = {<w, b>, <w, w>}.
__global__ void k_start_scale(long long n, const double* __restrict__ d, double* __restrict__ x,
                              double* __restrict__ w)
{
    const double a = d[1] > 0.0 ? d[0] / d[1] : 0.0;
    const double f = (a > 0.0 && isfinite(a)) ? a : 0.0;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        x[i] = f != 0.0 ? x[i] * f : 0.0;  // 0 * NaN would stay NaN
        w[i] = f != 0.0 ? w[i] * f : 0.0;
    }
}

// r = b - r  (r holds A x on input)
__global__ void k_residual(long long n, const double* __restrict__ b, double* __restrict__ r)
{
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) r[i] = b[i] - r[i];
}

// x += u
__global__ void k_axpy1(long long n, const double* __restrict__ u, double* __restrict__ x)
{
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) x[i] += u[i];
}

// u = V[:, 0..k) y
__global__ void k_combine(long long n, int k, const double* __restrict__ V, const double* __restrict__ y,
                          double* __restrict__ u)
{
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        double s = 0.0;
        for (int c = 0; c < k; ++c) s += V[(size_t)c * n + i] * y[c];
        u[i] = s;
    }
}

// Small dense state of GMRES(m) on the device: H (column-major (m+1) x m), Givens cs/sn, g.
struct GmState {
    double* H;
    double* cs;
    double* sn;
    double* g;
    double* y;
    double* hcol;  // h[0..j] and ||w||^2 of the current step
    double* res;   // |g_{j+1}|
};

// start of a cycle: g = (beta, 0, ...), beta = sqrt(hcol[0])
__global__ void k_gm_start(int m, GmState s)
{
    for (int i = 0; i <= m; ++i) s.g[i] = 0.0;
    s.g[0] = sqrt(s.hcol[0]);
    s.res[0] = s.g[0];
}

// step j: H[:, j] = (hcol[0..j], sqrt(hcol[j+1])); apply rotations; new rotation; residual.
// The entry that rotation i - 1 left for rotation i stays in a register (a round trip through
// global memory per rotation made this serial loop latency-bound).
__device__ __forceinline__ void gm_givens_step(int m, int j, GmState s)
{
    double* Hj = s.H + (size_t)j * (m + 1);
    double a = s.hcol[0];
    for (int i = 0; i < j; ++i) {
        const double b = s.hcol[i + 1];
        Hj[i] = s.cs[i] * a + s.sn[i] * b;
        a = -s.sn[i] * a + s.cs[i] * b;
    }
    const double b = sqrt(s.hcol[j + 1]);
    double r = hypot(a, b);
    double c = r > 0 ? a / r : 1.0, sn = r > 0 ? b / r : 0.0;
    s.cs[j] = c;
    s.sn[j] = sn;
    Hj[j] = r;
    Hj[j + 1] = 0.0;
    s.g[j + 1] = -sn * s.g[j];
    s.g[j] = c * s.g[j];
    s.res[0] = fabs(s.g[j + 1]);
}

__global__ void k_gm_givens(int m, int j, GmState s) { gm_givens_step(m, j, s); }

// back substitution: H[0..k, 0..k) y = g
__global__ void k_gm_solve(int m, int k, GmState s)
{
    for (int i = k - 1; i >= 0; --i) {
        double v = s.g[i];
        for (int q = i + 1; q < k; ++q) v -= s.H[(size_t)q * (m + 1) + i] * s.y[q];
        double d = s.H[(size_t)i * (m + 1) + i];
        s.y[i] = d != 0.0 ? v / d : 0.0;
    }
}

static int grid_for(long long n) { return (int)std::min<long long>((n + KB - 1) / KB, 4 * 152 * 4); }

// ---------- float-float Krylov basis (mixed precision) ----------
// On this GPU FP64 arithmetic runs at 1/64 of the FP32 rate, and CGS2 over a basis of FP64
// vectors (one FP64 FMA per element and column, four passes per Arnoldi step) is bound by it,
// not by HBM. In mixed precision the basis and the vector being orthogonalised are kept as
// float-float pairs (hi, lo) instead, 8 bytes per element as before, and every dot product
// and update runs on the FP32 pipe (about 15 FP32 instructions per element and column, a
// 48-bit significand), which leaves the passes bound by the HBM reads of the basis. The
// Hessenberg entries, norms and Givens rotations stay FP64; the product and the
// preconditioner still see FP64 vectors (a copy of v_j written beside its float-float form).
// The kernels serve the host-driven loop (explicit column counts) and the device-driven graph
// (jdev = the device's step index; right-hand side r = the last grid dimension).
#define FFK_CG 2         // basis vectors per block of the float-float dot products
#define FFK_MAXCOL 201   // restart length <= 200

// s += a b in float-float, renormalised once
__device__ __forceinline__ void ffk_acc(float& sh, float& sl, float ah, float al, float bh, float bl)
{
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float t = sh + p;
    const float bb = t - sh;
    sl += ((sh - (t - bb)) + (p - bb)) + e;
    sh = t + sl;
    sl -= sh - t;
}

__device__ __forceinline__ double ffk_to(float h, float l) { return (double)h + (double)l; }
__device__ __forceinline__ float2 ffk_from(double x)
{
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

// part_r[col * gridDim.x + blk] = partial of <V_r[col], w_r> over the block's elements for the
// FFK_CG columns blockIdx.y * FFK_CG + q < ncol (ncol = *jdev + 1 when jdev is given); with
// V == nullptr, <w_r, w_r> into column 0. Each thread takes two elements a stride apart per
// iteration, their loads issued before the sums (two columns x two elements measured 6.2 TB/s
// on 70 basis vectors of 3.67 M elements; four columns x one element 5.5 TB/s).
__global__ void __launch_bounds__(KB) k_ffdot(long long n, int ncol, const int* __restrict__ jdev,
                                              const float2* __restrict__ V, long long vstr,
                                              const float2* __restrict__ w, double* __restrict__ part, long long pstr)
{
    __shared__ double red[FFK_CG][KB / 32];
    const int r = blockIdx.z;
    if (jdev) ncol = *jdev + 1;
    const int c0 = blockIdx.y * FFK_CG;
    const int nc = V ? min(FFK_CG, ncol - c0) : (blockIdx.y == 0 ? 1 : 0);
    if (nc <= 0) return;
    w += r * n;
    part += r * pstr;
    const float2* v = V ? V + r * vstr + (size_t)c0 * n : w;
    float sh[FFK_CG] = {}, sl[FFK_CG] = {};
    const long long stride = (long long)gridDim.x * KB;
    const float2 zero = make_float2(0.f, 0.f);
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += 2 * stride) {
        const long long i2 = i + stride;
        const bool two = i2 < n;
        const float2 b0 = w[i], b1 = two ? w[i2] : zero;
        float2 a0[FFK_CG], a1[FFK_CG];
#pragma unroll
        for (int q = 0; q < FFK_CG; ++q) {
            a0[q] = q < nc ? v[(size_t)q * n + i] : zero;
            a1[q] = (q < nc && two) ? v[(size_t)q * n + i2] : zero;
        }
#pragma unroll
        for (int q = 0; q < FFK_CG; ++q) {
            ffk_acc(sh[q], sl[q], a0[q].x, a0[q].y, b0.x, b0.y);
            ffk_acc(sh[q], sl[q], a1[q].x, a1[q].y, b1.x, b1.y);
        }
    }
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < FFK_CG; ++q) {
        double s = ffk_to(sh[q], sl[q]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[q][wi] = s;
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        double s = 0.0;
        for (int k = 0; k < KB / 32; ++k) s += red[threadIdx.x][k];
        part[(size_t)(c0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
}

// wf_r (float-float) = w_r (FP64), the vectors the product wrote
__global__ void k_to_ff(long long n, const double* __restrict__ w, float2* __restrict__ wf)
{
    const long long o = blockIdx.y * n;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB)
        wf[o + i] = ffk_from(w[o + i]);
}

// w_r -= V_r[:, 0..ncol) h_r in float-float (h FP64, split once per block; ncol = *jdev + 1 when
// jdev is given)
__global__ void __launch_bounds__(KB) k_fforth(long long n, int ncol, const int* __restrict__ jdev,
                                               const float2* __restrict__ V, long long vstr,
                                               const double* __restrict__ h, long long hstr, float2* __restrict__ w)
{
    __shared__ float2 hs[FFK_MAXCOL];
    const int r = blockIdx.y;
    if (jdev) ncol = *jdev + 1;
    V += r * vstr;
    h += r * hstr;
    w += r * n;
    for (int q = threadIdx.x; q < ncol; q += KB) hs[q] = ffk_from(h[q]);
    __syncthreads();
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        float sh = 0.f, sl = 0.f;
        int q = 0;
        for (; q + 4 <= ncol; q += 4) {
            const float2 a0 = V[(size_t)q * n + i], a1 = V[(size_t)(q + 1) * n + i];
            const float2 a2 = V[(size_t)(q + 2) * n + i], a3 = V[(size_t)(q + 3) * n + i];
            ffk_acc(sh, sl, a0.x, a0.y, hs[q].x, hs[q].y);
            ffk_acc(sh, sl, a1.x, a1.y, hs[q + 1].x, hs[q + 1].y);
            ffk_acc(sh, sl, a2.x, a2.y, hs[q + 2].x, hs[q + 2].y);
            ffk_acc(sh, sl, a3.x, a3.y, hs[q + 3].x, hs[q + 3].y);
        }
        for (; q < ncol; ++q) {
            const float2 a = V[(size_t)q * n + i];
            ffk_acc(sh, sl, a.x, a.y, hs[q].x, hs[q].y);
        }
        // w - s: two-sum of the high parts, then the low parts, renormalised
        const float2 b = w[i];
        const float t = b.x - sh;
        const float bb = t - b.x;
        float e = ((b.x - (t - bb)) + (-sh - bb)) + (b.y - sl);
        const float s = t + e;
        e -= s - t;
        w[i] = make_float2(s, e);
    }
}

// V_r[:, c] = w_r / sqrt(small_r[hoff + c]) in float-float, and vd_r = the same in FP64 (the next
// product's input), c = 0 for the start of a cycle (first), else (the step index) + 1 with the
// step from *jdev or jhost. The source is w64_r (FP64) when given, else wf_r.
__global__ void k_ffscale(long long n, const float2* __restrict__ wf, const double* __restrict__ w64,
                          const double* __restrict__ small, long long sstr, long long hoff, const int* __restrict__ jdev,
                          int jhost, int first, float2* __restrict__ V, long long vstr, double* __restrict__ vd)
{
    const int r = blockIdx.y;
    const int c = first ? 0 : (jdev ? *jdev : jhost) + 1;
    const double f = 1.0 / sqrt(small[r * sstr + hoff + c]);
    const float fh = (float)f, fl = (float)(f - (double)fh);
    float2* dst = V + r * vstr + (size_t)c * n;
    vd += r * n;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        const float2 a = w64 ? ffk_from(w64[r * n + i]) : wf[r * n + i];
        float sh = 0.f, sl = 0.f;
        ffk_acc(sh, sl, a.x, a.y, fh, fl);
        dst[i] = make_float2(sh, sl);
        vd[i] = ffk_to(sh, sl);
    }
}

// u_r = V_r[:, 0..k) y_r (FP64 out), k = ksteps[r] when given, else khost
__global__ void __launch_bounds__(KB) k_ffcombine(long long n, int khost, const int* __restrict__ ksteps,
                                                  const float2* __restrict__ V, long long vstr,
                                                  const double* __restrict__ y, long long ystr, double* __restrict__ u)
{
    __shared__ float2 ys[FFK_MAXCOL];
    const int r = blockIdx.y;
    const int k = ksteps ? ksteps[r] : khost;
    V += r * vstr;
    y += r * ystr;
    u += r * n;
    for (int q = threadIdx.x; q < k; q += KB) ys[q] = ffk_from(y[q]);
    __syncthreads();
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        float sh = 0.f, sl = 0.f;
        for (int q = 0; q < k; ++q) {
            const float2 a = V[(size_t)q * n + i];
            ffk_acc(sh, sl, a.x, a.y, ys[q].x, ys[q].y);
        }
        u[i] = ffk_to(sh, sl);
    }
}

int pb_gmres_sorted(pb_ctx* c, double* xs, const double* bs, double tol, int max_iter, int restart,
                    pb_solve_info* info, bool x_zero)
{
    const long long n = 2LL * c->nu;
    const int m = restart;
    const int G = grid_for(n);
    int rc;
    // workspace, kept with the mesh and regrown when the restart length grows
    if (m > c->gm_m) {
        c->gmV = (double*)pb_alloc(c, sizeof(double) * n * (m + 1));
        c->gmw = (double*)pb_alloc(c, sizeof(double) * n);
        c->gmz = (double*)pb_alloc(c, sizeof(double) * n);
        c->gmpart = (double*)pb_alloc(c, sizeof(double) * DOT_BLOCKS * (m + 2));
        c->gmsmall = (double*)pb_alloc(c, sizeof(double) * ((m + 1) * m + 6 * (m + 2)));
        if (c->prm.precision == PB_MIXED) {  // float-float work vector, FP64 copy of v_j
            c->gmwf = (float2*)pb_alloc(c, sizeof(float2) * n);
            c->gmvd = (double*)pb_alloc(c, sizeof(double) * n);
            if (!c->gmwf || !c->gmvd) c->gmV = nullptr;
        }
        if (!c->gmV || !c->gmw || !c->gmz || !c->gmpart || !c->gmsmall) {
            c->gm_m = 0;
            return pb_fail(c, PB_ERR_NOMEM, "gmres: out of memory");
        }
        c->gm_m = m;
    }
    double *V = c->gmV, *w = c->gmw, *z = c->gmz, *part = c->gmpart, *small = c->gmsmall;
    // mixed precision: the basis as float-float pairs in the same storage
    const bool ffb = c->prm.precision == PB_MIXED;
    float2 *Vf = (float2*)c->gmV, *wf = c->gmwf;
    double* vd = c->gmvd;
    GmState s;
    s.H = small;
    s.cs = s.H + (size_t)(m + 1) * m;
    s.sn = s.cs + (m + 2);
    s.g = s.sn + (m + 2);
    s.y = s.g + (m + 2);
    s.hcol = s.y + (m + 2);
    s.res = s.hcol + (m + 2);
    pb_solve_info inf = {0, 0, 0.0, PB_OK, 1.0};
    // ||b||
    k_multidot<<<dim3(DOT_BLOCKS, 1), KB, 0, c->st>>>(n, nullptr, bs, part);
    PB_LAUNCH(c);
    k_finish<<<1, KB, 0, c->st>>>(DOT_BLOCKS, part, s.hcol, 0);
    PB_LAUNCH(c);
    PB_CUDA(c, cudaMemcpyAsync(c->hscal, s.hcol, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    const double bnorm = sqrt(c->hscal[0]);
    if (!isfinite(bnorm)) {  // an overflowing or non-finite right-hand side
        inf.status = PB_ERR_NONFINITE;
        inf.rel_residual = bnorm;
        if (info) *info = inf;
        return PB_ERR_NONFINITE;
    }
    if (!(bnorm > 0)) {
        PB_CUDA(c, cudaMemsetAsync(xs, 0, sizeof(double) * n, c->st));
        if (info) *info = inf;
        return PB_OK;
    }
    int it = 0;
    double rel = 1.0;
    bool done = false, converged = false;
    bool first = true;
    while (!done) {
        // r0 = b - A x ; V0 = r0 / ||r0||  (A x = 0 for a start the caller zeroed)
        if (first && x_zero) {
            PB_CUDA(c, cudaMemsetAsync(w, 0, sizeof(double) * n, c->st));
        } else {
            if ((rc = pb_matvec_sorted(c, xs, w, 0))) return rc;
            inf.matvecs++;
            if (first) {
                // a given start (a learned guess, say) is first rescaled by the least-squares
                // factor along it: two dot products, no extra product
                k_multidot<<<dim3(DOT_BLOCKS, 1), KB, 0, c->st>>>(n, bs, w, part);
                PB_LAUNCH(c);
                k_finish<<<1, KB, 0, c->st>>>(DOT_BLOCKS, part, s.hcol, 0);
                PB_LAUNCH(c);
                k_multidot<<<dim3(DOT_BLOCKS, 1), KB, 0, c->st>>>(n, nullptr, w, part);
                PB_LAUNCH(c);
                k_finish<<<1, KB, 0, c->st>>>(DOT_BLOCKS, part, s.hcol + 1, 0);
                PB_LAUNCH(c);
                k_start_scale<<<G, KB, 0, c->st>>>(n, s.hcol, xs, w);
                PB_LAUNCH(c);
            }
        }
        k_residual<<<G, KB, 0, c->st>>>(n, bs, w);
        PB_LAUNCH(c);
        k_multidot<<<dim3(DOT_BLOCKS, 1), KB, 0, c->st>>>(n, nullptr, w, part);
        PB_LAUNCH(c);
        k_finish<<<1, KB, 0, c->st>>>(DOT_BLOCKS, part, s.hcol, 0);
        PB_LAUNCH(c);
        if (ffb)
            k_ffscale<<<dim3(G, 1), KB, 0, c->st>>>(n, nullptr, w, s.hcol, 0, 0, nullptr, 0, 1, Vf, 0, vd);
        else
            k_scale<<<G, KB, 0, c->st>>>(n, w, s.hcol, V);
        PB_LAUNCH(c);
        k_gm_start<<<1, 1, 0, c->st>>>(m, s);
        PB_LAUNCH(c);
        PB_CUDA(c, cudaMemcpyAsync(c->hscal, s.res, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
        rel = c->hscal[0] / bnorm;
        if (first) inf.initial_residual = rel;
        first = false;
        if (!isfinite(rel)) {
            inf.status = PB_ERR_NONFINITE;
            break;
        }
        if (rel <= tol) {
            converged = true;
            break;
        }
        int k = 0;
        for (int j = 0; j < m && it < max_iter; ++j) {
            double* vj = ffb ? vd : V + (size_t)j * n;
            if ((rc = pb_precond_apply_sorted(c, vj, z))) return rc;
            if ((rc = pb_matvec_sorted(c, z, w, 0))) return rc;
            inf.matvecs++;
            pb_tic(c, PB_T_ARNOLDI);
            // CGS2
            if (ffb) {
                k_to_ff<<<dim3(G, 1), KB, 0, c->st>>>(n, w, wf);
                PB_LAUNCH(c);
                const unsigned ng = (unsigned)((j + 1 + FFK_CG - 1) / FFK_CG);
                for (int pass = 0; pass < 2; ++pass) {
                    double* h = pass ? s.y : s.hcol;
                    k_ffdot<<<dim3(DOT_BLOCKS, ng, 1), KB, 0, c->st>>>(n, j + 1, nullptr, Vf, 0, wf, part, 0);
                    PB_LAUNCH(c);
                    k_finish<<<j + 1, KB, 0, c->st>>>(DOT_BLOCKS, part, h, 0);
                    PB_LAUNCH(c);
                    k_fforth<<<dim3(G, 1), KB, 0, c->st>>>(n, j + 1, nullptr, Vf, 0, h, 0, wf);
                    PB_LAUNCH(c);
                }
                k_axpy1<<<1, KB, 0, c->st>>>(j + 1, s.y, s.hcol);
                PB_LAUNCH(c);
                k_ffdot<<<dim3(DOT_BLOCKS, 1, 1), KB, 0, c->st>>>(n, 1, nullptr, nullptr, 0, wf, part, 0);
                PB_LAUNCH(c);
                k_finish<<<1, KB, 0, c->st>>>(DOT_BLOCKS, part, s.hcol + j + 1, 0);
                PB_LAUNCH(c);
                k_ffscale<<<dim3(G, 1), KB, 0, c->st>>>(n, wf, nullptr, s.hcol, 0, 0, nullptr, j, 0, Vf, 0, vd);
                PB_LAUNCH(c);
            }
            for (int pass = 0; pass < 2 && !ffb; ++pass) {
                k_multidot<<<dim3(DOT_BLOCKS, j + 1), KB, 0, c->st>>>(n, V, w, part);
                PB_LAUNCH(c);
                k_finish<<<j + 1, KB, 0, c->st>>>(DOT_BLOCKS, part, pass ? s.y : s.hcol, 0);
                PB_LAUNCH(c);
                k_orth_update<<<G, KB, 0, c->st>>>(n, j + 1, V, pass ? s.y : s.hcol, w);
                PB_LAUNCH(c);
            }
            if (!ffb) {
                // merge the two passes: hcol[i] += y[i]
                k_axpy1<<<1, KB, 0, c->st>>>(j + 1, s.y, s.hcol);
                PB_LAUNCH(c);
                k_multidot<<<dim3(DOT_BLOCKS, 1), KB, 0, c->st>>>(n, nullptr, w, part);
                PB_LAUNCH(c);
                k_finish<<<1, KB, 0, c->st>>>(DOT_BLOCKS, part, s.hcol + j + 1, 0);
                PB_LAUNCH(c);
                k_scale<<<G, KB, 0, c->st>>>(n, w, s.hcol + j + 1, V + (size_t)(j + 1) * n);
                PB_LAUNCH(c);
            }
            k_gm_givens<<<1, 1, 0, c->st>>>(m, j, s);
            PB_LAUNCH(c);
            pb_toc(c, PB_T_ARNOLDI);
            PB_CUDA(c, cudaMemcpyAsync(c->hscal, s.res, sizeof(double), cudaMemcpyDeviceToHost, c->st));
            PB_CUDA(c, cudaStreamSynchronize(c->st));
            ++it;
            k = j + 1;
            rel = c->hscal[0] / bnorm;
            if (!isfinite(rel)) {
                inf.status = PB_ERR_NONFINITE;
                done = true;
                break;
            }
            if (rel <= tol) {
                converged = done = true;
                break;
            }
        }
        if (k > 0 && inf.status == PB_OK) {
            // x += M^-1 V y
            k_gm_solve<<<1, 1, 0, c->st>>>(m, k, s);
            PB_LAUNCH(c);
            if (ffb)
                k_ffcombine<<<dim3(G, 1), KB, 0, c->st>>>(n, k, nullptr, Vf, 0, s.y, 0, w);
            else
                k_combine<<<G, KB, 0, c->st>>>(n, k, V, s.y, w);
            PB_LAUNCH(c);
            if ((rc = pb_precond_apply_sorted(c, w, z))) return rc;
            k_axpy1<<<G, KB, 0, c->st>>>(n, z, xs);
            PB_LAUNCH(c);
        }
        if (it >= max_iter) done = true;
        if (inf.status != PB_OK) break;
    }
    // true residual
    if ((rc = pb_matvec_sorted(c, xs, w, 0))) return rc;
    inf.matvecs++;
    k_residual<<<G, KB, 0, c->st>>>(n, bs, w);
    PB_LAUNCH(c);
    k_multidot<<<dim3(DOT_BLOCKS, 1), KB, 0, c->st>>>(n, nullptr, w, part);
    PB_LAUNCH(c);
    k_finish<<<1, KB, 0, c->st>>>(DOT_BLOCKS, part, s.hcol, 0);
    PB_LAUNCH(c);
    PB_CUDA(c, cudaMemcpyAsync(c->hscal, s.hcol, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    inf.iterations = it;
    inf.rel_residual = sqrt(c->hscal[0]) / bnorm;
    if (inf.status == PB_OK && !converged) inf.status = PB_ERR_NOT_CONVERGED;
    if (inf.status == PB_OK && !isfinite(inf.rel_residual)) inf.status = PB_ERR_NONFINITE;
    // a kernel whose bounded wait gave up leaves its flag set; report it instead of a result
    int derr = 0;
    PB_CUDA(c, cudaMemcpyAsync(&derr, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    if (derr) {
        inf.status = PB_ERR_TIMEOUT;
        pb_fail(c, PB_ERR_TIMEOUT, "a bounded wait in the MtL kernel gave up");
    }
    if (info) *info = inf;
    return inf.status;
}

// ---------- several right-hand sides in lockstep ----------
// nr independent right-preconditioned GMRES(m) iterations advance together: each Arnoldi step
// applies one batched product (pb_matvec_sorted_multi) to the nr current basis vectors, and the
// orthogonalisation, Givens rotations and updates run batched over the right-hand sides
// (grid dimension y or z = right-hand side). Every right-hand side keeps its own Krylov basis,
// Hessenberg matrix and residual, so each one computes exactly what its own GMRES would; one
// that has converged stops at its own step count and its later steps are discarded.

// part[r][col][blk] = partial of <V_r[col], w_r> (or <w_r, w_r> when V == nullptr)
__global__ void k_bdot(long long n, const double* __restrict__ V, long long vstr, const double* __restrict__ w,
                       double* __restrict__ part, long long pstr)
{
    __shared__ double red[KB];
    const int col = blockIdx.y, r = blockIdx.z;
    w += r * n;
    const double* v = V ? V + r * vstr + (size_t)col * n : w;
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) s += v[i] * w[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = KB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[r * pstr + (size_t)col * gridDim.x + blockIdx.x] = red[0];
}

// out_r[col] = sum of the partials of column col of right-hand side r
__global__ void k_bfinish(int nparts, const double* __restrict__ part, long long pstr, double* __restrict__ out,
                          long long ostr)
{
    __shared__ double red[KB];
    const int col = blockIdx.x, r = blockIdx.y;
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += KB) s += part[r * pstr + (size_t)col * nparts + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = KB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r * ostr + col] = red[0];
}

// w_r -= V_r[:, 0..ncol) h_r
__global__ void k_borth(long long n, int ncol, const double* __restrict__ V, long long vstr,
                        const double* __restrict__ h, long long hstr, double* __restrict__ w)
{
    const int r = blockIdx.y;
    V += r * vstr;
    h += r * hstr;
    w += r * n;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        double s = 0.0;
        for (int c = 0; c < ncol; ++c) s += V[(size_t)c * n + i] * h[c];
        w[i] -= s;
    }
}

// dst_r = src_r / sqrt(*nrm_r)
__global__ void k_bscale(long long n, const double* __restrict__ src, long long sstr, const double* __restrict__ nrm,
                         long long nstr, double* __restrict__ dst, long long dstr)
{
    const int r = blockIdx.y;
    src += r * sstr;
    dst += r * dstr;
    const double f = 1.0 / sqrt(nrm[r * nstr]);
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) dst[i] = src[i] * f;
}

// r_q = b_q - r_q for all q
__global__ void k_bresidual(long long n, const double* __restrict__ b, double* __restrict__ w)
{
    b += blockIdx.y * n;
    w += blockIdx.y * n;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) w[i] = b[i] - w[i];
}

// hcol_r[i] += y_r[i], i <= j
__global__ void k_bmerge(int k, double* __restrict__ small, long long sstr, long long yoff, long long hoff)
{
    double* s = small + blockIdx.x * sstr;
    for (int i = threadIdx.x; i < k; i += blockDim.x) s[hoff + i] += s[yoff + i];
}

static GmState gm_state(double* small, int m)
{
    GmState s;
    s.H = small;
    s.cs = s.H + (size_t)(m + 1) * m;
    s.sn = s.cs + (m + 2);
    s.g = s.sn + (m + 2);
    s.y = s.g + (m + 2);
    s.hcol = s.y + (m + 2);
    s.res = s.hcol + (m + 2);
    return s;
}

// right-hand side r = blockIdx.x: the single-vector kernels on its own small state
__global__ void k_bgm_start(int m, GmState s, long long sstr)
{
    const long long o = blockIdx.x * sstr;
    GmState t = {s.H + o, s.cs + o, s.sn + o, s.g + o, s.y + o, s.hcol + o, s.res + o};
    for (int i = 0; i <= m; ++i) t.g[i] = 0.0;
    t.g[0] = sqrt(t.hcol[0]);
    t.res[0] = t.g[0];
}

__global__ void k_bgm_givens(int m, int j, GmState s, long long sstr)
{
    const long long o = blockIdx.x * sstr;
    GmState t = {s.H + o, s.cs + o, s.sn + o, s.g + o, s.y + o, s.hcol + o, s.res + o};
    gm_givens_step(m, j, t);
}

__global__ void k_dg_start_scale(long long n, const double* __restrict__ small, long long sstr, long long hoff,
                                 double* __restrict__ X, double* __restrict__ W);

int pb_gmres_batch_sorted(pb_ctx* c, double* X, const double* B, int nr, double tol, int max_iter, int restart,
                          pb_solve_info* infos)
{
    const long long n = 2LL * c->nu;
    const int m = restart;
    const int G = grid_for(n);
    const long long S = (long long)(m + 1) * m + 6 * (m + 2);  // small state per right-hand side
    const long long vstr = (long long)(m + 1) * n;               // Krylov basis per right-hand side
    const long long pstr = (long long)DOT_BLOCKS * (m + 2);      // dot partials per right-hand side
    if (nr > c->gb_nr || m > c->gb_m) {
        c->gbV = (double*)pb_alloc(c, sizeof(double) * (size_t)(vstr * nr));
        c->gbW = (double*)pb_alloc(c, sizeof(double) * (size_t)(n * nr));
        c->gbZ = (double*)pb_alloc(c, sizeof(double) * (size_t)(n * nr));
        c->gbpart = (double*)pb_alloc(c, sizeof(double) * (size_t)(pstr * nr));
        c->gbsmall = (double*)pb_alloc(c, sizeof(double) * (size_t)(S * nr));
        if (!c->gbV || !c->gbW || !c->gbZ || !c->gbpart || !c->gbsmall) {
            c->gb_nr = c->gb_m = 0;
            return pb_fail(c, PB_ERR_NOMEM, "batched gmres: out of memory");
        }
        c->gb_nr = nr;
        c->gb_m = m;
    }
    double *V = c->gbV, *W = c->gbW, *Z = c->gbZ, *part = c->gbpart, *small = c->gbsmall;
    const GmState st = gm_state(small, m);
    const long long hoff = st.hcol - small, yoff = st.y - small, roff = st.res - small;
    std::vector<double> hv(nr), bnorm(nr), rel(nr, 1.0);
    std::vector<int> active(nr, 1), steps(nr, 0), its(nr, 0), mvs(nr, 0), status(nr, PB_OK), conv(nr, 0);
    std::vector<double> init(nr, 1.0);
    auto read = [&](long long off) -> int {
        PB_CUDA(c, cudaMemcpy2DAsync(hv.data(), sizeof(double), small + off, sizeof(double) * S, sizeof(double), nr,
                                     cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
        return PB_OK;
    };
    int rc;
    // ||b_r||
    k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, nullptr, 0, B, part, pstr);
    PB_LAUNCH(c);
    k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff, S);
    PB_LAUNCH(c);
    if ((rc = read(hoff))) return rc;
    for (int r = 0; r < nr; ++r) {
        bnorm[r] = sqrt(hv[r]);
        if (!(bnorm[r] > 0)) {
            active[r] = 0;
            conv[r] = 1;
            PB_CUDA(c, cudaMemsetAsync(X + r * n, 0, sizeof(double) * n, c->st));
        }
    }
    // One Arnoldi step of all right-hand sides: z = M^-1 v_j, w = A z, CGS2, normalisation,
    // Givens rotation (finished right-hand sides are carried along and discarded).
    auto step_launches = [&](int j) -> int {
        int rc2;
        if ((rc2 = pb_precond_apply_multi(c, V + (size_t)j * n, vstr, Z, n, nr))) return rc2;
        if ((rc2 = pb_matvec_sorted_multi(c, Z, W, nr))) return rc2;
        pb_tic(c, PB_T_ARNOLDI);
        for (int pass = 0; pass < 2; ++pass) {
            k_bdot<<<dim3(DOT_BLOCKS, j + 1, nr), KB, 0, c->st>>>(n, V, vstr, W, part, pstr);
            PB_LAUNCH(c);
            k_bfinish<<<dim3(j + 1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + (pass ? yoff : hoff), S);
            PB_LAUNCH(c);
            k_borth<<<dim3(G, nr), KB, 0, c->st>>>(n, j + 1, V, vstr, small + (pass ? yoff : hoff), S, W);
            PB_LAUNCH(c);
        }
        k_bmerge<<<nr, 64, 0, c->st>>>(j + 1, small, S, yoff, hoff);
        PB_LAUNCH(c);
        k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, nullptr, 0, W, part, pstr);
        PB_LAUNCH(c);
        k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff + j + 1, S);
        PB_LAUNCH(c);
        k_bscale<<<dim3(G, nr), KB, 0, c->st>>>(n, W, n, small + hoff + j + 1, S, V + (size_t)(j + 1) * n, vstr);
        PB_LAUNCH(c);
        k_bgm_givens<<<nr, 1, 0, c->st>>>(m, j, st, S);
        PB_LAUNCH(c);
        pb_toc(c, PB_T_ARNOLDI);
        return PB_OK;
    };
    // Each step's launches (about 40, over both streams) are captured once into a CUDA graph
    // per step index and replayed; the graphs stay valid while the build and this workspace do.
    // With timing enabled (events per phase) the launches are issued directly.
    if ((rc = pb_matvec_reserve(c, nr))) return rc;
    const bool use_graphs = !c->timing;
    if (c->gb_graph_key != (void*)V || (int)c->gb_graphs.size() != m || c->gb_graph_nr != nr) {
        pb_drop_graphs(c);
        c->gb_graphs.assign(m, nullptr);
        c->gb_graph_n.assign(m, 0);
        c->gb_graph_key = V;
        c->gb_graph_nr = nr;
    }
    auto arnoldi_step = [&](int j) -> int {
        if (!use_graphs || c->gb_graph_failed) return step_launches(j);
        if (!c->gb_graphs[j]) {
            cudaStream_t keep = c->st;
            c->st = c->cap_st;  // capture on the context's private stream
            long long n0 = c->nlaunch;
            cudaGraph_t g = nullptr;
            int rc2 = PB_OK;
            if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                rc2 = -1;
            } else {
                rc2 = step_launches(j);
                if (cudaStreamEndCapture(c->st, &g) != cudaSuccess) rc2 = -1;
            }
            c->st = keep;
            c->gb_graph_n[j] = c->nlaunch - n0;
            c->nlaunch = n0;
            cudaGraphExec_t ex = nullptr;
            if (rc2 == PB_OK && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
                c->gb_graphs[j] = ex;
            } else {
                // capture not possible here: issue the launches directly from now on
                cudaGetLastError();
                c->gb_graph_failed = true;
                c->err = "no error";
            }
            if (g) cudaGraphDestroy(g);
            if (!c->gb_graphs[j]) return step_launches(j);
        }
        PB_CUDA(c, cudaGraphLaunch(c->gb_graphs[j], c->st));
        c->nlaunch += c->gb_graph_n[j];
        ++c->graph_launches;
        return PB_OK;
    };
    int it = 0, first = 1;
    auto any_active = [&]() {
        for (int r = 0; r < nr; ++r)
            if (active[r]) return true;
        return false;
    };
    while (any_active() && it < max_iter) {
        // r = b - A x, V_0 = r / ||r||
        if ((rc = pb_matvec_sorted_multi(c, X, W, nr))) return rc;
        for (int r = 0; r < nr; ++r) mvs[r] += active[r];
        if (first) {
            // each given start is first scaled by its least-squares factor (zero if none is
            // positive): two dot products per right-hand side, no extra product
            k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, B, n, W, part, pstr);
            PB_LAUNCH(c);
            k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff, S);
            PB_LAUNCH(c);
            k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, nullptr, 0, W, part, pstr);
            PB_LAUNCH(c);
            k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff + 1, S);
            PB_LAUNCH(c);
            k_dg_start_scale<<<dim3(G, nr), KB, 0, c->st>>>(n, small, S, hoff, X, W);
            PB_LAUNCH(c);
        }
        k_bresidual<<<dim3(G, nr), KB, 0, c->st>>>(n, B, W);
        PB_LAUNCH(c);
        k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, nullptr, 0, W, part, pstr);
        PB_LAUNCH(c);
        k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff, S);
        PB_LAUNCH(c);
        k_bscale<<<dim3(G, nr), KB, 0, c->st>>>(n, W, n, small + hoff, S, V, vstr);
        PB_LAUNCH(c);
        k_bgm_start<<<nr, 1, 0, c->st>>>(m, st, S);
        PB_LAUNCH(c);
        if ((rc = read(roff))) return rc;
        for (int r = 0; r < nr; ++r) {
            if (!active[r]) continue;
            rel[r] = hv[r] / bnorm[r];
            if (first) init[r] = rel[r];
            if (!isfinite(rel[r])) {
                status[r] = PB_ERR_NONFINITE;
                active[r] = 0;
            } else if (rel[r] <= tol) {
                conv[r] = 1;
                active[r] = 0;
            }
            steps[r] = 0;
        }
        first = 0;
        std::vector<int> cyc(nr, 0);  // right-hand sides iterating in this cycle
        for (int r = 0; r < nr; ++r) cyc[r] = active[r];
        int j = 0;
        for (; j < m && it < max_iter && any_active(); ++j) {
            if ((rc = arnoldi_step(j))) return rc;
            if ((rc = read(roff))) return rc;
            ++it;
            for (int r = 0; r < nr; ++r) {
                if (!active[r]) continue;
                ++its[r];
                ++mvs[r];
                steps[r] = j + 1;
                rel[r] = hv[r] / bnorm[r];
                if (!isfinite(rel[r])) {
                    status[r] = PB_ERR_NONFINITE;
                    active[r] = 0;
                    steps[r] = 0;  // no update from a broken cycle
                } else if (rel[r] <= tol) {
                    conv[r] = 1;
                    active[r] = 0;
                }
            }
        }
        // x_r += M^-1 V_r y_r over the steps r took in this cycle
        for (int r = 0; r < nr; ++r) {
            if (!cyc[r] || steps[r] == 0) continue;
            GmState t = st;
            const long long o = r * S;
            t.H += o;
            t.cs += o;
            t.sn += o;
            t.g += o;
            t.y += o;
            t.hcol += o;
            t.res += o;
            k_gm_solve<<<1, 1, 0, c->st>>>(m, steps[r], t);
            PB_LAUNCH(c);
            k_combine<<<G, KB, 0, c->st>>>(n, steps[r], V + r * vstr, t.y, W + r * n);
            PB_LAUNCH(c);
            if ((rc = pb_precond_apply_multi(c, W + r * n, 0, Z + r * n, 0, 1))) return rc;
            k_axpy1<<<G, KB, 0, c->st>>>(n, Z + r * n, X + r * n);
            PB_LAUNCH(c);
        }
    }
    // true residuals
    if ((rc = pb_matvec_sorted_multi(c, X, W, nr))) return rc;
    k_bresidual<<<dim3(G, nr), KB, 0, c->st>>>(n, B, W);
    PB_LAUNCH(c);
    k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, nullptr, 0, W, part, pstr);
    PB_LAUNCH(c);
    k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff, S);
    PB_LAUNCH(c);
    if ((rc = read(hoff))) return rc;
    int derr = 0;
    PB_CUDA(c, cudaMemcpyAsync(&derr, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    int worst = PB_OK;
    for (int r = 0; r < nr; ++r) {
        pb_solve_info inf = {its[r], mvs[r] + 1, bnorm[r] > 0 ? sqrt(hv[r]) / bnorm[r] : 0.0, status[r], init[r]};
        if (inf.status == PB_OK && !conv[r]) inf.status = PB_ERR_NOT_CONVERGED;
        if (inf.status == PB_OK && !isfinite(inf.rel_residual)) inf.status = PB_ERR_NONFINITE;
        if (derr) inf.status = PB_ERR_TIMEOUT;
        if (infos) infos[r] = inf;
        if (inf.status != PB_OK && worst == PB_OK) worst = inf.status;
    }
    if (derr) pb_fail(c, PB_ERR_TIMEOUT, "a bounded wait in the MtL kernel gave up");
    return worst;
}

// ---------- GMRES driven from the device: one CUDA graph launch per solve ----------
// The same right-preconditioned GMRES(m) for nr right-hand sides (CGS2, Givens rotations, the
// true residual recomputed at the end of every cycle), with every control decision taken on the
// device instead of the host. A control block holds the step index, the shared iteration count
// and each right-hand side's state; two conditional WHILE nodes of a CUDA graph repeat the
// Arnoldi step (inner) and the restart cycle (outer) until every right-hand side has converged,
// failed or run out of iterations. Kernels whose work depends on the step index read it from
// the control block (grids sized for the largest step; blocks past the current one leave at
// once), and the current basis vector is also kept in a fixed buffer so that the
// preconditioner and the product read one address in every replay. The graph is built from
// sequential stream captures on the context's private stream joined by the conditional nodes,
// so it can be appended as one branch of a larger graph (several molecules in one launch).
struct DgCtl {
    int j;          // Arnoldi step within the current cycle
    int it;         // Arnoldi steps taken (shared by the right-hand sides)
    int cycles;     // completed restart cycles
    int max_iter, m, nr;
    double tol;
    int active[PB_MAX_RHS], conv[PB_MAX_RHS], status[PB_MAX_RHS], its[PB_MAX_RHS], mvs[PB_MAX_RHS];
    int steps[PB_MAX_RHS], cyc[PB_MAX_RHS];
    double bnorm[PB_MAX_RHS], init[PB_MAX_RHS], rel[PB_MAX_RHS];
};

// part[r][col][blk] = partial of <V_r[col], w_r>, columns 0..j
__global__ void k_dg_dot(long long n, const double* __restrict__ V, long long vstr, const double* __restrict__ w,
                         double* __restrict__ part, long long pstr, const DgCtl* __restrict__ ctl)
{
    const int col = blockIdx.y, r = blockIdx.z;
    if (col > ctl->j) return;
    __shared__ double red[KB];
    w += r * n;
    const double* v = V + r * vstr + (size_t)col * n;
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) s += v[i] * w[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = KB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[r * pstr + (size_t)col * DOT_BLOCKS + blockIdx.x] = red[0];
}

// out_r[col] = sum of the partials of column col, columns 0..j (at = 0), or, for at = 1, the
// single column 0 of the partials into out_r[j + 1]
__global__ void k_dg_finish(const double* __restrict__ part, long long pstr, double* __restrict__ out,
                            long long ostr, const DgCtl* __restrict__ ctl, int at)
{
    const int col = blockIdx.x, r = blockIdx.y;
    const int j = ctl->j;
    if (col > (at ? 0 : j)) return;
    __shared__ double red[KB];
    double s = 0.0;
    for (int i = threadIdx.x; i < DOT_BLOCKS; i += KB) s += part[r * pstr + (size_t)col * DOT_BLOCKS + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = KB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r * ostr + (at ? j + 1 : col)] = red[0];
}

// w_r -= V_r[:, 0..j] h_r
__global__ void k_dg_orth(long long n, const double* __restrict__ V, long long vstr, const double* __restrict__ h,
                          long long hstr, double* __restrict__ w, const DgCtl* __restrict__ ctl)
{
    const int r = blockIdx.y, ncol = ctl->j + 1;
    V += r * vstr;
    h += r * hstr;
    w += r * n;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        double s = 0.0;
        for (int c = 0; c < ncol; ++c) s += V[(size_t)c * n + i] * h[c];
        w[i] -= s;
    }
}

// hcol_r[i] += y_r[i], i <= j
__global__ void k_dg_merge(double* __restrict__ small, long long sstr, long long yoff, long long hoff,
                           const DgCtl* __restrict__ ctl)
{
    double* s = small + blockIdx.x * sstr;
    const int k = ctl->j + 1;
    for (int i = threadIdx.x; i < k; i += blockDim.x) s[hoff + i] += s[yoff + i];
}

// V_r[c] = Vcur_r = w_r / sqrt(hcol_r[c]) with c = j + 1 (an Arnoldi step) or c = 0 (first = 1,
// the start of a cycle)
__global__ void k_dg_scale(long long n, const double* __restrict__ W, const double* __restrict__ small, long long sstr,
                           long long hoff, double* __restrict__ V, long long vstr, double* __restrict__ Vcur,
                           const DgCtl* __restrict__ ctl, int first)
{
    const int r = blockIdx.y;
    const int c = first ? 0 : ctl->j + 1;
    const double f = 1.0 / sqrt(small[r * sstr + hoff + c]);
    const double* src = W + r * n;
    double* dst = V + r * vstr + (size_t)c * n;
    double* cur = Vcur + r * n;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        const double v = src[i] * f;
        dst[i] = v;
        cur[i] = v;
    }
}

// step j of right-hand side r = blockIdx.x (k_bgm_givens with the step index from the device)
__global__ void k_dg_givens(int m, GmState s, long long sstr, const DgCtl* __restrict__ ctl)
{
    const long long o = blockIdx.x * sstr;
    GmState t = {s.H + o, s.cs + o, s.sn + o, s.g + o, s.y + o, s.hcol + o, s.res + o};
    gm_givens_step(m, ctl->j, t);
}

// After an Arnoldi step: each active right-hand side counts the step and checks its residual
// estimate; the inner loop continues while one is active, the cycle has room and the iteration
// budget is not spent. One block of PB_MAX_RHS threads.
__global__ void k_dg_step_ctl(DgCtl* __restrict__ ctl, const double* __restrict__ small, long long sstr,
                              long long roff, cudaGraphConditionalHandle h)
{
    const int r = threadIdx.x;
    const int j = ctl->j;
    int act = 0;
    if (r < ctl->nr && ctl->active[r]) {
        ctl->its[r]++;
        ctl->mvs[r]++;
        ctl->steps[r] = j + 1;
        const double rel = small[r * sstr + roff] / ctl->bnorm[r];
        ctl->rel[r] = rel;
        if (!isfinite(rel)) {
            ctl->status[r] = PB_ERR_NONFINITE;
            ctl->active[r] = 0;
            ctl->steps[r] = 0;  // no update from a broken cycle
        } else if (rel <= ctl->tol) {
            ctl->conv[r] = 1;
            ctl->active[r] = 0;
        } else {
            act = 1;
        }
    }
    act = __syncthreads_or(act);
    if (r == 0) {
        const int it = ctl->it + 1;
        ctl->it = it;
        ctl->j = j + 1;
        cudaGraphSetConditional(h, (act && j + 1 < ctl->m && it < ctl->max_iter) ? 1u : 0u);
    }
}

// Start of a cycle's Arnoldi loop: enter while a right-hand side is active and iterations are left.
__global__ void k_dg_enter(const DgCtl* __restrict__ ctl, cudaGraphConditionalHandle h)
{
    int act = 0;
    for (int r = 0; r < ctl->nr; ++r) act |= ctl->active[r];
    cudaGraphSetConditional(h, (act && ctl->j < ctl->m && ctl->it < ctl->max_iter) ? 1u : 0u);
}

// Before anything else: ||b_r|| (hcol_r[0] holds ||b_r||^2), the counters, and the host's
// settings (tol, max_iter, m, nr stay as uploaded). start = 1: the product of the given start
// counts for every right-hand side.
__global__ void k_dg_init(DgCtl* __restrict__ ctl, const double* __restrict__ small, long long sstr, long long hoff,
                          int start)
{
    const int r = threadIdx.x;
    if (r == 0) {
        ctl->j = 0;
        ctl->it = 0;
        ctl->cycles = 0;
    }
    if (r >= ctl->nr) return;
    const double bn = sqrt(small[r * sstr + hoff]);
    ctl->bnorm[r] = bn;
    ctl->its[r] = 0;
    ctl->mvs[r] = start;
    ctl->steps[r] = 0;
    ctl->conv[r] = 0;
    ctl->cyc[r] = 0;
    ctl->status[r] = PB_OK;
    ctl->init[r] = 1.0;
    ctl->rel[r] = 1.0;
    ctl->active[r] = 1;
    if (!isfinite(bn)) {  // an overflowing or non-finite right-hand side
        ctl->status[r] = PB_ERR_NONFINITE;
        ctl->active[r] = 0;
        ctl->rel[r] = bn;
    } else if (!(bn > 0)) {  // b = 0: x = 0 solves it exactly
        ctl->active[r] = 0;
        ctl->conv[r] = 1;
        ctl->rel[r] = 0.0;
        ctl->init[r] = 0.0;
    }
}

// x_r = 0 where b_r = 0 (or is not finite)
__global__ void k_dg_zero_x(long long n, double* __restrict__ X, const DgCtl* __restrict__ ctl)
{
    const int r = blockIdx.y;
    if (ctl->bnorm[r] > 0 && isfinite(ctl->bnorm[r])) return;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) X[r * n + i] = 0.0;
}

// k_start_scale per right-hand side: d_r = hcol_r[0..1] = {<w, b>, <w, w>}
__global__ void k_dg_start_scale(long long n, const double* __restrict__ small, long long sstr, long long hoff,
                                 double* __restrict__ X, double* __restrict__ W)
{
    const int r = blockIdx.y;
    const double* d = small + r * sstr + hoff;
    const double a = d[1] > 0.0 ? d[0] / d[1] : 0.0;
    const double f = (a > 0.0 && isfinite(a)) ? a : 0.0;
    X += r * n;
    W += r * n;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        X[i] = f != 0.0 ? X[i] * f : 0.0;
        W[i] = f != 0.0 ? W[i] * f : 0.0;
    }
}

// End of a cycle (first = 0) or end of the start (first = 1): the residual of the current x is
// in res_r (true residual, from a product). Records it, retires converged or broken right-hand
// sides, opens the next cycle for the others and decides whether the outer loop runs again.
__global__ void k_dg_cycle_ctl(DgCtl* __restrict__ ctl, const double* __restrict__ small, long long sstr,
                               long long roff, cudaGraphConditionalHandle h, int first)
{
    const int r = threadIdx.x;
    int act = 0;
    if (r < ctl->nr) {
        const double bn = ctl->bnorm[r];
        const bool live = bn > 0 && isfinite(bn);
        const double rel = small[r * sstr + roff] / bn;
        if (!first && ctl->cyc[r]) ctl->mvs[r]++;  // the product that closed its cycle
        if (live) {
            ctl->rel[r] = rel;
            if (first) ctl->init[r] = rel;
        }
        if (ctl->active[r]) {
            if (!isfinite(rel)) {
                ctl->status[r] = PB_ERR_NONFINITE;
                ctl->active[r] = 0;
            } else if (rel <= ctl->tol) {
                ctl->conv[r] = 1;
                ctl->active[r] = 0;
            }
        }
        ctl->cyc[r] = ctl->active[r];
        ctl->steps[r] = 0;
        act = ctl->active[r];
    }
    act = __syncthreads_or(act);
    if (r == 0) {
        ctl->j = 0;
        if (!first) ctl->cycles++;
        cudaGraphSetConditional(h, (act && ctl->it < ctl->max_iter) ? 1u : 0u);
    }
}

// back substitution of right-hand side r = blockIdx.x over the steps it took in this cycle
__global__ void k_dg_solve(int m, GmState s, long long sstr, const DgCtl* __restrict__ ctl)
{
    const long long o = blockIdx.x * sstr;
    const int k = ctl->steps[blockIdx.x];
    const double* H = s.H + o;
    const double* g = s.g + o;
    double* y = s.y + o;
    for (int i = k - 1; i >= 0; --i) {
        double v = g[i];
        for (int q = i + 1; q < k; ++q) v -= H[(size_t)q * (m + 1) + i] * y[q];
        const double d = H[(size_t)i * (m + 1) + i];
        y[i] = d != 0.0 ? v / d : 0.0;
    }
}

// u_r = V_r[:, 0..steps_r) y_r (zero for a right-hand side without steps)
__global__ void k_dg_combine(long long n, const double* __restrict__ V, long long vstr, const double* __restrict__ small,
                             long long sstr, long long yoff, double* __restrict__ U, const DgCtl* __restrict__ ctl)
{
    const int r = blockIdx.y;
    const int k = ctl->steps[r];
    V += r * vstr;
    const double* y = small + r * sstr + yoff;
    U += r * n;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
        double s = 0.0;
        for (int c = 0; c < k; ++c) s += V[(size_t)c * n + i] * y[c];
        U[i] = s;
    }
}

// x_r += z_r for the right-hand sides that took steps in this cycle
__global__ void k_dg_axpy(long long n, const double* __restrict__ Z, double* __restrict__ X, const DgCtl* __restrict__ ctl)
{
    const int r = blockIdx.y;
    if (ctl->steps[r] == 0) return;
    for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB)
        X[r * n + i] += Z[r * n + i];
}

// device workspace of the device-driven solver: the batched Krylov workspace (shared with the
// host-driven batched solver) for nr right-hand sides, the current-vector buffer and nctl
// control blocks
int pb_dg_reserve(pb_ctx* c, int nr, int m, int nctl)
{
    const long long n = 2LL * c->nu;
    const long long S = (long long)(m + 1) * m + 6 * (m + 2);
    if (nr > c->gb_nr || m > c->gb_m) {
        const int nr2 = std::max(nr, c->gb_nr), m2 = std::max(m, c->gb_m);
        const long long S2 = (long long)(m2 + 1) * m2 + 6 * (m2 + 2);
        c->gbV = (double*)pb_alloc(c, sizeof(double) * (size_t)((m2 + 1) * n * nr2));
        c->gbW = (double*)pb_alloc(c, sizeof(double) * (size_t)(n * nr2));
        c->gbZ = (double*)pb_alloc(c, sizeof(double) * (size_t)(n * nr2));
        c->gbpart = (double*)pb_alloc(c, sizeof(double) * (size_t)(DOT_BLOCKS * (m2 + 2) * nr2));
        c->gbsmall = (double*)pb_alloc(c, sizeof(double) * (size_t)(S2 * nr2));
        if (!c->gbV || !c->gbW || !c->gbZ || !c->gbpart || !c->gbsmall) {
            c->gb_nr = c->gb_m = 0;
            return pb_fail(c, PB_ERR_NOMEM, "gmres workspace: out of memory");
        }
        c->gb_nr = nr2;
        c->gb_m = m2;
        pb_drop_graphs(c);
    }
    (void)S;
    if (nr > c->dg_nr) {
        c->dgVcur = (double*)pb_alloc(c, sizeof(double) * (size_t)(n * nr));
        c->dgWf = c->prm.precision == PB_MIXED ? (float2*)pb_alloc(c, sizeof(float2) * (size_t)(n * nr)) : nullptr;
        if (!c->dgVcur || (c->prm.precision == PB_MIXED && !c->dgWf))
            return pb_fail(c, PB_ERR_NOMEM, "gmres workspace: out of memory");
        c->dg_nr = nr;
    }
    if (nctl > c->dg_nctl) {
        c->dgctl = pb_alloc(c, sizeof(DgCtl) * nctl);
        if (!c->dgctl) return pb_fail(c, PB_ERR_NOMEM, "gmres workspace: out of memory");
        if (c->dgctl_h) cudaFreeHost(c->dgctl_h);
        c->dgctl_h = nullptr;
        if (cudaMallocHost(&c->dgctl_h, sizeof(DgCtl) * nctl) != cudaSuccess) {
            c->dgctl_h = nullptr;
            return pb_fail(c, PB_ERR_NOMEM, "gmres workspace: out of pinned host memory");
        }
        memset(c->dgctl_h, 0, sizeof(DgCtl) * nctl);
        c->dg_nctl = nctl;
    }
    return PB_OK;
}

// one capture segment on the context's private stream into graph g after deps
static bool seg_begin(pb_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd)
{
    return cudaStreamBeginCaptureToGraph(c->st, g, nd ? deps : nullptr, nullptr, nd, cudaStreamCaptureModeThreadLocal) ==
           cudaSuccess;
}
static bool seg_end(pb_ctx* c, std::vector<cudaGraphNode_t>* leaves)
{
    cudaStreamCaptureStatus stt;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    bool ok = cudaStreamGetCaptureInfo(c->st, &stt, nullptr, nullptr, &d, nullptr, &nd) == cudaSuccess &&
              stt == cudaStreamCaptureStatusActive;
    if (ok && leaves) leaves->assign(d, d + nd);
    cudaGraph_t out = nullptr;
    ok = (cudaStreamEndCapture(c->st, &out) == cudaSuccess) && ok;
    return ok;
}
static bool add_while(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle h,
                      cudaGraphNode_t* node, cudaGraph_t* body)
{
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    if (cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p) != cudaSuccess)
        return false;
    *body = p.conditional.phGraph_out[0];
    return true;
}

// Append one device-driven solve of nr right-hand sides (X, B: nr x 2N in tree order, vector r
// at + 2 N r) to graph g after deps; its last nodes go to leaves. start: 0 = from zero (X is
// zeroed inside), 1 = from the given X, scaled per right-hand side by its least-squares
// factor. ictl selects the control block. Must run with the context's private stream as c->st
// and every buffer reserved. The captured launch counts go to cnt (prologue, per cycle, per
// step).
int pb_dg_append(pb_ctx* c, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, double* X, const double* B,
                 int nr, int m, int start, int ictl, std::vector<cudaGraphNode_t>* leaves, long long cnt[3])
{
    const long long n = 2LL * c->nu;
    const int G = grid_for(n);
    const long long S = (long long)(m + 1) * m + 6 * (m + 2);
    const long long vstr = (long long)(m + 1) * n, pstr = (long long)DOT_BLOCKS * (m + 2);
    double *V = c->gbV, *W = c->gbW, *Z = c->gbZ, *part = c->gbpart, *small = c->gbsmall, *Vc = c->dgVcur;
    DgCtl* ctl = (DgCtl*)c->dgctl + ictl;
    // mixed precision: float-float basis in the same storage (the step index and the per-vector
    // step counts read by the kernels from the control block)
    const bool ffb = c->prm.precision == PB_MIXED;
    float2 *Vf = (float2*)c->gbV, *Wf = c->dgWf;
    const int* jdev = (const int*)((const char*)ctl + offsetof(DgCtl, j));
    const int* ksteps = (const int*)((const char*)ctl + offsetof(DgCtl, steps));
    const GmState st = gm_state(small, m);
    const long long hoff = st.hcol - small, yoff = st.y - small, roff = st.res - small;
    cudaGraphConditionalHandle hO, hI;
    if (cudaGraphConditionalHandleCreate(&hO, g, 0, 0) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> lv;
    int rc = PB_OK;
    long long n0 = c->nlaunch;
    // prologue: ||b||, the start, the first residual and its normalisation
    if (!seg_begin(c, g, deps.data(), deps.size())) return -1;
    do {
        if (start == 0) PB_CUDA(c, cudaMemsetAsync(X, 0, sizeof(double) * n * nr, c->st));
        k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, nullptr, 0, B, part, pstr);
        PB_LAUNCH(c);
        k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff, S);
        PB_LAUNCH(c);
        k_dg_init<<<1, PB_MAX_RHS, 0, c->st>>>(ctl, small, S, hoff, start);
        PB_LAUNCH(c);
        if (start == 0) {
            PB_CUDA(c, cudaMemcpyAsync(W, B, sizeof(double) * n * nr, cudaMemcpyDeviceToDevice, c->st));
        } else {
            if ((rc = pb_matvec_sorted_multi(c, X, W, nr))) break;
            k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, B, n, W, part, pstr);
            PB_LAUNCH(c);
            k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff, S);
            PB_LAUNCH(c);
            k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, nullptr, 0, W, part, pstr);
            PB_LAUNCH(c);
            k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff + 1, S);
            PB_LAUNCH(c);
            k_dg_start_scale<<<dim3(G, nr), KB, 0, c->st>>>(n, small, S, hoff, X, W);
            PB_LAUNCH(c);
            k_bresidual<<<dim3(G, nr), KB, 0, c->st>>>(n, B, W);
            PB_LAUNCH(c);
        }
        k_dg_zero_x<<<dim3(G, nr), KB, 0, c->st>>>(n, X, ctl);
        PB_LAUNCH(c);
        k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, nullptr, 0, W, part, pstr);
        PB_LAUNCH(c);
        k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff, S);
        PB_LAUNCH(c);
        if (ffb)
            k_ffscale<<<dim3(G, nr), KB, 0, c->st>>>(n, nullptr, W, small, S, hoff, nullptr, 0, 1, Vf, vstr, Vc);
        else
            k_dg_scale<<<dim3(G, nr), KB, 0, c->st>>>(n, W, small, S, hoff, V, vstr, Vc, ctl, 1);
        PB_LAUNCH(c);
        k_bgm_start<<<nr, 1, 0, c->st>>>(m, st, S);
        PB_LAUNCH(c);
        k_dg_cycle_ctl<<<1, PB_MAX_RHS, 0, c->st>>>(ctl, small, S, roff, hO, 1);
        PB_LAUNCH(c);
    } while (0);
    if (!seg_end(c, &lv) || rc) return rc ? rc : -1;
    cnt[0] = c->nlaunch - n0;
    // outer loop: one restart cycle per pass
    cudaGraphNode_t wO, wI;
    cudaGraph_t bO, bI;
    if (!add_while(g, lv, hO, &wO, &bO)) return -1;
    if (cudaGraphConditionalHandleCreate(&hI, bO, 0, 0) != cudaSuccess) return -1;
    n0 = c->nlaunch;
    if (!seg_begin(c, bO, nullptr, 0)) return -1;
    k_dg_enter<<<1, 1, 0, c->st>>>(ctl, hI);
    PB_LAUNCH(c);
    if (!seg_end(c, &lv)) return -1;
    if (!add_while(bO, lv, hI, &wI, &bI)) return -1;
    long long n1 = c->nlaunch - n0;
    // inner loop: one Arnoldi step per pass
    n0 = c->nlaunch;
    if (!seg_begin(c, bI, nullptr, 0)) return -1;
    do {
        if ((rc = pb_precond_apply_multi(c, Vc, n, Z, n, nr))) break;
        if ((rc = pb_matvec_sorted_multi(c, Z, W, nr))) break;
        if (ffb) {
            k_to_ff<<<dim3(G, nr), KB, 0, c->st>>>(n, W, Wf);
            PB_LAUNCH(c);
        }
        for (int pass = 0; pass < 2; ++pass) {
            double* h = small + (pass ? yoff : hoff);
            if (ffb)
                k_ffdot<<<dim3(DOT_BLOCKS, (m + FFK_CG - 1) / FFK_CG, nr), KB, 0, c->st>>>(n, 0, jdev, Vf, vstr, Wf,
                                                                                           part, pstr);
            else
                k_dg_dot<<<dim3(DOT_BLOCKS, m, nr), KB, 0, c->st>>>(n, V, vstr, W, part, pstr, ctl);
            PB_LAUNCH(c);
            k_dg_finish<<<dim3(m, nr), KB, 0, c->st>>>(part, pstr, h, S, ctl, 0);
            PB_LAUNCH(c);
            if (ffb)
                k_fforth<<<dim3(G, nr), KB, 0, c->st>>>(n, 0, jdev, Vf, vstr, h, S, Wf);
            else
                k_dg_orth<<<dim3(G, nr), KB, 0, c->st>>>(n, V, vstr, h, S, W, ctl);
            PB_LAUNCH(c);
        }
        k_dg_merge<<<nr, 64, 0, c->st>>>(small, S, yoff, hoff, ctl);
        PB_LAUNCH(c);
        if (ffb)
            k_ffdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, 1, nullptr, nullptr, 0, Wf, part, pstr);
        else
            k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, nullptr, 0, W, part, pstr);
        PB_LAUNCH(c);
        k_dg_finish<<<dim3(1, nr), KB, 0, c->st>>>(part, pstr, small + hoff, S, ctl, 1);
        PB_LAUNCH(c);
        if (ffb)
            k_ffscale<<<dim3(G, nr), KB, 0, c->st>>>(n, Wf, nullptr, small, S, hoff, jdev, 0, 0, Vf, vstr, Vc);
        else
            k_dg_scale<<<dim3(G, nr), KB, 0, c->st>>>(n, W, small, S, hoff, V, vstr, Vc, ctl, 0);
        PB_LAUNCH(c);
        k_dg_givens<<<nr, 1, 0, c->st>>>(m, st, S, ctl);
        PB_LAUNCH(c);
        k_dg_step_ctl<<<1, PB_MAX_RHS, 0, c->st>>>(ctl, small, S, roff, hI);
        PB_LAUNCH(c);
    } while (0);
    if (!seg_end(c, nullptr) || rc) return rc ? rc : -1;
    cnt[2] = c->nlaunch - n0;
    // end of the cycle: update, true residual, next cycle's start
    n0 = c->nlaunch;
    std::vector<cudaGraphNode_t> after = {wI};
    if (!seg_begin(c, bO, after.data(), 1)) return -1;
    do {
        k_dg_solve<<<nr, 1, 0, c->st>>>(m, st, S, ctl);
        PB_LAUNCH(c);
        if (ffb)
            k_ffcombine<<<dim3(G, nr), KB, 0, c->st>>>(n, 0, ksteps, Vf, vstr, small + yoff, S, W);
        else
            k_dg_combine<<<dim3(G, nr), KB, 0, c->st>>>(n, V, vstr, small, S, yoff, W, ctl);
        PB_LAUNCH(c);
        if ((rc = pb_precond_apply_multi(c, W, n, Z, n, nr))) break;
        k_dg_axpy<<<dim3(G, nr), KB, 0, c->st>>>(n, Z, X, ctl);
        PB_LAUNCH(c);
        if ((rc = pb_matvec_sorted_multi(c, X, W, nr))) break;
        k_bresidual<<<dim3(G, nr), KB, 0, c->st>>>(n, B, W);
        PB_LAUNCH(c);
        k_bdot<<<dim3(DOT_BLOCKS, 1, nr), KB, 0, c->st>>>(n, nullptr, 0, W, part, pstr);
        PB_LAUNCH(c);
        k_bfinish<<<dim3(1, nr), KB, 0, c->st>>>(DOT_BLOCKS, part, pstr, small + hoff, S);
        PB_LAUNCH(c);
        if (ffb)
            k_ffscale<<<dim3(G, nr), KB, 0, c->st>>>(n, nullptr, W, small, S, hoff, nullptr, 0, 1, Vf, vstr, Vc);
        else
            k_dg_scale<<<dim3(G, nr), KB, 0, c->st>>>(n, W, small, S, hoff, V, vstr, Vc, ctl, 1);
        PB_LAUNCH(c);
        k_bgm_start<<<nr, 1, 0, c->st>>>(m, st, S);
        PB_LAUNCH(c);
        k_dg_cycle_ctl<<<1, PB_MAX_RHS, 0, c->st>>>(ctl, small, S, roff, hO, 0);
        PB_LAUNCH(c);
    } while (0);
    if (!seg_end(c, nullptr) || rc) return rc ? rc : -1;
    cnt[1] = n1 + c->nlaunch - n0;
    if (leaves) leaves->assign(1, wO);
    return PB_OK;
}

void pb_dg_drop(pb_ctx* c)
{
    if (c->dg_exec) cudaGraphExecDestroy(c->dg_exec);
    c->dg_exec = nullptr;
}

// host side of one control block after the graph ran: solve records and launch count
void pb_dg_results(pb_ctx* c, int ictl, int nr, const long long cnt[3], pb_solve_info* infos, int* worst)
{
    const DgCtl* h = (const DgCtl*)c->dgctl_h + ictl;
    c->nlaunch += cnt[0] + (long long)h->cycles * cnt[1] + (long long)h->it * cnt[2];
    for (int r = 0; r < nr; ++r) {
        pb_solve_info inf = {h->its[r], h->mvs[r], h->rel[r], h->status[r], h->init[r]};
        if (inf.status == PB_OK && !h->conv[r]) inf.status = PB_ERR_NOT_CONVERGED;
        if (inf.status == PB_OK && !isfinite(inf.rel_residual)) inf.status = PB_ERR_NONFINITE;
        if (infos) infos[r] = inf;
        if (inf.status != PB_OK && *worst == PB_OK) *worst = inf.status;
    }
}

// the host's settings of a control block (uploaded before the graph launch)
void pb_dg_settings(pb_ctx* c, int ictl, int nr, int m, double tol, int max_iter)
{
    DgCtl* h = (DgCtl*)c->dgctl_h + ictl;
    h->nr = nr;
    h->m = m;
    h->tol = tol;
    h->max_iter = max_iter;
}

int pb_dg_upload(pb_ctx* c, int nctl)
{
    PB_CUDA(c, cudaMemcpyAsync(c->dgctl, c->dgctl_h, sizeof(DgCtl) * nctl, cudaMemcpyHostToDevice, c->st));
    return PB_OK;
}

int pb_dg_download(pb_ctx* c, int nctl)
{
    PB_CUDA(c, cudaMemcpyAsync(c->dgctl_h, c->dgctl, sizeof(DgCtl) * nctl, cudaMemcpyDeviceToHost, c->st));
    return PB_OK;
}

// Device-driven GMRES of nr right-hand sides on this context (one graph, cached while the
// build, the workspace and the shape of the call stay the same). Returns -1 when the graph
// cannot be built here (the caller then takes the host-driven loop).
int pb_gmres_dev(pb_ctx* c, double* X, const double* B, int nr, double tol, int max_iter, int restart, int start,
                 pb_solve_info* infos)
{
    int rc;
    if ((rc = pb_matvec_reserve(c, nr))) return rc;
    if ((rc = pb_dg_reserve(c, nr, restart, 1))) return rc;
    const void* key[6] = {(void*)X, (void*)B, (void*)c->gbV, (void*)c->dgVcur, (void*)c->dgctl,
                          (void*)(long long)c->build_gen};
    const int ikey[3] = {nr, restart, start};
    bool same = c->dg_exec && !memcmp(key, c->dg_key, sizeof(key)) && !memcmp(ikey, c->dg_ikey, sizeof(ikey));
    if (!same) {
        if (c->dg_exec) cudaGraphExecDestroy(c->dg_exec);
        c->dg_exec = nullptr;
        cudaGraph_t g = nullptr;
        if (cudaGraphCreate(&g, 0) != cudaSuccess) return -1;
        cudaStream_t keep = c->st;
        c->st = c->cap_st;
        const long long nl = c->nlaunch;
        std::vector<cudaGraphNode_t> leaves;
        rc = pb_dg_append(c, g, {}, X, B, nr, restart, start, 0, &leaves, c->dg_cnt);
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(c->st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;  // a failed segment left its capture open
            cudaStreamEndCapture(c->st, &junk);
            if (junk && junk != g) cudaGraphDestroy(junk);
        }
        c->st = keep;
        c->nlaunch = nl;
        if (rc == PB_OK && cudaGraphInstantiate(&c->dg_exec, g, 0) != cudaSuccess) rc = -1;
        cudaGraphDestroy(g);
        if (rc != PB_OK) {
            c->dg_exec = nullptr;
            if (rc > 0) return rc;
            cudaGetLastError();
            return -1;
        }
        memcpy(c->dg_key, key, sizeof(key));
        memcpy(c->dg_ikey, ikey, sizeof(ikey));
    }
    pb_dg_settings(c, 0, nr, restart, tol, max_iter);
    if ((rc = pb_dg_upload(c, 1))) return rc;
    PB_CUDA(c, cudaGraphLaunch(c->dg_exec, c->st));
    ++c->graph_launches;
    if ((rc = pb_dg_download(c, 1))) return rc;
    int derr = 0;
    PB_CUDA(c, cudaMemcpyAsync(&derr, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    int worst = PB_OK;
    pb_dg_results(c, 0, nr, c->dg_cnt, infos, &worst);
    if (derr) {
        for (int r = 0; r < nr; ++r)
            if (infos) infos[r].status = PB_ERR_TIMEOUT;
        return pb_fail(c, PB_ERR_TIMEOUT, "a bounded wait in the MtL kernel gave up");
    }
    return worst;
}
