// Far field of the FMM matrix-vector product (Section 2.4, steps 2-6): leaf moments,
// upward MtM pass (eqMtM), interaction phase MtL (eqcoeff) with kernel derivatives by
// recurrence, downward LtL pass and LtP evaluation (LtP).
//
// The four kernels regroup into two expansions. With densities f0 = dphi m - phi m_nu (for
// G0) and fk = -dphi m + eps phi m_nu (for Gk), where m^b(psi_i) = A_i (c_i - x_c)^b and
// m_nu^b(psi_i) = A_i n_i . grad (y - x_c)^b at y = c_i (one-point rule, eqmoment), the
// far-field rows are
//   y1_i -= A_i sum_a (lam0 + lamk)^a (c_i - x_c)^a
//   y2_i -= A_i sum_a (lam0 + lamk / eps)^a n_i . grad (x - x_c)^a
// since K1 + K2 pair G0 and Gk single and double layers, and K3 + K4 are their normal
// derivatives at the target (Eq_K1/Eq_K2).
//
// Kernel derivatives (MtL). With phi = exp(-kappa r)/(4 pi r), psi = exp(-kappa r)/(4 pi)
// and Taylor coefficients F_k = D^k phi(d)/k!, Psi_k = D^k psi(d)/k!, the identities
// r^2 grad phi = -(phi + kappa psi) x and grad psi = -kappa phi x, applied to the Euler
// operator h . grad of the expansion in h, give for n = |k| >= 1
//   |d|^2 n F_k = -(2n - 1) sum_i d_i F_{k-e_i} - (n - 1) sum_i F_{k-2e_i}
//                 - kappa sum_i d_i Psi_{k-e_i} - kappa sum_i Psi_{k-2e_i}
//   n Psi_k     = -kappa (sum_i d_i F_{k-e_i} + sum_i F_{k-2e_i})
// (terms with a negative index vanish). kappa = 0 gives the Coulomb recurrence.
// The MtL sum is evaluated as  a! lam^a = sum_b D^{a+b} G(d) * [(-1)^|b| m^b / b!].
#include <math.h>

#include <algorithm>
#include <vector>

#include "ff.cuh"
#include "pb_internal.cuh"

#include "m2l_unrolled.cuh"

#define FAR_T 128
#define NT_MAX 455  // nterms(12)

__constant__ int c_mi[NT_MAX];          // multi-index exponents a | b << 8 | c << 16
__constant__ double c_fact[25];         // n!
__constant__ double c_binom[13][13];    // C(n, k)
__constant__ float c_ifact[NT_MAX];     // 1 / (a1! a2! a3!) of multi-index a (FP32)
__constant__ double c_ifact64[NT_MAX];  // the same in FP64
__constant__ float c_i1f[PB_PMAX + 1];  // 1 / k! (one axis), FP32
__constant__ double c_i1d[PB_PMAX + 1]; // the same in FP64
template <class R>
__device__ __forceinline__ R inv_fact1(int k)
{
    return sizeof(R) == 4 ? (R)c_i1f[k] : (R)c_i1d[k];
}

__device__ __forceinline__ void mi_unpack(int v, int& a, int& b, int& c)
{
    a = v & 0xff;
    b = (v >> 8) & 0xff;
    c = v >> 16;
}

// ---------- step 2: leaf moments ----------
// Stored form of every moment array: m~[b] = (-1)^|b| m[b] / b!, the form the MtL contraction
// uses (eqcoeff), so that MtL reads the moments as they are and MtM is a plain shift.
// With d' = x_c - y (cluster centre minus source point), (-1)^|b| (y - x_c)^b = d'^b.
// With e_j[b] = d'_j^b / b! (d' = x_c - y_j, one factor per axis) the stored moments are
//   m~0[b] = S[b] + sum_i G_i[b - e_i],   m~k[b] = -S[b] - eps sum_i G_i[b - e_i],
//   S[b] = sum_j A_j dphi_j e_j[b],   G_i[b] = sum_j A_j phi_j n_j,i e_j[b],
// because the normal derivative of d'^b / b! is sum_i n_i e[b - e_i] up to the sign of d'.
// Thread q owns the multi-indices q, q + P2M_T, ...; the sources are staged P2M_S at a time
// with their per-axis tables d'^k / k! (one row of 3 (p + 1) values per source, so that the
// threads of a warp, which differ in k, read different banks) and their four weights (dynamic
// shared memory, p2m_smem bytes).
template <class R>
struct __align__(4 * sizeof(R)) P2mW {
    R a, b, c, d;
};
#define P2M_T 192
#define P2M_S 96
#define P2M_R 3  // multi-indices per thread: nterms(12) = 455 <= 3 * 192
template <class R>
static size_t p2m_smem(int p)
{
    return sizeof(R) * ((size_t)3 * (p + 1) * P2M_S + 4 * P2M_S);
}
template <class R>
__global__ void __launch_bounds__(P2M_T) k_p2m(int nt, int p, const int* __restrict__ begin,
                                               const double* __restrict__ xc, const double4_32a* __restrict__ ep,
                                               const double4_32a* __restrict__ en, const double* __restrict__ xs,
                                               double eps, R* __restrict__ sig0, R* __restrict__ sigk,
                                               long long xstr, long long sstr)
{
    // right-hand side blockIdx.y: its density at xs + y xstr, its moments at sig + y sstr
    xs += blockIdx.y * xstr;
    sig0 += blockIdx.y * sstr;
    sigk += blockIdx.y * sstr;
    extern __shared__ __align__(32) unsigned char p2m_sm[];
    R* ex = (R*)p2m_sm;                   // [P2M_S][3][p + 1]: (source, axis, power)
    // [P2M_S] records (A dphi, A phi n_x, A phi n_y, A phi n_z): one broadcast load per source
    P2mW<R>* wt = (P2mW<R>*)(ex + 3 * (p + 1) * P2M_S);
    const int c = blockIdx.x;
    const int T = pb_nterms(p);
    R* Ssh = ex;                          // after the sources: S and G_x, G_y, G_z, [4][T]
    const int rs = 3 * (p + 1);  // row of one source
    auto EX = [&](int a, int k, int q) -> R& { return ex[q * rs + a * (p + 1) + k]; };
    const int b = begin[c], e = begin[c + 1];
    const double cx = xc[3 * c], cy = xc[3 * c + 1], cz = xc[3 * c + 2];
    int xi[P2M_R][3];
#pragma unroll
    for (int r = 0; r < P2M_R; ++r) {
        const int q = threadIdx.x + r * P2M_T;
        mi_unpack(c_mi[q < T ? q : 0], xi[r][0], xi[r][1], xi[r][2]);
    }
    R acc[P2M_R][4] = {};
    for (int s0 = b; s0 < e; s0 += P2M_S) {
        const int ns = min(P2M_S, e - s0);
        __syncthreads();
        if (threadIdx.x < ns) {
            const int j = s0 + threadIdx.x;
            const double4_32a P = ep[j], Nn = en[j];
            const R d[3] = {(R)(cx - P.x), (R)(cy - P.y), (R)(cz - P.z)};
            for (int a = 0; a < 3; ++a) {
                R v = 1;
                for (int k = 0; k <= p; ++k) {
                    EX(a, k, threadIdx.x) = v * inv_fact1<R>(k);
                    v *= d[a];
                }
            }
            const R wphi = (R)(P.w * xs[j]), wdphi = (R)(P.w * xs[nt + j]);
            wt[threadIdx.x] = {wdphi, wphi * (R)Nn.x, wphi * (R)Nn.y, wphi * (R)Nn.z};
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < P2M_R; ++r) {
            if (threadIdx.x + r * P2M_T >= T) continue;
            const R* e1 = &EX(0, xi[r][0], 0);
            const R* e2 = &EX(1, xi[r][1], 0);
            const R* e3 = &EX(2, xi[r][2], 0);
            R s = 0, g0 = 0, g1 = 0, g2 = 0;
            for (int q = 0; q < ns; ++q) {
                const R m = e1[q * rs] * e2[q * rs] * e3[q * rs];
                const P2mW<R> w = wt[q];
                s += w.a * m;
                g0 += w.b * m;
                g1 += w.c * m;
                g2 += w.d * m;
            }
            acc[r][0] += s;
            acc[r][1] += g0;
            acc[r][2] += g1;
            acc[r][3] += g2;
        }
    }
    __syncthreads();  // the source tables are done with: S and G reuse their space
#pragma unroll
    for (int r = 0; r < P2M_R; ++r) {
        const int q = threadIdx.x + r * P2M_T;
        if (q >= T) continue;
        Ssh[q] = acc[r][0];
        Ssh[T + q] = acc[r][1];
        Ssh[2 * T + q] = acc[r][2];
        Ssh[3 * T + q] = acc[r][3];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < P2M_R; ++r) {
        const int q = threadIdx.x + r * P2M_T;
        if (q >= T) continue;
        const int a1 = xi[r][0], a2 = xi[r][1], a3 = xi[r][2];
        R g = 0;
        if (a1) g += Ssh[T + pb_midx(a1 - 1, a2, a3)];
        if (a2) g += Ssh[2 * T + pb_midx(a1, a2 - 1, a3)];
        if (a3) g += Ssh[3 * T + pb_midx(a1, a2, a3 - 1)];
        sig0[(size_t)c * T + q] = Ssh[q] + g;
        sigk[(size_t)c * T + q] = -Ssh[q] - (R)eps * g;
    }
}

// ---------- step 3: MtM, children (order pc) into parent (order pp) ----------
// With t = x_child - x_parent, M_parent[a] = sum_{b <= a} C(a, b) t^(a - b) M_child[b]. In the
// stored form m~ = (-1)^|b| M / b! this is m~_parent[a] = sum_{b <= a} e[a - b] m~_child[b] with
// e[g] = (-t)^g / g!, a product of one factor per axis, so the sum over b <= a is three
// one-dimensional shifts: along x, then y, then z (at most p + 1 terms each instead of up to
// (a1 + 1)(a2 + 1)(a3 + 1)). One block per parent; thread q owns the multi-indices q, q + 256;
// children are taken one after the other in child order, so the result does not depend on
// scheduling. All intermediate arrays use the layout of degree <= pp.
#define M2M_T 256

template <class R>
__global__ void __launch_bounds__(M2M_T) k_m2m(int pp, int pc, const int* __restrict__ cbeg,
                                               const double* __restrict__ xp, const double* __restrict__ xch,
                                               const R* __restrict__ c0, const R* __restrict__ ck,
                                               R* __restrict__ s0, R* __restrict__ sk, long long cstr, long long pstr)
{
    c0 += blockIdx.y * cstr;
    ck += blockIdx.y * cstr;
    s0 += blockIdx.y * pstr;
    sk += blockIdx.y * pstr;
    __shared__ R e[3][PB_PMAX + 1];
    extern __shared__ __align__(128) unsigned char dsm[];
    const int Tp = pb_nterms(pp), Tc = pb_nterms(pc);
    R* A0 = (R*)dsm;  // [Tp] each
    R* Ak = A0 + Tp;
    R* B0 = Ak + Tp;
    R* Bk = B0 + Tp;
    const int c = blockIdx.x;
    const int cb = cbeg[c], nch = min(cbeg[c + 1] - cb, 8);
    int xi[2][3];
    bool own[2];
    R acc0[2] = {0, 0}, acck[2] = {0, 0};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int q = threadIdx.x + r * M2M_T;
        own[r] = q < Tp;
        mi_unpack(c_mi[own[r] ? q : 0], xi[r][0], xi[r][1], xi[r][2]);
    }
    for (int ch = 0; ch < nch; ++ch) {
        __syncthreads();  // the previous child's last pass has read A
        if (threadIdx.x < 3) {
            const int d = threadIdx.x;
            const R t = (R)(xp[3 * c + d] - xch[3 * (cb + ch) + d]);  // -(x_child - x_parent)
            R v = 1;
            for (int k = 0; k <= pp; ++k) {
                e[d][k] = v * inv_fact1<R>(k);
                v *= t;
            }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int q = threadIdx.x + r * M2M_T;
            if (!own[r]) continue;
            // child moments exist up to degree pc (the layouts of degree <= pc and <= pp agree on
            // their common prefix)
            A0[q] = q < Tc ? c0[(size_t)(cb + ch) * Tc + q] : R(0);
            Ak[q] = q < Tc ? ck[(size_t)(cb + ch) * Tc + q] : R(0);
        }
        __syncthreads();
        // x: B[x1, x2, x3] = sum_{b1 <= x1} e_x[x1 - b1] A[b1, x2, x3]
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!own[r]) continue;
            const int x1 = xi[r][0], x2 = xi[r][1], x3 = xi[r][2];
            R v0 = 0, vk = 0;
            for (int b1 = 0; b1 <= x1; ++b1) {
                const int q = pb_midx(b1, x2, x3);
                const R w = e[0][x1 - b1];
                v0 += w * A0[q];
                vk += w * Ak[q];
            }
            B0[threadIdx.x + r * M2M_T] = v0;
            Bk[threadIdx.x + r * M2M_T] = vk;
        }
        __syncthreads();
        // y: A[x1, x2, x3] = sum_{b2 <= x2} e_y[x2 - b2] B[x1, b2, x3]
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!own[r]) continue;
            const int x1 = xi[r][0], x2 = xi[r][1], x3 = xi[r][2];
            R v0 = 0, vk = 0;
            for (int b2 = 0; b2 <= x2; ++b2) {
                const int q = pb_midx(x1, b2, x3);
                const R w = e[1][x2 - b2];
                v0 += w * B0[q];
                vk += w * Bk[q];
            }
            A0[threadIdx.x + r * M2M_T] = v0;
            Ak[threadIdx.x + r * M2M_T] = vk;
        }
        __syncthreads();
        // z: the parent's moment gains sum_{b3 <= x3} e_z[x3 - b3] A[x1, x2, b3]
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!own[r]) continue;
            const int x1 = xi[r][0], x2 = xi[r][1], x3 = xi[r][2];
            R v0 = 0, vk = 0;
            for (int b3 = 0; b3 <= x3; ++b3) {
                const int q = pb_midx(x1, x2, b3);
                const R w = e[2][x3 - b3];
                v0 += w * A0[q];
                vk += w * Ak[q];
            }
            acc0[r] += v0;
            acck[r] += vk;
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int q = threadIdx.x + r * M2M_T;
        if (!own[r]) continue;
        s0[(size_t)c * Tp + q] = acc0[r];
        sk[(size_t)c * Tp + q] = acck[r];
    }
}

// ---------- step 4: MtL over the interaction lists of one level ----------
template <class R>
__global__ void __launch_bounds__(FAR_T) k_m2l(int p, double kappa, const int* __restrict__ ioff,
                                               const int* __restrict__ iidx, const double* __restrict__ xc,
                                               const R* __restrict__ s0, const R* __restrict__ sk,
                                               R* __restrict__ l0, R* __restrict__ lk, long long str)
{
    s0 += blockIdx.y * str;
    sk += blockIdx.y * str;
    l0 += blockIdx.y * str;
    lk += blockIdx.y * str;
    __shared__ R F0[NT_MAX], Fk[NT_MAX], Pk[NT_MAX];
    __shared__ R M0[NT_MAX], Mk[NT_MAX];
    const int c = blockIdx.x;
    const int T = pb_nterms(p);
    R L0[4] = {0, 0, 0, 0}, Lk[4] = {0, 0, 0, 0};
    const double i4pi = 0.07957747154594767;
    for (int t = ioff[c]; t < ioff[c + 1]; ++t) {
        const int c2 = iidx[t];
        const R dx = (R)(xc[3 * c] - xc[3 * c2]), dy = (R)(xc[3 * c + 1] - xc[3 * c2 + 1]),
                dz = (R)(xc[3 * c + 2] - xc[3 * c2 + 2]);
        const R d2 = dx * dx + dy * dy + dz * dz;
        const R kap = (R)kappa;
        __syncthreads();
        // source moments (stored already scaled by (-1)^|b| / b!)
        for (int b = threadIdx.x; b < T; b += FAR_T) {
            M0[b] = s0[(size_t)c2 * T + b];
            Mk[b] = sk[(size_t)c2 * T + b];
        }
        if (threadIdx.x == 0) {
            R r = sqrt(d2);
            R ex = exp(-kap * r);
            F0[0] = (R)i4pi / r;
            Fk[0] = (R)i4pi * ex / r;
            Pk[0] = (R)i4pi * ex;
        }
        __syncthreads();
        // Taylor coefficients degree by degree
        for (int n = 1; n <= p; ++n) {
            const int lo = pb_nterms(n - 1), hi = pb_nterms(n);
            for (int k = lo + threadIdx.x; k < hi; k += FAR_T) {
                int k1, k2, k3;
                mi_unpack(c_mi[k], k1, k2, k3);
                R d[3] = {dx, dy, dz};
                int kk[3] = {k1, k2, k3};
                R a0 = 0, a1 = 0, ak0 = 0, ak1 = 0, ap0 = 0, ap1 = 0;
                for (int i = 0; i < 3; ++i) {
                    if (kk[i] >= 1) {
                        int q = pb_midx(k1 - (i == 0), k2 - (i == 1), k3 - (i == 2));
                        a0 += d[i] * F0[q];
                        ak0 += d[i] * Fk[q];
                        ap0 += d[i] * Pk[q];
                    }
                    if (kk[i] >= 2) {
                        int q = pb_midx(k1 - 2 * (i == 0), k2 - 2 * (i == 1), k3 - 2 * (i == 2));
                        a1 += F0[q];
                        ak1 += Fk[q];
                        ap1 += Pk[q];
                    }
                }
                R nn = (R)n;
                F0[k] = (-(R)(2 * n - 1) * a0 - (nn - 1) * a1) / (d2 * nn);
                Fk[k] = (-(R)(2 * n - 1) * ak0 - (nn - 1) * ak1 - kap * ap0 - kap * ap1) / (d2 * nn);
                Pk[k] = -kap * (ak0 + ak1) / nn;
            }
            __syncthreads();
        }
        // raw derivatives D^k = k! F_k
        for (int k = threadIdx.x; k < T; k += FAR_T) {
            int k1, k2, k3;
            mi_unpack(c_mi[k], k1, k2, k3);
            R f = (R)(c_fact[k1] * c_fact[k2] * c_fact[k3]);
            F0[k] *= f;
            Fk[k] *= f;
        }
        __syncthreads();
        for (int r = 0; r < 4; ++r) {
            int al = threadIdx.x + r * FAR_T;
            if (al >= T) break;
            int a1, a2, a3;
            mi_unpack(c_mi[al], a1, a2, a3);
            int nb = pb_nterms(p - (a1 + a2 + a3));
            R v0 = 0, vk = 0;
            for (int b = 0; b < nb; ++b) {
                int b1, b2, b3;
                mi_unpack(c_mi[b], b1, b2, b3);
                int g = pb_midx(a1 + b1, a2 + b2, a3 + b3);
                v0 += F0[g] * M0[b];
                vk += Fk[g] * Mk[b];
            }
            L0[r] += v0;
            Lk[r] += vk;
        }
    }
    for (int r = 0; r < 4; ++r) {
        int al = threadIdx.x + r * FAR_T;
        if (al >= T) break;
        int a1, a2, a3;
        mi_unpack(c_mi[al], a1, a2, a3);
        R f = (R)(1.0 / (c_fact[a1] * c_fact[a2] * c_fact[a3]));
        l0[(size_t)c * T + al] = L0[r] * f;
        lk[(size_t)c * T + al] = Lk[r] * f;
    }
}

// ---------- step 4, precomputed form ----------
// Setup: the kernel derivatives D^g G0 and D^g Gk of every interaction slot depend only on
// the geometry, so they are evaluated once (FP64 recurrence, stored in the working
// precision) in the interleaved slot layout the contraction reads.
// One warp per slot (target cluster, source cluster): the lanes share the terms of each order
// of the recurrence, so orders are separated by warp barriers only and eight slots of a block
// proceed independently. Per-warp scratch: three FP64 term arrays in dynamic shared memory.
template <class R>
__global__ void __launch_bounds__(256) k_m2l_setup(int nslots, int p, double kappa, const int* __restrict__ stgt,
                                                   const int* __restrict__ ssrc, const double* __restrict__ xc,
                                                   const int* __restrict__ mirror, R* __restrict__ D0,
                                                   R* __restrict__ Dk)
{
    extern __shared__ double m2ls[];
    const int T = pb_nterms(p);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * 8 + warp;
    if (s >= nslots) return;
    double* F0 = m2ls + (size_t)warp * 3 * T;
    double* Fk = F0 + T;
    double* Pk = Fk + T;
    const double i4pi = 0.07957747154594767;
    const int c = stgt[s], c2 = ssrc[s];
    const size_t base = ((size_t)(s >> 5) * T) * 32 + (s & 31);
    if (c2 < 0) {
        for (int k = lane; k < T; k += 32) {
            D0[base + (size_t)k * 32] = R(0);
            Dk[base + (size_t)k * 32] = R(0);
        }
        return;
    }
    // a pair and its reverse are computed once, by the slot with the smaller index (only when
    // the two slots name each other); the reverse differs by (-1)^|g|
    int ms = mirror[s];
    if (ms >= 0 && mirror[ms] != s) ms = -1;
    if (ms >= 0 && ms < s) return;
    const size_t mbase = ms >= 0 ? ((size_t)(ms >> 5) * T) * 32 + (ms & 31) : 0;
    const double d[3] = {xc[3 * c] - xc[3 * c2], xc[3 * c + 1] - xc[3 * c2 + 1], xc[3 * c + 2] - xc[3 * c2 + 2]};
    const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (lane == 0) {
        double r = sqrt(d2), ex = exp(-kappa * r);
        F0[0] = i4pi / r;
        Fk[0] = i4pi * ex / r;
        Pk[0] = i4pi * ex;
    }
    __syncwarp();
    for (int n = 1; n <= p; ++n) {
        for (int k = pb_nterms(n - 1) + lane; k < pb_nterms(n); k += 32) {
            int kk[3];
            mi_unpack(c_mi[k], kk[0], kk[1], kk[2]);
            double a0 = 0, a1 = 0, ak0 = 0, ak1 = 0, ap0 = 0, ap1 = 0;
            for (int i = 0; i < 3; ++i) {
                if (kk[i] >= 1) {
                    int q = pb_midx(kk[0] - (i == 0), kk[1] - (i == 1), kk[2] - (i == 2));
                    a0 += d[i] * F0[q];
                    ak0 += d[i] * Fk[q];
                    ap0 += d[i] * Pk[q];
                }
                if (kk[i] >= 2) {
                    int q = pb_midx(kk[0] - 2 * (i == 0), kk[1] - 2 * (i == 1), kk[2] - 2 * (i == 2));
                    a1 += F0[q];
                    ak1 += Fk[q];
                    ap1 += Pk[q];
                }
            }
            F0[k] = (-(2.0 * n - 1.0) * a0 - (n - 1.0) * a1) / (d2 * n);
            Fk[k] = (-(2.0 * n - 1.0) * ak0 - (n - 1.0) * ak1 - kappa * ap0 - kappa * ap1) / (d2 * n);
            Pk[k] = -kappa * (ak0 + ak1) / n;
        }
        __syncwarp();
    }
    for (int k = lane; k < T; k += 32) {
        int k1, k2, k3;
        mi_unpack(c_mi[k], k1, k2, k3);
        double f = c_fact[k1] * c_fact[k2] * c_fact[k3];
        D0[base + (size_t)k * 32] = (R)(F0[k] * f);
        Dk[base + (size_t)k * 32] = (R)(Fk[k] * f);
        if (ms >= 0) {
            const double sg = (k1 + k2 + k3) & 1 ? -f : f;
            D0[mbase + (size_t)k * 32] = (R)(F0[k] * sg);
            Dk[mbase + (size_t)k * 32] = (R)(Fk[k] * sg);
        }
    }
}

// Contraction, precomputed form: one warp per target cluster, one lane per interaction slot,
// the order-P local coefficients of the lane in registers (straight-line bodies of
// m2l_unrolled.cuh). Per chunk of 32 slots the derivative block D and the gathered scaled
// moments M (both T x 32, contiguous) are read from shared memory; the per-lane partial sums
// are added across the warp at the end.
//
// Scaled moments gathered into the chunk layout: M[((s / 32) * T + b) * 32 + s % 32] =
// (-1)^|b| sigma^b(src(s)) / b!, zero for padding slots.
// The same recurrence in float-float on the FP32 pipe, for the FP32 tables of mixed
// precision: ~1e-13 relative before the final rounding to FP32, at a fraction of the FP64
// pipe's time. The starting values come from FP64 once per slot.
__device__ __forceinline__ ff ld_ffs(const float2* p)
{
    const float2 v = *p;
    return {v.x, v.y};
}

// Mirror slots: the interaction lists are symmetric (c' in I(c) exactly when c in I(c')), and the
// tensors of the two directions differ only by (-1)^|g| (G is even in x_c - x_c'). mirror[s] is
// the slot of the reversed pair, or -1 for padding (or if none is found).
__global__ void k_m2l_mirror(int nslots, const int* __restrict__ soff, const int* __restrict__ stgt,
                             const int* __restrict__ ssrc, int* __restrict__ mirror)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    const int q = ssrc[s], t = stgt[s];
    int m = -1;
    if (q >= 0)
        for (int u = soff[q]; u < soff[q + 1]; ++u)
            if (ssrc[u] == t) {
                m = u;
                break;
            }
    mirror[s] = m;
}

__global__ void __launch_bounds__(256) k_m2l_setup_ff(int nslots, int p, double kappa, const int* __restrict__ stgt,
                                                      const int* __restrict__ ssrc, const double* __restrict__ xc,
                                                      const int* __restrict__ mirror, float* __restrict__ D0,
                                                      float* __restrict__ Dk)
{
    extern __shared__ float2 m2lf[];
    const int T = pb_nterms(p);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * 8 + warp;
    if (s >= nslots) return;
    float2* F0 = m2lf + (size_t)warp * 3 * T;
    float2* Fk = F0 + T;
    float2* Pk = Fk + T;
    const int c = stgt[s], c2 = ssrc[s];
    const size_t base = ((size_t)(s >> 5) * T) * 32 + (s & 31);
    if (c2 < 0) {
        for (int k = lane; k < T; k += 32) {
            D0[base + (size_t)k * 32] = 0.f;
            Dk[base + (size_t)k * 32] = 0.f;
        }
        return;
    }
    // a pair and its reverse are computed once, by the slot with the smaller index (only when
    // the two slots name each other)
    int ms = mirror[s];
    if (ms >= 0 && mirror[ms] != s) ms = -1;
    if (ms >= 0 && ms < s) return;
    const size_t mbase = ms >= 0 ? ((size_t)(ms >> 5) * T) * 32 + (ms & 31) : 0;
    const ff d[3] = {ff_from(xc[3 * c] - xc[3 * c2]), ff_from(xc[3 * c + 1] - xc[3 * c2 + 1]),
                     ff_from(xc[3 * c + 2] - xc[3 * c2 + 2])};
    const ff d2 = ff_add(ff_add(ff_sqr(d[0]), ff_sqr(d[1])), ff_sqr(d[2]));
    const ff kap = ff_from(kappa);
    if (lane == 0) {
        const double dd[3] = {xc[3 * c] - xc[3 * c2], xc[3 * c + 1] - xc[3 * c2 + 1], xc[3 * c + 2] - xc[3 * c2 + 2]};
        const double r = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]), ex = exp(-kappa * r);
        const double i4pi = 0.07957747154594767;
        const ff a = ff_from(i4pi / r), b = ff_from(i4pi * ex / r), e = ff_from(i4pi * ex);
        F0[0] = make_float2(a.h, a.l);
        Fk[0] = make_float2(b.h, b.l);
        Pk[0] = make_float2(e.h, e.l);
    }
    // 1 / d2 to float-float accuracy: FP32 estimate and one Newton step
    const float y0 = 1.0f / d2.h;
    const ff id2 = ff_add_f(ff_mul_f(ff_neg(ff_add_f(ff_mul_f(d2, y0), -1.0f)), y0), y0);
    __syncwarp();
    for (int n = 1; n <= p; ++n) {
        const float fn = (float)n, in = 1.0f / fn;
        const ff inv_n = ff_add_f(ff_mul_f(ff_neg(ff{fn * in - 1.0f, fmaf(fn, in, -(fn * in))}), in), in);
        const ff scale = ff_mul(id2, inv_n);
        for (int k = pb_nterms(n - 1) + lane; k < pb_nterms(n); k += 32) {
            int kk[3];
            mi_unpack(c_mi[k], kk[0], kk[1], kk[2]);
            ff a0 = {0.f, 0.f}, a1 = a0, ak0 = a0, ak1 = a0, ap0 = a0, ap1 = a0;
            for (int i = 0; i < 3; ++i) {
                if (kk[i] >= 1) {
                    const int q = pb_midx(kk[0] - (i == 0), kk[1] - (i == 1), kk[2] - (i == 2));
                    a0 = ff_add(a0, ff_mul(d[i], ld_ffs(F0 + q)));
                    ak0 = ff_add(ak0, ff_mul(d[i], ld_ffs(Fk + q)));
                    ap0 = ff_add(ap0, ff_mul(d[i], ld_ffs(Pk + q)));
                }
                if (kk[i] >= 2) {
                    const int q = pb_midx(kk[0] - 2 * (i == 0), kk[1] - 2 * (i == 1), kk[2] - 2 * (i == 2));
                    a1 = ff_add(a1, ld_ffs(F0 + q));
                    ak1 = ff_add(ak1, ld_ffs(Fk + q));
                    ap1 = ff_add(ap1, ld_ffs(Pk + q));
                }
            }
            const float c1 = -(2.0f * fn - 1.0f), c2 = -(fn - 1.0f);
            const ff f0 = ff_mul(ff_add(ff_mul_f(a0, c1), ff_mul_f(a1, c2)), scale);
            const ff fk = ff_mul(ff_sub(ff_add(ff_mul_f(ak0, c1), ff_mul_f(ak1, c2)), ff_mul(kap, ff_add(ap0, ap1))),
                                 scale);
            const ff pk = ff_neg(ff_mul(ff_mul(kap, ff_add(ak0, ak1)), inv_n));
            F0[k] = make_float2(f0.h, f0.l);
            Fk[k] = make_float2(fk.h, fk.l);
            Pk[k] = make_float2(pk.h, pk.l);
        }
        __syncwarp();
    }
    for (int k = lane; k < T; k += 32) {
        int k1, k2, k3;
        mi_unpack(c_mi[k], k1, k2, k3);
        const float f = (float)(c_fact[k1] * c_fact[k2] * c_fact[k3]);  // at most 12!, exact in FP32 up to 8!
        const ff a = ff_mul_f(ld_ffs(F0 + k), f), b = ff_mul_f(ld_ffs(Fk + k), f);
        D0[base + (size_t)k * 32] = a.h + a.l;
        Dk[base + (size_t)k * 32] = b.h + b.l;
        if (ms >= 0) {  // the reversed pair: (-1)^|g|
            const float sg = (k1 + k2 + k3) & 1 ? -1.f : 1.f;
            D0[mbase + (size_t)k * 32] = sg * (a.h + a.l);
            Dk[mbase + (size_t)k * 32] = sg * (b.h + b.l);
        }
    }
}

template <class R>
__global__ void k_m2l_gather(int T, const int* __restrict__ ssrc, const R* __restrict__ s0, const R* __restrict__ sk,
                             R* __restrict__ M0, R* __restrict__ Mk, long long sstr, long long mstr)
{
    s0 += blockIdx.y * sstr;
    sk += blockIdx.y * sstr;
    M0 += blockIdx.y * mstr;
    Mk += blockIdx.y * mstr;
    // one block per chunk of 32 slots; thread (b, lane) pairs walk the T x 32 block (the
    // moments are stored already scaled by (-1)^|b| / b!)
    const long long chunk = blockIdx.x;
    const size_t base = (size_t)chunk * T * 32;
    const int src = ssrc[chunk * 32 + (threadIdx.x & 31)];
    for (int t = threadIdx.x; t < T * 32; t += blockDim.x) {
        const int b = t >> 5;
        M0[base + t] = src >= 0 ? s0[(size_t)src * T + b] : R(0);
        Mk[base + t] = src >= 0 ? sk[(size_t)src * T + b] : R(0);
    }
}

// warp-level sum of the lanes' coefficients, scaled by 1/a!, written to out[c * T + a]
template <int P, class R>
__device__ __forceinline__ void m2l_flush(R* L, R* scratch, R* __restrict__ out, int c, int lane)
{
    constexpr int T = (P + 1) * (P + 2) * (P + 3) / 6;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < T; ++i) scratch[i * 33 + lane] = L[i];
    __syncwarp();
    for (int i = lane; i < T; i += 32) {
        R s = 0;
        for (int l = 0; l < 32; ++l) s += scratch[i * 33 + l];
        int a1, a2, a3;
        mi_unpack(c_mi[i], a1, a2, a3);
        out[(size_t)c * T + i] = s * (sizeof(R) == 4 ? (R)c_ifact[i] : (R)c_ifact64[i]);
    }
    __syncwarp();
}

// ---- TMA bulk copies and mbarriers (FP32 path) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* bar, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// 4-byte asynchronous global -> shared copy (zero-filled when !valid: no bytes are read)
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
// this thread's asynchronous copies have landed
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
// bounded wait: gives up after PB_WAIT_LIMIT polls (each poll may itself block briefly)
#define PB_WAIT_LIMIT (1u << 24)
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned phase)
{
    for (unsigned it = 0; it < PB_WAIT_LIMIT; ++it)
        if (mbar_try(bar, phase)) return true;
    return false;
}

// FP32: one block of two warps per chunk of 32 slots and per kernel (G0 for blockIdx.z = 0, Gk
// for 1). Under mixed precision the slots of a level are packed without padding (the
// interaction lists of consecutive targets follow one another; only the level's end is padded
// to 32), so a chunk's lanes may belong to several targets. The chunk's derivative block (T x 32
// floats, 21 KB at p = 8) arrives by TMA bulk copy (mbarrier completion, every wait bounded)
// while the warps load the 32 source clusters' moments straight from the level's moment array
// (L2-resident, stored already scaled by (-1)^|b| / b!; the source indices come from one
// coalesced load and a shuffle per row), one coalesced row per source, into shared memory rows
// of 33 words (conflict-free in both directions). Warp w accumulates its half of the local
// coefficients (M2LWarp<P, w>: equal FMA counts, moments held in registers a block at a time).
// After the chunk, the lanes' coefficients are summed per run of lanes with the same target and
// scaled by 1/a!: a target whose list lies inside the chunk is written directly; the run that
// opens the chunk and the run that closes it, when their target's list crosses the chunk's
// edge, go to the staging rows part[2 k] and part[2 k + 1], which k_m2l_runs adds up per
// target in chunk order. No atomics: the result does not depend on scheduling.
template <int P>
__global__ void __launch_bounds__(64, 5) k_m2l_seg(int nch, const int* __restrict__ soff,
                                                   const int* __restrict__ ssrc, const int* __restrict__ stgt,
                                                   const float* __restrict__ D0, const float* __restrict__ Dk,
                                                   const float* __restrict__ s0, const float* __restrict__ sk,
                                                   float* __restrict__ l0, float* __restrict__ lk,
                                                   float* __restrict__ p0, float* __restrict__ pk,
                                                   int* __restrict__ err, long long sstr, int nr)
{
    // block x = chunk * nr + right-hand side r: the nr blocks of a chunk are adjacent in launch
    // order, so its derivative block comes from HBM once and from L2 for the other vectors
    const int kern = blockIdx.z;
    const int r = (int)(blockIdx.x % (unsigned)nr);
    const int k = (int)(blockIdx.x / (unsigned)nr);
    const float* D = kern ? Dk : D0;
    constexpr int T = (P + 1) * (P + 2) * (P + 3) / 6;
    const float* sig = (kern ? sk : s0) + r * sstr;
    float* out = (kern ? lk : l0) + r * sstr;
    float* part = (kern ? pk : p0) + (size_t)r * nch * 2 * T;
    constexpr unsigned CH = T * 32 * sizeof(float);  // bytes of one derivative block (multiple of 16)
    constexpr int NL = M2LWarp<P, 0>::n > M2LWarp<P, 1>::n ? M2LWarp<P, 0>::n : M2LWarp<P, 1>::n;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) unsigned long long bar;
    // the chunk's runs of slots with the same target (targets are sorted, so each is one run):
    // first lane, target (-1: padding) and whether it began in an earlier chunk (1) or goes on
    // in a later one (2)
    __shared__ int rs[33], rt[32], rf[32];
    __shared__ int nrun;
    float* Ds = (float*)dsm;    // [T * 32]
    float* Ms = Ds + T * 32;    // [T * 33]; with Ds, the reduction scratch [T * 33]
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    if (k >= nch) return;
    const int jl = ssrc[(size_t)k * 32 + lane];
    if (wi == 0) {
        const int t = jl >= 0 ? stgt[(size_t)k * 32 + lane] : -1;
        const int tp = __shfl_up_sync(0xffffffffu, t, 1);
        const bool st = lane == 0 || tp != t;
        const unsigned m = __ballot_sync(0xffffffffu, st);
        if (st) {
            const int q = __popc(m & ((1u << lane) - 1));
            const unsigned later = lane == 31 ? 0u : (m >> (lane + 1)) << (lane + 1);
            const int end = later ? __ffs(later) - 1 : 32;
            const long long s0k = 32LL * k;  // first slot of the chunk
            int f = 0;
            if (t >= 0) {
                if (lane == 0 && soff[t] < s0k) f |= 1;
                if (end == 32 && soff[t + 1] > s0k + 32) f |= 2;
            }
            rs[q] = lane;
            rt[q] = t;
            rf[q] = f;
        }
        if (lane == 0) {
            nrun = __popc(m);
            rs[__popc(m)] = 32;
        }
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();  // the barrier is initialised before any thread waits on it
    if (threadIdx.x == 0) {
        mbar_expect(&bar, CH);
        bulk_g2s(Ds, D + (size_t)k * T * 32, CH, &bar);
    }
    // the moments of the chunk's sources (padding slots: zero), two rows at a time, by
    // asynchronous copies that overlap the derivative block's copy
#pragma unroll 4
    for (int s = wi; s < 32; s += 2) {
        const int j = __shfl_sync(0xffffffffu, jl, s);
        const float* row = sig + (size_t)(j < 0 ? 0 : j) * T;
        for (int b = lane; b < T; b += 32) cp_async4(Ms + b * 33 + s, row + b, j >= 0);
    }
    cp_async_wait_all();
    // the block agrees on the outcome, so that no thread leaves while another waits
    if (!__syncthreads_and(mbar_wait(&bar, 0u))) {
        // the copy never completed: record it, give it a bounded time to land, and stop
        if (threadIdx.x == 0) atomicExch(err, 1);
        mbar_wait(&bar, 0u);
        return;
    }
    float L[NL];
#pragma unroll
    for (int i = 0; i < NL; ++i) L[i] = 0.f;
    if (wi == 0) M2LWarp<P, 0>::run(Ds + lane, Ms + lane, L);
    else M2LWarp<P, 1>::run(Ds + lane, Ms + lane, L);
    __syncthreads();
    // per-lane coefficients into disjoint rows of the scratch, then sums over runs of lanes
    // with the same target
    float* scratch = Ds;
    if (wi == 0) {
#pragma unroll
        for (int i = 0; i < M2LWarp<P, 0>::n; ++i) scratch[M2LWarp<P, 0>::alpha(i) * 33 + lane] = L[i];
    } else {
#pragma unroll
        for (int i = 0; i < M2LWarp<P, 1>::n; ++i) scratch[M2LWarp<P, 1>::alpha(i) * 33 + lane] = L[i];
    }
    __syncthreads();
    // per coefficient, the sum of each run in lane order: a run inside the chunk is the
    // target's coefficient; one that crosses an edge is staged for k_m2l_runs
    const int nrn = nrun;
    for (int i = threadIdx.x; i < T; i += 64) {
        const float sc = c_ifact[i];
        const float* row = scratch + i * 33;
        for (int q = 0; q < nrn; ++q) {
            const int l1 = rs[q + 1];
            int l = rs[q];
            float acc = 0.f;
            for (; l + 4 <= l1; l += 4) acc = (((acc + row[l]) + row[l + 1]) + row[l + 2]) + row[l + 3];
            for (; l < l1; ++l) acc += row[l];
            const int t = rt[q];
            if (t >= 0) {
                const int f = rf[q];
                if (f & 1) part[(2LL * k) * T + i] = acc * sc;
                if (f & 2) part[(2LL * k + 1) * T + i] = acc * sc;
                if (!f) out[(size_t)t * T + i] = acc * sc;
            }
        }
    }
}

// the local coefficients of the targets whose lists cross a chunk edge (the closing run of the
// first chunk, the opening run of every later one, in chunk order), and zeros for the targets
// without an interaction
__global__ void k_m2l_runs(int ncl, int T, int nch, const int* __restrict__ soff, const float* __restrict__ p0,
                           const float* __restrict__ pk, float* __restrict__ l0, float* __restrict__ lk,
                           long long sstr)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)ncl * T) return;
    const int c = (int)(e / T), i = (int)(e % T);
    const float* part = (blockIdx.z ? pk : p0) + (size_t)blockIdx.y * nch * 2 * T;
    float* out = (blockIdx.z ? lk : l0) + blockIdx.y * sstr;
    const int b = soff[c], en = soff[c + 1];
    if (b == en) {
        out[e] = 0.f;
        return;
    }
    const int k0 = b >> 5, k1 = (en - 1) >> 5;
    if (k0 == k1) return;  // written by the chunk kernel
    float s = part[(2LL * k0 + 1) * T + i];
    for (int k = k0 + 1; k <= k1; ++k) s += part[(2LL * k) * T + i];
    out[e] = s;
}

// FP64 (and fallback): D read from global memory, the moment chunk copied to shared memory.
template <int P, class R>
__global__ void __launch_bounds__(32) k_m2l_chunks(int ncl, const int* __restrict__ soff, const R* __restrict__ D0,
                                                   const R* __restrict__ Dk, const R* __restrict__ M0,
                                                   const R* __restrict__ Mk, R* __restrict__ l0, R* __restrict__ lk,
                                                   long long mstr, long long lstr)
{
    M0 += blockIdx.y * mstr;
    Mk += blockIdx.y * mstr;
    l0 += blockIdx.y * lstr;
    lk += blockIdx.y * lstr;
    constexpr int T = (P + 1) * (P + 2) * (P + 3) / 6;
    extern __shared__ __align__(128) unsigned char dsm[];
    R* Ms = (R*)dsm;  // [T * 33] (also the reduction scratch)
    const int lane = threadIdx.x;
    const int c = blockIdx.x;
    if (c >= ncl) return;
    const int sb = soff[c], se = soff[c + 1];
#pragma unroll 1
    for (int kern = 0; kern < 2; ++kern) {
        const R* D = kern ? Dk : D0;
        const R* M = kern ? Mk : M0;
        R* out = kern ? lk : l0;
        R L[T];
#pragma unroll
        for (int i = 0; i < T; ++i) L[i] = R(0);
#pragma unroll 1
        for (int s = sb; s < se; s += 32) {
            const R* Mc = M + (size_t)(s >> 5) * T * 32;
            __syncwarp();
            for (int t = lane; t < T * 32; t += 32) Ms[t] = Mc[t];
            __syncwarp();
            M2LBody<P, 0>::run(D + (size_t)(s >> 5) * T * 32 + lane, Ms + lane, L);
        }
        m2l_flush<P, R>(L, Ms, out, c, lane);
    }
}

// ---------- step 5: LtL, parent (order pp) into child (order pc) ----------
// With t = x_child - x_parent, L_child[b] += sum_g C(b + g, b) t^g L_parent[b + g]. With the
// scaled coefficients L^[a] = a! L[a] the weights become t^g / g!, one factor per axis, so the
// sum is three one-dimensional shifts (x, then y, then z), each over the indices above b on
// its axis. One block per child cluster; intermediate arrays in the layout of degree <= pp.
template <class R>
__global__ void __launch_bounds__(FAR_T) k_l2l(int pp, int pc, const int* __restrict__ parent,
                                               const double* __restrict__ xp, const double* __restrict__ xch,
                                               const R* __restrict__ lp0, const R* __restrict__ lpk,
                                               R* __restrict__ lc0, R* __restrict__ lck, long long pstr, long long cstr)
{
    lp0 += blockIdx.y * pstr;
    lpk += blockIdx.y * pstr;
    lc0 += blockIdx.y * cstr;
    lck += blockIdx.y * cstr;
    __shared__ R e[3][PB_PMAX + 1];
    __shared__ R A0[NT_MAX], Ak[NT_MAX], B0[NT_MAX], Bk[NT_MAX];
    const int c = blockIdx.x;
    const int P = parent[c];
    const int Tp = pb_nterms(pp), Tc = pb_nterms(pc);
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        const R t = (R)(xch[3 * c + d] - xp[3 * P + d]);
        R v = 1;
        for (int k = 0; k <= pp; ++k) {
            e[d][k] = v * inv_fact1<R>(k);
            v *= t;
        }
    }
    for (int q = threadIdx.x; q < Tp; q += FAR_T) {
        int a1, a2, a3;
        mi_unpack(c_mi[q], a1, a2, a3);
        const R f = (R)(c_fact[a1] * c_fact[a2] * c_fact[a3]);
        A0[q] = lp0[(size_t)P * Tp + q] * f;
        Ak[q] = lpk[(size_t)P * Tp + q] * f;
    }
    __syncthreads();
    // x: B[b1, x2, x3] = sum_{a1 >= b1, a1 + x2 + x3 <= pp} e_x[a1 - b1] A[a1, x2, x3]
    for (int q = threadIdx.x; q < Tp; q += FAR_T) {
        int x1, x2, x3;
        mi_unpack(c_mi[q], x1, x2, x3);
        R v0 = 0, vk = 0;
        for (int a1 = x1; a1 + x2 + x3 <= pp; ++a1) {
            const int s = pb_midx(a1, x2, x3);
            const R w = e[0][a1 - x1];
            v0 += w * A0[s];
            vk += w * Ak[s];
        }
        B0[q] = v0;
        Bk[q] = vk;
    }
    __syncthreads();
    // y: A[x1, b2, x3] = sum_{a2 >= b2} e_y[a2 - b2] B[x1, a2, x3]
    for (int q = threadIdx.x; q < Tp; q += FAR_T) {
        int x1, x2, x3;
        mi_unpack(c_mi[q], x1, x2, x3);
        R v0 = 0, vk = 0;
        for (int a2 = x2; x1 + a2 + x3 <= pp; ++a2) {
            const int s = pb_midx(x1, a2, x3);
            const R w = e[1][a2 - x2];
            v0 += w * B0[s];
            vk += w * Bk[s];
        }
        A0[q] = v0;
        Ak[q] = vk;
    }
    __syncthreads();
    // z, then unscale by 1/b! into the child's coefficients (degree <= pc)
    for (int q = threadIdx.x; q < Tc; q += FAR_T) {
        int x1, x2, x3;
        mi_unpack(c_mi[q], x1, x2, x3);
        R v0 = 0, vk = 0;
        for (int a3 = x3; x1 + x2 + a3 <= pp; ++a3) {
            const int s = pb_midx(x1, x2, a3);
            const R w = e[2][a3 - x3];
            v0 += w * A0[s];
            vk += w * Ak[s];
        }
        const R f = sizeof(R) == 4 ? (R)c_ifact[q] : (R)c_ifact64[q];
        lc0[(size_t)c * Tc + q] += v0 * f;
        lck[(size_t)c * Tc + q] += vk * f;
    }
}

// ---------- step 6: LtP ----------
// With the scaled coefficients L^[a] = a! L[a] and e[a] = d^a / a! (d = y - x_c), the local
// expansion is sum_a L^[a] e[a] and its normal derivative sum_b e[b] sum_i n_i L^[b + e_i]. Per
// cluster the three shifted arrays G_i[b] = L^[b + e_i] (potential combination of the normal
// derivative) are formed once; each thread then evaluates one target with per-axis tables
// (dynamic shared memory, l2p_smem bytes).
template <class R>
static size_t l2p_smem(int p)
{
    return sizeof(R) * (2 * (size_t)pb_nterms(p) + 3 * (size_t)pb_nterms(p - 1) + 3 * (size_t)(p + 1) * FAR_T);
}
template <class R>
__global__ void __launch_bounds__(FAR_T) k_l2p(int nt, int p, double eps, const int* __restrict__ begin,
                                               const double* __restrict__ xc, const double4_32a* __restrict__ ep,
                                               const double4_32a* __restrict__ en, const R* __restrict__ l0,
                                               const R* __restrict__ lk, double* __restrict__ ys, long long lstr,
                                               long long ystr)
{
    l0 += blockIdx.y * lstr;
    lk += blockIdx.y * lstr;
    ys += blockIdx.y * ystr;
    extern __shared__ __align__(16) unsigned char l2p_sm[];
    const int c = blockIdx.x;
    const int T = pb_nterms(p), Tm = pb_nterms(p - 1);
    R* A1 = (R*)l2p_sm;  // [T]
    R* A2 = A1 + T;      // [T]
    R* G = A2 + T;       // [3][Tm]
    R* pw = G + 3 * Tm;  // [3][p + 1][FAR_T]: (axis, power, target), conflict-free by target
    for (int a = threadIdx.x; a < T; a += FAR_T) {
        int a1, a2, a3;
        mi_unpack(c_mi[a], a1, a2, a3);
        const R f = (R)(c_fact[a1] * c_fact[a2] * c_fact[a3]);
        const R u = l0[(size_t)c * T + a], v = lk[(size_t)c * T + a];
        A1[a] = (u + v) * f;
        A2[a] = (u + v * (R)(1.0 / eps)) * f;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < Tm; a += FAR_T) {
        int a1, a2, a3;
        mi_unpack(c_mi[a], a1, a2, a3);
        G[a] = A2[pb_midx(a1 + 1, a2, a3)];
        G[Tm + a] = A2[pb_midx(a1, a2 + 1, a3)];
        G[2 * Tm + a] = A2[pb_midx(a1, a2, a3 + 1)];
    }
    const double cx = xc[3 * c], cy = xc[3 * c + 1], cz = xc[3 * c + 2];
    __syncthreads();
    for (int k = begin[c] + threadIdx.x; k < begin[c + 1]; k += FAR_T) {
        double4_32a P = ep[k], Nn = en[k];
        const R d[3] = {(R)(P.x - cx), (R)(P.y - cy), (R)(P.z - cz)};
        const R nx = (R)Nn.x, ny = (R)Nn.y, nz = (R)Nn.z;
        for (int a = 0; a < 3; ++a) {
            R v = 1;
            for (int q = 0; q <= p; ++q) {
                pw[(a * (p + 1) + q) * FAR_T + threadIdx.x] = v * inv_fact1<R>(q);
                v *= d[a];
            }
        }
        R s1 = 0, s2 = 0;
        for (int al = 0; al < T; ++al) {
            int a, b, cc;
            mi_unpack(c_mi[al], a, b, cc);
            const R m = pw[a * FAR_T + threadIdx.x] * pw[((p + 1) + b) * FAR_T + threadIdx.x] *
                        pw[(2 * (p + 1) + cc) * FAR_T + threadIdx.x];
            s1 += A1[al] * m;
            if (al < Tm) s2 += (nx * G[al] + ny * G[Tm + al] + nz * G[2 * Tm + al]) * m;
        }
        ys[k] = -(P.w * (double)s1);  // every element lies in one leaf: the far-field part is set here
        ys[nt + k] = -(P.w * (double)s2);
    }
}

// LtP in FP32 for a compile-time order P (the mixed-precision path): per leaf the coefficients
// are staged once as (L^[a], G_1[a], G_2[a], G_3[a]) records, one 16-byte shared-memory
// broadcast per term; per target the per-axis tables d^q / q! live in registers and the loops
// over the multi-indices are unrolled in layout order, so a term costs one product, one load
// and four FMAs instead of an index unpack and three table loads.
template <int P>
__global__ void __launch_bounds__(FAR_T) k_l2p_f(int nt, double eps, const int* __restrict__ begin,
                                                 const double* __restrict__ xc, const double4_32a* __restrict__ ep,
                                                 const double4_32a* __restrict__ en, const float* __restrict__ l0,
                                                 const float* __restrict__ lk, double* __restrict__ ys, long long lstr,
                                                 long long ystr)
{
    constexpr int T = (P + 1) * (P + 2) * (P + 3) / 6, Tm = P * (P + 1) * (P + 2) / 6;
    __shared__ float A2[T];
    __shared__ float4 cf[T];
    l0 += blockIdx.y * lstr;
    lk += blockIdx.y * lstr;
    ys += blockIdx.y * ystr;
    const int c = blockIdx.x;
    const float ieps = (float)(1.0 / eps);
    for (int a = threadIdx.x; a < T; a += FAR_T) {
        int a1, a2, a3;
        mi_unpack(c_mi[a], a1, a2, a3);
        const float f = (float)(c_fact[a1] * c_fact[a2] * c_fact[a3]);
        const float u = l0[(size_t)c * T + a], v = lk[(size_t)c * T + a];
        cf[a].x = (u + v) * f;
        A2[a] = (u + v * ieps) * f;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < T; a += FAR_T) {
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        if (a < Tm) {
            int a1, a2, a3;
            mi_unpack(c_mi[a], a1, a2, a3);
            g0 = A2[pb_midx(a1 + 1, a2, a3)];
            g1 = A2[pb_midx(a1, a2 + 1, a3)];
            g2 = A2[pb_midx(a1, a2, a3 + 1)];
        }
        cf[a].y = g0;
        cf[a].z = g1;
        cf[a].w = g2;
    }
    const double cx = xc[3 * c], cy = xc[3 * c + 1], cz = xc[3 * c + 2];
    __syncthreads();
    for (int k = begin[c] + threadIdx.x; k < begin[c + 1]; k += FAR_T) {
        const double4_32a Pp = ep[k], Nn = en[k];
        const float dx = (float)(Pp.x - cx), dy = (float)(Pp.y - cy), dz = (float)(Pp.z - cz);
        float ex[P + 1], ey[P + 1], ez[P + 1];
        {
            float vx = 1.f, vy = 1.f, vz = 1.f;
#pragma unroll
            for (int q = 0; q <= P; ++q) {
                const float f = c_i1f[q];
                ex[q] = vx * f;
                ey[q] = vy * f;
                ez[q] = vz * f;
                vx *= dx;
                vy *= dy;
                vz *= dz;
            }
        }
        float s1 = 0.f, t0 = 0.f, t1 = 0.f, t2 = 0.f;
        // an offset the compiler cannot see through, so that the coefficient loads stay in the
        // target loop (hoisted out of it they would need 4 T registers)
        int z;
        asm volatile("mov.u32 %0, 0;" : "=r"(z));
        const float4* cfz = cf + z;
        int al = 0;
#pragma unroll
        for (int n = 0; n <= P; ++n)
#pragma unroll
            for (int a = n; a >= 0; --a)
#pragma unroll
                for (int b = n - a; b >= 0; --b) {
                    const float m = ex[a] * (ey[b] * ez[n - a - b]);
                    const float4 k4 = cfz[al];
                    s1 = fmaf(k4.x, m, s1);
                    if (n < P) {
                        t0 = fmaf(k4.y, m, t0);
                        t1 = fmaf(k4.z, m, t1);
                        t2 = fmaf(k4.w, m, t2);
                    }
                    ++al;
                }
        const float s2 = (float)Nn.x * t0 + (float)Nn.y * t1 + (float)Nn.z * t2;
        ys[k] = -(Pp.w * (double)s1);  // every element lies in one leaf: the far-field part is set here
        ys[nt + k] = -(Pp.w * (double)s2);
    }
}

template <int P>
static void l2p_f_launch(dim3 g, cudaStream_t st, int nt, double eps, const int* begin, const double* xc,
                         const double4_32a* ep, const double4_32a* en, const float* l0, const float* lk, double* ys,
                         long long lstr, long long ystr)
{
    k_l2p_f<P><<<g, FAR_T, 0, st>>>(nt, eps, begin, xc, ep, en, l0, lk, ys, lstr, ystr);
}

// the fixed-order FP32 LtP for orders 1..12; false for other orders (the generic kernel then)
static bool l2p_f(int p, dim3 g, cudaStream_t st, int nt, double eps, const int* begin, const double* xc,
                  const double4_32a* ep, const double4_32a* en, const float* l0, const float* lk, double* ys,
                  long long lstr, long long ystr)
{
#define PB_L2P_F(P)                                                                     \
    case P:                                                                             \
        l2p_f_launch<P>(g, st, nt, eps, begin, xc, ep, en, l0, lk, ys, lstr, ystr); \
        return true;
    switch (p) {
        PB_L2P_F(1) PB_L2P_F(2) PB_L2P_F(3) PB_L2P_F(4) PB_L2P_F(5) PB_L2P_F(6)
        PB_L2P_F(7) PB_L2P_F(8) PB_L2P_F(9) PB_L2P_F(10) PB_L2P_F(11) PB_L2P_F(12)
    }
#undef PB_L2P_F
    return false;
}


static int upload_tables(pb_ctx* c)
{
    int mi[NT_MAX];
    for (int n = 0, pos = 0; n <= PB_PMAX; ++n)
        for (int a = n; a >= 0; --a)
            for (int b = n - a; b >= 0; --b) mi[pos++] = a | (b << 8) | ((n - a - b) << 16);
    double f[25];
    f[0] = 1;
    for (int i = 1; i < 25; ++i) f[i] = f[i - 1] * i;
    double bn[13][13] = {};
    for (int n = 0; n <= 12; ++n) {
        bn[n][0] = 1;
        for (int k = 1; k <= n; ++k) bn[n][k] = bn[n - 1][k - 1] + (k <= n - 1 ? bn[n - 1][k] : 0);
    }
    PB_CUDA(c, cudaMemcpyToSymbol(c_mi, mi, sizeof(mi)));
    PB_CUDA(c, cudaMemcpyToSymbol(c_fact, f, sizeof(f)));
    PB_CUDA(c, cudaMemcpyToSymbol(c_binom, bn, sizeof(bn)));
    float iff[NT_MAX];
    double iff64[NT_MAX];
    for (int k = 0; k < NT_MAX; ++k) {
        const int a1 = mi[k] & 0xff, a2 = (mi[k] >> 8) & 0xff, a3 = mi[k] >> 16;
        iff64[k] = 1.0 / (f[a1] * f[a2] * f[a3]);
        iff[k] = (float)iff64[k];
    }
    PB_CUDA(c, cudaMemcpyToSymbol(c_ifact, iff, sizeof(iff)));
    float i1f[PB_PMAX + 1];
    double i1d[PB_PMAX + 1];
    for (int k = 0; k <= PB_PMAX; ++k) {
        i1d[k] = 1.0 / f[k];
        i1f[k] = (float)i1d[k];
    }
    PB_CUDA(c, cudaMemcpyToSymbol(c_i1f, i1f, sizeof(i1f)));
    PB_CUDA(c, cudaMemcpyToSymbol(c_i1d, i1d, sizeof(i1d)));
    PB_CUDA(c, cudaMemcpyToSymbol(c_ifact64, iff64, sizeof(iff64)));
    c->tables_ready = true;
    return PB_OK;
}

static bool m2l_fast_order(int p) { return p == 4 || p == 6 || p == 8; }

// interaction lists as slots (host work and uploads; no kernels): each target's list padded to
// a multiple of 32 slots for the FP64 contraction (one block per target), packed one after the
// other under mixed precision (the chunk kernel sums per target run), the level's end padded
static int m2l_fast_plan(pb_ctx* c, PbLevel& lv)
{
    cudaStream_t fs = c->st2;  // the whole far-field setup runs on the second stream
    std::vector<int> off(lv.ncl + 1), idx(lv.ninter);
    PB_CUDA(c, cudaMemcpyAsync(off.data(), lv.int_off, sizeof(int) * (lv.ncl + 1), cudaMemcpyDeviceToHost, fs));
    PB_CUDA(c, cudaMemcpyAsync(idx.data(), lv.int_idx, sizeof(int) * lv.ninter, cudaMemcpyDeviceToHost, fs));
    PB_CUDA(c, cudaStreamSynchronize(fs));
    std::vector<int>& soff = lv.h_slot[0];
    std::vector<int>& ssrc = lv.h_slot[1];
    std::vector<int>& stgt = lv.h_slot[2];
    const bool packed = c->prm.precision == PB_MIXED;
    soff.assign(lv.ncl + 1, 0);
    for (int k = 0; k < lv.ncl; ++k) {
        const int n = off[k + 1] - off[k];
        soff[k + 1] = soff[k] + (packed ? n : ((n + 31) / 32) * 32);
    }
    const int ns = ((soff[lv.ncl] + 31) / 32) * 32;
    ssrc.assign(ns, -1);
    stgt.assign(ns, -1);
    for (int k = 0; k < lv.ncl; ++k) {
        for (int t = off[k]; t < off[k + 1]; ++t) ssrc[soff[k] + (t - off[k])] = idx[t];
        for (int t = soff[k]; t < soff[k + 1]; ++t) stgt[t] = k;
    }
    lv.nslots = ns;
    if (packed) {  // the chunk kernel's staging rows, one vector (pb_far_reserve grows them)
        lv.Mp0 = pb_alloc_on(c, sizeof(float) * (size_t)(ns / 32) * 2 * pb_nterms(lv.p), fs);
        lv.Mpk = pb_alloc_on(c, sizeof(float) * (size_t)(ns / 32) * 2 * pb_nterms(lv.p), fs);
        if (!lv.Mp0 || !lv.Mpk) return pb_fail(c, PB_ERR_NOMEM, "m2l setup: out of memory");
    }
    const int T = pb_nterms(lv.p);
    size_t rs = c->prm.precision == PB_MIXED ? sizeof(float) : sizeof(double);
    lv.slot_off = (int*)pb_alloc_on(c, sizeof(int) * (lv.ncl + 1), fs);
    lv.slot_src = (int*)pb_alloc_on(c, sizeof(int) * (lv.nslots + 1), fs);
    lv.slot_tgt = (int*)pb_alloc_on(c, sizeof(int) * (lv.nslots + 1), fs);
    lv.slot_mirror = (int*)pb_alloc_on(c, sizeof(int) * (lv.nslots + 1), fs);
    lv.D0 = pb_alloc_on(c, rs * (size_t)lv.nslots * T, fs);
    lv.Dk = pb_alloc_on(c, rs * (size_t)lv.nslots * T, fs);
    // gathered moments: the FP64 contraction only (the FP32 kernel reads the moments itself)
    const bool gath = c->prm.precision != PB_MIXED;
    lv.Mg0 = gath ? pb_alloc_on(c, rs * (size_t)lv.nslots * T, fs) : nullptr;
    lv.Mgk = gath ? pb_alloc_on(c, rs * (size_t)lv.nslots * T, fs) : nullptr;
    if (!lv.slot_off || !lv.slot_src || !lv.slot_tgt || !lv.slot_mirror || !lv.D0 || !lv.Dk || (gath && (!lv.Mg0 || !lv.Mgk)))
        return pb_fail(c, PB_ERR_NOMEM, "m2l setup: out of memory");
    // (the host vectors live in the level until the next build, so no synchronisation)
    PB_CUDA(c, cudaMemcpyAsync(lv.slot_off, soff.data(), sizeof(int) * (lv.ncl + 1), cudaMemcpyHostToDevice, fs));
    PB_CUDA(c, cudaMemcpyAsync(lv.slot_src, ssrc.data(), sizeof(int) * lv.nslots, cudaMemcpyHostToDevice, fs));
    PB_CUDA(c, cudaMemcpyAsync(lv.slot_tgt, stgt.data(), sizeof(int) * lv.nslots, cudaMemcpyHostToDevice, fs));
    return PB_OK;
}

// the derivative tensors per slot
static int m2l_fast_tables(pb_ctx* c, PbLevel& lv)
{
    cudaStream_t fs = c->st2;
    const int T = pb_nterms(lv.p);
    const size_t smem = sizeof(double) * 3 * (size_t)T * 8;
    const unsigned nb = (unsigned)((lv.nslots + 7) / 8);
    if (nb == 0) return PB_OK;
    k_m2l_mirror<<<(unsigned)((lv.nslots + 255) / 256), 256, 0, fs>>>((int)lv.nslots, lv.slot_off, lv.slot_tgt,
                                                                  lv.slot_src, lv.slot_mirror);
    PB_LAUNCH(c);
    if (c->prm.precision == PB_MIXED) {
        PB_CUDA(c, cudaFuncSetAttribute(k_m2l_setup_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_m2l_setup_ff<<<nb, 256, smem, fs>>>(lv.nslots, lv.p, c->prm.kappa, lv.slot_tgt, lv.slot_src, lv.xc,
                                                  lv.slot_mirror, (float*)lv.D0, (float*)lv.Dk);
    } else {
        PB_CUDA(c, cudaFuncSetAttribute(k_m2l_setup<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_m2l_setup<double><<<nb, 256, smem, fs>>>(lv.nslots, lv.p, c->prm.kappa, lv.slot_tgt, lv.slot_src, lv.xc,
                                                       lv.slot_mirror, (double*)lv.D0, (double*)lv.Dk);
    }
    PB_LAUNCH(c);
    return PB_OK;
}

template <int P, class R>
static int m2l_fast_launch(pb_ctx* c, PbLevel& lv, int nr, cudaStream_t st)
{
    constexpr int T = (P + 1) * (P + 2) * (P + 3) / 6;
    const long long sstr = (long long)lv.ncl * T, mstr = (long long)lv.nslots * T;
    if constexpr (sizeof(R) == sizeof(float)) {
        // the kernel reads the source moments itself (no gathered copy); the targets whose
        // lists cross a chunk edge are summed by a second pass
        const int nch = (int)(lv.nslots / 32);
        size_t smem = (size_t)T * (32 + 33) * sizeof(float);
        if (nch > 0) {
            if ((long long)nch * nr > 0x7fffffffLL) return pb_fail(c, PB_ERR_ARG, "far field: too many chunks x vectors");
            PB_CUDA(c, cudaFuncSetAttribute(k_m2l_seg<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_m2l_seg<P><<<dim3((unsigned)(nch * nr), 1, 2), 64, smem, st>>>(
                nch, lv.slot_off, lv.slot_src, lv.slot_tgt, (const float*)lv.D0, (const float*)lv.Dk,
                (const float*)lv.sig0, (const float*)lv.sigk, (float*)lv.lam0, (float*)lv.lamk, (float*)lv.Mp0,
                (float*)lv.Mpk, c->dev_err, sstr, nr);
            PB_LAUNCH(c);
        }
        const long long ne = (long long)lv.ncl * T;
        k_m2l_runs<<<dim3((unsigned)((ne + 255) / 256), nr, 2), 256, 0, st>>>(
            lv.ncl, T, nch, lv.slot_off, (const float*)lv.Mp0, (const float*)lv.Mpk, (float*)lv.lam0,
            (float*)lv.lamk, sstr);
    } else {
        k_m2l_gather<R><<<dim3((unsigned)(lv.nslots / 32), nr), 256, 0, st>>>(
            T, lv.slot_src, (const R*)lv.sig0, (const R*)lv.sigk, (R*)lv.Mg0, (R*)lv.Mgk, sstr, mstr);
        PB_LAUNCH(c);
        size_t smem = (size_t)T * 33 * sizeof(R);
        PB_CUDA(c, cudaFuncSetAttribute(k_m2l_chunks<P, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_m2l_chunks<P, R><<<dim3(lv.ncl, nr), 32, smem, st>>>(lv.ncl, lv.slot_off, (const R*)lv.D0,
                                                                  (const R*)lv.Dk, (const R*)lv.Mg0, (const R*)lv.Mgk,
                                                                  (R*)lv.lam0, (R*)lv.lamk, mstr, sstr);
    }
    PB_LAUNCH(c);
    return PB_OK;
}

// moments, local coefficients (and, for FP64, gathered moments) for nr right-hand sides at once
int pb_far_reserve(pb_ctx* c, int nr)
{
    if (nr <= c->far_nr) return PB_OK;
    size_t rs = c->prm.precision == PB_MIXED ? sizeof(float) : sizeof(double);
    for (int l = 1; l <= c->L; ++l) {
        PbLevel& lv = c->lev[l];
        const size_t T = pb_nterms(lv.p), n = (size_t)lv.ncl * T * nr;
        lv.sig0 = pb_alloc(c, rs * n);
        lv.sigk = pb_alloc(c, rs * n);
        lv.lam0 = pb_alloc(c, rs * n);
        lv.lamk = pb_alloc(c, rs * n);
        if (!lv.sig0 || !lv.sigk || !lv.lam0 || !lv.lamk) return pb_fail(c, PB_ERR_NOMEM, "far field: out of memory");
        if (lv.D0 && c->prm.precision != PB_MIXED) {  // gathered moments: FP64 contraction only
            lv.Mg0 = pb_alloc(c, rs * (size_t)lv.nslots * T * nr);
            lv.Mgk = pb_alloc(c, rs * (size_t)lv.nslots * T * nr);
            if (!lv.Mg0 || !lv.Mgk) return pb_fail(c, PB_ERR_NOMEM, "far field: out of memory");
        }
        if (lv.D0 && c->prm.precision == PB_MIXED) {  // staging rows of the chunk kernel
            lv.Mp0 = pb_alloc(c, sizeof(float) * (size_t)(lv.nslots / 32) * 2 * T * nr);
            lv.Mpk = pb_alloc(c, sizeof(float) * (size_t)(lv.nslots / 32) * 2 * T * nr);
            if (!lv.Mp0 || !lv.Mpk) return pb_fail(c, PB_ERR_NOMEM, "far field: out of memory");
        }
    }
    c->far_nr = nr;
    return PB_OK;
}

int pb_far_setup(pb_ctx* c)
{
    c->far_nr = 1;
    // on the second stream, after the tree (ev_tree); the host work overlaps the singular pass
    cudaStream_t fs = c->st2;
    PB_CUDA(c, cudaStreamWaitEvent(fs, c->ev_tree, 0));
    // the constant tables never change: uploaded by the first build of a context (a blocking
    // copy, done before any of its streams has work in flight)
    int rc = c->tables_ready ? PB_OK : upload_tables(c);
    if (rc) return rc;
    size_t rs = c->prm.precision == PB_MIXED ? sizeof(float) : sizeof(double);
    {
        // the root's moments: only the treecode energy uses them
        PbLevel& lv = c->lev[0];
        size_t n = (size_t)lv.ncl * pb_nterms(lv.p);
        lv.sig0 = pb_alloc_on(c, rs * n, fs);
        lv.sigk = pb_alloc_on(c, rs * n, fs);
        if (!lv.sig0 || !lv.sigk) return pb_fail(c, PB_ERR_NOMEM, "far field: out of memory");
    }
    for (int l = 1; l <= c->L; ++l) {
        PbLevel& lv = c->lev[l];
        size_t n = (size_t)lv.ncl * pb_nterms(lv.p);
        lv.sig0 = pb_alloc_on(c, rs * n, fs);
        lv.sigk = pb_alloc_on(c, rs * n, fs);
        lv.lam0 = pb_alloc_on(c, rs * n, fs);
        lv.lamk = pb_alloc_on(c, rs * n, fs);
        if (!lv.sig0 || !lv.sigk || !lv.lam0 || !lv.lamk) return pb_fail(c, PB_ERR_NOMEM, "far field: out of memory");
        if (lv.ninter > 0 && m2l_fast_order(lv.p)) {
            int rc2 = m2l_fast_plan(c, lv);
            if (rc2) return rc2;
        }
    }
    // The table kernels wait for the singular pass: long-lived singular blocks would otherwise
    // hold every SM slot while these kernels queue for them. Afterwards they run beside the
    // preconditioner's factorisation.
    PB_CUDA(c, cudaStreamWaitEvent(fs, c->ev_sing, 0));
    pb_tic_on(c, PB_T_FARSETUP, fs);
    for (int l = 1; l <= c->L; ++l) {
        PbLevel& lv = c->lev[l];
        if (lv.ninter > 0 && m2l_fast_order(lv.p)) {
            int rc2 = m2l_fast_tables(c, lv);
            if (rc2) return rc2;
        }
    }
    pb_toc_on(c, PB_T_FARSETUP, fs);
    PB_CUDA(c, cudaEventRecord(c->ev_join, c->st2));
    return PB_OK;
}

// nr right-hand sides: xs and ys hold nr vectors of 2 nt, one after the other; ys receives the
// far-field part of the product (overwritten). All work is queued on stream st.
template <class R>
static int far_apply(pb_ctx* c, const double* xs, double* ys, int nr, cudaStream_t st)
{
    const int L = c->L;
    if (L < 1) {
        PB_CUDA(c, cudaMemsetAsync(ys, 0, sizeof(double) * 2 * c->nt * nr, st));
        return PB_OK;
    }
    int rc0 = pb_far_reserve(c, nr);
    if (rc0) return rc0;
    double eps = c->prm.eps_out / c->prm.eps_in;
    const long long vstr = 2LL * c->nt;
    auto sstr = [](const PbLevel& lv) { return (long long)lv.ncl * pb_nterms(lv.p); };
    // coarsest level with an interaction list: moments above it and local expansions there
    // would only ever be zero or unused
    int lmin = 1;
    while (lmin <= L && c->lev[lmin].ninter == 0) ++lmin;
    if (lmin > L) {  // every pair is near
        PB_CUDA(c, cudaMemsetAsync(ys, 0, sizeof(double) * 2 * c->nt * nr, st));
        return PB_OK;
    }
    // a regular rule of order > 1 (one vector at a time): moments and evaluation on its points
    const bool pts = c->q2 > 1;
    const int np = c->nt * c->q2;
    const long long pvstr = pts ? 2LL * np : vstr;
    pb_tic_on(c, PB_T_UP, st);
    {
        PbLevel& lv = c->lev[L];
        const size_t psm = p2m_smem<R>(lv.p);
        if (pts && xs) {  // (xs == nullptr: the caller has filled the point densities)
            int rc1 = pb_to_points(c, xs, c->xq, st);
            if (rc1) return rc1;
        }
        PB_CUDA(c, cudaFuncSetAttribute(k_p2m<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
        k_p2m<R><<<dim3(lv.ncl, nr), P2M_T, psm, st>>>(np, lv.p, pts ? c->begin_q : lv.begin, lv.xc,
                                                        pts ? c->pts_p : c->e64p, pts ? c->pts_n : c->e64n,
                                                        pts ? c->xq : xs, eps, (R*)lv.sig0, (R*)lv.sigk, pvstr,
                                                        sstr(lv));
        PB_LAUNCH(c);
    }
    for (int l = L - 1; l >= lmin; --l) {
        PbLevel& lv = c->lev[l];
        PbLevel& ch = c->lev[l + 1];
        const size_t msm = 4 * (size_t)pb_nterms(lv.p) * sizeof(R);
        PB_CUDA(c, cudaFuncSetAttribute(k_m2m<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm));
        k_m2m<R><<<dim3(lv.ncl, nr), M2M_T, msm, st>>>(lv.p, ch.p, lv.cbeg, lv.xc, ch.xc, (R*)ch.sig0,
                                                        (R*)ch.sigk, (R*)lv.sig0, (R*)lv.sigk, sstr(ch), sstr(lv));
        PB_LAUNCH(c);
    }
    pb_toc_on(c, PB_T_UP, st);
    pb_tic_on(c, PB_T_M2L, st);
    for (int l = lmin; l <= L; ++l) {
        PbLevel& lv = c->lev[l];
        int rc = -1;
        if (lv.D0) {
            if (lv.p == 4) rc = m2l_fast_launch<4, R>(c, lv, nr, st);
            else if (lv.p == 6) rc = m2l_fast_launch<6, R>(c, lv, nr, st);
            else if (lv.p == 8) rc = m2l_fast_launch<8, R>(c, lv, nr, st);
        }
        if (rc > 0) return rc;
        if (rc == 0) continue;
        k_m2l<R><<<dim3(lv.ncl, nr), FAR_T, 0, st>>>(lv.p, c->prm.kappa, lv.int_off, lv.int_idx, lv.xc,
                                                        (R*)lv.sig0, (R*)lv.sigk, (R*)lv.lam0, (R*)lv.lamk, sstr(lv));
        PB_LAUNCH(c);
    }
    pb_toc_on(c, PB_T_M2L, st);
    pb_tic_on(c, PB_T_DOWN, st);
    for (int l = lmin; l < L; ++l) {
        PbLevel& lv = c->lev[l];
        PbLevel& ch = c->lev[l + 1];
        k_l2l<R><<<dim3(ch.ncl, nr), FAR_T, 0, st>>>(lv.p, ch.p, ch.parent, lv.xc, ch.xc, (R*)lv.lam0,
                                                        (R*)lv.lamk, (R*)ch.lam0, (R*)ch.lamk, sstr(lv), sstr(ch));
        PB_LAUNCH(c);
    }
    {
        PbLevel& lv = c->lev[L];
        const int* tb = pts ? c->begin_q : lv.begin;
        const double4_32a *tp = pts ? c->pts_p : c->e64p, *tn = pts ? c->pts_n : c->e64n;
        double* ty = pts ? c->yq : ys;
        bool done = false;
        if constexpr (sizeof(R) == sizeof(float))
            done = l2p_f(lv.p, dim3(lv.ncl, nr), st, np, eps, tb, lv.xc, tp, tn, (const float*)lv.lam0,
                         (const float*)lv.lamk, ty, sstr(lv), pvstr);
        if (!done) {
            const size_t lsm = l2p_smem<R>(lv.p);
            PB_CUDA(c, cudaFuncSetAttribute(k_l2p<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm));
            k_l2p<R><<<dim3(lv.ncl, nr), FAR_T, lsm, st>>>(np, lv.p, eps, tb, lv.xc, tp, tn, (R*)lv.lam0, (R*)lv.lamk,
                                                            ty, sstr(lv), pvstr);
        }
        PB_LAUNCH(c);
        if (pts) {
            int rc1 = pb_from_points(c, c->yq, ys, 0, st);
            if (rc1) return rc1;
        }
    }
    pb_toc_on(c, PB_T_DOWN, st);
    return PB_OK;
}

int pb_far_apply(pb_ctx* c, const double* xs, double* ys, int nr, cudaStream_t st)
{
    if (c->prm.precision == PB_MIXED) return far_apply<float>(c, xs, ys, nr, st);
    return far_apply<double>(c, xs, ys, nr, st);
}

// ---------- solvation energy by the Cartesian treecode (Section 2.5) ----------
// E = 1/2 * 4 pi 332.0716 * sum_n q_n V_n with V_n = sum_i A_i [K1(x_n, c_i) dphi_i +
// K2(x_n, c_i) phi_i] (eqsolengdis, one-point rule). Per charge, addCluster from the root: a
// cluster c that satisfies the MAC (eqMAC) r_c / R <= theta, tested in FP64 as
// rho_c^2 <= theta^2 |x_n - x_c|^2 with rho_c the shrink-box half diagonal (it bounds every
// point of the cluster), contributes its Taylor series (eqsolengformTree)
//   sum_b D^b G0(x_n - x_c) m~0[b] + D^b Gk(x_n - x_c) m~k[b],
// with the FMM's own moments in their stored form m~ = (-1)^|b| m / b! (the same densities as
// the product's y1 rows, whose kernels K1 + K2 the energy uses); otherwise its children are
// visited, and a leaf that fails is summed directly. The moments come from the same P2M and
// MtM kernels as the product, run on the solution up to the root.
//
// One warp per (charge, level-1 cluster): the warp first makes the root's test (a charge far
// from the whole surface takes the root's series once, in the warp of the first level-1
// cluster), then runs addCluster on its subtree with a stack in shared memory. The lanes share
// each order of the derivative recurrence (warp barriers between orders) and split the
// contraction and the direct sums. Results per warp, summed in a fixed order afterwards.
struct TcLevels {
    const double* xc[PB_MAXL + 1];
    const double* rho[PB_MAXL + 1];
    const int* cbeg[PB_MAXL + 1];
    const void* s0[PB_MAXL + 1];
    const void* sk[PB_MAXL + 1];
    int p[PB_MAXL + 1];
    const int* leaf_begin;
    int L, n1;
};
#define TC_W 4
#define TC_STACK 96  // <= 8 children per level, 10 levels

template <class R>
__device__ double tc_series(const TcLevels& tl, int l, int c, const double* xn, double kappa, R* F0, R* Fk, R* Pk,
                            int lane)
{
    const int p = tl.p[l];
    const int T = pb_nterms(p);
    const R dx = (R)(xn[0] - tl.xc[l][3 * c]), dy = (R)(xn[1] - tl.xc[l][3 * c + 1]),
            dz = (R)(xn[2] - tl.xc[l][3 * c + 2]);
    const R d2 = dx * dx + dy * dy + dz * dz;
    const R kap = (R)kappa;
    if (lane == 0) {
        const R r = sqrt(d2), ex = exp(-kap * r), i4pi = (R)0.07957747154594767;
        F0[0] = i4pi / r;
        Fk[0] = i4pi * ex / r;
        Pk[0] = i4pi * ex;
    }
    __syncwarp();
    // Taylor coefficients F = D^k G / k! degree by degree (the MtL recurrence)
    for (int n = 1; n <= p; ++n) {
        const int lo = pb_nterms(n - 1), hi = pb_nterms(n);
        for (int k = lo + lane; k < hi; k += 32) {
            int k1, k2, k3;
            mi_unpack(c_mi[k], k1, k2, k3);
            const R d[3] = {dx, dy, dz};
            const int kk[3] = {k1, k2, k3};
            R a0 = 0, a1 = 0, ak0 = 0, ak1 = 0, ap0 = 0, ap1 = 0;
            for (int i = 0; i < 3; ++i) {
                if (kk[i] >= 1) {
                    const int q = pb_midx(k1 - (i == 0), k2 - (i == 1), k3 - (i == 2));
                    a0 += d[i] * F0[q];
                    ak0 += d[i] * Fk[q];
                    ap0 += d[i] * Pk[q];
                }
                if (kk[i] >= 2) {
                    const int q = pb_midx(k1 - 2 * (i == 0), k2 - 2 * (i == 1), k3 - 2 * (i == 2));
                    a1 += F0[q];
                    ak1 += Fk[q];
                    ap1 += Pk[q];
                }
            }
            const R nn = (R)n;
            F0[k] = (-(R)(2 * n - 1) * a0 - (nn - 1) * a1) / (d2 * nn);
            Fk[k] = (-(R)(2 * n - 1) * ak0 - (nn - 1) * ak1 - kap * ap0 - kap * ap1) / (d2 * nn);
            Pk[k] = -kap * (ak0 + ak1) / nn;
        }
        __syncwarp();
    }
    // sum_b D^b G m~[b] with D^b = b! F_b
    const R* m0 = (const R*)tl.s0[l] + (size_t)c * T;
    const R* mk = (const R*)tl.sk[l] + (size_t)c * T;
    R acc = 0;
    for (int k = lane; k < T; k += 32) {
        int k1, k2, k3;
        mi_unpack(c_mi[k], k1, k2, k3);
        const R f = (R)(c_fact[k1] * c_fact[k2] * c_fact[k3]);
        acc += f * (F0[k] * m0[k] + Fk[k] * mk[k]);
    }
    __syncwarp();  // F0, Fk, Pk are reused by the next cluster
    return (double)acc;
}

template <class R>
__global__ void __launch_bounds__(32 * TC_W) k_tc_energy(int nc, TcLevels tl, const double* __restrict__ qpos,
                                                         const double* __restrict__ q,
                                                         const double4_32a* __restrict__ ep,
                                                         const double4_32a* __restrict__ en,
                                                         const double* __restrict__ xs, int nt, double eps,
                                                         double kappa, double theta2, int tmax,
                                                         double* __restrict__ vpart)
{
    extern __shared__ __align__(16) unsigned char tsm[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    R* F0 = (R*)tsm + (size_t)wib * 3 * tmax;
    R* Fk = F0 + tmax;
    R* Pk = Fk + tmax;
    __shared__ int stk[TC_W][TC_STACK];
    const long long w = (long long)blockIdx.x * TC_W + wib;
    if (w >= (long long)nc * tl.n1) return;
    const int n = (int)(w / tl.n1), s = (int)(w % tl.n1);
    const double xn[3] = {qpos[3 * n], qpos[3 * n + 1], qpos[3 * n + 2]};
    auto mac = [&](int l, int c) {
        const double dx = xn[0] - tl.xc[l][3 * c], dy = xn[1] - tl.xc[l][3 * c + 1], dz = xn[2] - tl.xc[l][3 * c + 2];
        const double R2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        const double rh = tl.rho[l][c];
        return __dmul_rn(rh, rh) <= __dmul_rn(theta2, R2);
    };
    double V = 0.0;  // lane partial
    const R kap = (R)kappa, ep_ = (R)eps, i4pi = (R)0.07957747154594767;
    auto leaf = [&](int c) {
        const int b = tl.leaf_begin[c], e = tl.leaf_begin[c + 1];
        R acc = 0;
        for (int k = b + lane; k < e; k += 32) {
            const double4_32a y = ep[k], nv = en[k];
            const R dx = (R)(xn[0] - y.x), dy = (R)(xn[1] - y.y), dz = (R)(xn[2] - y.z);
            const R r2 = dx * dx + dy * dy + dz * dz, r = sqrt(r2);
            const R ex = exp(-kap * r);
            const R k1 = -expm1(-kap * r) * i4pi / r;
            const R nd = (R)nv.x * dx + (R)nv.y * dy + (R)nv.z * dz;
            const R k2 = nd * i4pi / (r2 * r) * (ep_ * ((R)1 + kap * r) * ex - (R)1);
            acc += (R)y.w * (k1 * (R)xs[nt + k] + k2 * (R)xs[k]);
        }
        return (double)acc;
    };
    if (mac(0, 0)) {
        if (s == 0) V += tc_series<R>(tl, 0, 0, xn, kappa, F0, Fk, Pk, lane);
    } else if (tl.L == 0) {
        if (s == 0) V += leaf(0);
    } else {
        int sp = 0;
        if (lane == 0) stk[wib][0] = (1 << 24) | s;
        sp = 1;
        __syncwarp();
        while (sp > 0) {
            const int e = stk[wib][sp - 1];
            --sp;
            const int l = e >> 24, c = e & 0xffffff;
            if (mac(l, c)) {
                V += tc_series<R>(tl, l, c, xn, kappa, F0, Fk, Pk, lane);
            } else if (l < tl.L) {
                const int cb = tl.cbeg[l][c], ce = tl.cbeg[l][c + 1];
                __syncwarp();
                // children in reverse, so that they are taken in order
                for (int ch = ce - 1; ch >= cb; --ch) {
                    if (lane == 0 && sp < TC_STACK) stk[wib][sp] = ((l + 1) << 24) | ch;
                    ++sp;
                }
                if (sp > TC_STACK) sp = TC_STACK;  // cannot happen for <= 8 children and 10 levels
                __syncwarp();
            } else {
                V += leaf(c);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) V += __shfl_xor_sync(0xffffffffu, V, o);
    if (lane == 0) vpart[w] = q[n] * V;
}

__global__ void k_tc_sum(long long n, const double* __restrict__ part, double* __restrict__ out, double scale)
{
    __shared__ double red[256];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += 256) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * scale;
}

template <class R>
static int tc_energy(pb_ctx* c, const double* xs, double theta, double* E)
{
    const int L = c->L;
    double eps = c->prm.eps_out / c->prm.eps_in;
    const long long vstr = 2LL * c->nt;
    auto sstr = [](const PbLevel& lv) { return (long long)lv.ncl * pb_nterms(lv.p); };
    pb_tic(c, PB_T_ENERGY);
    // a regular rule of order > 1: moments and leaf sums on its points
    const bool pts = c->q2 > 1;
    const int np = c->nt * c->q2;
    if (pts) {
        int rc1 = pb_to_points(c, xs, c->xq, c->st);
        if (rc1) return rc1;
        xs = c->xq;
    }
    const long long pvstr = 2LL * np;
    (void)vstr;
    // moments of the solution on every level, up to the root (P2M, MtM)
    {
        PbLevel& lv = c->lev[L];
        const size_t psm = p2m_smem<R>(lv.p);
        PB_CUDA(c, cudaFuncSetAttribute(k_p2m<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
        k_p2m<R><<<dim3(lv.ncl, 1), P2M_T, psm, c->st>>>(np, lv.p, pts ? c->begin_q : lv.begin, lv.xc,
                                                          pts ? c->pts_p : c->e64p, pts ? c->pts_n : c->e64n, xs, eps,
                                                          (R*)lv.sig0, (R*)lv.sigk, pvstr, sstr(lv));
        PB_LAUNCH(c);
    }
    for (int l = L - 1; l >= 0; --l) {
        PbLevel& lv = c->lev[l];
        PbLevel& ch = c->lev[l + 1];
        const size_t msm = 4 * (size_t)pb_nterms(lv.p) * sizeof(R);
        PB_CUDA(c, cudaFuncSetAttribute(k_m2m<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm));
        k_m2m<R><<<dim3(lv.ncl, 1), M2M_T, msm, c->st>>>(lv.p, ch.p, lv.cbeg, lv.xc, ch.xc, (R*)ch.sig0,
                                                          (R*)ch.sigk, (R*)lv.sig0, (R*)lv.sigk, sstr(ch), sstr(lv));
        PB_LAUNCH(c);
    }
    TcLevels tl;
    memset(&tl, 0, sizeof(tl));
    int pmax = 0;
    for (int l = 0; l <= L; ++l) {
        tl.xc[l] = c->lev[l].xc;
        tl.rho[l] = c->lev[l].rho;
        tl.cbeg[l] = c->lev[l].cbeg;
        tl.s0[l] = c->lev[l].sig0;
        tl.sk[l] = c->lev[l].sigk;
        tl.p[l] = c->lev[l].p;
        pmax = std::max(pmax, c->lev[l].p);
    }
    tl.leaf_begin = pts ? c->begin_q : c->lev[L].begin;
    tl.L = L;
    tl.n1 = L > 0 ? c->lev[1].ncl : 1;
    const long long nw = (long long)c->nc * tl.n1;
    if (nw > c->tc_nw) {
        c->tc_part = (double*)pb_alloc(c, sizeof(double) * (size_t)(nw + 1));
        if (!c->tc_part) return pb_fail(c, PB_ERR_NOMEM, "treecode energy: out of memory");
        c->tc_nw = nw;
    }
    const int tmax = pb_nterms(pmax);
    const size_t sm = sizeof(R) * 3 * (size_t)tmax * TC_W;
    PB_CUDA(c, cudaFuncSetAttribute(k_tc_energy<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (nw > 0) {
        k_tc_energy<R><<<(unsigned)((nw + TC_W - 1) / TC_W), 32 * TC_W, sm, c->st>>>(
            c->nc, tl, c->qpos, c->q, pts ? c->pts_p : c->e64p, pts ? c->pts_n : c->e64n, xs, np, eps, c->prm.kappa,
            theta * theta, tmax, c->tc_part);
        PB_LAUNCH(c);
    }
    k_tc_sum<<<1, 256, 0, c->st>>>(nw, c->tc_part, c->tc_part + nw, 0.5 * 4.0 * PB_PI * 332.0716);
    PB_LAUNCH(c);
    pb_toc(c, PB_T_ENERGY);
    PB_CUDA(c, cudaMemcpyAsync(c->hscal, c->tc_part + nw, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    *E = c->hscal[0];
    return PB_OK;
}

int pb_energy_treecode_sorted(pb_ctx* c, const double* xs, double theta, double* E)
{
    if (c->prm.precision == PB_MIXED) return tc_energy<float>(c, xs, theta, E);
    return tc_energy<double>(c, xs, theta, E);
}
