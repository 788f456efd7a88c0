// Near field of the FMM matrix-vector product (Section 2.4, step 1 "Nearfield Calculation"):
// for every leaf c and every neighbour leaf c' in N(c), the Galerkin block of A between their
// elements is applied directly. Regular pairs use the one-point (centroid) rule
// A_i A_j K_m(c_i, c_j); identical and adjacent pairs receive their Sauter-Schwab
// correction afterwards (k_corrections). The mass terms 1/2 (1 + eps) A_i and
// 1/2 (1 + 1/eps) A_i of eq_linsysEntry are added here.
//
// Row signs follow eqbim_5/eqbim_6:
//   y1_i = 1/2 (1 + eps) A_i phi_i     - sum_j (I1_ij dphi_j + I2_ij phi_j)
//   y2_i = 1/2 (1 + 1/eps) A_i dphi_i  - sum_j (I3_ij dphi_j + I4_ij phi_j)
//
// Layout (FP64): one CTA per target leaf, one thread per target element. Source leaves are
// staged tile by tile in shared memory (centroid, area, normal, A_j phi_j, A_j dphi_j) and read
// as warp-wide broadcasts. Mixed precision: one warp per chunk of up to 32 targets, which
// evaluates each pair of distinct chunks once for both directions (k_near_tile; several
// right-hand sides: k_near32m, one direction, up to 16 densities per pair evaluation). In
// mixed precision each source leaf's partial sums are kept in FP32
// and added into FP64 accumulators per leaf (compensated leaf sums), and coordinates are
// carried as FP32 hi + lo pairs so that d = (x_hi - y_hi) + (x_lo - y_lo) keeps the
// separation of close elements to FP32 relative accuracy instead of losing digits to the
// size of the coordinates.
#include <algorithm>
#include <vector>

#include "f32x2.cuh"
#include "kernels.cuh"
#include "pb_internal.cuh"


#define NEAR_T 128
#define NEAR_ITEM 6    // pair tiles per warp of the mixed-precision near field
#define NEAR_ITEM_M 8  // directed tiles per warp of the several-vector near field

template <class R, class PV, bool HILO>
__global__ void __launch_bounds__(NEAR_T) k_near(int nt, const int* __restrict__ begin,
                                                 const int* __restrict__ noff, const int* __restrict__ nidx,
                                                 const PV* __restrict__ ep, const PV* __restrict__ en,
                                                 const float4* __restrict__ elo, const double* __restrict__ xs,
                                                 double eps_d, double kappa_d, double* __restrict__ ys)
{
    __shared__ R sx[NEAR_T], sy[NEAR_T], sz[NEAR_T], snx[NEAR_T], sny[NEAR_T], snz[NEAR_T];
    __shared__ R sphi[NEAR_T], sdphi[NEAR_T];
    __shared__ R slx[HILO ? NEAR_T : 1], sly[HILO ? NEAR_T : 1], slz[HILO ? NEAR_T : 1];
    const int c = blockIdx.x;
    const int tb = begin[c], te = begin[c + 1];
    const R eps = (R)eps_d, inv_eps = (R)(1.0 / eps_d), kappa = (R)kappa_d;
    for (int t0 = tb; t0 < te; t0 += NEAR_T) {
        const int k = t0 + threadIdx.x;
        const bool act = k < te;
        R px = 0, py = 0, pz = 0, qx = 0, qy = 0, qz = 0, lx = 0, ly = 0, lz = 0;
        if (act) {
            PV p = ep[k], n = en[k];
            if (HILO) {
                float4 l = elo[k];
                lx = l.x;
                ly = l.y;
                lz = l.z;
            }
            px = (R)p.x;
            py = (R)p.y;
            pz = (R)p.z;
            qx = (R)n.x;
            qy = (R)n.y;
            qz = (R)n.z;
        }
        double acc1 = 0.0, acc2 = 0.0;
        for (int t = noff[c]; t < noff[c + 1]; ++t) {
            const int c2 = nidx[t];
            const int sb = begin[c2], se = begin[c2 + 1];
            R s1 = 0, s2 = 0;
            for (int s0 = sb; s0 < se; s0 += NEAR_T) {
                const int ns = min(NEAR_T, se - s0);
                __syncthreads();
                if (threadIdx.x < ns) {
                    const int j = s0 + threadIdx.x;
                    PV p = ep[j], n = en[j];
                    sx[threadIdx.x] = (R)p.x;
                    sy[threadIdx.x] = (R)p.y;
                    sz[threadIdx.x] = (R)p.z;
                    snx[threadIdx.x] = (R)n.x;
                    sny[threadIdx.x] = (R)n.y;
                    snz[threadIdx.x] = (R)n.z;
                    sphi[threadIdx.x] = (R)(p.w * xs[j]);
                    sdphi[threadIdx.x] = (R)(p.w * xs[nt + j]);
                    if (HILO) {
                        float4 l = elo[j];
                        slx[threadIdx.x] = l.x;
                        sly[threadIdx.x] = l.y;
                        slz[threadIdx.x] = l.z;
                    }
                }
                __syncthreads();
                if (act) {
#pragma unroll 4
                    for (int q = 0; q < ns; ++q) {
                        if (s0 + q == k) continue;
                        R K[4];
                        R dx = px - sx[q], dy = py - sy[q], dz = pz - sz[q];
                        if (HILO) {
                            dx += lx - slx[q];
                            dy += ly - sly[q];
                            dz += lz - slz[q];
                        }
                        pb_kernels<R>(dx, dy, dz, qx, qy, qz, snx[q], sny[q], snz[q], eps, inv_eps, kappa, K);
                        s1 += K[0] * sdphi[q] + K[1] * sphi[q];
                        s2 += K[2] * sdphi[q] + K[3] * sphi[q];
                    }
                }
            }
            acc1 += (double)s1;
            acc2 += (double)s2;
        }
        if (act) {
            double A = (double)ep[k].w;
            ys[k] = 0.5 * (1.0 + eps_d) * A * xs[k] - A * acc1;
            ys[nt + k] = 0.5 * (1.0 + 1.0 / eps_d) * A * xs[nt + k] - A * acc2;
        }
    }
}

// ---------- mixed precision near field ----------
// Per matrix-vector product the sources are packed once as FP32 records
// (x_hi, y_hi, z_hi, A phi), (n_x, n_y, n_z, A dphi) beside the fixed (x_lo, y_lo, z_lo).
__global__ void k_near_pack(int nt, const float4* __restrict__ e32p, const float4* __restrict__ e32n,
                            const double* __restrict__ xs, float4* __restrict__ sp, float4* __restrict__ sn)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    float4 p = e32p[k], n = e32n[k];
    double A = (double)p.w;
    sp[k] = make_float4(p.x, p.y, p.z, (float)(A * xs[k]));
    sn[k] = make_float4(n.x, n.y, n.z, (float)(A * xs[nt + k]));
}


// ---------- the tile kernel (mixed precision) ----------
// Both directions of a pair at once, by tiles of one target chunk A (up to 32 targets, lane l
// holds A_l) and one source chunk B of nb <= 32 sources. K1 and K4 are symmetric in (x, y),
// and with d = x_i - x_j the double-layer kernels of the reversed pair follow from the same
// radial factors: K2(j, i) = -(n_i.d) ri3 (eps e1 - 1), K3(j, i) = (n_j.d) ri3 (1 - e1/eps).
// The tiles (A, B) -- every source chunk B of the neighbour leaves c2 >= c that follows A (B
// after A within A's own leaf) -- are cut into work items of at most NEAR_ITEM tiles of one A;
// one warp per item, so that the warps carry nearly equal work whatever the leaf order. B's
// records are staged in shared memory as packed pairs (below); at step s (s < ceil(nb / 2)) lane
// l pairs A_l with B_((l + s) mod nb) and B_((l + s + h) mod nb), h = ceil(nb / 2), and keeps
// the forward terms. The reverse terms of a full tile of another chunk (nb = 32) ride in
// registers that move one lane down after every step (shuffles), so that after 16 steps lane l
// holds the sums of sources (l + 16) mod 32 and l; partial tiles add them to B's shared-memory
// accumulators instead (FP32 shared atomics). Forward sums of a chunk and reverse sums of a
// tile are FP32, added into FP64 (atomics for the reverse terms and the final forward sums; ys
// starts at zero). The tile of A with itself keeps only the forward terms and drops the
// identical pair.
// Q2 > 1: the records are the points of a regular rule (Q2 per element, consecutive; Q2 divides
// 32 and every leaf starts at an element, so no chunk splits an element): the pairs of points of
// one element are dropped, which can only happen in the tile of a chunk with itself.
//
// Packed pairs: entry m of a staged tile holds source m in the low halves and source
// (m + h) mod nb in the high halves, as F0 = (x, y), F1 = (z, A phi), F2 = (n_x, n_y),
// F3 = (n_z, -A dphi) of the high coordinate parts and F4 = (x, y), F5 = (z, 0) of the low
// parts. Every FP32 operation of the two pairs of a step is one f32x2 instruction; only the
// reciprocal square root, the exponential and the branch of the screening function run per
// half. (The packed instructions do not raise the FP32 rate; they halve the issue slots that
// bound this loop.)
struct NearTgt2 {
    f2x px, py, pz, lx, ly, lz, nx, ny, nz, phi, dphi;
};

// s1, s2 += forward terms; q1n -= first reverse term, q2 += second reverse term (per half).
// bump is added to r^2 of dropped pairs (so that r stays finite), scale = 1 / (4 pi) or 0.
template <bool BUMP>
__device__ __forceinline__ void near_pair_x2(const NearTgt2& T, const float4* __restrict__ e, f2x bump, f2x scale,
                                             f2x eps2, f2x nieps2, f2x kappa2, f2x& s1, f2x& s2, f2x& q1n, f2x& q2)
{
    const float4 g0 = e[0], g1 = e[32], g2 = e[64], g3 = e[96], g4 = e[128], g5 = e[160];
    const f2x ax = x2_pack(g0.x, g0.y), ay = x2_pack(g0.z, g0.w), az = x2_pack(g1.x, g1.y);
    const f2x aphi = x2_pack(g1.z, g1.w);
    const f2x bx = x2_pack(g2.x, g2.y), by = x2_pack(g2.z, g2.w), bz = x2_pack(g3.x, g3.y);
    const f2x nadphi = x2_pack(g3.z, g3.w);
    const f2x lx = x2_pack(g4.x, g4.y), ly = x2_pack(g4.z, g4.w), lz = x2_pack(g5.x, g5.y);
    const f2x one = x2_dup(1.f), mone = x2_dup(-1.f), three = x2_dup(3.f);
    const f2x dx = x2_add(x2_sub(T.px, ax), x2_sub(T.lx, lx));
    const f2x dy = x2_add(x2_sub(T.py, ay), x2_sub(T.ly, ly));
    const f2x dz = x2_add(x2_sub(T.pz, az), x2_sub(T.lz, lz));
    f2x r2 = x2_fma(dz, dz, x2_fma(dy, dy, x2_mul(dx, dx)));
    if (BUMP) r2 = x2_add(r2, bump);
    float ra, rb;
    x2_unpack(r2, ra, rb);
    const f2x rinv = x2_pack(rsqrtf(ra), rsqrtf(rb));
    const f2x tt = x2_mul(kappa2, x2_mul(r2, rinv));
    // g / t^2 = 1/2 - t/6 + t^2/24 - ... (the Taylor series of e^-t - 1 + t), for small t
    f2x sg = x2_fma(x2_dup(1.f / 40320.f), tt, x2_dup(-1.f / 5040.f));
    sg = x2_fma(sg, tt, x2_dup(1.f / 720.f));
    sg = x2_fma(sg, tt, x2_dup(-1.f / 120.f));
    sg = x2_fma(sg, tt, x2_dup(1.f / 24.f));
    sg = x2_fma(sg, tt, x2_dup(-1.f / 6.f));
    sg = x2_fma(sg, tt, x2_dup(0.5f));
    const f2x gs = x2_mul(x2_mul(sg, tt), tt);
    float ta, tb;
    x2_unpack(tt, ta, tb);
    const f2x ed = x2_add(x2_pack(__expf(-ta), __expf(-tb)), mone);
    const f2x ga = x2_add(ed, tt), eb = x2_sub(gs, tt);
    float gsa, gsb, gaa, gab, eba, ebb, eda, edb;
    x2_unpack(gs, gsa, gsb);
    x2_unpack(ga, gaa, gab);
    x2_unpack(eb, eba, ebb);
    x2_unpack(ed, eda, edb);
    const bool sa = ta < 0.125f, sb = tb < 0.125f;
    const f2x g = x2_pack(sa ? gsa : gaa, sb ? gsb : gab);
    const f2x E = x2_pack(sa ? eba : eda, sb ? ebb : edb);
    const f2x tE = x2_mul(tt, E);
    const f2x c1n = x2_add(g, tE);                                            // -c1
    const f2x c3n = x2_fma(tE, x2_add(three, tt), x2_fma(tt, tt, x2_mul(three, g)));  // -c3
    const f2x ri = x2_mul(rinv, scale);
    const f2x ri3 = x2_mul(x2_mul(ri, rinv), rinv);
    const f2x nxd = x2_fma(T.nz, dz, x2_fma(T.ny, dy, x2_mul(T.nx, dx)));
    const f2x nyd = x2_fma(bz, dz, x2_fma(by, dy, x2_mul(bx, dx)));
    const f2x nxny = x2_fma(T.nz, bz, x2_fma(T.ny, by, x2_mul(T.nx, bx)));
    const f2x e1 = x2_add(one, c1n);
    const f2x f2 = x2_mul(ri3, x2_fma(eps2, e1, mone));   // ri3 (eps e1 - 1)
    const f2x f3 = x2_mul(ri3, x2_fma(nieps2, e1, one));  // ri3 (1 - e1 / eps)
    const f2x k1n = x2_mul(E, ri);                       // -K1
    const f2x u = x2_mul(x2_mul(nxd, nyd), x2_mul(rinv, rinv));
    const f2x k4 = x2_mul(ri3, x2_sub(x2_mul(c1n, nxny), x2_mul(c3n, u)));
    s1 = x2_fma(k1n, nadphi, x2_fma(x2_mul(nyd, f2), aphi, s1));
    s2 = x2_fma(k4, aphi, x2_fma(x2_mul(nxd, f3), nadphi, s2));
    q1n = x2_fma(k1n, T.dphi, x2_fma(x2_mul(nxd, f2), T.phi, q1n));
    q2 = x2_fma(k4, T.phi, x2_fma(x2_mul(nyd, f3), T.dphi, q2));
}

__device__ __forceinline__ f2x x2_shfl_down1(f2x v, int lane)
{
    float a, b;
    x2_unpack(v, a, b);
    a = __shfl_sync(0xffffffffu, a, (lane + 1) & 31);
    b = __shfl_sync(0xffffffffu, b, (lane + 1) & 31);
    return x2_pack(a, b);
}

template <int Q2>
__global__ void __launch_bounds__(256, 3) k_near_tile(int nt, int nitems, const int4* __restrict__ items,
                                                    const int* __restrict__ tiles, const int* __restrict__ chunk_leaf,
                                                    const int* __restrict__ chunk_first, const int* __restrict__ begin,
                                                    const float4* __restrict__ sp, const float4* __restrict__ sn,
                                                    const float4* __restrict__ sl, double eps_d, double kappa_d,
                                                    double* __restrict__ ys)
{
    __shared__ float4 fq[8][6 * 32];
    __shared__ float rv1[8][32], rv2[8][32];
    const float i4pi = 0.07957747154594767f;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    if (w >= nitems) return;
    const int4 item = items[w];
    const int ca = item.x;
    const int c = chunk_leaf[ca], a0 = chunk_first[ca];
    const int k = a0 + lane;
    const bool act = k < begin[c + 1];
    const int kk = act ? k : a0;
    NearTgt2 T;
    {
        const float4 tp = sp[kk], tn = sn[kk], tl = sl[kk];
        T.px = x2_dup(tp.x);
        T.py = x2_dup(tp.y);
        T.pz = x2_dup(tp.z);
        T.lx = x2_dup(tl.x);
        T.ly = x2_dup(tl.y);
        T.lz = x2_dup(tl.z);
        T.nx = x2_dup(tn.x);
        T.ny = x2_dup(tn.y);
        T.nz = x2_dup(tn.z);
        T.phi = x2_dup(act ? tp.w : 0.f);
        T.dphi = x2_dup(act ? tn.w : 0.f);
    }
    const f2x eps2 = x2_dup((float)eps_d), nieps2 = x2_dup((float)(-1.0 / eps_d)), kappa2 = x2_dup((float)kappa_d);
    const f2x zero = x2_dup(0.f);
    double acc1 = 0.0, acc2 = 0.0;
    float4* F = fq[wi];
    for (int ti = item.y; ti < item.z; ++ti) {
        const int cb = tiles[ti];
        const int b0 = chunk_first[cb], se = begin[chunk_leaf[cb] + 1];
        const bool diag = cb == ca;
        const int nb = min(32, se - b0);
        if (nb <= 0) continue;  // no chunk is empty; the test keeps the indexing below in range
        const int h = (nb + 1) >> 1;
        // stage the tile: lane l < nb writes entry l = (source l, source (l + h) mod nb)
        {
            const int j = b0 + min(lane, nb - 1);
            const float4 p = sp[j], n = sn[j], lo = sl[j];
            int src = lane + h;
            if (src >= nb) src -= nb;
            if (lane >= nb) src = lane;
            const float Px = __shfl_sync(0xffffffffu, p.x, src), Py = __shfl_sync(0xffffffffu, p.y, src);
            const float Pz = __shfl_sync(0xffffffffu, p.z, src), Pw = __shfl_sync(0xffffffffu, p.w, src);
            const float Nx = __shfl_sync(0xffffffffu, n.x, src), Ny = __shfl_sync(0xffffffffu, n.y, src);
            const float Nz = __shfl_sync(0xffffffffu, n.z, src), Nw = __shfl_sync(0xffffffffu, n.w, src);
            const float Lx = __shfl_sync(0xffffffffu, lo.x, src), Ly = __shfl_sync(0xffffffffu, lo.y, src);
            const float Lz = __shfl_sync(0xffffffffu, lo.z, src);
            __syncwarp();
            if (lane < nb) {
                F[lane] = make_float4(p.x, Px, p.y, Py);
                F[32 + lane] = make_float4(p.z, Pz, p.w, Pw);
                F[64 + lane] = make_float4(n.x, Nx, n.y, Ny);
                F[96 + lane] = make_float4(n.z, Nz, -n.w, -Nw);
                F[128 + lane] = make_float4(lo.x, Lx, lo.y, Ly);
                F[160 + lane] = make_float4(lo.z, Lz, 0.f, 0.f);
            }
            __syncwarp();
        }
        f2x s1 = zero, s2 = zero;
        if (!diag && nb == 32) {
            // full tile of another chunk: lane l meets sources (l + s) mod 32 and (l + s + 16)
            // mod 32 at step s; the reverse sums move one lane down after every step
            const f2x sc = x2_dup(act ? i4pi : 0.f);
            f2x q1n = zero, q2 = zero;
            int m = lane;
#pragma unroll 4
            for (int s = 0; s < 16; ++s) {
                near_pair_x2<false>(T, F + m, zero, sc, eps2, nieps2, kappa2, s1, s2, q1n, q2);
                q1n = x2_shfl_down1(q1n, lane);
                q2 = x2_shfl_down1(q2, lane);
                m = (m + 1) & 31;
            }
            // lane l: the low halves belong to source (l + 16) mod 32, the high halves to l
            float a1, b1, a2, b2;
            x2_unpack(q1n, a1, b1);
            x2_unpack(q2, a2, b2);
            const float t1 = b1 + __shfl_sync(0xffffffffu, a1, (lane + 16) & 31);
            const float t2 = b2 + __shfl_sync(0xffffffffu, a2, (lane + 16) & 31);
            atomicAdd(&ys[b0 + lane], -(double)t1);
            atomicAdd(&ys[nt + b0 + lane], (double)t2);
        } else {
            rv1[wi][lane] = 0.f;
            rv2[wi][lane] = 0.f;
            __syncwarp();
            int m = lane % nb;
            int m2 = m + h;
            if (m2 >= nb) m2 -= nb;
            const bool odd = nb & 1;
            for (int s = 0; s < h; ++s) {
                // drop the identical pair (the correction's), padding targets and, for odd nb,
                // the repeated source of the last step
                const bool okl = act && !(diag && (Q2 == 1 ? m == lane : m / Q2 == lane / Q2));
                const bool okh = act && !(odd && s == h - 1) && !(diag && (Q2 == 1 ? m2 == lane : m2 / Q2 == lane / Q2));
                const f2x bump = x2_pack(okl ? 0.f : 1.f, okh ? 0.f : 1.f);
                const f2x sc = x2_pack(okl ? i4pi : 0.f, okh ? i4pi : 0.f);
                f2x q1n = zero, q2 = zero;
                near_pair_x2<true>(T, F + m, bump, sc, eps2, nieps2, kappa2, s1, s2, q1n, q2);
                if (!diag) {
                    float a1, b1, a2, b2;
                    x2_unpack(q1n, a1, b1);
                    x2_unpack(q2, a2, b2);
                    atomicAdd(&rv1[wi][m], -a1);
                    atomicAdd(&rv1[wi][m2], -b1);
                    atomicAdd(&rv2[wi][m], a2);
                    atomicAdd(&rv2[wi][m2], b2);
                }
                m = m + 1 == nb ? 0 : m + 1;
                m2 = m2 + 1 == nb ? 0 : m2 + 1;
            }
            __syncwarp();
            if (!diag && lane < nb) {
                atomicAdd(&ys[b0 + lane], (double)rv1[wi][lane]);
                atomicAdd(&ys[nt + b0 + lane], (double)rv2[wi][lane]);
            }
        }
        float a, b;
        x2_unpack(s1, a, b);
        acc1 += (double)(a + b);
        x2_unpack(s2, a, b);
        acc2 += (double)(a + b);
    }
    if (act) {
        atomicAdd(&ys[k], acc1);
        atomicAdd(&ys[nt + k], acc2);
    }
}

// ---------- several right-hand sides at once (mixed precision) ----------
// The pair kernels depend on the geometry only, so one evaluation serves NR densities: the
// source's geometry records are loaded once per pair and each right-hand side adds four FMAs.
// dens[r nt + j] = (A_j phi_j, A_j dphi_j) of right-hand side r.
__global__ void k_near_dens(int nt, const float4* __restrict__ e32p, const double* __restrict__ xs,
                            float2* __restrict__ dens)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const double A = (double)e32p[k].w;
    const double* x = xs + 2LL * nt * blockIdx.y;
    dens[(size_t)nt * blockIdx.y + k] = make_float2((float)(A * x[k]), (float)(A * x[nt + k]));
}

// Work items of at most NEAR_ITEM_M directed tiles (target chunk A, source chunk B of any
// neighbour leaf), one warp each; the item's sums are added into ys (zeroed first) with FP64
// atomics, so that items of one target chunk may run on different warps. Each tile's source
// records and its NR densities are staged in shared memory by coalesced loads (one per lane
// and record), so the pair loop reads them as shared-memory broadcasts.
template <int NR>
__global__ void __launch_bounds__(256, 2) k_near32m(int nt, int nitems, const int4* __restrict__ items,
                                                    const int* __restrict__ tiles, const int* __restrict__ chunk_leaf,
                                                    const int* __restrict__ chunk_first,
                                                    const int* __restrict__ begin, const float4* __restrict__ sp,
                                                    const float4* __restrict__ sn, const float4* __restrict__ sl,
                                                    const float2* __restrict__ dens, double eps_d, double kappa_d,
                                                    double* __restrict__ ys, int nvalid)
{
    // dynamic shared memory (near32m_smem<NR>()): per warp the tile's source records, its NR
    // densities, and the item's FP64 sums (kept here rather than in registers)
    extern __shared__ __align__(16) unsigned char nsm[];
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    float4* s_p = (float4*)nsm + wi * 32;
    float4* s_n = (float4*)nsm + 256 + wi * 32;
    float4* s_l = (float4*)nsm + 512 + wi * 32;
    float2* s_d = (float2*)((float4*)nsm + 768) + wi * NR * 32;
    double* s_acc = (double*)((float2*)((float4*)nsm + 768) + 8 * NR * 32) + wi * 2 * NR * 32;
    if (w >= nitems) return;
    const int4 item = items[w];
    const int c = chunk_leaf[item.x];
    const int k = chunk_first[item.x] + lane;
    const bool act = k < begin[c + 1];
    const int kk = act ? k : chunk_first[item.x];
    const float4 tp = sp[kk], tn = sn[kk], tl = sl[kk];
    const float eps = (float)eps_d, inv_eps = (float)(1.0 / eps_d), kappa = (float)kappa_d;
#pragma unroll
    for (int r = 0; r < 2 * NR; ++r) s_acc[r * 32 + lane] = 0.0;
    for (int ti = item.y; ti < item.z; ++ti) {
        const int cb = tiles[ti];
        const int sb = chunk_first[cb], se = min(sb + 32, begin[chunk_leaf[cb] + 1]);
        const int nb = se - sb;
        __syncwarp();
        if (lane < nb) {
            const int j = sb + lane;
            s_p[lane] = sp[j];
            s_n[lane] = sn[j];
            s_l[lane] = sl[j];
#pragma unroll
            for (int r = 0; r < NR; ++r) s_d[r * 32 + lane] = dens[(size_t)nt * r + j];
        }
        __syncwarp();
        float s1[NR], s2[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) s1[r] = s2[r] = 0.f;
#pragma unroll 2
        for (int q = 0; q < nb; ++q) {
            const int j = sb + q;
            const float4 a = s_p[q], b = s_n[q], l = s_l[q];
            float K[4];
            float dx = (tp.x - a.x) + (tl.x - l.x);
            float dy = (tp.y - a.y) + (tl.y - l.y);
            float dz = (tp.z - a.z) + (tl.z - l.z);
            if (j == k) dx = 1.0f;  // the identical pair is the correction's; keep r finite
            pb_kernels<float>(dx, dy, dz, tn.x, tn.y, tn.z, b.x, b.y, b.z, eps, inv_eps, kappa, K,
                              (j == k) ? 0.f : 1.f);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float2 d = s_d[r * 32 + q];
                s1[r] = fmaf(K[0], d.y, fmaf(K[1], d.x, s1[r]));
                s2[r] = fmaf(K[2], d.y, fmaf(K[3], d.x, s2[r]));
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            s_acc[r * 32 + lane] += (double)s1[r];
            s_acc[(NR + r) * 32 + lane] += (double)s2[r];
        }
    }
    // densities beyond nvalid are padding of the group (finite, unused): only nvalid are added
    if (act)
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r < nvalid) {
                atomicAdd(&ys[2LL * nt * r + k], s_acc[r * 32 + lane]);
                atomicAdd(&ys[2LL * nt * r + nt + k], s_acc[(NR + r) * 32 + lane]);
            }
}

// y1 = 1/2 (1 + eps) A phi - A acc1, y2 = 1/2 (1 + 1/eps) A dphi - A acc2 (FP64)
__global__ void k_near_finish(int nt, const double4_32a* __restrict__ ep, const double* __restrict__ xs,
                              double eps, double* __restrict__ ys)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    xs += 2LL * nt * blockIdx.y;
    ys += 2LL * nt * blockIdx.y;
    double A = ep[k].w;
    ys[k] = 0.5 * (1.0 + eps) * A * xs[k] - A * ys[k];
    ys[nt + k] = 0.5 * (1.0 + 1.0 / eps) * A * xs[nt + k] - A * ys[nt + k];
}

// Sauter-Schwab corrections of identical and adjacent pairs (FP64), and the far-field part of
// the product when yf is given (xs == nullptr: the far field alone)
__global__ void k_corrections(int nt, const int* __restrict__ toff, const int* __restrict__ tj,
                              const double* __restrict__ corr, const double* __restrict__ xs,
                              double* __restrict__ ys, const double* __restrict__ yf)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const long long o = 2LL * nt * blockIdx.y;
    ys += o;
    double y1 = 0.0, y2 = 0.0;
    if (xs) {
        xs += o;
        // the four values of a pair as two 16-byte loads
        const double2* c2 = reinterpret_cast<const double2*>(corr);
        for (int t = toff[k]; t < toff[k + 1]; ++t) {
            int j = tj[t];
            double ph = xs[j], dph = xs[nt + j];
            const double2 a = c2[2 * t], b = c2[2 * t + 1];
            y1 += a.x * dph + a.y * ph;
            y2 += b.x * dph + b.y * ph;
        }
    }
    if (yf) {
        y1 -= yf[o + k];
        y2 -= yf[o + nt + k];
    }
    ys[k] -= y1;
    ys[nt + k] -= y2;
}

// chunks of at most 32 targets per leaf and the packed source buffers (mixed precision)
int pb_near_setup(pb_ctx* c)
{
    if (c->prm.precision != PB_MIXED) return PB_OK;
    const PbLevel& lv = c->lev[c->L];
    const std::vector<int>& b = c->h_leaf_begin;  // the leaf ranges, read back by the tree build
    std::vector<int>& cl = c->h_up_i[0];
    std::vector<int>& cf = c->h_up_i[1];
    cl.clear();
    cf.clear();
    for (int k = 0; k < lv.ncl; ++k)
        for (int s = b[k]; s < b[k + 1]; s += 32) {
            cl.push_back(k);
            cf.push_back(s);
        }
    c->nchunks = (int)cl.size();
    // pair tiles (A, B), B a chunk of a neighbour leaf c2 >= leaf(A) and B >= A, cut into work
    // items of at most NEAR_ITEM tiles that share A
    {
        std::vector<int> first_chunk(lv.ncl + 1, 0);
        for (int k = 0; k < lv.ncl; ++k) first_chunk[k + 1] = first_chunk[k] + (b[k + 1] - b[k] + 31) / 32;
        std::vector<int>& tl = c->h_up_i[4];
        std::vector<int4>& it = c->h_up_i4;
        tl.clear();
        it.clear();
        const std::vector<int>& no = c->h_near_off;
        const std::vector<int>& ni = c->h_near_idx;
        for (int k = 0; k < lv.ncl; ++k)
            for (int a = first_chunk[k]; a < first_chunk[k + 1]; ++a) {
                int start = (int)tl.size();
                for (int t = no[k]; t < no[k + 1]; ++t) {
                    const int c2 = ni[t];
                    if (c2 < k) continue;
                    for (int bq = (c2 == k ? a : first_chunk[c2]); bq < first_chunk[c2 + 1]; ++bq) {
                        tl.push_back(bq);
                        if ((int)tl.size() - start == NEAR_ITEM) {
                            it.push_back(make_int4(a, start, (int)tl.size(), 0));
                            start = (int)tl.size();
                        }
                    }
                }
                if ((int)tl.size() > start) it.push_back(make_int4(a, start, (int)tl.size(), 0));
            }
        c->near_nitems = (int)it.size();
        c->near_mitems = 0;  // the several-vector items are made on first use (pb_near_reserve)
        c->near_mitem = nullptr;
        c->near_mtiles = nullptr;
        c->near_items = (int4*)pb_alloc(c, sizeof(int4) * (it.size() + 1));
        c->near_tiles = (int*)pb_alloc(c, sizeof(int) * (tl.size() + 1));
        if (!c->near_items || !c->near_tiles) return pb_fail(c, PB_ERR_NOMEM, "near setup: out of memory");
        PB_CUDA(c, cudaMemcpyAsync(c->near_items, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice, c->st));
        PB_CUDA(c, cudaMemcpyAsync(c->near_tiles, tl.data(), sizeof(int) * tl.size(), cudaMemcpyHostToDevice, c->st));
    }
    c->chunk_leaf = (int*)pb_alloc(c, sizeof(int) * cl.size());
    c->chunk_first = (int*)pb_alloc(c, sizeof(int) * cf.size());
    c->near_sp = (float4*)pb_alloc(c, sizeof(float4) * c->nt);
    c->near_sn = (float4*)pb_alloc(c, sizeof(float4) * c->nt);
    if (!c->chunk_leaf || !c->chunk_first || !c->near_sp || !c->near_sn)
        return pb_fail(c, PB_ERR_NOMEM, "near setup: out of memory");
    PB_CUDA(c, cudaMemcpyAsync(c->chunk_leaf, cl.data(), sizeof(int) * cl.size(), cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyAsync(c->chunk_first, cf.data(), sizeof(int) * cf.size(), cudaMemcpyHostToDevice, c->st));
    return PB_OK;
}

int pb_near_apply(pb_ctx* c, const double* xs, double* ys)
{
    const PbLevel& lv = c->lev[c->L];
    double eps = c->prm.eps_out / c->prm.eps_in;
    if (c->prm.precision == PB_MIXED) {
        const int nt = c->nt;
        k_near_pack<<<(nt + 255) / 256, 256, 0, c->st>>>(nt, c->e32p, c->e32n, xs, c->near_sp, c->near_sn);
        PB_LAUNCH(c);
        PB_CUDA(c, cudaMemsetAsync(ys, 0, sizeof(double) * 2 * nt, c->st));
        k_near_tile<1><<<(c->near_nitems * 32 + 255) / 256, 256, 0, c->st>>>(
            nt, c->near_nitems, c->near_items, c->near_tiles, c->chunk_leaf, c->chunk_first, lv.begin, c->near_sp,
            c->near_sn, c->e32l, eps, c->prm.kappa, ys);
        PB_LAUNCH(c);
        k_near_finish<<<(nt + 255) / 256, 256, 0, c->st>>>(nt, c->e64p, xs, eps, ys);
    } else
        k_near<double, double4_32a, false><<<lv.ncl, NEAR_T, 0, c->st>>>(c->nt, lv.begin, lv.near_off,
                                                                         lv.near_idx, c->e64p, c->e64n, nullptr, xs,
                                                                         eps, c->prm.kappa, ys);
    PB_LAUNCH(c);
    return PB_OK;
}

// Several right-hand sides: four per thread (blockIdx.y = group of four), so each correction
// is read once per four vectors instead of once per vector.
__global__ void k_corrections4(int nt, int nr, const int* __restrict__ toff, const int* __restrict__ tj,
                               const double* __restrict__ corr, const double* __restrict__ xs,
                               double* __restrict__ ys, const double* __restrict__ yf)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const int q0 = 4 * blockIdx.y, nq = min(4, nr - q0);
    const long long vs = 2LL * nt;
    double y1[4] = {0, 0, 0, 0}, y2[4] = {0, 0, 0, 0};
    if (xs)
        for (int t = toff[k]; t < toff[k + 1]; ++t) {
            const int j = tj[t];
            const double2 a = reinterpret_cast<const double2*>(corr)[2 * t];
            const double2 b = reinterpret_cast<const double2*>(corr)[2 * t + 1];
            const double c0 = a.x, c1 = a.y, c2 = b.x, c3 = b.y;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nq) {
                    const double* x = xs + (q0 + q) * vs;
                    const double ph = x[j], dph = x[nt + j];
                    y1[q] += c0 * dph + c1 * ph;
                    y2[q] += c2 * dph + c3 * ph;
                }
        }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (q < nq) {
            const long long o = (q0 + q) * vs;
            double a = y1[q], b = y2[q];
            if (yf) {
                a -= yf[o + k];
                b -= yf[o + nt + k];
            }
            ys[o + k] -= a;
            ys[o + nt + k] -= b;
        }
}

int pb_corr_apply(pb_ctx* c, const double* xs, double* ys, int nr, const double* yfar)
{
    if (nr > 1) {
        k_corrections4<<<dim3((c->nt + 255) / 256, (nr + 3) / 4), 256, 0, c->st>>>(c->nt, nr, c->touch_off, c->touch_j,
                                                                                c->corr, xs, ys, yfar);
        PB_LAUNCH(c);
        return PB_OK;
    }
    k_corrections<<<dim3((c->nt + 255) / 256, nr), 256, 0, c->st>>>(c->nt, c->touch_off, c->touch_j, c->corr, xs,
                                                                     ys, yfar);
    PB_LAUNCH(c);
    return PB_OK;
}

template <int NR>
static constexpr size_t near32m_smem()
{
    return 768 * sizeof(float4) + 8 * NR * 32 * sizeof(float2) + 8 * 2 * NR * 32 * sizeof(double);
}

template <int NR>
static int near_multi_launch(pb_ctx* c, const float2* dens, double* ys, double eps, int nvalid)
{
    const PbLevel& lv = c->lev[c->L];
    PB_CUDA(c, cudaFuncSetAttribute(k_near32m<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)near32m_smem<NR>()));
    k_near32m<NR><<<(c->near_mitems * 32 + 255) / 256, 256, near32m_smem<NR>(), c->st>>>(
        c->nt, c->near_mitems, c->near_mitem, c->near_mtiles, c->chunk_leaf, c->chunk_first, lv.begin, c->e32p,
        c->e32n, c->e32l, dens, eps, c->prm.kappa, ys, nvalid);
    PB_LAUNCH(c);
    return PB_OK;
}

// directed tiles for the several-vector kernel: every chunk of every neighbour leaf, cut into
// work items of at most NEAR_ITEM_M tiles of one target chunk
static int near_multi_items(pb_ctx* c)
{
    const PbLevel& lv = c->lev[c->L];
    const std::vector<int>& b = c->h_leaf_begin;
    const std::vector<int>& no = c->h_near_off;
    const std::vector<int>& ni = c->h_near_idx;
    std::vector<int> first_chunk(lv.ncl + 1, 0);
    for (int k = 0; k < lv.ncl; ++k) first_chunk[k + 1] = first_chunk[k] + (b[k + 1] - b[k] + 31) / 32;
    std::vector<int>& tm = c->h_up_i[5];
    std::vector<int4>& im = c->h_up_i4m;
    tm.clear();
    im.clear();
    for (int k = 0; k < lv.ncl; ++k)
        for (int a = first_chunk[k]; a < first_chunk[k + 1]; ++a) {
            int start = (int)tm.size();
            for (int t = no[k]; t < no[k + 1]; ++t)
                for (int bq = first_chunk[ni[t]]; bq < first_chunk[ni[t] + 1]; ++bq) {
                    tm.push_back(bq);
                    if ((int)tm.size() - start == NEAR_ITEM_M) {
                        im.push_back(make_int4(a, start, (int)tm.size(), 0));
                        start = (int)tm.size();
                    }
                }
            if ((int)tm.size() > start) im.push_back(make_int4(a, start, (int)tm.size(), 0));
        }
    c->near_mitems = (int)im.size();
    c->near_mitem = (int4*)pb_alloc(c, sizeof(int4) * (im.size() + 1));
    c->near_mtiles = (int*)pb_alloc(c, sizeof(int) * (tm.size() + 1));
    if (!c->near_mitem || !c->near_mtiles) return pb_fail(c, PB_ERR_NOMEM, "near setup: out of memory");
    PB_CUDA(c, cudaMemcpyAsync(c->near_mitem, im.data(), sizeof(int4) * im.size(), cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyAsync(c->near_mtiles, tm.data(), sizeof(int) * tm.size(), cudaMemcpyHostToDevice, c->st));
    return PB_OK;
}

// density buffer of the multi-vector near field and its work items (build lifetime, grown on
// demand)
int pb_near_reserve(pb_ctx* c, int nr)
{
    if (c->prm.precision != PB_MIXED || nr < 2) return PB_OK;
    if (!c->near_mitem) {
        int rc = near_multi_items(c);
        if (rc) return rc;
    }
    if (nr <= c->dens_nr) return PB_OK;
    nr = (nr + 15) / 16 * 16;  // groups read whole padded widths
    c->near_dens = (float2*)pb_alloc(c, sizeof(float2) * (size_t)c->nt * nr);
    if (!c->near_dens) return pb_fail(c, PB_ERR_NOMEM, "near field: out of memory");
    c->dens_nr = nr;
    return PB_OK;
}

// nr right-hand sides: xs and ys hold nr vectors of 2 nt; mixed precision evaluates each pair
// once for up to 16 of them, FP64 applies the single-vector kernel per right-hand side
int pb_near_apply_multi(pb_ctx* c, const double* xs, double* ys, int nr)
{
    const int nt = c->nt;
    const double eps = c->prm.eps_out / c->prm.eps_in;
    if (c->prm.precision != PB_MIXED) {
        for (int r = 0; r < nr; ++r) {
            int rc = pb_near_apply(c, xs + 2LL * nt * r, ys + 2LL * nt * r);
            if (rc) return rc;
        }
        return PB_OK;
    }
    int rc0 = pb_near_reserve(c, nr);
    if (rc0) return rc0;
    k_near_dens<<<dim3((nt + 255) / 256, nr), 256, 0, c->st>>>(nt, c->e32p, xs, c->near_dens);
    PB_LAUNCH(c);
    PB_CUDA(c, cudaMemsetAsync(ys, 0, sizeof(double) * 2 * (size_t)nt * nr, c->st));
    // groups of up to 16 right-hand sides, each one launch of the smallest width that holds it
    // (the density buffer is padded to a multiple of 16 vectors)
    for (int r0 = 0; r0 < nr;) {
        const int v = std::min(16, nr - r0);
        const int g = v > 8 ? 16 : v > 4 ? 8 : v > 2 ? 4 : v > 1 ? 2 : 1;
        const float2* d = c->near_dens + (size_t)nt * r0;
        double* y = ys + 2LL * nt * r0;
        const int rc = g == 16  ? near_multi_launch<16>(c, d, y, eps, v)
                       : g == 8 ? near_multi_launch<8>(c, d, y, eps, v)
                       : g == 4 ? near_multi_launch<4>(c, d, y, eps, v)
                       : g == 2 ? near_multi_launch<2>(c, d, y, eps, v)
                                : near_multi_launch<1>(c, d, y, eps, v);
        if (rc) return rc;
        r0 += v;
    }
    k_near_finish<<<dim3((nt + 255) / 256, nr), 256, 0, c->st>>>(nt, c->e64p, xs, eps, ys);
    PB_LAUNCH(c);
    return PB_OK;
}

// ---------- the near field on the points of a regular rule (mixed precision) ----------
// The same pair-tile kernel over the q2 points of every element (q2 = 4 or 16), so the order-q
// rule's near field (both bases) runs at the element kernel's rate: point chunks of 32 within
// each leaf's point range, the tiles of the element plan's neighbour lists, FP32 hi/lo point
// records built once per build.
__global__ void k_pts32(long long np, const double4_32a* __restrict__ pp, const double4_32a* __restrict__ pn,
                        float4* __restrict__ p32, float4* __restrict__ l32, float4* __restrict__ n32)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double4_32a x = pp[p], n = pn[p];
    const float hx = (float)x.x, hy = (float)x.y, hz = (float)x.z;
    p32[p] = make_float4(hx, hy, hz, (float)x.w);
    l32[p] = make_float4((float)(x.x - (double)hx), (float)(x.y - (double)hy), (float)(x.z - (double)hz), 0.f);
    n32[p] = make_float4((float)n.x, (float)n.y, (float)n.z, 0.f);
}

// point records with densities: W_p times the point's values, from the element values xs
// (piecewise constant: every point of element p / q2) or from per-point values xq
__global__ void k_pts_pack(long long np, int q2, int nt, const float4* __restrict__ p32, const float4* __restrict__ n32,
                           const double4_32a* __restrict__ pp, const double* __restrict__ xs,
                           const double* __restrict__ xq, float4* __restrict__ sp, float4* __restrict__ sn)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double W = pp[p].w;
    double u1, u2;
    if (xq) {
        u1 = xq[p];
        u2 = xq[np + p];
    } else {
        const int k = (int)(p / q2);
        u1 = xs[k];
        u2 = xs[nt + k];
    }
    const float4 a = p32[p], b = n32[p];
    sp[p] = make_float4(a.x, a.y, a.z, (float)(W * u1));
    sn[p] = make_float4(b.x, b.y, b.z, (float)(W * u2));
}

// ys[k] = mass - sum over element k's points of W_a y_a (both halves), y the point sums
__global__ void k_pts_finish_elem(int nt, int q2, const double4_32a* __restrict__ ep,
                                  const double4_32a* __restrict__ pp, const double* __restrict__ xs,
                                  const double* __restrict__ ypt, double eps, double* __restrict__ ys)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const long long np = (long long)nt * q2;
    double s1 = 0.0, s2 = 0.0;
    for (int a = 0; a < q2; ++a) {
        const long long p = (long long)k * q2 + a;
        const double W = pp[p].w;
        s1 += W * ypt[p];
        s2 += W * ypt[np + p];
    }
    const double A = ep[k].w;
    ys[k] = 0.5 * (1.0 + eps) * A * xs[k] - s1;
    ys[nt + k] = 0.5 * (1.0 + 1.0 / eps) * A * xs[nt + k] - s2;
}

bool pb_near_points_ok(const pb_ctx* c) { return c->prm.precision == PB_MIXED && (c->q2 == 4 || c->q2 == 16); }

int pb_near_points_setup(pb_ctx* c)
{
    if (!pb_near_points_ok(c)) return PB_OK;
    const PbLevel& lv = c->lev[c->L];
    const int q2 = c->q2;
    const long long np = (long long)c->nt * q2;
    const std::vector<int>& b = c->h_leaf_begin;
    std::vector<int> cl, cf, tl;
    std::vector<int4> it;
    std::vector<int> first_chunk(lv.ncl + 1, 0);
    for (int k = 0; k < lv.ncl; ++k) {
        const long long s0 = (long long)b[k] * q2, s1 = (long long)b[k + 1] * q2;
        for (long long s = s0; s < s1; s += 32) {
            cl.push_back(k);
            cf.push_back((int)s);
        }
        first_chunk[k + 1] = (int)cl.size();
    }
    const std::vector<int>& no = c->h_near_off;
    const std::vector<int>& ni = c->h_near_idx;
    for (int k = 0; k < lv.ncl; ++k)
        for (int a = first_chunk[k]; a < first_chunk[k + 1]; ++a) {
            int start = (int)tl.size();
            for (int t = no[k]; t < no[k + 1]; ++t) {
                const int c2 = ni[t];
                if (c2 < k) continue;
                for (int bq = (c2 == k ? a : first_chunk[c2]); bq < first_chunk[c2 + 1]; ++bq) {
                    tl.push_back(bq);
                    if ((int)tl.size() - start == NEAR_ITEM) {
                        it.push_back(make_int4(a, start, (int)tl.size(), 0));
                        start = (int)tl.size();
                    }
                }
            }
            if ((int)tl.size() > start) it.push_back(make_int4(a, start, (int)tl.size(), 0));
        }
    c->pn_nitems = (int)it.size();
    c->h_pn_i[0].swap(cl);
    c->h_pn_i[1].swap(cf);
    c->h_pn_i[2].swap(tl);
    c->h_pn_i4.swap(it);
    c->pn_items = (int4*)pb_alloc(c, sizeof(int4) * (c->h_pn_i4.size() + 1));
    c->pn_tiles = (int*)pb_alloc(c, sizeof(int) * (c->h_pn_i[2].size() + 1));
    c->pn_chunk_leaf = (int*)pb_alloc(c, sizeof(int) * (c->h_pn_i[0].size() + 1));
    c->pn_chunk_first = (int*)pb_alloc(c, sizeof(int) * (c->h_pn_i[1].size() + 1));
    c->pn_begin = (int*)pb_alloc(c, sizeof(int) * (lv.ncl + 1));
    c->pn_p32 = (float4*)pb_alloc(c, sizeof(float4) * np);
    c->pn_l32 = (float4*)pb_alloc(c, sizeof(float4) * np);
    c->pn_n32 = (float4*)pb_alloc(c, sizeof(float4) * np);
    c->pn_sp = (float4*)pb_alloc(c, sizeof(float4) * np);
    c->pn_sn = (float4*)pb_alloc(c, sizeof(float4) * np);
    c->pn_y = (double*)pb_alloc(c, sizeof(double) * 2 * np);
    if (!c->pn_items || !c->pn_tiles || !c->pn_chunk_leaf || !c->pn_chunk_first || !c->pn_begin || !c->pn_p32 ||
        !c->pn_l32 || !c->pn_n32 || !c->pn_sp || !c->pn_sn || !c->pn_y)
        return pb_fail(c, PB_ERR_NOMEM, "point near field: out of memory");
    // (the host vectors live in the context until the next build: no synchronisation needed)
    PB_CUDA(c, cudaMemcpyAsync(c->pn_items, c->h_pn_i4.data(), sizeof(int4) * c->h_pn_i4.size(),
                               cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyAsync(c->pn_tiles, c->h_pn_i[2].data(), sizeof(int) * c->h_pn_i[2].size(),
                               cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyAsync(c->pn_chunk_leaf, c->h_pn_i[0].data(), sizeof(int) * c->h_pn_i[0].size(),
                               cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyAsync(c->pn_chunk_first, c->h_pn_i[1].data(), sizeof(int) * c->h_pn_i[1].size(),
                               cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyAsync(c->pn_begin, c->begin_q, sizeof(int) * (lv.ncl + 1), cudaMemcpyDeviceToDevice, c->st));
    k_pts32<<<(unsigned)((np + 255) / 256), 256, 0, c->st>>>(np, c->pts_p, c->pts_n, c->pn_p32, c->pn_l32, c->pn_n32);
    PB_LAUNCH(c);
    return PB_OK;
}

// ypt (2 np) = per point sum over the near points of other elements of K (W u), in FP64; the
// densities from element values xs or point values xq (one of them null)
int pb_near_points_apply(pb_ctx* c, const double* xs, const double* xq, double* ypt)
{
    const long long np = (long long)c->nt * c->q2;
    const double eps = c->prm.eps_out / c->prm.eps_in;
    k_pts_pack<<<(unsigned)((np + 255) / 256), 256, 0, c->st>>>(np, c->q2, c->nt, c->pn_p32, c->pn_n32, c->pts_p, xs,
                                                                 xq, c->pn_sp, c->pn_sn);
    PB_LAUNCH(c);
    PB_CUDA(c, cudaMemsetAsync(ypt, 0, sizeof(double) * 2 * np, c->st));
    const unsigned nb = (unsigned)(((long long)c->pn_nitems * 32 + 255) / 256);
    if (c->q2 == 4)
        k_near_tile<4><<<nb, 256, 0, c->st>>>((int)np, c->pn_nitems, c->pn_items, c->pn_tiles, c->pn_chunk_leaf,
                                               c->pn_chunk_first, c->pn_begin, c->pn_sp, c->pn_sn, c->pn_l32, eps,
                                               c->prm.kappa, ypt);
    else
        k_near_tile<16><<<nb, 256, 0, c->st>>>((int)np, c->pn_nitems, c->pn_items, c->pn_tiles, c->pn_chunk_leaf,
                                                c->pn_chunk_first, c->pn_begin, c->pn_sp, c->pn_sn, c->pn_l32, eps,
                                                c->prm.kappa, ypt);
    PB_LAUNCH(c);
    return PB_OK;
}

// the piecewise-constant order-q near field with the mass terms from the point tiles
int pb_near_points_elem(pb_ctx* c, const double* xs, double* ys)
{
    int rc;
    if ((rc = pb_near_points_apply(c, xs, nullptr, c->pn_y))) return rc;
    const double eps = c->prm.eps_out / c->prm.eps_in;
    k_pts_finish_elem<<<(c->nt + 255) / 256, 256, 0, c->st>>>(c->nt, c->q2, c->e64p, c->pts_p, xs, c->pn_y, eps, ys);
    PB_LAUNCH(c);
    return PB_OK;
}
