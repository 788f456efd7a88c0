// Preconditioners of Section 2.6 (and the diagonal one Table 4 compares against).
//
// Block-diagonal ("bd"): M keeps the entries of A whose two elements lie in the same cube of
// the designated level -- here the leaf level -- and is zero elsewhere. Permuting the unknowns
// leaf by leaf makes M = diag(M_1, ..., M_nL); each M_c (order [phi of the leaf; dphi of the
// leaf], size m = 2 n_c) is assembled from the same one-point entries and Sauter-Schwab
// corrections as the near field (evaluated in FP64) and inverted once, in place, by
// Gauss-Jordan elimination with partial pivoting. Applying M^-1 is then one dense
// matrix-vector product per leaf, a bandwidth-bound pass instead of two latency-bound
// triangular solves. The inverse is stored and applied in the working precision (FP32 in
// mixed mode): a preconditioner only has to be a fixed linear operator close to A^-1, and
// right-preconditioned GMRES measures convergence on the true residual of A.
//
// Diagonal ("d"): the 2x2 blocks [[A11_ii, A12_ii], [A21_ii, A22_ii]] of every element.
#include <math.h>

#include <algorithm>
#include <vector>

#include "kernels.cuh"
#include "pb_internal.cuh"

#define GJ_T 256
#define GJ_SMEM_BYTES (200 * 1024)
#define PB_PC_BMAX 96  // largest preconditioner block, in elements

// Assemble the block of leaf c, row-major m x m, into minv + moff[c]: the one-point entries
// of every pair (evaluated in the working precision R from FP64 separations) and the mass
// terms, then the Sauter-Schwab corrections of the touching pairs inside the block.
template <class R>
__global__ void k_blk_fill(const int* __restrict__ begin, const long long* __restrict__ moff,
                           const double4_32a* __restrict__ ep, const double4_32a* __restrict__ en,
                           const int* __restrict__ toff, const int* __restrict__ tj,
                           const double* __restrict__ corr, double eps, double kappa, R* __restrict__ minv)
{
    // the block's element records staged once in shared memory (n <= PB_PC_BMAX)
    __shared__ double4_32a sp_[PB_PC_BMAX], sn_[PB_PC_BMAX];
    const int c = blockIdx.x;
    const int b = begin[c], n = begin[c + 1] - begin[c], m = 2 * n;
    R* Mc = minv + moff[c];
    const double inv_eps = 1.0 / eps;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sp_[i] = ep[b + i];
        sn_[i] = en[b + i];
    }
    __syncthreads();
    for (int i = threadIdx.x / 32; i < n; i += blockDim.x / 32) {
        const double4_32a pi = sp_[i], ni = sn_[i];
        for (int j = threadIdx.x & 31; j < n; j += 32) {
            const double4_32a pj = sp_[j], nj = sn_[j];
            R K[4] = {0, 0, 0, 0};
            if (i != j) {
                pb_kernels<R>((R)(pi.x - pj.x), (R)(pi.y - pj.y), (R)(pi.z - pj.z), (R)ni.x, (R)ni.y, (R)ni.z,
                              (R)nj.x, (R)nj.y, (R)nj.z, (R)eps, (R)inv_eps, (R)kappa, K);
                const R aa = (R)(pi.w * pj.w);
                for (int q = 0; q < 4; ++q) K[q] *= aa;
            }
            R m11 = -K[1], m12 = -K[0], m21 = -K[3], m22 = -K[2];
            if (i == j) {
                m11 += (R)(0.5 * (1.0 + eps) * pi.w);
                m22 += (R)(0.5 * (1.0 + inv_eps) * pi.w);
            }
            Mc[(size_t)i * m + j] = m11;
            Mc[(size_t)i * m + n + j] = m12;
            Mc[(size_t)(n + i) * m + j] = m21;
            Mc[(size_t)(n + i) * m + n + j] = m22;
        }
    }
    __syncthreads();
    // corrections: each touching pair of the block once, from the target's list
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int t = toff[b + i]; t < toff[b + i + 1]; ++t) {
            const int j = tj[t] - b;
            if (j < 0 || j >= n) continue;
            const double* cr = corr + 4 * (size_t)t;
            Mc[(size_t)i * m + j] -= (R)cr[1];
            Mc[(size_t)i * m + n + j] -= (R)cr[0];
            Mc[(size_t)(n + i) * m + j] -= (R)cr[3];
            Mc[(size_t)(n + i) * m + n + j] -= (R)cr[2];
        }
}

// In-place Gauss-Jordan inversion with partial pivoting. Blocks with m <= mfit are worked
// on in shared memory; larger ones in place in global memory (L2 resident).
template <class R>
__global__ void __launch_bounds__(GJ_T) k_blk_gj(const int* __restrict__ begin, const long long* __restrict__ moff,
                                                 R* __restrict__ minv, int mcap, int mfit, int* __restrict__ singular)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ R sv[GJ_T];
    __shared__ int si[GJ_T];
    R* colk = (R*)dsm;
    R* rowk = colk + mcap;
    int* perm = (int*)(rowk + mcap);
    R* smat = (R*)(perm + mcap + (mcap & 1)) ;
    const int c = blockIdx.x;
    const int m = 2 * (begin[c + 1] - begin[c]);
    R* g = minv + moff[c];
    const bool in_smem = m <= mfit;
    R* a = in_smem ? smat : g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x / 32, nw = GJ_T / 32;
    if (in_smem)
        for (int t = threadIdx.x; t < m * m; t += GJ_T) a[t] = g[t];
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        R best = R(-1);
        int bi = k;
        for (int i = k + threadIdx.x; i < m; i += GJ_T) {
            R v = fabs(a[(size_t)i * m + k]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            R ov = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            sv[warp] = best;
            si[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < nw; ++q)
                if (sv[q] > sv[0] || (sv[q] == sv[0] && si[q] < si[0])) {
                    sv[0] = sv[q];
                    si[0] = si[q];
                }
        }
        __syncthreads();
        const int p = si[0];
        if (threadIdx.x == 0) perm[k] = p;
        if (p != k)
            for (int j = threadIdx.x; j < m; j += GJ_T) {
                R t = a[(size_t)k * m + j];
                a[(size_t)k * m + j] = a[(size_t)p * m + j];
                a[(size_t)p * m + j] = t;
            }
        __syncthreads();
        R piv = a[(size_t)k * m + k];
        if (!(fabs(piv) > R(0))) {
            if (threadIdx.x == 0) atomicExch(singular, 1);
            piv = R(1);
        }
        const R ip = R(1) / piv;
        for (int j = threadIdx.x; j < m; j += GJ_T) {
            R v = (j == k) ? ip : a[(size_t)k * m + j] * ip;
            rowk[j] = v;
            colk[j] = a[(size_t)j * m + k];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += GJ_T) a[(size_t)k * m + j] = rowk[j];
        for (int i = warp; i < m; i += nw) {
            if (i == k) continue;
            const R f = colk[i];
            R* ai = a + (size_t)i * m;
            for (int j = lane; j < m; j += 32) ai[j] = (j == k ? R(0) : ai[j]) - f * rowk[j];
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, in reverse order
    for (int i = threadIdx.x; i < m; i += GJ_T) {
        R* ai = a + (size_t)i * m;
        for (int k = m - 1; k >= 0; --k) {
            int p = perm[k];
            if (p != k) {
                R t = ai[k];
                ai[k] = ai[p];
                ai[p] = t;
            }
        }
    }
    __syncthreads();
    if (in_smem)
        for (int t = threadIdx.x; t < m * m; t += GJ_T) g[t] = a[t];
}

// Register-resident Gauss-Jordan inversion by pivot exchanges (FP32, m <= 32 MA and m <= 8 MB),
// laid out so that a column belongs to one warp: lane l of warp w holds rows l + 32 a (a < MA)
// of columns w + 8 b (b < MB). Step k: the warp owning column k finds the pivot row p (the
// unused row of largest |entry|) with warp shuffles and publishes the column, p and the pivot
// to shared memory -- the step's only barrier follows -- and every warp takes row p of its own
// columns from the lane holding it by a shuffle, then applies the exchange
//   T[p][k] <- 1/a, T[p][j] <- -T[p][j]/a, T[i][k] <- T[i][k]/a, T[i][j] -= T[i][k] T[p][j]/a.
// After m exchanges T[p_k][k'] = (A^-1)[k][p_k'], which the final store applies.
template <int MA, int MB, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_blk_gj_w(const int* __restrict__ ids, const int* __restrict__ begin,
                                                       const long long* __restrict__ moff, float* __restrict__ minv,
                                                       int* __restrict__ singular)
{
    __shared__ float colb[2][32 * MA], pivv[2];
    __shared__ int pivs[2], perm[32 * MA], inv[32 * MA];
    const int c = ids[blockIdx.x];
    const int m = 2 * (begin[c + 1] - begin[c]);
    float* g = minv + moff[c];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float v[MA][MB];
#pragma unroll
    for (int a = 0; a < MA; ++a)
#pragma unroll
        for (int b = 0; b < MB; ++b) {
            const int i = lane + 32 * a, j = warp + NW * b;
            v[a][b] = (i < m && j < m) ? g[(size_t)i * m + j] : 0.f;
        }
    unsigned used = 0;  // bit a: row lane + 32 a has been a pivot row
#pragma unroll
    for (int kb = 0; kb < MB; ++kb) {
        for (int kw = 0; kw < NW; ++kw) {
            const int k = NW * kb + kw;
            if (k >= m) break;
            const int s = k & 1;
            if (warp == kw) {
                float best = -1.f;
                int bi = 0x7fffffff;
#pragma unroll
                for (int a = 0; a < MA; ++a) {
                    const int i = lane + 32 * a;
                    const float x = v[a][kb];
                    if (i < m) {
                        colb[s][i] = x;
                        float ax = fabsf(x);
                        if (!(ax >= 0.f)) ax = 0.f;  // a NaN still yields a valid (singular) pivot row
                        if (!((used >> a) & 1u) && ax > best) {
                            best = ax;
                            bi = i;
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                }
                if (lane == (bi & 31)) {
                    // the lane holding the pivot row publishes it and its entry in column k
                    float pv = 0.f;
#pragma unroll
                    for (int a = 0; a < MA; ++a)
                        if (lane + 32 * a == bi) pv = v[a][kb];
                    pivs[s] = bi;
                    pivv[s] = pv;
                }
            }
            __syncthreads();
            const int p = pivs[s];
            float piv = pivv[s];
            if (threadIdx.x == 0) {
                perm[k] = p;
                inv[p] = k;
                if (!(fabsf(piv) > 0.f)) atomicExch(singular, 1);
            }
            if (!(fabsf(piv) > 0.f)) piv = 1.f;
            const float ia = 1.f / piv;
            const int pa = p >> 5, pl = p & 31;
            if (lane == pl) used |= 1u << pa;
            // row p of this warp's columns, from the lane that holds it
            float rk[MB];
#pragma unroll
            for (int b = 0; b < MB; ++b) {
                float x = v[0][b];
#pragma unroll
                for (int a = 1; a < MA; ++a)
                    if (a == pa) x = v[a][b];
                rk[b] = __shfl_sync(0xffffffffu, x, pl) * ia;
            }
            const bool ownk = warp == kw;
#pragma unroll
            for (int a = 0; a < MA; ++a) {
                const int i = lane + 32 * a;
                if (i == p) {
#pragma unroll
                    for (int b = 0; b < MB; ++b) v[a][b] = (b == kb && ownk) ? ia : -v[a][b] * ia;
                } else {
                    const float ck = i < m ? colb[s][i] : 0.f;
#pragma unroll
                    for (int b = 0; b < MB; ++b)
                        v[a][b] = (b == kb && ownk) ? ck * ia : fmaf(-ck, rk[b], v[a][b]);
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < MA; ++a)
#pragma unroll
        for (int b = 0; b < MB; ++b) {
            const int i = lane + 32 * a, j = warp + NW * b;
            if (i < m && j < m) g[(size_t)inv[i] * m + perm[j]] = v[a][b];
        }
}

// z = M^-1 r per leaf: the block's slice of r staged once in shared memory (in the working
// precision), then one warp per row (FP32: two rows) with lanes striding the columns
template <class R>
__global__ void k_blk_apply(int nt, const int* __restrict__ begin, const long long* __restrict__ moff,
                            const R* __restrict__ minv, const double* __restrict__ r, double* __restrict__ z,
                            long long rstr, long long zstr)
{
    __shared__ __align__(16) R rv[2 * PB_PC_BMAX];
    r += blockIdx.y * rstr;  // right-hand side blockIdx.y
    z += blockIdx.y * zstr;
    const int c = blockIdx.x;
    const int b = begin[c], n = begin[c + 1] - begin[c], m = 2 * n;
    const R* Mc = minv + moff[c];
    for (int j = threadIdx.x; j < m; j += blockDim.x) rv[j] = (R)(j < n ? r[b + j] : r[nt + b + j - n]);
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31, nw = blockDim.x / 32;
    if constexpr (sizeof(R) == sizeof(float)) {
        // m is even and every block starts at a multiple of 4 entries (the orders m^2 of the
        // blocks before it are multiples of 4): rows and the staged slice read in pairs; two rows
        // per warp at a time, so that twice the loads are in flight
        const float2* rv2 = reinterpret_cast<const float2*>(rv);
        for (int i = warp; i < m; i += 2 * nw) {
            const int i2 = i + nw;
            const bool two = i2 < m;
            const float2* row = reinterpret_cast<const float2*>(Mc + (size_t)i * m);
            const float2* row2 = reinterpret_cast<const float2*>(Mc + (size_t)(two ? i2 : i) * m);
            float s = 0.f, s2 = 0.f;
            for (int j = lane; j < m / 2; j += 32) {
                const float2 a = row[j], a2 = row2[j], v = rv2[j];
                s += a.x * v.x + a.y * v.y;
                s2 += a2.x * v.x + a2.y * v.y;
            }
            for (int o = 16; o > 0; o >>= 1) {
                s += __shfl_xor_sync(0xffffffffu, s, o);
                s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            }
            if (lane == 0) {
                if (i < n) z[b + i] = (double)s;
                else z[nt + b + i - n] = (double)s;
                if (two) {
                    if (i2 < n) z[b + i2] = (double)s2;
                    else z[nt + b + i2 - n] = (double)s2;
                }
            }
        }
        return;
    }
    for (int i = warp; i < m; i += nw) {
        R s = 0;
        for (int j = lane; j < m; j += 32) s += Mc[(size_t)i * m + j] * rv[j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (i < n) z[b + i] = (double)s;
            else z[nt + b + i - n] = (double)s;
        }
    }
}

// The same for up to 16 right-hand sides at once (q0 = 16 blockIdx.y, nq of them): each block
// row is read once for all of them. The vectors' slices sit in shared memory as rv[j][q]; lane
// (h, q) of a warp sums column parity h of row i for vector q (lanes of one half read the same
// matrix entry, and the two halves hit different banks), then the halves are added.
template <class R>
__global__ void k_blk_apply_m(int nt, const int* __restrict__ begin, const long long* __restrict__ moff,
                              const R* __restrict__ minv, const double* __restrict__ r, double* __restrict__ z,
                              long long rstr, long long zstr, int nr)
{
    __shared__ R rv[2 * PB_PC_BMAX * 16];
    const int q0 = 16 * blockIdx.y, nq = min(16, nr - q0);
    const int c = blockIdx.x;
    const int b = begin[c], n = begin[c + 1] - begin[c], m = 2 * n;
    const R* Mc = minv + moff[c];
    for (int t = threadIdx.x; t < m * 16; t += blockDim.x) {
        const int j = t >> 4, q = t & 15;
        const double* rq = r + (long long)(q0 + q) * rstr;
        rv[t] = q < nq ? (R)(j < n ? rq[b + j] : rq[nt + b + j - n]) : R(0);
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31, nw = blockDim.x / 32;
    const int h = lane >> 4, q = lane & 15;
    for (int i = warp; i < m; i += nw) {
        const R* row = Mc + (size_t)i * m;
        R s = 0;
        for (int j = h; j < m; j += 2) s += row[j] * rv[j * 16 + q];
        s += __shfl_xor_sync(0xffffffffu, s, 16);
        if (h == 0 && q < nq) {
            double* zq = z + (long long)(q0 + q) * zstr;
            if (i < n) zq[b + i] = (double)s;
            else zq[nt + b + i - n] = (double)s;
        }
    }
}

// 2x2 element blocks (diagonal preconditioner): uses the (i, i) correction entry
__global__ void k_diag_build(int nt, const double4_32a* __restrict__ ep, const int* __restrict__ toff,
                             const int* __restrict__ tj, const double* __restrict__ corr, double eps,
                             double* __restrict__ dinv)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    double I[4] = {0, 0, 0, 0};
    for (int t = toff[k]; t < toff[k + 1]; ++t)
        if (tj[t] == k)
            for (int q = 0; q < 4; ++q) I[q] = corr[4 * t + q];
    double A = ep[k].w;
    double a11 = 0.5 * (1.0 + eps) * A - I[1], a12 = -I[0], a21 = -I[3], a22 = 0.5 * (1.0 + 1.0 / eps) * A - I[2];
    double det = a11 * a22 - a12 * a21;
    dinv[4 * k] = a22 / det;
    dinv[4 * k + 1] = -a12 / det;
    dinv[4 * k + 2] = -a21 / det;
    dinv[4 * k + 3] = a11 / det;
}

__global__ void k_diag_apply(int nt, const double* __restrict__ dinv, const double* __restrict__ r,
                             double* __restrict__ z, long long rstr, long long zstr)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    r += blockIdx.y * rstr;
    z += blockIdx.y * zstr;
    double a = r[k], b = r[nt + k];
    z[k] = dinv[4 * k] * a + dinv[4 * k + 1] * b;
    z[nt + k] = dinv[4 * k + 2] * a + dinv[4 * k + 3] * b;
}

template <class R>
static int blk_build(pb_ctx* c, const long long* dmoff, long long ntot, int mcap, int ncl)
{
    double eps = c->prm.eps_out / c->prm.eps_in;
    R* M = (R*)pb_alloc(c, sizeof(R) * (size_t)ntot);
    int* sing = (int*)pb_alloc(c, sizeof(int));
    if (!M || !sing) return pb_fail(c, PB_ERR_NOMEM, "precond: out of memory");
    c->minv = M;
    k_blk_fill<R><<<ncl, 256, 0, c->st>>>(c->pc_begin, dmoff, c->e64p, c->e64n, c->touch_off, c->touch_j, c->corr, eps,
                                           c->prm.kappa, M);
    PB_LAUNCH(c);
    if (sizeof(R) == 4 && mcap <= 192) {
        // one launch per size class, each with a register tile that just covers its blocks
        const int* ids = c->pc_ids;
        const int* cl = c->pc_cls;
        if (cl[1] > cl[0]) {
            k_blk_gj_w<2, 8, 8, 4><<<cl[1] - cl[0], 256, 0, c->st>>>(ids + cl[0], c->pc_begin, dmoff, (float*)M, sing);
            PB_LAUNCH(c);
        }
        if (cl[2] > cl[1]) {
            k_blk_gj_w<4, 8, 16, 2><<<cl[2] - cl[1], 512, 0, c->st>>>(ids + cl[1], c->pc_begin, dmoff, (float*)M, sing);
            PB_LAUNCH(c);
        }
        if (cl[3] > cl[2]) {
            k_blk_gj_w<6, 12, 16, 1><<<cl[3] - cl[2], 512, 0, c->st>>>(ids + cl[2], c->pc_begin, dmoff, (float*)M, sing);
            PB_LAUNCH(c);
        }
        int hs = 0;
        PB_CUDA(c, cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
        if (hs) return pb_fail(c, PB_ERR_MESH, "a preconditioner block is singular");
        return PB_OK;
    }
    // shared memory: col, row, perm (mcap each) + the block itself when it fits
    size_t fixed = sizeof(R) * 2 * (size_t)mcap + sizeof(int) * ((size_t)mcap + 1) + 16;
    int mfit = 0;
    while ((size_t)(mfit + 1) * (mfit + 1) * sizeof(R) + fixed <= GJ_SMEM_BYTES) ++mfit;
    size_t smem = fixed + (size_t)std::min(mfit, mcap) * std::min(mfit, mcap) * sizeof(R);
    PB_CUDA(c, cudaFuncSetAttribute(k_blk_gj<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_blk_gj<R><<<ncl, GJ_T, smem, c->st>>>(c->pc_begin, dmoff, M, mcap, std::min(mfit, mcap), sing);
    PB_LAUNCH(c);
    int hs = 0;
    PB_CUDA(c, cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    if (hs) return pb_fail(c, PB_ERR_MESH, "a preconditioner block is singular");
    return PB_OK;
}

// The block partition, from the leaf ranges the tree build read back to the host.
int pb_precond_plan(pb_ctx* c)
{
    const int nt = c->nt;
    if (c->prm.precond != PB_PRECOND_BLOCK) return PB_OK;
    // blocks: the leaves of the tree; a leaf with more than bmax elements (pc_block, at most
    // PB_PC_BMAX) is split into nearly equal consecutive (Morton-ordered) parts of at most bmax
    const PbLevel& lv = c->lev[c->L];
    const std::vector<int>& hb = c->h_leaf_begin;
    std::vector<int>& pb_ = c->h_up_i[2];
    const int bmax = c->prm.pc_block > 0 ? std::min(c->prm.pc_block, PB_PC_BMAX) : PB_PC_BMAX;
    pb_.clear();
    for (int k = 0; k < lv.ncl; ++k) {
        int n = hb[k + 1] - hb[k];
        int parts = (n + bmax - 1) / bmax;
        int base = n / parts, extra = n % parts, s = hb[k];
        for (int q = 0; q < parts; ++q) {
            pb_.push_back(s);
            s += base + (q < extra ? 1 : 0);
        }
    }
    pb_.push_back(nt);
    const int nb = (int)pb_.size() - 1;
    std::vector<long long>& moff = c->h_up_l;
    moff.assign(nb + 1, 0);
    moff[0] = 0;
    int mcap = 0;
    for (int k = 0; k < nb; ++k) {
        long long m = 2LL * (pb_[k + 1] - pb_[k]);
        moff[k + 1] = moff[k] + m * m;
        mcap = std::max(mcap, (int)m);
    }
    c->npcblk = nb;
    c->pc_max = mcap;
    c->pc_sum_m3 = 0;
    for (int k = 0; k < nb; ++k) {
        const double m = 2.0 * (pb_[k + 1] - pb_[k]);
        c->pc_sum_m3 += m * m * m;
    }
    // size classes of the FP32 register-tile inversion: order <= 64, <= 128, larger
    std::vector<int>& ids = c->h_up_i[3];
    ids.clear();
    const int lim[3] = {64, 128, 1 << 30};
    for (int q = 0; q < 3; ++q) {
        c->pc_cls[q] = (int)ids.size();
        for (int k = 0; k < nb; ++k) {
            const int m = 2 * (pb_[k + 1] - pb_[k]);
            if (m <= lim[q] && (q == 0 || m > lim[q - 1])) ids.push_back(k);
        }
        // largest blocks first, so that the last wave of a class holds the shortest inversions
        std::stable_sort(ids.begin() + c->pc_cls[q], ids.end(), [&](int x, int y) {
            return pb_[x + 1] - pb_[x] > pb_[y + 1] - pb_[y];
        });
    }
    c->pc_cls[3] = (int)ids.size();
    c->pc_begin = (int*)pb_alloc(c, sizeof(int) * (nb + 1));
    c->blk_off = (long long*)pb_alloc(c, sizeof(long long) * (nb + 1));
    c->pc_ids = (int*)pb_alloc(c, sizeof(int) * (nb + 1));
    if (!c->blk_off || !c->pc_begin || !c->pc_ids) return pb_fail(c, PB_ERR_NOMEM, "precond: out of memory");
    PB_CUDA(c, cudaMemcpyAsync(c->pc_begin, pb_.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyAsync(c->blk_off, moff.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyAsync(c->pc_ids, ids.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c->st));
    c->pc_total = moff[nb];
    return PB_OK;
}

// Assemble and invert the blocks (or the 2x2 diagonal blocks): needs the singular entries.
int pb_precond_factor(pb_ctx* c)
{
    const int nt = c->nt;
    double eps = c->prm.eps_out / c->prm.eps_in;
    if (c->prm.precond == PB_PRECOND_DIAG) {
        c->dinv = (double*)pb_alloc(c, sizeof(double) * 4 * nt);
        if (!c->dinv) return pb_fail(c, PB_ERR_NOMEM, "precond: out of memory");
        k_diag_build<<<(nt + 255) / 256, 256, 0, c->st>>>(nt, c->e64p, c->touch_off, c->touch_j, c->corr, eps, c->dinv);
        PB_LAUNCH(c);
        return PB_OK;
    }
    if (c->prm.precond != PB_PRECOND_BLOCK) return PB_OK;
    return c->prm.precision == PB_MIXED ? blk_build<float>(c, c->blk_off, c->pc_total, c->pc_max, c->npcblk)
                                        : blk_build<double>(c, c->blk_off, c->pc_total, c->pc_max, c->npcblk);
}

// z_q = M^-1 r_q for nr vectors r_q = r + q rstr, z_q = z + q zstr
int pb_precond_apply_multi(pb_ctx* c, const double* r, long long rstr, double* z, long long zstr, int nr)
{
    if (c->prm.basis == PB_BASIS_LINEAR) {
        for (int q = 0; q < nr; ++q) {
            int rc = pb_p1_precond(c, r + q * rstr, z + q * zstr);
            if (rc) return rc;
        }
        return PB_OK;
    }
    const int nt = c->nt;
    pb_tic(c, PB_T_PRECOND);
    if (c->prm.precond == PB_PRECOND_BLOCK) {
        const dim3 gm(c->npcblk, (nr + 15) / 16);
        if (c->prm.precision == PB_MIXED) {
            if (nr == 1)
                k_blk_apply<float><<<c->npcblk, 256, 0, c->st>>>(nt, c->pc_begin, c->blk_off, (const float*)c->minv,
                                                                 r, z, rstr, zstr);
            else
                k_blk_apply_m<float><<<gm, 256, 0, c->st>>>(nt, c->pc_begin, c->blk_off, (const float*)c->minv, r,
                                                            z, rstr, zstr, nr);
        } else {
            if (nr == 1)
                k_blk_apply<double><<<c->npcblk, 256, 0, c->st>>>(nt, c->pc_begin, c->blk_off,
                                                                  (const double*)c->minv, r, z, rstr, zstr);
            else
                k_blk_apply_m<double><<<gm, 256, 0, c->st>>>(nt, c->pc_begin, c->blk_off,
                                                             (const double*)c->minv, r, z, rstr, zstr, nr);
        }
    } else if (c->prm.precond == PB_PRECOND_DIAG) {
        k_diag_apply<<<dim3((nt + 255) / 256, nr), 256, 0, c->st>>>(nt, c->dinv, r, z, rstr, zstr);
    } else {
        for (int q = 0; q < nr; ++q)
            PB_CUDA(c, cudaMemcpyAsync(z + q * zstr, r + q * rstr, sizeof(double) * 2 * nt, cudaMemcpyDeviceToDevice,
                                       c->st));
        pb_toc(c, PB_T_PRECOND);
        return PB_OK;
    }
    PB_LAUNCH(c);
    pb_toc(c, PB_T_PRECOND);
    return PB_OK;
}

int pb_precond_apply_sorted(pb_ctx* c, const double* r, double* z)
{
    if (c->prm.basis == PB_BASIS_LINEAR) return pb_p1_precond(c, r, z);
    return pb_precond_apply_multi(c, r, 0, z, 0, 1);
}
