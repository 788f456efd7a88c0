// Preconditioners of Section 2.6 (and the diagonal one Table 4 compares against).
//
// Block-diagonal ("bd"): M keeps the entries of A whose two elements lie in the same cube of
// the designated level -- here the leaf level -- and is zero elsewhere. Permuting the unknowns
// leaf by leaf makes M = diag(M_1, ..., M_nL); each M_c (order [phi of the leaf; dphi of the
// leaf], size 2 n_c) is assembled in FP64 from the same one-point entries and Sauter-Schwab
// corrections as the near field, and inverted once by Gauss-Jordan elimination with partial
// pivoting. Applying M^-1 is then one dense matrix-vector product per leaf, a bandwidth-bound
// pass instead of two latency-bound triangular solves.
//
// Diagonal ("d"): the 2x2 blocks [[A11_ii, A12_ii], [A21_ii, A22_ii]] of every element.
#include <math.h>

#include <vector>

#include "kernels.cuh"
#include "pb_internal.cuh"

// Assemble the block of leaf c into W (2n rows, 4n columns: [M | I]).
__global__ void k_blk_fill(const int* __restrict__ begin, const long long* __restrict__ woff,
                           const double4_32a* __restrict__ ep, const double4_32a* __restrict__ en,
                           const int* __restrict__ toff, const int* __restrict__ tj,
                           const double* __restrict__ corr, double eps, double kappa, double* __restrict__ W)
{
    const int c = blockIdx.x;
    const int b = begin[c], n = begin[c + 1] - begin[c], m = 2 * n, ld = 4 * n;
    double* Wc = W + woff[c];
    const double inv_eps = 1.0 / eps;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        int i = (int)(t / n), j = (int)(t % n);
        double4_32a pi = ep[b + i], pj = ep[b + j], ni = en[b + i], nj = en[b + j];
        double I[4] = {0, 0, 0, 0};
        if (i != j) {
            double K[4];
            pb_kernels<double>(pi.x - pj.x, pi.y - pj.y, pi.z - pj.z, ni.x, ni.y, ni.z, nj.x, nj.y, nj.z, eps,
                               inv_eps, kappa, K);
            for (int q = 0; q < 4; ++q) I[q] = pi.w * pj.w * K[q];
        }
        Wc[(size_t)i * ld + j] = -I[1];
        Wc[(size_t)i * ld + n + j] = -I[0];
        Wc[(size_t)(n + i) * ld + j] = -I[3];
        Wc[(size_t)(n + i) * ld + n + j] = -I[2];
        Wc[(size_t)i * ld + m + j] = (i == j);
        Wc[(size_t)i * ld + m + n + j] = 0.0;
        Wc[(size_t)(n + i) * ld + m + j] = 0.0;
        Wc[(size_t)(n + i) * ld + m + n + j] = (i == j);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double A = ep[b + i].w;
        Wc[(size_t)i * ld + i] += 0.5 * (1.0 + eps) * A;
        Wc[(size_t)(n + i) * ld + n + i] += 0.5 * (1.0 + inv_eps) * A;
        for (int t = toff[b + i]; t < toff[b + i + 1]; ++t) {
            int j = tj[t] - b;
            if (j < 0 || j >= n) continue;
            Wc[(size_t)i * ld + j] -= corr[4 * t + 1];
            Wc[(size_t)i * ld + n + j] -= corr[4 * t];
            Wc[(size_t)(n + i) * ld + j] -= corr[4 * t + 3];
            Wc[(size_t)(n + i) * ld + n + j] -= corr[4 * t + 2];
        }
    }
}

// Gauss-Jordan with partial pivoting on [M | I] -> [I | M^-1]; copies M^-1 to minv.
__global__ void __launch_bounds__(256) k_blk_invert(const int* __restrict__ begin, const long long* __restrict__ woff,
                                                    const long long* __restrict__ moff, double* __restrict__ W,
                                                    double* __restrict__ minv, int* __restrict__ singular)
{
    __shared__ double sv[256];
    __shared__ int si[256];
    __shared__ double prow_scale;
    const int c = blockIdx.x;
    const int n = begin[c + 1] - begin[c], m = 2 * n, ld = 4 * n;
    double* Wc = W + woff[c];
    for (int k = 0; k < m; ++k) {
        // pivot search in column k, rows k..m-1
        double best = -1.0;
        int bi = k;
        for (int i = k + threadIdx.x; i < m; i += blockDim.x) {
            double v = fabs(Wc[(size_t)i * ld + k]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        sv[threadIdx.x] = best;
        si[threadIdx.x] = bi;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) {
                double o = sv[threadIdx.x + h];
                int oi = si[threadIdx.x + h];
                if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                    sv[threadIdx.x] = o;
                    si[threadIdx.x] = oi;
                }
            }
            __syncthreads();
        }
        const int piv = si[0];
        if (threadIdx.x == 0) {
            double pv = Wc[(size_t)piv * ld + k];
            if (!(fabs(pv) > 0.0)) {
                atomicExch(singular, 1);
                pv = 1.0;
            }
            prow_scale = 1.0 / pv;
        }
        __syncthreads();
        // swap rows k and piv, scale row k
        for (int j = threadIdx.x; j < ld; j += blockDim.x) {
            double a = Wc[(size_t)k * ld + j], b2 = Wc[(size_t)piv * ld + j];
            if (piv != k) Wc[(size_t)piv * ld + j] = a;
            Wc[(size_t)k * ld + j] = b2 * prow_scale;
        }
        __syncthreads();
        // eliminate column k from every other row
        for (long long t = threadIdx.x; t < (long long)m * ld; t += blockDim.x) {
            int i = (int)(t / ld), j = (int)(t % ld);
            if (i == k || j < k) continue;
            double f = Wc[(size_t)i * ld + k];
            if (j == k) continue;
            Wc[(size_t)i * ld + j] -= f * Wc[(size_t)k * ld + j];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            if (i != k) Wc[(size_t)i * ld + k] = 0.0;
        __syncthreads();
    }
    double* Mc = minv + moff[c];
    for (long long t = threadIdx.x; t < (long long)m * m; t += blockDim.x) {
        int i = (int)(t / m), j = (int)(t % m);
        Mc[t] = Wc[(size_t)i * ld + m + j];
    }
}

// z = M^-1 r per leaf: one warp per row, lanes stride the columns
__global__ void k_blk_apply(int nt, const int* __restrict__ begin, const long long* __restrict__ moff,
                            const double* __restrict__ minv, const double* __restrict__ r, double* __restrict__ z)
{
    const int c = blockIdx.x;
    const int b = begin[c], n = begin[c + 1] - begin[c], m = 2 * n;
    const double* Mc = minv + moff[c];
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31, nw = blockDim.x / 32;
    for (int i = warp; i < m; i += nw) {
        double s = 0.0;
        for (int j = lane; j < m; j += 32) {
            double rv = j < n ? r[b + j] : r[nt + b + j - n];
            s += Mc[(size_t)i * m + j] * rv;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (i < n) z[b + i] = s;
            else z[nt + b + i - n] = s;
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
                             double* __restrict__ z)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    double a = r[k], b = r[nt + k];
    z[k] = dinv[4 * k] * a + dinv[4 * k + 1] * b;
    z[nt + k] = dinv[4 * k + 2] * a + dinv[4 * k + 3] * b;
}

int pb_precond_build(pb_ctx* c)
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
    const PbLevel& lv = c->lev[c->L];
    std::vector<int> hb(lv.ncl + 1);
    PB_CUDA(c, cudaMemcpyAsync(hb.data(), lv.begin, sizeof(int) * (lv.ncl + 1), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    std::vector<long long> woff(lv.ncl + 1), moff(lv.ncl + 1);
    woff[0] = moff[0] = 0;
    for (int k = 0; k < lv.ncl; ++k) {
        long long n = hb[k + 1] - hb[k];
        woff[k + 1] = woff[k] + (2 * n) * (4 * n);
        moff[k + 1] = moff[k] + (2 * n) * (2 * n);
    }
    long long* dwoff = (long long*)pb_alloc(c, sizeof(long long) * (lv.ncl + 1));
    c->blk_off = (long long*)pb_alloc(c, sizeof(long long) * (lv.ncl + 1));
    c->minv = (double*)pb_alloc(c, sizeof(double) * moff[lv.ncl]);
    int* sing = (int*)pb_alloc(c, sizeof(int));
    double* W = nullptr;
    if (!dwoff || !c->blk_off || !c->minv || !sing) return pb_fail(c, PB_ERR_NOMEM, "precond: out of memory");
    if (cudaMallocAsync((void**)&W, sizeof(double) * woff[lv.ncl], c->st) != cudaSuccess) {
        cudaGetLastError();
        return pb_fail(c, PB_ERR_NOMEM, "precond: out of memory (work)");
    }
    PB_CUDA(c, cudaMemcpyAsync(dwoff, woff.data(), sizeof(long long) * (lv.ncl + 1), cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyAsync(c->blk_off, moff.data(), sizeof(long long) * (lv.ncl + 1), cudaMemcpyHostToDevice, c->st));
    k_blk_fill<<<lv.ncl, 256, 0, c->st>>>(lv.begin, dwoff, c->e64p, c->e64n, c->touch_off, c->touch_j, c->corr, eps,
                                          c->prm.kappa, W);
    PB_LAUNCH(c);
    k_blk_invert<<<lv.ncl, 256, 0, c->st>>>(lv.begin, dwoff, c->blk_off, W, c->minv, sing);
    PB_LAUNCH(c);
    PB_CUDA(c, cudaFreeAsync(W, c->st));
    int hs = 0;
    PB_CUDA(c, cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    if (hs) return pb_fail(c, PB_ERR_MESH, "a preconditioner block is singular");
    return PB_OK;
}

int pb_precond_apply_sorted(pb_ctx* c, const double* r, double* z)
{
    const int nt = c->nt;
    pb_tic(c, PB_T_PRECOND);
    if (c->prm.precond == PB_PRECOND_BLOCK) {
        const PbLevel& lv = c->lev[c->L];
        k_blk_apply<<<lv.ncl, 256, 0, c->st>>>(nt, lv.begin, c->blk_off, c->minv, r, z);
    } else if (c->prm.precond == PB_PRECOND_DIAG) {
        k_diag_apply<<<(nt + 255) / 256, 256, 0, c->st>>>(nt, c->dinv, r, z);
    } else {
        PB_CUDA(c, cudaMemcpyAsync(z, r, sizeof(double) * 2 * nt, cudaMemcpyDeviceToDevice, c->st));
        pb_toc(c, PB_T_PRECOND);
        return PB_OK;
    }
    PB_LAUNCH(c);
    pb_toc(c, PB_T_PRECOND);
    return PB_OK;
}
