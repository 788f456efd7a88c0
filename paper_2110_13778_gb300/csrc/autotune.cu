// Autotuner of the tree and expansion parameters for one uploaded molecule.
//
// The paper fixes the leaf size and the order by hand for each test (Section 3, "adjust L for
// N"). Here the context tries leaf sizes and orders on the molecule itself: for every
// candidate it builds the tree, times the matrix-vector product with CUDA events, and measures
// its error against a reference product of order 10 on a fixed pseudo-random density; it
// keeps the cheapest candidate (build time + expected products x product time) whose error
// stays within the tolerance; then it lowers the order of single levels, finest first, while
// the error stays within the tolerance and the cost falls, and leaves the context built with
// the result. Products are timed on as many vectors at once as the caller will solve for.
#include <math.h>

#include <algorithm>
#include <vector>

#include "pb_internal.cuh"

__global__ void k_tune_fill(long long n, unsigned long long seed, double* __restrict__ x)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z = z ^ (z >> 31);
        x[i] = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
}

// out[0] += sum (a - b)^2, out[1] += sum b^2
__global__ void k_tune_err(long long n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out)
{
    __shared__ double s0[256], s1[256];
    double e = 0, r = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double d = a[i] - b[i];
        e += d * d;
        r += b[i] * b[i];
    }
    s0[threadIdx.x] = e;
    s1[threadIdx.x] = r;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s0[threadIdx.x] += s0[threadIdx.x + h];
            s1[threadIdx.x] += s1[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&out[0], s0[0]);
        atomicAdd(&out[1], s1[0]);
    }
}

// build with the current parameters; returns the build time in ms through *ms
static int timed_build(pb_ctx* c, cudaEvent_t e0, cudaEvent_t e1, float* ms)
{
    PB_CUDA(c, cudaEventRecord(e0, c->st));
    int rc = pb_build_tree(c);
    if (rc) return rc;
    PB_CUDA(c, cudaEventRecord(e1, c->st));
    PB_CUDA(c, cudaEventSynchronize(e1));
    PB_CUDA(c, cudaEventElapsedTime(ms, e0, e1));
    return PB_OK;
}

// one timed product of nr vectors (X, Y: nr x 2N, element order): the median of three after a
// warm-up
static int timed_products(pb_ctx* c, const double* X, double* Y, int nr, cudaEvent_t e0, cudaEvent_t e1,
                          float* med)
{
    auto prod = [&]() { return nr == 1 ? pb_matvec(c, X, Y) : pb_matvec_multi(c, X, Y, nr); };
    int rc = prod();
    if (rc) return rc;
    float t[3];
    for (int r = 0; r < 3; ++r) {
        PB_CUDA(c, cudaEventRecord(e0, c->st));
        if ((rc = prod())) return rc;
        PB_CUDA(c, cudaEventRecord(e1, c->st));
        PB_CUDA(c, cudaEventSynchronize(e1));
        PB_CUDA(c, cudaEventElapsedTime(&t[r], e0, e1));
    }
    std::sort(t, t + 3);
    *med = t[1];
    return PB_OK;
}

extern "C" int pb_autotune(pb_ctx* c, double tol, int matvecs_per_solve, int nrhs, pb_tune_result* out)
{
    if (!c) return PB_ERR_ARG;
    if (c->dead) return PB_ERR_CUDA;
    if (!c->verts) return pb_fail(c, PB_ERR_STATE, "autotune before mesh_upload");
    if (!(tol > 0) || matvecs_per_solve < 1 || nrhs < 1 || nrhs > PB_MAX_RHS || !out)
        return pb_fail(c, PB_ERR_ARG, "autotune: bad arguments");
    if (c->prm.basis != PB_BASIS_CONSTANT) return pb_fail(c, PB_ERR_ARG, "autotune: piecewise-constant basis only");
    const pb_params keep = c->prm;
    c->p_level_L = -1;  // candidates use one order on every level
    const long long n = 2LL * c->nt;
    double *x = nullptr, *yref = nullptr, *y = nullptr, *acc = nullptr;
    if (cudaMallocFromPoolAsync(&x, sizeof(double) * n * nrhs, c->pool, c->st) != cudaSuccess ||
        cudaMallocFromPoolAsync(&yref, sizeof(double) * n, c->pool, c->st) != cudaSuccess ||
        cudaMallocFromPoolAsync(&y, sizeof(double) * n * nrhs, c->pool, c->st) != cudaSuccess ||
        cudaMallocFromPoolAsync(&acc, sizeof(double) * 2, c->pool, c->st) != cudaSuccess) {
        cudaGetLastError();
        return pb_fail(c, PB_ERR_NOMEM, "autotune: out of memory");
    }
    cudaEvent_t e0, e1;
    PB_CUDA(c, cudaEventCreate(&e0));
    PB_CUDA(c, cudaEventCreate(&e1));
    int rc = PB_OK;
    const int G = (int)std::min<long long>((n + 255) / 256, 1024);
    auto fail = [&](int r) {
        if (r) c->p_level_L = -1;  // a failed tuning leaves no per-level orders behind
        cudaFreeAsync(x, c->st);
        cudaFreeAsync(yref, c->st);
        cudaFreeAsync(y, c->st);
        cudaFreeAsync(acc, c->st);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return r;
    };
    // nrhs pseudo-random vectors in element order; every product goes through the public entry
    // points, and the error is measured on the first vector
    for (int r = 0; r < nrhs; ++r) {
        k_tune_fill<<<G, 256, 0, c->st>>>(n, 0x5EEDULL + 7919ULL * r, x + n * r);
        PB_LAUNCH(c);
    }
    // reference: order 10 at the caller's leaf size
    c->prm.p = 10;
    c->prm.adaptive = 0;
    float ms = 0;
    if ((rc = timed_build(c, e0, e1, &ms)) || (rc = pb_matvec(c, x, yref))) {
        c->prm = keep;
        return fail(rc);
    }
    // relative L2 error of y (first vector) against the reference
    auto rel_err = [&](double* err) -> int {
        PB_CUDA(c, cudaMemsetAsync(acc, 0, sizeof(double) * 2, c->st));
        k_tune_err<<<G, 256, 0, c->st>>>(n, y, yref, acc);
        PB_LAUNCH(c);
        double h[2];
        PB_CUDA(c, cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
        *err = sqrt(h[0] / (h[1] > 0 ? h[1] : 1.0));
        return PB_OK;
    };
    const int leaves[5] = {32, 48, 64, 96, 128};
    const int orders[3] = {4, 6, 8};
    double best_cost = 1e300, best_err = 1e300, best_ms = 0, best_bms = 0;
    int best_leaf = keep.leaf_size, best_p = keep.p, tried = 0;
    bool best_ok = false;
    for (int li = 0; li < 5; ++li) {
        for (int pi = 0; pi < 3; ++pi) {
            c->prm.leaf_size = leaves[li];
            c->prm.levels = 0;
            c->prm.p = orders[pi];
            float bms = 0, t = 0;
            double err = 0;
            if ((rc = timed_build(c, e0, e1, &bms)) || (rc = timed_products(c, x, y, nrhs, e0, e1, &t)) ||
                (rc = rel_err(&err))) {
                c->prm = keep;
                return fail(rc);
            }
            const double cost = bms + (double)matvecs_per_solve * t;
            ++tried;
            const bool ok = err <= tol;
            if ((ok && (!best_ok || cost < best_cost)) || (!ok && !best_ok && err < best_err)) {
                best_ok = ok;
                best_cost = cost;
                best_err = err;
                best_leaf = leaves[li];
                best_p = orders[pi];
                best_ms = t;
                best_bms = bms;
            }
            if (ok) break;  // higher orders at this leaf size only cost more
        }
    }
    c->prm = keep;
    c->prm.leaf_size = best_leaf;
    c->prm.levels = 0;
    c->prm.p = best_p;
    c->prm.adaptive = 0;
    if ((rc = timed_build(c, e0, e1, &ms))) return fail(rc);
    // Per-level orders: from the finest level with a far field upwards, lower that level's
    // order by 2 (not below 4) while the product stays within tol and the cost falls.
    if (best_ok) {
        const int L = c->L;
        int po[PB_MAXL + 1];
        for (int l = 0; l <= L; ++l) po[l] = c->lev[l].p;
        for (int l = L; l >= 1; --l) {
            if (c->lev[l].ninter == 0 || po[l] <= 4) continue;
            for (int q = 0; q <= L; ++q) c->p_level[q] = po[q];
            c->p_level[l] = po[l] - 2;
            c->p_level_L = L;
            float bms = 0, t = 0;
            double err = 0;
            if ((rc = timed_build(c, e0, e1, &bms)) || (rc = timed_products(c, x, y, nrhs, e0, e1, &t)) ||
                (rc = rel_err(&err)))
                return fail(rc);
            ++tried;
            const double cost = bms + (double)matvecs_per_solve * t;
            if (c->L == L && err <= tol && cost < best_cost) {
                po[l] -= 2;
                best_cost = cost;
                best_err = err;
                best_ms = t;
                best_bms = bms;
            }
        }
        for (int q = 0; q <= L; ++q) c->p_level[q] = po[q];
        c->p_level_L = L;
        if ((rc = timed_build(c, e0, e1, &ms))) return fail(rc);
    }
    out->leaf_size = best_leaf;
    out->p = best_p;
    out->matvec_ms = best_ms;
    out->build_ms = best_bms;
    out->rel_err = best_err;
    out->tried = tried;
    out->met_tolerance = best_ok ? 1 : 0;
    for (int l = 0; l < 11; ++l) out->order[l] = l <= c->L ? c->lev[l].p : 0;
    fail(PB_OK);
    return PB_OK;
}
