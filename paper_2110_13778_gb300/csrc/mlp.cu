// Learned warm start for GMRES: a per-element multilayer perceptron that maps local
// geometry and source-term features to the element's (phi, dphi/dn), trained on solutions
// the solver itself produces. GMRES started from its prediction still converges to the same
// residual, so the network only changes the number of iterations, never the answer.
//
// Arithmetic: BF16 weights and activations, FP32 accumulation, on the fifth-generation tensor
// cores (tcgen05.mma with tensor-memory accumulators): the fused inference of the default shape
// (width 128) and a generic tiled GEMM for the training passes and other shapes; FP32 master
// weights and Adam moments. Hidden layers use ReLU, the output layer is linear, the loss is the
// mean squared error.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "pb_internal.cuh"

#define MLP_MAXL 8

struct pb_mlp {
    int nin = 0, width = 0, depth = 0, nout = 0;  // depth = number of hidden layers
    int nl = 0;                                   // weight layers = depth + 1
    int din[MLP_MAXL] = {}, dout[MLP_MAXL] = {};  // padded dimensions (multiples of 16)
    long long woff[MLP_MAXL + 1] = {}, boff[MLP_MAXL + 1] = {};
    cudaStream_t st = nullptr;
    float *W = nullptr, *Wm = nullptr, *Wv = nullptr, *G = nullptr;  // all weights then biases
    __nv_bfloat16* Wb = nullptr;                                      // BF16 copy of the weights
    // training buffers (grown on demand): per layer pre-activations and BF16 activations
    int cap = 0;
    float* Z[MLP_MAXL] = {};
    __nv_bfloat16* Ab[MLP_MAXL + 1] = {};
    float* dA = nullptr;
    __nv_bfloat16* dZb = nullptr;
    float* lossbuf = nullptr;
    int* derr = nullptr;  // set by the tensor-core inference when a bounded wait gives up
    long long nparam = 0;
    int adam_t = 0;
    std::string err;
};

static int mlp_fail(pb_mlp* m, int code, const char* msg)
{
    if (m) m->err = msg;
    return code;
}
static int mlp_check_err(pb_mlp* m);

// ---------- tcgen05 helpers ----------
#define TC_ROWS 128
__device__ __forceinline__ unsigned tc_su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// shared-memory matrix descriptor: start address, leading (K) and stride (8-row) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M = 128
__device__ __forceinline__ unsigned tc_idesc(int nn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(nn >> 3) << 17) | ((unsigned)(TC_ROWS >> 4) << 24);
}
__device__ __forceinline__ bool tc_wait(unsigned bar, unsigned ph)
{
    for (unsigned it = 0; it < (1u << 24); ++it) {
        unsigned ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(bar), "r"(ph) : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// byte offset of element (r, k) in the no-swizzle K-major layout of a matrix with K columns
__device__ __forceinline__ unsigned tc_off(int r, int k, int K) { return (r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }
// 32 consecutive FP32 accumulator columns of this warp's 32 lanes (rows)
__device__ __forceinline__ void tc_ld32(unsigned taddr, float* v)
{
    unsigned r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}


// ---------- generic BF16 GEMM on the fifth-generation tensor cores ----------
// C[M x N] (FP32, ldc) = sum_k A(i, k) B(k, j) with A(i, k) = A[i * sAi + k * sAk] and
// B(k, j) = B[k * sBk + j * sBj] (BF16, any strides; the training passes read transposed
// operands). One block of four warps per 128 x 128 tile of C and per slice of K (gridDim.z
// slices that add into C with atomicAdd when ksplit > 1): chunks of 64 along K are staged by
// plain loads into shared memory in the no-swizzle K-major layout (zero outside A, B and the
// slice), four tcgen05.mma (M = N = 128, K = 16) per chunk accumulate into 128 columns of tensor
// memory, committed to an mbarrier; each warp then reads its 32 rows back with tcgen05.ld.
// Every wait is bounded (a wait that gives up sets *err, waits once more and stops).
#define GT_K 64
__device__ __forceinline__ unsigned gt_off(int r, int k) { return (r >> 3) * (GT_K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }
__device__ __forceinline__ unsigned gt_su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__global__ void __launch_bounds__(128, 1) k_gemm_tc(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                    long long sAi, long long sAk, const __nv_bfloat16* __restrict__ B,
                                                    long long sBk, long long sBj, float* __restrict__ C, long long ldc,
                                                    int accumulate, int* __restrict__ err)
{
    __shared__ __align__(128) __nv_bfloat16 As[128 * GT_K], Bs[128 * GT_K];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.x * 128, j0 = blockIdx.y * 128;
    const int kslice = (K + gridDim.z - 1) / gridDim.z;
    const int kb = blockIdx.z * kslice, ke = min(K, kb + kslice);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(gt_su32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gt_su32(&tslot)),
                     "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned taddr = tslot;
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
    const unsigned sbo = (GT_K / 8) * 128;
    const __nv_bfloat16 z = __float2bfloat16(0.f);
    unsigned ph = 0u;
    bool alive = true, any = false;
    for (int k0 = kb; k0 < ke && alive; k0 += GT_K) {
        for (int e = tid; e < 128 * GT_K; e += 128) {
            const int r = e / GT_K, kk = e % GT_K, k = k0 + kk;
            const int i = i0 + r, j = j0 + r;
            const bool kin = k < ke;
            *(__nv_bfloat16*)((char*)As + gt_off(r, kk)) = (kin && i < M) ? A[(long long)i * sAi + (long long)k * sAk] : z;
            *(__nv_bfloat16*)((char*)Bs + gt_off(r, kk)) = (kin && j < N) ? B[(long long)k * sBk + (long long)j * sBj] : z;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            for (int ks = 0; ks < GT_K / 16; ++ks) {
                const uint64_t ad = tc_desc(gt_su32(As) + ks * 256, 128, sbo);
                const uint64_t bd = tc_desc(gt_su32(Bs) + ks * 256, 128, sbo);
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"((unsigned)(any || ks > 0)) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(gt_su32(&bar)) : "memory");
        }
        any = true;
        if (!__syncthreads_and(tc_wait(gt_su32(&bar), ph))) {
            if (tid == 0) atomicExch(err, 1);
            tc_wait(gt_su32(&bar), ph);
            alive = false;
            break;
        }
        ph ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (alive && (any || !accumulate)) {
        const int i = i0 + 32 * warp + lane;
        for (int c0 = 0; c0 < 128; c0 += 32) {
            float v[32];
            if (any) tc_ld32(taddr + ((unsigned)(32 * warp) << 16) + c0, v);
            else
                for (int q = 0; q < 32; ++q) v[q] = 0.f;
            if (i < M)
                for (int q = 0; q < 32; ++q) {
                    const int j = j0 + c0 + q;
                    if (j < N) {
                        float* c = C + (long long)i * ldc + j;
                        if (accumulate) atomicAdd(c, v[q]);
                        else *c = v[q];
                    }
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(128) : "memory");
}

static void gemm(cudaStream_t st, int M, int N, int K, const __nv_bfloat16* A, long long sAi, long long sAk,
                 const __nv_bfloat16* B, long long sBk, long long sBj, float* C, long long ldc, int ksplit, int* err)
{
    dim3 grid((M + 127) / 128, (N + 127) / 128, ksplit);
    k_gemm_tc<<<grid, 128, 0, st>>>(M, N, K, A, sAi, sAk, B, sBk, sBj, C, ldc, ksplit > 1, err);
}

// ---------- elementwise pieces ----------
__global__ void k_to_bf16(long long n, const float* __restrict__ x, __nv_bfloat16* __restrict__ y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// input rows (n x nin, FP32) into a zero-padded BF16 matrix (n x dpad)
__global__ void k_pack_input(int n, int nin, int dpad, const float* __restrict__ X, __nv_bfloat16* __restrict__ Y)
{
    long long tot = (long long)n * dpad;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        int r = (int)(i / dpad), c = (int)(i % dpad);
        Y[i] = __float2bfloat16(c < nin ? X[(long long)r * nin + c] : 0.f);
    }
}

// Z += bias; A = relu(Z) (hidden) or Z (output), as BF16 for the next layer
__global__ void k_bias_act(int n, int d, const float* __restrict__ b, float* __restrict__ Z,
                           __nv_bfloat16* __restrict__ Ab, int relu)
{
    long long tot = (long long)n * d;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        float v = Z[i] + b[i % d];
        Z[i] = v;
        if (Ab) Ab[i] = __float2bfloat16(relu ? fmaxf(v, 0.f) : v);
    }
}

// output layer: dZ = 2 (Y - T) / (n nout) on the real outputs, loss partial sums
__global__ void k_mse(int n, int nout, int dpad, const float* __restrict__ Y, const float* __restrict__ T,
                      float* __restrict__ dZ, float* __restrict__ loss)
{
    __shared__ float red[256];
    float s = 0.f;
    long long tot = (long long)n * dpad;
    const float sc = 2.f / ((float)n * (float)nout);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        int r = (int)(i / dpad), c = (int)(i % dpad);
        float g = 0.f;
        if (c < nout) {
            float e = Y[i] - T[(long long)r * nout + c];
            s += e * e;
            g = sc * e;
        }
        dZ[i] = g;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / ((float)n * (float)nout));
}

// dZ = dA * relu'(Z)
__global__ void k_relu_back(long long n, const float* __restrict__ Z, const float* __restrict__ dA,
                            __nv_bfloat16* __restrict__ dZb)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dZb[i] = __float2bfloat16(Z[i] > 0.f ? dA[i] : 0.f);
}

// bias gradient: column sums of dZ (n x d)
__global__ void k_colsum(int n, int d, const __nv_bfloat16* __restrict__ dZ, float* __restrict__ gb)
{
    int c = blockIdx.x;
    float s = 0.f;
    for (int r = threadIdx.x; r < n; r += blockDim.x) s += __bfloat162float(dZ[(long long)r * d + c]);
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[c] = red[0];
}

__global__ void k_adam(long long n, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float c1, float c2, float eps)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// deterministic initialisation: uniform(-s, s) with s = sqrt(6 / (fan_in + fan_out)) (SplitMix64)
__global__ void k_init(long long n, float* __restrict__ w, float s, unsigned long long seed)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z = z ^ (z >> 31);
        double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        w[i] = (float)((2.0 * u - 1.0) * s);
    }
}

static int grid1(long long n) { return (int)std::min<long long>((n + 255) / 256, 152 * 8); }

static int ensure_cap(pb_mlp* m, int n)
{
    if (n <= m->cap) return PB_OK;
    cudaStreamSynchronize(m->st);
    for (int l = 0; l < m->nl; ++l) {
        cudaFree(m->Z[l]);
        m->Z[l] = nullptr;
    }
    for (int l = 0; l <= m->nl; ++l) {
        cudaFree(m->Ab[l]);
        m->Ab[l] = nullptr;
    }
    cudaFree(m->dA);
    cudaFree(m->dZb);
    int dmax = 16;
    for (int l = 0; l < m->nl; ++l) dmax = std::max(dmax, std::max(m->din[l], m->dout[l]));
    bool ok = true;
    for (int l = 0; l < m->nl; ++l) ok &= cudaMalloc(&m->Z[l], sizeof(float) * (size_t)n * m->dout[l]) == cudaSuccess;
    ok &= cudaMalloc(&m->Ab[0], sizeof(__nv_bfloat16) * (size_t)n * m->din[0]) == cudaSuccess;
    for (int l = 0; l < m->nl; ++l)
        ok &= cudaMalloc(&m->Ab[l + 1], sizeof(__nv_bfloat16) * (size_t)n * m->dout[l]) == cudaSuccess;
    ok &= cudaMalloc(&m->dA, sizeof(float) * (size_t)n * dmax) == cudaSuccess;
    ok &= cudaMalloc(&m->dZb, sizeof(__nv_bfloat16) * (size_t)n * dmax) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        m->cap = 0;
        return mlp_fail(m, PB_ERR_NOMEM, "mlp: out of memory");
    }
    m->cap = n;
    return PB_OK;
}

// forward pass over n rows; keeps Z and BF16 activations for a backward pass
static int mlp_forward(pb_mlp* m, const float* X, int n)
{
    int rc = ensure_cap(m, n);
    if (rc) return rc;
    k_to_bf16<<<grid1(m->nparam), 256, 0, m->st>>>(m->nparam, m->W, m->Wb);
    k_pack_input<<<grid1((long long)n * m->din[0]), 256, 0, m->st>>>(n, m->nin, m->din[0], X, m->Ab[0]);
    for (int l = 0; l < m->nl; ++l) {
        const int k = m->din[l], d = m->dout[l];
        // Z = A W^T: B(kk, j) = W[j][kk]
        gemm(m->st, n, d, k, m->Ab[l], k, 1, m->Wb + m->woff[l], 1, k, m->Z[l], d, 1, m->derr);
        k_bias_act<<<grid1((long long)n * d), 256, 0, m->st>>>(n, d, m->W + m->boff[l], m->Z[l], m->Ab[l + 1],
                                                               l + 1 < m->nl);
    }
    return cudaGetLastError() == cudaSuccess ? PB_OK : mlp_fail(m, PB_ERR_CUDA, "mlp forward launch failed");
}

// backward pass after mlp_forward: gradients into m->G, loss into m->lossbuf
static int mlp_backward(pb_mlp* m, const float* T, int n)
{
    const int L = m->nl;
    cudaMemsetAsync(m->G, 0, sizeof(float) * m->nparam, m->st);
    cudaMemsetAsync(m->lossbuf, 0, sizeof(float), m->st);
    const int dl = m->dout[L - 1];
    k_mse<<<grid1((long long)n * dl), 256, 0, m->st>>>(n, m->nout, dl, m->Z[L - 1], T, m->dA, m->lossbuf);
    k_to_bf16<<<grid1((long long)n * dl), 256, 0, m->st>>>((long long)n * dl, m->dA, m->dZb);
    for (int l = L - 1; l >= 0; --l) {
        const int k = m->din[l], d = m->dout[l];
        // dW = dZ^T A: A-operand (i = out unit, kk = row) = dZ[kk][i]; B(kk = row, j = in) = A[kk][j]
        const int ks = std::max(1, std::min(64, n / 2048));
        gemm(m->st, d, k, n, m->dZb, 1, d, m->Ab[l], k, 1, m->G + m->woff[l], k, ks, m->derr);
        k_colsum<<<d, 256, 0, m->st>>>(n, d, m->dZb, m->G + m->boff[l]);
        if (l > 0) {
            // dA_prev = dZ W: A(i = row, kk = out) = dZ[i][kk]; B(kk = out, j = in) = W[kk][j]
            gemm(m->st, n, k, d, m->dZb, d, 1, m->Wb + m->woff[l], k, 1, m->dA, k, 1, m->derr);
            k_relu_back<<<grid1((long long)n * k), 256, 0, m->st>>>((long long)n * k, m->Z[l - 1], m->dA, m->dZb);
        }
    }
    return cudaGetLastError() == cudaSuccess ? PB_OK : mlp_fail(m, PB_ERR_CUDA, "mlp backward launch failed");
}

extern "C" int pb_mlp_create(int nin, int width, int depth, int nout, unsigned long long seed, void* stream,
                             pb_mlp** out)
{
    if (!out || nin < 1 || width < 16 || width % 16 || depth < 1 || depth + 1 > MLP_MAXL || nout < 1 || nout > 64)
        return PB_ERR_ARG;
    pb_mlp* m = new pb_mlp();
    m->nin = nin;
    m->width = width;
    m->depth = depth;
    m->nout = nout;
    m->nl = depth + 1;
    m->st = (cudaStream_t)stream;
    auto pad = [](int x) { return (x + 15) / 16 * 16; };
    long long o = 0;
    for (int l = 0; l < m->nl; ++l) {
        m->din[l] = l == 0 ? pad(nin) : width;
        m->dout[l] = l + 1 < m->nl ? width : pad(nout);
        m->woff[l] = o;
        o += (long long)m->din[l] * m->dout[l];
    }
    m->woff[m->nl] = o;
    for (int l = 0; l < m->nl; ++l) {
        m->boff[l] = o;
        o += m->dout[l];
    }
    m->boff[m->nl] = o;
    m->nparam = o;
    bool ok = cudaMalloc(&m->W, sizeof(float) * o) == cudaSuccess;
    ok &= cudaMalloc(&m->Wm, sizeof(float) * o) == cudaSuccess;
    ok &= cudaMalloc(&m->Wv, sizeof(float) * o) == cudaSuccess;
    ok &= cudaMalloc(&m->G, sizeof(float) * o) == cudaSuccess;
    ok &= cudaMalloc(&m->Wb, sizeof(__nv_bfloat16) * o) == cudaSuccess;
    ok &= cudaMalloc(&m->lossbuf, sizeof(float)) == cudaSuccess;
    ok &= cudaMalloc(&m->derr, sizeof(int)) == cudaSuccess;
    ok &= ok && cudaMemset(m->derr, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        delete m;
        return PB_ERR_NOMEM;
    }
    cudaMemsetAsync(m->W, 0, sizeof(float) * o, m->st);
    cudaMemsetAsync(m->Wm, 0, sizeof(float) * o, m->st);
    cudaMemsetAsync(m->Wv, 0, sizeof(float) * o, m->st);
    for (int l = 0; l < m->nl; ++l) {
        long long n = (long long)m->din[l] * m->dout[l];
        float s = sqrtf(6.f / (float)((l == 0 ? nin : width) + (l + 1 < m->nl ? width : nout)));
        k_init<<<grid1(n), 256, 0, m->st>>>(n, m->W + m->woff[l], s, seed + 7919ULL * l);
    }
    // padded input columns and output rows carry zero weights
    std::vector<float> h(o);
    cudaMemcpyAsync(h.data(), m->W, sizeof(float) * o, cudaMemcpyDeviceToHost, m->st);
    cudaStreamSynchronize(m->st);
    for (int l = 0; l < m->nl; ++l) {
        int realin = l == 0 ? nin : width, realout = l + 1 < m->nl ? width : nout;
        for (int j = 0; j < m->dout[l]; ++j)
            for (int kk = 0; kk < m->din[l]; ++kk)
                if (j >= realout || kk >= realin) h[m->woff[l] + (long long)j * m->din[l] + kk] = 0.f;
    }
    cudaMemcpyAsync(m->W, h.data(), sizeof(float) * o, cudaMemcpyHostToDevice, m->st);
    if (cudaStreamSynchronize(m->st) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return PB_ERR_CUDA;
    }
    *out = m;
    return PB_OK;
}

extern "C" int pb_mlp_destroy(pb_mlp* m)
{
    if (!m) return PB_OK;
    cudaStreamSynchronize(m->st);
    cudaFree(m->W);
    cudaFree(m->Wm);
    cudaFree(m->Wv);
    cudaFree(m->G);
    cudaFree(m->Wb);
    cudaFree(m->lossbuf);
    cudaFree(m->derr);
    for (int l = 0; l < MLP_MAXL; ++l) cudaFree(m->Z[l]);
    for (int l = 0; l <= MLP_MAXL; ++l) cudaFree(m->Ab[l]);
    cudaFree(m->dA);
    cudaFree(m->dZb);
    delete m;
    return PB_OK;
}

extern "C" const char* pb_mlp_last_error(const pb_mlp* m) { return m ? m->err.c_str() : "null network"; }

extern "C" int pb_mlp_param_count(pb_mlp* m, long long* n)
{
    if (!m || !n) return PB_ERR_ARG;
    *n = m->nparam;
    return PB_OK;
}

extern "C" int pb_mlp_get_params(pb_mlp* m, float* host)
{
    if (!m || !host) return PB_ERR_ARG;
    if (cudaMemcpyAsync(host, m->W, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
        return mlp_fail(m, PB_ERR_CUDA, "mlp: copy failed");
    return PB_OK;
}

extern "C" int pb_mlp_set_params(pb_mlp* m, const float* host)
{
    if (!m || !host) return PB_ERR_ARG;
    if (cudaMemcpyAsync(m->W, host, sizeof(float) * m->nparam, cudaMemcpyHostToDevice, m->st) != cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
        return mlp_fail(m, PB_ERR_CUDA, "mlp: copy failed");
    return PB_OK;
}

// ---------- fused inference: every layer in one kernel ----------
// For width 128, a first layer of at most 32 padded inputs and at most 16 padded outputs: all
// weights are converted to BF16 once per block and every tile of rows runs through all layers
// inside the kernel, so the features are read once and two outputs written per row.
#define FUSED_W 128
struct MlpDesc {
    long long woff[MLP_MAXL], boff[MLP_MAXL];
    int nin, din0, nl, nout;  // inputs, padded inputs (row length of W_0), layers, outputs
};

// ---------- fused inference on the fifth-generation tensor cores (tcgen05) ----------
// The layers and rounding points of the layer-by-layer path, one tile of 128 rows at a time: the
// tile's BF16 activations sit in shared memory in the K-major layout without swizzle that the
// MMA reads through matrix descriptors (8 x 16-byte core matrices: the next core matrix along K
// 128 bytes on, the next group of 8 rows K / 8 x 128 bytes on); one thread issues the layer's
// tcgen05.mma instructions (M = 128, N = 128 or 16, K = 16 each, BF16 in, FP32 accumulate) into a
// 128-column tensor-memory accumulator and commits them to an mbarrier; each warp then reads its
// 32 rows back with tcgen05.ld, adds the bias, applies ReLU, rounds to BF16 and writes the next
// layer's operand in place. Every wait is bounded: a wait that gives up sets *err, lets the MMAs
// in flight finish (bounded again), frees the tensor memory and leaves.
static size_t tc_smem(int nl, int din0)
{
    return sizeof(__nv_bfloat16) * ((size_t)FUSED_W * din0 + (size_t)(nl - 2) * FUSED_W * FUSED_W + 16 * FUSED_W +
                                    (size_t)TC_ROWS * FUSED_W) +
           sizeof(float) * ((size_t)(nl - 1) * FUSED_W + 16) + 128;
}

__global__ void __launch_bounds__(128, 1) k_mlp_tc(int n, const float* __restrict__ X, const float* __restrict__ W,
                                                   MlpDesc md, float* __restrict__ Y, int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned tslot;
    const int nl = md.nl, din0 = md.din0;
    __nv_bfloat16* w0 = (__nv_bfloat16*)tsm;                           // [128 x din0]
    __nv_bfloat16* wh = w0 + FUSED_W * din0;                           // [nl-2][128 x 128]
    __nv_bfloat16* wl = wh + (size_t)(nl - 2) * FUSED_W * FUSED_W;     // [16 x 128]
    __nv_bfloat16* as = wl + 16 * FUSED_W;                             // [128 x 128] activations
    float* bs = (float*)(as + TC_ROWS * FUSED_W);                      // [nl-1][128] then [16]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // weights (row o of layer l is output o: the B operand, K-major) and biases
    for (int i = tid; i < FUSED_W * din0; i += 128)
        *(__nv_bfloat16*)((char*)w0 + tc_off(i / din0, i % din0, din0)) = __float2bfloat16(W[md.woff[0] + i]);
    for (int l = 1; l < nl - 1; ++l)
        for (int i = tid; i < FUSED_W * FUSED_W; i += 128)
            *(__nv_bfloat16*)((char*)(wh + (size_t)(l - 1) * FUSED_W * FUSED_W) + tc_off(i / FUSED_W, i % FUSED_W, FUSED_W)) =
                __float2bfloat16(W[md.woff[l] + i]);
    for (int i = tid; i < 16 * FUSED_W; i += 128)
        *(__nv_bfloat16*)((char*)wl + tc_off(i / FUSED_W, i % FUSED_W, FUSED_W)) = __float2bfloat16(W[md.woff[nl - 1] + i]);
    for (int l = 0; l < nl - 1; ++l)
        for (int i = tid; i < FUSED_W; i += 128) bs[l * FUSED_W + i] = W[md.boff[l] + i];
    for (int i = tid; i < 16; i += 128) bs[(nl - 1) * FUSED_W + i] = W[md.boff[nl - 1] + i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_su32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_su32(&tslot)),
                     "r"(FUSED_W)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned taddr = tslot, tw = taddr + ((unsigned)(32 * warp) << 16);
    unsigned ph = 0u;
    bool alive = true;
    const int ntiles = (n + TC_ROWS - 1) / TC_ROWS;
    for (int tile = blockIdx.x; tile < ntiles && alive; tile += gridDim.x) {
        // the tile's features, BF16, zero beyond nin and beyond n, in the layer-0 layout
        {
            const int r = tid, row = tile * TC_ROWS + r;
            for (int k0 = 0; k0 < din0; k0 += 8) {
                __align__(16) __nv_bfloat16 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int c = k0 + q;
                    v[q] = __float2bfloat16(row < n && c < md.nin ? X[(size_t)row * md.nin + c] : 0.f);
                }
                *(uint4*)((char*)as + tc_off(r, k0, din0)) = *(const uint4*)v;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        for (int l = 0; l < nl && alive; ++l) {
            const bool last = l == nl - 1;
            const int K = l == 0 ? din0 : FUSED_W, nn = last ? 16 : FUSED_W;
            const __nv_bfloat16* wb = l == 0 ? w0 : last ? wl : wh + (size_t)(l - 1) * FUSED_W * FUSED_W;
            if (tid == 0) {
                const unsigned sbo = (K / 8) * 128, id = tc_idesc(nn);
                for (int ks = 0; ks < K / 16; ++ks) {
                    const uint64_t ad = tc_desc(tc_su32(as) + ks * 256, 128, sbo);
                    const uint64_t bd = tc_desc(tc_su32(wb) + ks * 256, 128, sbo);
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                 ::"r"(taddr), "l"(ad), "l"(bd), "r"(id), "r"((unsigned)(ks > 0)) : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(tc_su32(&bar)) : "memory");
            }
            if (!__syncthreads_and(tc_wait(tc_su32(&bar), ph))) {
                if (tid == 0) atomicExch(err, 1);
                tc_wait(tc_su32(&bar), ph);  // let the MMAs in flight finish before the memory goes
                alive = false;
                break;
            }
            ph ^= 1u;
            tc_fence_after();
            const float* bias = bs + l * FUSED_W;
            const int r = 32 * warp + lane, row = tile * TC_ROWS + r;
            if (last) {
                float v[32];
                tc_ld32(tw, v);  // (columns 16..31 are not part of this layer's result)
                for (int c = 0; c < md.nout; ++c)
                    if (row < n) Y[(size_t)row * md.nout + c] = v[c] + bias[c];
            } else {
                for (int c0 = 0; c0 < FUSED_W; c0 += 32) {
                    float v[32];
                    tc_ld32(tw + c0, v);
#pragma unroll
                    for (int q0 = 0; q0 < 32; q0 += 8) {
                        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) o[q] = __float2bfloat16(fmaxf(v[q0 + q] + bias[c0 + q0 + q], 0.f));
                        *(uint4*)((char*)as + tc_off(r, c0 + q0, FUSED_W)) = *(const uint4*)o;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(FUSED_W) : "memory");
}

static bool fused_ok(const pb_mlp* m)
{
    return m->width == FUSED_W && m->din[0] <= 32 && m->dout[m->nl - 1] == 16 && m->nl >= 2 &&
           tc_smem(m->nl, m->din[0]) <= 200 * 1024;
}

static int mlp_forward_fused(pb_mlp* m, const float* X, int n, float* Y)
{
    MlpDesc md;
    for (int l = 0; l < MLP_MAXL; ++l) {
        md.woff[l] = l < m->nl ? m->woff[l] : 0;
        md.boff[l] = l < m->nl ? m->boff[l] : 0;
    }
    md.nin = m->nin;
    md.din0 = m->din[0];
    md.nl = m->nl;
    md.nout = m->nout;
    const size_t smem = tc_smem(m->nl, m->din[0]);
    if (cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return mlp_fail(m, PB_ERR_CUDA, "mlp: shared memory attribute failed");
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (n + TC_ROWS - 1) / TC_ROWS;
    const int grid = std::max(1, std::min(tiles, nsm));  // one block per SM (its tensor memory and shared memory)
    k_mlp_tc<<<grid, 128, smem, m->st>>>(n, X, m->W, md, Y, m->derr);
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(m, PB_ERR_CUDA, "mlp fused forward launch failed");
    return mlp_check_err(m);
}

extern "C" int pb_mlp_forward(pb_mlp* m, const float* X, int n, float* Y)
{
    if (!m || !X || !Y || n < 1) return PB_ERR_ARG;
    if (fused_ok(m)) return mlp_forward_fused(m, X, n, Y);
    int rc = mlp_forward(m, X, n);
    if (rc) return rc;
    // real outputs of the last layer, row-major n x nout
    const int L = m->nl, dl = m->dout[L - 1];
    if (cudaMemcpy2DAsync(Y, sizeof(float) * m->nout, m->Z[L - 1], sizeof(float) * dl, sizeof(float) * m->nout, n,
                          cudaMemcpyDeviceToDevice, m->st) != cudaSuccess)
        return mlp_fail(m, PB_ERR_CUDA, "mlp: output copy failed");
    return PB_OK;
}

// PB_ERR_TIMEOUT (and the flag cleared) if a bounded wait of a tensor-core kernel gave up
static int mlp_check_err(pb_mlp* m)
{
    int herr = 0;
    if (cudaMemcpyAsync(&herr, m->derr, sizeof(int), cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
        return mlp_fail(m, PB_ERR_CUDA, "mlp: sync failed");
    if (!herr) return PB_OK;
    cudaMemsetAsync(m->derr, 0, sizeof(int), m->st);
    return mlp_fail(m, PB_ERR_TIMEOUT, "mlp: a bounded wait on the tensor cores gave up");
}

extern "C" int pb_mlp_gradient(pb_mlp* m, const float* X, const float* T, int n, float* loss, float* grad_host)
{
    if (!m || !X || !T || n < 1) return PB_ERR_ARG;
    int rc = mlp_forward(m, X, n);
    if (!rc) rc = mlp_backward(m, T, n);
    if (rc) return rc;
    if (loss && cudaMemcpyAsync(loss, m->lossbuf, sizeof(float), cudaMemcpyDeviceToHost, m->st) != cudaSuccess)
        return mlp_fail(m, PB_ERR_CUDA, "mlp: copy failed");
    if (grad_host &&
        cudaMemcpyAsync(grad_host, m->G, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->st) != cudaSuccess)
        return mlp_fail(m, PB_ERR_CUDA, "mlp: copy failed");
    if (cudaStreamSynchronize(m->st) != cudaSuccess) return mlp_fail(m, PB_ERR_CUDA, "mlp: sync failed");
    return mlp_check_err(m);
}

extern "C" int pb_mlp_train_step(pb_mlp* m, const float* X, const float* T, int n, float lr, float* loss)
{
    if (!m || !X || !T || n < 1 || !(lr > 0)) return PB_ERR_ARG;
    int rc = mlp_forward(m, X, n);
    if (!rc) rc = mlp_backward(m, T, n);
    if (rc) return rc;
    m->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
    k_adam<<<grid1(m->nparam), 256, 0, m->st>>>(m->nparam, m->W, m->Wm, m->Wv, m->G, lr, b1, b2, c1, c2, 1e-8f);
    if (loss && cudaMemcpyAsync(loss, m->lossbuf, sizeof(float), cudaMemcpyDeviceToHost, m->st) != cudaSuccess)
        return mlp_fail(m, PB_ERR_CUDA, "mlp: copy failed");
    if (loss && cudaStreamSynchronize(m->st) != cudaSuccess) return mlp_fail(m, PB_ERR_CUDA, "mlp: sync failed");
    return cudaGetLastError() == cudaSuccess ? PB_OK : mlp_fail(m, PB_ERR_CUDA, "mlp: launch failed");
}

// ---------- features of the learned warm start ----------
// Per element, in element order (16 columns; r = distance from the centroid c to charge k):
//   0-2   c minus the mean charge position, over the radius of gyration of the centroids
//   3-5   unit normal
//   6     log(A / mean A)
//   7     curvature: 1 - mean n_i . n_j over the other triangles sharing a vertex with i
//   8, 9  S1 and S2 at the centroid (the source terms of eqbim_3/eqbim_4)
//   10    U = sum_k |q_k| / (4 pi r)
//   11    distance to the nearest charge / 3 Angstrom
//   12    screened source sum_k q_k exp(-kappa r) / (4 pi eps_in r)
//   13,14 smoothed sources sum_k q_k / (4 pi eps_in sqrt(r^2 + a^2)), a = 4 and 8 Angstrom
//   15    charge density around c: sum_k exp(-r^2 / 50) / 10
//   16,17 smoothed normal fields -sum_k q_k n.(c - x_k) / (4 pi eps_in (r^2 + a^2)^(3/2)),
//         a = 4 and 8 Angstrom
// Columns 8, 9, 10, 12, 13, 14, 16 and 17 are divided by their root mean square over the
// molecule.
// Targets: phi / (rms S1 * 2 eps_in / (eps_in + eps_out)) and
// dphi / (rms S2 * 2 eps_out / (eps_in + eps_out)) -- the image-charge values at a flat
// dielectric interface, so that targets are O(1) for molecules of any size and charge.
#define NFEAT 18
#define NSTAT 20  // column normalisers [0, 18) and the two target scales [18], [19]

struct PoolTmp {
    pb_ctx* c;
    void* p = nullptr;
    PoolTmp(pb_ctx* cc, size_t bytes) : c(cc)
    {
        if (cudaMallocFromPoolAsync(&p, bytes, c->pool, c->st) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    ~PoolTmp()
    {
        if (p) cudaFreeAsync(p, c->st);
    }
};

// raw columns in sorted order. The charge sums run in FP32 (coordinates relative to the charge
// centre, charges staged through shared memory 256 at a time), each tile's partial sums added
// into FP64: the features only feed the network, and FP32 keeps this pass to a few ms even for
// 200k elements x 2000 charges.
#define FT 256
__global__ void __launch_bounds__(FT) k_feat_pass(int nt, int nc, const double4_32a* __restrict__ ep,
                                                  const double4_32a* __restrict__ en,
                                                  const double* __restrict__ qpos, const double* __restrict__ q,
                                                  const int* __restrict__ toff, const int* __restrict__ tj, double cx,
                                                  double cy, double cz, double eps_in, double kappa,
                                                  float* __restrict__ raw)
{
    __shared__ float4 sq[FT];
    const int k = blockIdx.x * FT + threadIdx.x;
    const bool act = k < nt;
    double4_32a p = {0, 0, 0, 0}, n = {0, 0, 0, 0};
    if (act) {
        p = ep[k];
        n = en[k];
    }
    const float px = (float)(p.x - cx), py = (float)(p.y - cy), pz = (float)(p.z - cz);
    const float nx = (float)n.x, ny = (float)n.y, nz = (float)n.z, kap = (float)kappa;
    double s1 = 0, s2 = 0, u = 0, sk = 0, sa4 = 0, sa8 = 0, dens = 0, e4 = 0, e8 = 0;
    float dmin2 = 3.0e38f;
    for (int t0 = 0; t0 < nc; t0 += FT) {
        __syncthreads();
        if (t0 + threadIdx.x < nc) {
            const int t = t0 + threadIdx.x;
            sq[threadIdx.x] = make_float4((float)(qpos[3 * t] - cx), (float)(qpos[3 * t + 1] - cy),
                                          (float)(qpos[3 * t + 2] - cz), (float)q[t]);
        }
        __syncthreads();
        const int m = min(FT, nc - t0);
        float f1 = 0, f2 = 0, fu = 0, fk = 0, f4 = 0, f8 = 0, fd = 0, g4 = 0, g8 = 0;
        for (int j = 0; j < m; ++j) {
            const float4 c = sq[j];
            const float dx = px - c.x, dy = py - c.y, dz = pz - c.z;
            const float r2 = dx * dx + dy * dy + dz * dz, ri = rsqrtf(r2);
            const float nd = nx * dx + ny * dy + nz * dz;
            const float w4 = rsqrtf(r2 + 16.f), w8 = rsqrtf(r2 + 64.f);
            f1 += c.w * ri;
            f2 -= c.w * nd * ri * ri * ri;
            fu += fabsf(c.w) * ri;
            fk += c.w * __expf(-kap * r2 * ri) * ri;
            f4 += c.w * w4;
            f8 += c.w * w8;
            g4 -= c.w * nd * w4 * w4 * w4;
            g8 -= c.w * nd * w8 * w8 * w8;
            fd += __expf(-r2 * 0.02f);
            dmin2 = fminf(dmin2, r2);
        }
        s1 += f1;
        s2 += f2;
        u += fu;
        sk += fk;
        sa4 += f4;
        sa8 += f8;
        e4 += g4;
        e8 += g8;
        dens += fd;
    }
    if (!act) return;
    double curv = 0;
    int cnt = 0;
    for (int t = toff[k]; t < toff[k + 1]; ++t) {
        int j = tj[t];
        if (j == k) continue;
        double4_32a m2 = en[j];
        curv += n.x * m2.x + n.y * m2.y + n.z * m2.z;
        ++cnt;
    }
    curv = cnt ? 1.0 - curv / cnt : 0.0;
    const double i4pi = 0.07957747154594767;
    float* r = raw + (size_t)k * NFEAT;
    r[0] = (float)(p.x - cx);
    r[1] = (float)(p.y - cy);
    r[2] = (float)(p.z - cz);
    r[3] = (float)n.x;
    r[4] = (float)n.y;
    r[5] = (float)n.z;
    r[6] = (float)p.w;
    r[7] = (float)curv;
    r[8] = (float)(s1 * i4pi / eps_in);
    r[9] = (float)(s2 * i4pi / eps_in);
    r[10] = (float)(u * i4pi);
    r[11] = sqrtf(dmin2) / 3.f;
    r[12] = (float)(sk * i4pi / eps_in);
    r[13] = (float)(sa4 * i4pi / eps_in);
    r[14] = (float)(sa8 * i4pi / eps_in);
    r[15] = (float)(dens / 10.0);
    r[16] = (float)(e4 * i4pi / eps_in);
    r[17] = (float)(e8 * i4pi / eps_in);
}

// the normalisers, one block: sums of squares (means for column 6) over the molecule
#define NRED 10
__global__ void k_feat_stats(int nt, const float* __restrict__ raw, double eps_in, double eps_out,
                             double* __restrict__ stats)
{
    const int cols[NRED] = {0, 6, 8, 9, 10, 12, 13, 14, 16, 17};
    __shared__ double red[NRED][256];
    double s[NRED];
    for (int c = 0; c < NRED; ++c) s[c] = 0;
    for (int k = threadIdx.x; k < nt; k += 256) {
        const float* r = raw + (size_t)k * NFEAT;
        s[0] += (double)r[0] * r[0] + (double)r[1] * r[1] + (double)r[2] * r[2];
        s[1] += r[6];
        for (int c = 2; c < NRED; ++c) s[c] += (double)r[cols[c]] * r[cols[c]];
    }
    for (int c = 0; c < NRED; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < NRED; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < NSTAT; ++c) stats[c] = 1.0;
        stats[0] = sqrt(red[0][0] / nt) + 1e-30;
        stats[6] = red[1][0] / nt;
        for (int c = 2; c < NRED; ++c) stats[cols[c]] = sqrt(red[c][0] / nt) + 1e-30;
        stats[18] = stats[8] * 2.0 * eps_in / (eps_in + eps_out);
        stats[19] = stats[9] * 2.0 * eps_out / (eps_in + eps_out);
    }
}

// normalise and scatter from sorted to element order; optionally the scaled targets
__global__ void k_feat_finish(int nt, const int* __restrict__ order, const float* __restrict__ raw,
                              const double* __restrict__ stats, float* __restrict__ F, const double* __restrict__ x,
                              float* __restrict__ T)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const float* r = raw + (size_t)k * NFEAT;
    const int e = order[k];
    float* f = F + (size_t)e * NFEAT;
#pragma unroll
    for (int c = 0; c < NFEAT; ++c) {
        const float s = (float)stats[c < 3 ? 0 : c];
        f[c] = c == 6 ? logf(r[6] / s) : r[c] / s;
    }
    if (T) {
        T[2 * (size_t)e] = (float)(x[e] / stats[18]);
        T[2 * (size_t)e + 1] = (float)(x[nt + e] / stats[19]);
    }
}

static int features(pb_ctx* c, float* F, const double* x, float* T, double* stats)
{
    const int nt = c->nt;
    std::vector<double> qp(3 * (size_t)std::max(c->nc, 1));
    double cx = 0, cy = 0, cz = 0;
    if (c->nc > 0) {
        PB_CUDA(c, cudaMemcpyAsync(qp.data(), c->qpos, sizeof(double) * 3 * c->nc, cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
        for (int k = 0; k < c->nc; ++k) {
            cx += qp[3 * k];
            cy += qp[3 * k + 1];
            cz += qp[3 * k + 2];
        }
        cx /= c->nc;
        cy /= c->nc;
        cz /= c->nc;
    }
    PoolTmp raw(c, sizeof(float) * (size_t)nt * NFEAT);
    if (!raw.p) return pb_fail(c, PB_ERR_NOMEM, "features: out of memory");
    k_feat_pass<<<(nt + FT - 1) / FT, FT, 0, c->st>>>(nt, c->nc, c->e64p, c->e64n, c->qpos, c->q, c->touch_off,
                                                     c->touch_j, cx, cy, cz, c->prm.eps_in, c->prm.kappa,
                                                     (float*)raw.p);
    PB_LAUNCH(c);
    k_feat_stats<<<1, 256, 0, c->st>>>(nt, (const float*)raw.p, c->prm.eps_in, c->prm.eps_out, stats);
    PB_LAUNCH(c);
    k_feat_finish<<<(nt + 255) / 256, 256, 0, c->st>>>(nt, c->order, (const float*)raw.p, stats, F, x, T);
    PB_LAUNCH(c);
    return PB_OK;
}

extern "C" int pb_features(pb_ctx* c, float* F, const double* x, float* T, double* scales)
{
    if (!c) return PB_ERR_ARG;
    if (c->dead) return PB_ERR_CUDA;
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "features before build_tree");
    if (c->prm.basis != PB_BASIS_CONSTANT) return pb_fail(c, PB_ERR_ARG, "features: piecewise-constant basis only");
    if (!F || (!x) != (!T)) return pb_fail(c, PB_ERR_ARG, "features: F is required, x and T go together");
    PoolTmp stats(c, sizeof(double) * NSTAT);
    if (!stats.p) return pb_fail(c, PB_ERR_NOMEM, "features: out of memory");
    int rc = features(c, F, x, T, (double*)stats.p);
    if (rc) return rc;
    if (scales) {
        PB_CUDA(c, cudaMemcpyAsync(scales, stats.p, sizeof(double) * NSTAT, cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
    }
    return PB_OK;
}

// x0 from the network output Y (element order, nt x 2) times the two target scales
__global__ void k_unscale(int nt, const float* __restrict__ Y, const double* __restrict__ stats,
                          double* __restrict__ x)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    x[k] = (double)Y[2 * (size_t)k] * stats[18];
    x[nt + k] = (double)Y[2 * (size_t)k + 1] * stats[19];
}

extern "C" int pb_learned_guess(pb_ctx* c, pb_mlp* m, double* x)
{
    if (!c || !m || !x) return PB_ERR_ARG;
    if (c->dead) return PB_ERR_CUDA;
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "learned guess before build_tree");
    if (c->prm.basis != PB_BASIS_CONSTANT) return pb_fail(c, PB_ERR_ARG, "learned guess: piecewise-constant basis only");
    if (m->nin != NFEAT || m->nout != 2) return pb_fail(c, PB_ERR_ARG, "learned guess: network must map 18 -> 2");
    const int nt = c->nt;
    PoolTmp F(c, sizeof(float) * (size_t)nt * NFEAT), Y(c, sizeof(float) * (size_t)nt * 2),
        stats(c, sizeof(double) * NSTAT);
    if (!F.p || !Y.p || !stats.p) return pb_fail(c, PB_ERR_NOMEM, "learned guess: out of memory");
    int rc = features(c, (float*)F.p, nullptr, nullptr, (double*)stats.p);
    if (rc) return rc;
    if (m->st != c->st) PB_CUDA(c, cudaStreamSynchronize(c->st));
    rc = pb_mlp_forward(m, (const float*)F.p, nt, (float*)Y.p);
    if (rc) return pb_fail(c, rc, "%s", m->err.c_str());
    if (m->st != c->st) PB_CUDA(c, cudaStreamSynchronize(m->st));
    k_unscale<<<(nt + 255) / 256, 256, 0, c->st>>>(nt, (const float*)Y.p, (const double*)stats.p, x);
    PB_LAUNCH(c);
    return PB_OK;
}
