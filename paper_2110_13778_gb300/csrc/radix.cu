// Prefix sums and the Morton-key radix sort of the tree build (Section 2.4, cluster
// hierarchy: elements ordered by the Morton code of their centroids).
//
// Exclusive scan: per-tile sums, a scan of the tile sums in one block, then each tile scans
// itself and adds its offset. Radix sort: least-significant-digit first, 8-bit digits; each
// pass counts the digits of every tile of 256 keys, scans the counts digit-major (digit d of
// tile t lands after every smaller digit and after digit d of the earlier tiles), and
// scatters. Within a tile the rank among equal digits keeps the input order (peers found by a
// warp match, earlier warps' counts from shared memory), so every pass is stable and ties keep
// the order of the element indices.
#include <algorithm>

#include "pb_internal.cuh"

#define SC_T 1024    // elements per scan tile (256 threads x 4)
#define RS_T 256     // keys per radix tile (one per thread)
#define RS_BINS 256

// ---------- exclusive scan ----------
__global__ void k_scan_tiles(int n, const int* __restrict__ in, int* __restrict__ tsum)
{
    __shared__ int red[256];
    const int base = blockIdx.x * SC_T;
    int s = 0;
    for (int q = 0; q < 4; ++q) {
        const int i = base + q * 256 + threadIdx.x;
        if (i < n) s += in[i];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) tsum[blockIdx.x] = red[0];
}

// exclusive scan of the tile sums in place (one block of 1024 threads, any count); the total
// goes to tsum[nt]
__global__ void k_scan_sums(int ntile, int* __restrict__ tsum)
{
    __shared__ int buf[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b = 0; b < ntile; b += 1024) {
        const int i = b + threadIdx.x;
        const int v = i < ntile ? tsum[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
            const int t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        const int c0 = carry;
        if (i < ntile) tsum[i] = c0 + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c0 + buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) tsum[ntile] = carry;
}

__global__ void k_scan_apply(int n, const int* __restrict__ in, const int* __restrict__ tsum, int* __restrict__ out)
{
    __shared__ int wsum[8];
    const int base = blockIdx.x * SC_T + threadIdx.x * 4;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int v[4], s = 0;
    for (int q = 0; q < 4; ++q) {
        v[q] = base + q < n ? in[base + q] : 0;
        s += v[q];
    }
    int inc = s;  // inclusive scan of the thread sums within the warp
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int woff = 0;
    for (int k = 0; k < w; ++k) woff += wsum[k];
    int run = tsum[blockIdx.x] + woff + inc - s;
    for (int q = 0; q < 4; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
}

__global__ void k_scan_total(int n, const int* __restrict__ tsum, int ntile, int* __restrict__ out)
{
    out[n] = tsum[ntile];
}

// out[i] = sum of in[0..i) for i = 0..n (out[n] the total); queued on c->st
int pb_scan_exclusive(pb_ctx* c, const int* in, int* out, int n)
{
    const int ntile = std::max(1, (n + SC_T - 1) / SC_T);
    int* tsum = nullptr;
    PB_CUDA(c, cudaMallocFromPoolAsync((void**)&tsum, sizeof(int) * (ntile + 1), c->pool, c->st));
    k_scan_tiles<<<ntile, 256, 0, c->st>>>(n, in, tsum);
    PB_LAUNCH(c);
    k_scan_sums<<<1, 1024, 0, c->st>>>(ntile, tsum);
    PB_LAUNCH(c);
    k_scan_apply<<<ntile, 256, 0, c->st>>>(n, in, tsum, out);
    PB_LAUNCH(c);
    k_scan_total<<<1, 1, 0, c->st>>>(n, tsum, ntile, out);
    PB_LAUNCH(c);
    PB_CUDA(c, cudaFreeAsync(tsum, c->st));
    return PB_OK;
}

// ---------- radix sort of (key, value) pairs ----------
// counts[d * ntile + t] = keys of tile t with digit d
__global__ void k_rs_count(int n, const unsigned* __restrict__ keys, int shift, unsigned dmask, int ntile,
                           int* __restrict__ counts)
{
    __shared__ int h[RS_BINS];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * RS_T + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & dmask], 1);
    __syncthreads();
    counts[threadIdx.x * ntile + blockIdx.x] = h[threadIdx.x];
}

// stable scatter of one tile: position = offs[d * ntile + t] + (earlier keys of digit d in
// the tile: earlier warps' counts + earlier peers in the own warp)
__global__ void k_rs_scatter(int n, const unsigned* __restrict__ kin, const int* __restrict__ vin, int shift,
                             unsigned dmask, int ntile, const int* __restrict__ offs, unsigned* __restrict__ kout,
                             int* __restrict__ vout)
{
    __shared__ int wc[RS_T / 32][RS_BINS];  // per warp: keys of each digit
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < (RS_T / 32) * RS_BINS; k += RS_T) (&wc[0][0])[k] = 0;
    __syncthreads();
    const int i = blockIdx.x * RS_T + threadIdx.x;
    const bool ok = i < n;
    const unsigned key = ok ? kin[i] : 0u;
    const int d = ok ? (int)((key >> shift) & dmask) : RS_BINS;  // padding: a digit of its own
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (ok && rank == 0) wc[w][d] = __popc(peers);
    __syncthreads();
    if (ok) {
        int before = 0;
        for (int k = 0; k < w; ++k) before += wc[k][d];
        const int pos = offs[d * ntile + blockIdx.x] + before + rank;
        kout[pos] = key;
        vout[pos] = vin[i];
    }
}

// Stable sort of n (key, value) pairs by the low `bits` bits of the key (1 <= bits <= 32);
// kin/vin are read, kout/vout receive the result. Queued on c->st.
int pb_radix_sort_pairs(pb_ctx* c, const unsigned* kin, const int* vin, unsigned* kout, int* vout, int n, int bits)
{
    const int ntile = std::max(1, (n + RS_T - 1) / RS_T);
    const int npass = (bits + 7) / 8;
    unsigned* kt = nullptr;
    int *vt = nullptr, *counts = nullptr, *offs = nullptr;
    const size_t nc = (size_t)RS_BINS * ntile;
    const size_t nn = (size_t)std::max(n, 1);
    PB_CUDA(c, cudaMallocFromPoolAsync((void**)&kt, sizeof(unsigned) * nn, c->pool, c->st));
    PB_CUDA(c, cudaMallocFromPoolAsync((void**)&vt, sizeof(int) * nn, c->pool, c->st));
    PB_CUDA(c, cudaMallocFromPoolAsync((void**)&counts, sizeof(int) * (nc + 1), c->pool, c->st));
    PB_CUDA(c, cudaMallocFromPoolAsync((void**)&offs, sizeof(int) * (nc + 1), c->pool, c->st));
    // pass p reads src and writes dst; the last pass writes kout/vout
    const unsigned* ks = kin;
    const int* vs = vin;
    int rc = PB_OK;
    for (int p = 0; p < npass && rc == PB_OK; ++p) {
        const bool to_out = ((npass - 1 - p) & 1) == 0;
        unsigned* kd = to_out ? kout : kt;
        int* vd = to_out ? vout : vt;
        const int nb = std::min(8, bits - 8 * p);  // digit bits of this pass
        const unsigned dmask = (1u << nb) - 1u;
        k_rs_count<<<ntile, RS_T, 0, c->st>>>(n, ks, 8 * p, dmask, ntile, counts);
        PB_LAUNCH(c);
        if ((rc = pb_scan_exclusive(c, counts, offs, (int)nc))) break;
        k_rs_scatter<<<ntile, RS_T, 0, c->st>>>(n, ks, vs, 8 * p, dmask, ntile, offs, kd, vd);
        PB_LAUNCH(c);
        ks = kd;
        vs = vd;
    }
    PB_CUDA(c, cudaFreeAsync(kt, c->st));
    PB_CUDA(c, cudaFreeAsync(vt, c->st));
    PB_CUDA(c, cudaFreeAsync(counts, c->st));
    PB_CUDA(c, cudaFreeAsync(offs, c->st));
    return rc;
}
