// Solvation energy without any device allocation, for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc: hosts that give this library a fixed device-memory
// budget and forbid allocations after start-up, or code that runs where an allocation is not
// allowed (an allocation may synchronise the device, or fail when memory is exhausted). For them
// pb_solvation_energy_noalloc evaluates the same energy as pb_solvation_energy from
// caller-owned device buffers, and keeps its only scratch -- one partial sum per thread
// block -- in a fixed file-scope device array instead of a context buffer.
//
// The array below is held by every GPU that loads this library, until the process exits.
// In host code its name is only a host-side stand-in: a kernel given that name faults, or
// on systems where the GPU can reach host memory silently uses the wrong memory. The device
// address is therefore looked up once per device, with that device current, by
// cudaGetSymbolAddress, and passed to the kernels.
#include <mutex>

#include "kernels.cuh"
#include "pb_internal.cuh"

#define NA_THREADS 256
#define NA_MAX_BLOCKS 8192  // 64 KiB of partial sums: at most 8192 * 256 = 2,097,152 triangles

static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[256] = {};  // device address of the scratch array, per device

// per element: A_i [K1(x_n, c_i) dphi_i + K2(x_n, c_i) phi_i], summed over charges
template <class R>
__global__ void __launch_bounds__(NA_THREADS)
    k_energy_noalloc(int nt, const double* __restrict__ V, const int* __restrict__ T, int nc,
                     const double* __restrict__ qpos, const double* __restrict__ q, double eps, double kappa,
                     const double* __restrict__ x, double* __restrict__ part)
{
    __shared__ double sq[NA_THREADS][4];
    __shared__ double red[NA_THREADS];
    int i = blockIdx.x * NA_THREADS + threadIdx.x;
    double c[3] = {0, 0, 0}, n[3] = {0, 0, 0}, A = 0.0, ph = 0.0, dph = 0.0;
    if (i < nt) {
        const double* u = V + 3 * T[3 * i];
        const double* v = V + 3 * T[3 * i + 1];
        const double* w = V + 3 * T[3 * i + 2];
        double a[3], b[3];
        for (int k = 0; k < 3; ++k) {
            a[k] = v[k] - u[k];
            b[k] = w[k] - u[k];
            c[k] = __ddiv_rn(__dadd_rn(__dadd_rn(u[k], v[k]), w[k]), 3.0);
        }
        double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        A = 0.5 * len;
        for (int k = 0; k < 3; ++k) n[k] = cr[k] / len;
        ph = x[i];
        dph = x[nt + i];
    }
    const R e = (R)eps, ie = (R)(1.0 / eps), kp = (R)kappa;
    double acc = 0.0;
    for (int t0 = 0; t0 < nc; t0 += NA_THREADS) {
        __syncthreads();
        if (t0 + threadIdx.x < nc) {
            int t = t0 + threadIdx.x;
            sq[threadIdx.x][0] = qpos[3 * t];
            sq[threadIdx.x][1] = qpos[3 * t + 1];
            sq[threadIdx.x][2] = qpos[3 * t + 2];
            sq[threadIdx.x][3] = q[t];
        }
        __syncthreads();
        int m = min(NA_THREADS, nc - t0);
        if (i < nt) {
            R s = 0;
            for (int t = 0; t < m; ++t) {
                R K[4];
                pb_kernels<R>((R)(sq[t][0] - c[0]), (R)(sq[t][1] - c[1]), (R)(sq[t][2] - c[2]), R(0), R(0), R(0),
                              (R)n[0], (R)n[1], (R)n[2], e, ie, kp, K);
                s += (R)sq[t][3] * (K[0] * (R)dph + K[1] * (R)ph);
            }
            acc += (double)s;
        }
    }
    red[threadIdx.x] = acc * A;
    __syncthreads();
    for (int h = NA_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];  // every slot that is read is written here first
}

__global__ void k_energy_noalloc_sum(int nb, const double* __restrict__ part, double scale, double* __restrict__ E)
{
    __shared__ double red[NA_THREADS];
    double s = 0.0;
    for (int k = threadIdx.x; k < nb; k += NA_THREADS) s += part[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = NA_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E = red[0] * scale;
}

static void na_msg(char* buf, int len, const char* s)
{
    if (buf && len > 0) {
        int k = 0;
        for (; s[k] && k < len - 1; ++k) buf[k] = s[k];
        buf[k] = 0;
    }
}

extern "C" int pb_solvation_energy_noalloc(const double* verts, const int32_t* tris, int nt, const double* qpos,
                                           const double* q, int nc, double eps_in, double eps_out, double kappa,
                                           int precision, const double* x, double* E, void* stream, char* errbuf,
                                           int errlen)
{
    if (!verts || !tris || !x || !E || nt < 1 || nc < 0 || (nc > 0 && (!qpos || !q))) {
        na_msg(errbuf, errlen, "pb_solvation_energy_noalloc: null pointer or nt < 1");
        return PB_ERR_ARG;
    }
    if (!(eps_in > 0) || !(eps_out > 0) || !(kappa >= 0) || (precision != PB_FP64 && precision != PB_MIXED)) {
        na_msg(errbuf, errlen, "pb_solvation_energy_noalloc: bad physical parameters or precision");
        return PB_ERR_ARG;
    }
    const int nb = (nt + NA_THREADS - 1) / NA_THREADS;
    if (nb > NA_MAX_BLOCKS) {
        na_msg(errbuf, errlen,
               "pb_solvation_energy_noalloc: nt exceeds the fixed scratch limit of 2097152 triangles");
        return PB_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        na_msg(errbuf, errlen, "pb_solvation_energy_noalloc: no current CUDA device");
        return PB_ERR_CUDA;
    }
    double* part = nullptr;
    {
        // first call on this device: look up the device address of the scratch array
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                na_msg(errbuf, errlen, "pb_solvation_energy_noalloc: cudaGetSymbolAddress failed");
                return PB_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = (double*)p;
        }
        part = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    double eps = eps_out / eps_in;
    // clear a launch error left by earlier, unrelated work, so that the check below reports
    // this call's launches only (an error that has made the context unusable stays and shows)
    cudaGetLastError();
    if (precision == PB_MIXED)
        k_energy_noalloc<float><<<nb, NA_THREADS, 0, st>>>(nt, verts, tris, nc, qpos, q, eps, kappa, x, part);
    else
        k_energy_noalloc<double><<<nb, NA_THREADS, 0, st>>>(nt, verts, tris, nc, qpos, q, eps, kappa, x, part);
    k_energy_noalloc_sum<<<1, NA_THREADS, 0, st>>>(nb, part, 0.5 * 4.0 * PB_PI * 332.0716, E);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        na_msg(errbuf, errlen, cudaGetErrorString(e));
        return PB_ERR_CUDA;
    }
    return PB_OK;
}
