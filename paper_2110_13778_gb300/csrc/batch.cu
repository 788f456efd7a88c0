// Several molecules and several charge states each, solved in one CUDA-graph launch.
//
// Each molecule has its own context (a context holds one mesh: the context is the mesh
// handle of this interface). The graph holds one independent branch per molecule, so the
// molecules' solves run side by side on the GPU; a branch is: the right-hand side of state 0
// and its device-driven GMRES from zero, then the right-hand sides of the other states and one
// device-driven GMRES over all of them (batched products, every state with its own Krylov basis
// and stopping test) started from state 0's solution scaled per state by its least-squares
// factor, then the energies of all states (eqsolengdis) and the solutions scattered to the
// caller's arrays. No host read happens until the whole graph has finished. The paper solves
// one molecule and one charge state at a time; this form of batching has no counterpart there.
#include <string.h>

#include <algorithm>
#include <vector>

#include "pb_internal.cuh"

__global__ void k_scatter_b(int n, const int* __restrict__ order, const double* __restrict__ xs, double* __restrict__ x)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    x += 2LL * n * blockIdx.y;
    xs += 2LL * n * blockIdx.y;
    if (k < n) {
        const int e = order[k];
        x[e] = xs[k];
        x[n + e] = xs[n + k];
    }
}

namespace {
struct Branch {
    pb_ctx* c;
    int R;                 // charge states
    int nchunk;            // batches of the states after the first
    long long cnt[1 + 16][3];
    long long extra;       // launches of the branch outside the two solves' loops
};
}  // namespace

static bool cap_begin(pb_ctx* c, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps)
{
    return cudaStreamBeginCaptureToGraph(c->st, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                         cudaStreamCaptureModeThreadLocal) == cudaSuccess;
}
static bool cap_end(pb_ctx* c, std::vector<cudaGraphNode_t>* leaves)
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

// one molecule's branch into g (c->st is the context's private capture stream)
static int branch(Branch& b, cudaGraph_t g, double* X, int m)
{
    pb_ctx* c = b.c;
    const size_t n2 = 2 * (size_t)c->nt;
    const int R = b.R;
    std::vector<cudaGraphNode_t> lv;
    int rc = PB_OK;
    // state 0: its right-hand side, then GMRES from zero
    if (!cap_begin(c, g, {})) return -1;
    rc = pb_rhs_states_sorted(c, c->qstates, c->ws, 1);
    if (!cap_end(c, &lv) || rc) return rc ? rc : -1;
    if ((rc = pb_dg_append(c, g, lv, c->xs, c->ws, 1, m, 0, 0, &lv, b.cnt[0]))) return rc;
    // the other states in batches of up to PB_MAX_RHS, each from state 0's solution
    for (int k = 0; k < b.nchunk; ++k) {
        const int s0 = 1 + k * PB_MAX_RHS, nr = std::min(PB_MAX_RHS, R - s0);
        if (!cap_begin(c, g, lv)) return -1;
        do {
            for (int q = 0; q < nr && !rc; q += 16)
                rc = pb_rhs_states_sorted(c, c->qstates + (size_t)(s0 + q) * c->nc, c->mys + q * n2, std::min(16, nr - q));
            if (rc) break;
            for (int r = 0; r < nr; ++r)
                PB_CUDA(c, cudaMemcpyAsync(c->mxs + r * n2, c->xs, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->st));
        } while (0);
        if (!cap_end(c, &lv) || rc) return rc ? rc : -1;
        if ((rc = pb_dg_append(c, g, lv, c->mxs, c->mys, nr, m, 1, 1 + k, &lv, b.cnt[1 + k]))) return rc;
        // this batch's energies and solutions before the next batch reuses the work vectors
        if (!cap_begin(c, g, lv)) return -1;
        do {
            for (int q = 0; q < nr && !rc; q += 16)
                rc = pb_energy_states_queue(c, c->qstates + (size_t)(s0 + q) * c->nc, c->mxs + q * n2,
                                            std::min(16, nr - q), c->bE + s0 + q);
            if (rc) break;
            k_scatter_b<<<dim3((c->nt + 255) / 256, nr), 256, 0, c->st>>>(c->nt, c->order, c->mxs, X + s0 * n2);
            PB_LAUNCH(c);
        } while (0);
        if (!cap_end(c, &lv) || rc) return rc ? rc : -1;
    }
    // state 0's energy and solution
    if (!cap_begin(c, g, lv)) return -1;
    do {
        if ((rc = pb_energy_states_queue(c, c->qstates, c->xs, 1, c->bE))) break;
        k_scatter_b<<<dim3((c->nt + 255) / 256, 1), 256, 0, c->st>>>(c->nt, c->order, c->xs, X);
        PB_LAUNCH(c);
    } while (0);
    if (!cap_end(c, nullptr) || rc) return rc ? rc : -1;
    return PB_OK;
}

extern "C" int pb_batch_solve_states(pb_ctx* const* ctxs, int nmol, const double* const* q, int nrhs,
                                     double* const* X, double* E, double tol, int max_iter, int restart,
                                     pb_solve_info* infos)
{
    if (!ctxs || nmol < 1 || !q || !X || nrhs < 1 || nrhs > 1 + 16 * PB_MAX_RHS || !(tol > 0) || max_iter < 1 ||
        restart < 1 || restart > 200)
        return PB_ERR_ARG;
    for (int k = 0; k < nmol; ++k) {
        pb_ctx* c = ctxs[k];
        if (!c || !q[k] || !X[k]) return PB_ERR_ARG;
        if (c->dead) return PB_ERR_CUDA;
        if (!c->built) return pb_fail(c, PB_ERR_STATE, "batch_solve_states before build_tree");
        if (c->timing) return pb_fail(c, PB_ERR_STATE, "batch_solve_states with per-phase timing enabled");
        if (c->q2 > 1) return pb_fail(c, PB_ERR_ARG, "batch_solve_states needs the one-point regular rule");
        for (long long i = 0; i < (long long)nrhs * c->nc; ++i)
            if (!isfinite(q[k][i])) return pb_fail(c, PB_ERR_MESH, "charge state value %lld not finite", i);
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == c) return pb_fail(c, PB_ERR_ARG, "batch_solve_states: a context appears twice");
    }
    const int nchunk = (nrhs - 1 + PB_MAX_RHS - 1) / PB_MAX_RHS;
    std::vector<Branch> br(nmol);
    int rc;
    // buffers first (nothing may be allocated while the graph is captured), charges uploaded
    for (int k = 0; k < nmol; ++k) {
        pb_ctx* c = ctxs[k];
        br[k].c = c;
        br[k].R = nrhs;
        br[k].nchunk = nchunk;
        const int nrm = std::max(1, std::min(PB_MAX_RHS, nrhs - 1));
        if ((rc = pb_matvec_reserve(c, nrm))) return rc;
        if ((rc = pb_dg_reserve(c, nrm, restart, 1 + nchunk))) return rc;
        if ((rc = pb_energy_reserve(c))) return rc;
        if (c->mv_nr < nrm) {
            c->mxs = (double*)pb_alloc(c, sizeof(double) * (size_t)nrm * 2 * c->nt);
            c->mys = (double*)pb_alloc(c, sizeof(double) * (size_t)nrm * 2 * c->nt);
            if (!c->mxs || !c->mys) return pb_fail(c, PB_ERR_NOMEM, "batch_solve_states: out of memory");
            c->mv_nr = nrm;
        }
        if (c->bE_n < nrhs) {
            c->bE = (double*)pb_alloc(c, sizeof(double) * nrhs);
            if (!c->bE) return pb_fail(c, PB_ERR_NOMEM, "batch_solve_states: out of memory");
            c->bE_n = nrhs;
        }
        if (c->qstates_n < nrhs) {
            c->qstates = (double*)pb_alloc(c, sizeof(double) * ((size_t)nrhs * c->nc + 1));
            if (!c->qstates) return pb_fail(c, PB_ERR_NOMEM, "batch_solve_states: out of memory");
            c->qstates_n = nrhs;
        }
        if (c->nc > 0)
            PB_CUDA(c, cudaMemcpyAsync(c->qstates, q[k], sizeof(double) * (size_t)nrhs * c->nc, cudaMemcpyHostToDevice,
                                       c->st));
        pb_dg_settings(c, 0, 1, restart, tol, max_iter);
        for (int j = 0; j < nchunk; ++j)
            pb_dg_settings(c, 1 + j, std::min(PB_MAX_RHS, nrhs - 1 - j * PB_MAX_RHS), restart, tol, max_iter);
        if ((rc = pb_dg_upload(c, 1 + nchunk))) return rc;
    }
    for (int k = 0; k < nmol; ++k) PB_CUDA(ctxs[k], cudaStreamSynchronize(ctxs[k]->st));
    // the graph: one branch per molecule
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return pb_fail(ctxs[0], PB_ERR_CUDA, "cudaGraphCreate failed");
    rc = PB_OK;
    for (int k = 0; k < nmol && rc == PB_OK; ++k) {
        pb_ctx* c = ctxs[k];
        cudaStream_t keep = c->st;
        c->st = c->cap_st;
        const long long nl = c->nlaunch;
        rc = branch(br[k], g, X[k], restart);
        br[k].extra = c->nlaunch - nl;
        for (int j = 0; j <= nchunk; ++j)
            br[k].extra -= br[k].cnt[j][0] + br[k].cnt[j][1] + br[k].cnt[j][2];
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(c->st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(c->st, &junk);
        }
        c->st = keep;
        c->nlaunch = nl;
    }
    cudaGraphExec_t ex = nullptr;
    if (rc == PB_OK && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) rc = -1;
    cudaGraphDestroy(g);
    if (rc != PB_OK) {
        cudaGetLastError();
        if (rc > 0) return rc;
        return pb_fail(ctxs[0], PB_ERR_CUDA, "batch_solve_states: the solve graph could not be built");
    }
    pb_ctx* c0 = ctxs[0];
    PB_CUDA(c0, cudaGraphLaunch(ex, c0->st));
    for (int k = 0; k < nmol; ++k) {
        pb_ctx* c = ctxs[k];
        ++c->graph_launches;
        if ((rc = pb_dg_download(c, 1 + nchunk))) break;
    }
    cudaError_t e1 = cudaStreamSynchronize(c0->st);
    cudaGraphExecDestroy(ex);
    if (rc) return rc;
    PB_CUDA(c0, e1);
    int worst = PB_OK;
    std::vector<double> Eh(nrhs);
    for (int k = 0; k < nmol; ++k) {
        pb_ctx* c = ctxs[k];
        PB_CUDA(c, cudaMemcpy(Eh.data(), c->bE, sizeof(double) * nrhs, cudaMemcpyDeviceToHost));
        int derr = 0;
        PB_CUDA(c, cudaMemcpy(&derr, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (E)
            for (int r = 0; r < nrhs; ++r) E[(size_t)k * nrhs + r] = Eh[r];
        pb_solve_info* inf = infos ? infos + (size_t)k * nrhs : nullptr;
        pb_dg_results(c, 0, 1, br[k].cnt[0], inf, &worst);
        for (int j = 0; j < nchunk; ++j)
            pb_dg_results(c, 1 + j, std::min(PB_MAX_RHS, nrhs - 1 - j * PB_MAX_RHS), br[k].cnt[1 + j],
                          inf ? inf + 1 + j * PB_MAX_RHS : nullptr, &worst);
        c->nlaunch += br[k].extra;  // right-hand sides, energies and scatters
        if (derr) {
            worst = PB_ERR_TIMEOUT;
            pb_fail(c, PB_ERR_TIMEOUT, "a bounded wait in the MtL kernel gave up");
        }
    }
    return worst;
}
