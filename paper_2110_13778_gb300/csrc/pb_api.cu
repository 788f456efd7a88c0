// C ABI entry points of libpb: context, mesh upload, orchestration of the solve.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pb_internal.cuh"

int pb_fail(pb_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

void* pb_alloc(pb_ctx* c, size_t bytes, bool build_lifetime) { return pb_alloc_on(c, bytes, c->st, build_lifetime); }

void* pb_alloc_on(pb_ctx* c, size_t bytes, cudaStream_t s, bool build_lifetime)
{
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    // stream-ordered allocation from the context's pool, which keeps released memory for reuse
    if (cudaMallocFromPoolAsync(&p, bytes, c->pool, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaMemsetAsync(p, 0, bytes, s) != cudaSuccess) {
        cudaFreeAsync(p, s);
        return nullptr;
    }
    (build_lifetime ? c->build_allocs : c->mesh_allocs).push_back(p);
    return p;
}

// drop everything pb_build_tree made (tree, lists, integrals, factors, work vectors)
static void pb_free_build(pb_ctx* c)
{
    for (void* p : c->build_allocs) cudaFreeAsync(p, c->st);
    c->build_allocs.clear();
    c->built = false;
    c->touch_class_dev = nullptr;
    c->canon_check = nullptr;
    c->canon_expect = 0;
    c->gm_m = 0;
    c->gmwf = nullptr;
    c->gmvd = nullptr;
    c->scratch = nullptr;
    c->escratch = nullptr;
    c->qstates = nullptr;
    c->qstates_n = 0;
    pb_drop_graphs(c);
    c->gb_graph_failed = false;
    c->mv_nr = c->gb_nr = c->gb_m = c->dens_nr = 0;
    c->far_nr = 1;
    c->mxs = c->mys = c->gbV = c->gbW = c->gbZ = c->gbB = c->gbpart = c->gbsmall = nullptr;
    pb_dg_drop(c);
    c->tc_part = nullptr;
    c->tc_nw = 0;
    c->bE = nullptr;
    c->bE_n = 0;
    c->q2 = 1;
    c->pts_p = c->pts_n = nullptr;
    c->begin_q = nullptr;
    c->xq = c->yq = nullptr;
    c->p1_voff = c->p1_vlist = nullptr;
    c->p1_corr = c->p1_diag = c->p1_pinv = c->p1_yqn = c->p1_yl = nullptr;
    c->pn_nitems = 0;
    c->pn_items = nullptr;
    c->pn_tiles = c->pn_chunk_leaf = c->pn_chunk_first = c->pn_begin = nullptr;
    c->pn_p32 = c->pn_l32 = c->pn_n32 = c->pn_sp = c->pn_sn = nullptr;
    c->pn_y = nullptr;
    c->dgVcur = nullptr;
    c->dgWf = nullptr;
    c->dgctl = nullptr;
    c->dg_nr = c->dg_nctl = 0;
    ++c->build_gen;
    c->near_dens = nullptr;
    c->yfar = nullptr;
    c->yfar_nr = 0;
    c->L = 0;
    for (auto& l : c->lev) l = PbLevel();
    c->cent = c->area = c->nrm = nullptr;
}

static void pb_free_mesh(pb_ctx* c)
{
    pb_free_build(c);
    for (void* p : c->mesh_allocs) cudaFreeAsync(p, c->st);
    c->mesh_allocs.clear();
    c->verts = c->qpos = c->q = nullptr;
    c->tris = nullptr;
    c->nt = c->nv = c->nc = 0;
}

extern "C" int pb_create(const pb_params* prm, void* stream, pb_ctx** out)
{
    if (!prm || !out) return PB_ERR_ARG;
    *out = nullptr;
    if (!(prm->eps_in > 0) || !(prm->eps_out > 0) || !(prm->kappa >= 0)) return PB_ERR_ARG;
    if (!(prm->eta0 > 0 && prm->eta0 < 1)) return PB_ERR_ARG;
    if (prm->p < 0 || prm->p > 10 || prm->qs < 1 || prm->qs > 8) return PB_ERR_ARG;
    if (prm->levels < 0 || prm->levels > PB_MAXL || (prm->levels == 0 && prm->leaf_size < 1))
        return PB_ERR_ARG;
    if (prm->precision != PB_FP64 && prm->precision != PB_MIXED) return PB_ERR_ARG;
    if (prm->singular < PB_SINGULAR_AUTO || prm->singular > PB_SINGULAR_FF) return PB_ERR_ARG;
    if (prm->precond < PB_PRECOND_NONE || prm->precond > PB_PRECOND_BLOCK) return PB_ERR_ARG;
    if (prm->pc_block != 0 && (prm->pc_block < 8 || prm->pc_block > 96)) return PB_ERR_ARG;
    if (prm->qr < 0 || prm->qr > 4) return PB_ERR_ARG;
    if (prm->basis != PB_BASIS_CONSTANT && prm->basis != PB_BASIS_LINEAR) return PB_ERR_ARG;
    if (prm->basis == PB_BASIS_LINEAR && prm->qr < 2) return PB_ERR_ARG;  // the points carry the linear functions
    pb_ctx* c = new pb_ctx();
    c->prm = *prm;
    c->st = (cudaStream_t)stream;
    void* h = nullptr;
    if (cudaMallocHost(&h, 64 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return PB_ERR_NOMEM;
    }
    c->hscal = (double*)h;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    if (cudaMemPoolCreate(&c->pool, &pp) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(h);
        delete c;
        return PB_ERR_NOMEM;
    }
    unsigned long long keep = ~0ULL;  // never hand released blocks back to the driver early
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    for (int i = 0; i < 10; ++i) cudaEventCreate(&c->ev[i]);
    // the far field runs on a second stream of the highest priority, overlapping the near field
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&c->st2, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_tree, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_sing, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        pb_destroy(c);
        return PB_ERR_CUDA;
    }
    *out = c;
    return PB_OK;
}

extern "C" int pb_destroy(pb_ctx* c)
{
    if (!c) return PB_OK;
    for (void* p : c->mesh_allocs) cudaFreeAsync(p, c->st);
    for (void* p : c->build_allocs) cudaFreeAsync(p, c->st);
    cudaStreamSynchronize(c->st);
    if (c->st2) {
        cudaStreamSynchronize(c->st2);
        cudaStreamDestroy(c->st2);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_tree) cudaEventDestroy(c->ev_tree);
    if (c->ev_sing) cudaEventDestroy(c->ev_sing);
    pb_drop_graphs(c);
    pb_dg_drop(c);
    if (c->dgctl_h) cudaFreeHost(c->dgctl_h);
    if (c->cap_st) cudaStreamDestroy(c->cap_st);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    for (int i = 0; i < 10; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->tev_ready)
        for (int a = 0; a < 2; ++a)
            for (int s = 0; s < PB_TIMING_SLOTS; ++s)
                for (int k = 0; k < PB_TMAX; ++k) cudaEventDestroy(c->tev[a][s][k]);
    if (c->hscal) cudaFreeHost(c->hscal);
    delete c;
    return PB_OK;
}

extern "C" const char* pb_last_error(const pb_ctx* c) { return c ? c->err.c_str() : "null context"; }

#define PB_ALIVE(c)                                                          \
    do {                                                                     \
        if (!(c)) return PB_ERR_ARG;                                         \
        if ((c)->dead) return pb_fail((c), PB_ERR_CUDA, "context is dead after a CUDA error"); \
    } while (0)

extern "C" int pb_mesh_upload(pb_ctx* c, const double* verts, int nv, const int32_t* tris, int nt,
                              const double* qpos, const double* q, int nc)
{
    PB_ALIVE(c);
    if (!verts || !tris || nv < 3 || nt < 1 || nc < 0 || (nc > 0 && (!qpos || !q)))
        return pb_fail(c, PB_ERR_ARG, "mesh_upload: need nv >= 3, nt >= 1 and non-null arrays");
    // host-side validation (indices, zero-area or non-finite triangles)
    for (int i = 0; i < nt; ++i) {
        int a = tris[3 * i], b = tris[3 * i + 1], d = tris[3 * i + 2];
        if (a < 0 || b < 0 || d < 0 || a >= nv || b >= nv || d >= nv || a == b || b == d || a == d)
            return pb_fail(c, PB_ERR_MESH, "triangle %d has a bad vertex index", i);
        const double *u = verts + 3 * a, *v = verts + 3 * b, *w = verts + 3 * d;
        double e1[3] = {v[0] - u[0], v[1] - u[1], v[2] - u[2]};
        double e2[3] = {w[0] - u[0], w[1] - u[1], w[2] - u[2]};
        double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                        e1[0] * e2[1] - e1[1] * e2[0]};
        double A2 = cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2];
        if (!(A2 > 0) || !isfinite(A2)) return pb_fail(c, PB_ERR_MESH, "triangle %d has zero area", i);
    }
    for (int k = 0; k < 3 * nc; ++k)
        if (!isfinite(qpos[k])) return pb_fail(c, PB_ERR_MESH, "charge position %d not finite", k / 3);
    for (int k = 0; k < nc; ++k)
        if (!isfinite(q[k])) return pb_fail(c, PB_ERR_MESH, "charge %d not finite", k);
    pb_free_mesh(c);
    c->verts = (double*)pb_alloc(c, sizeof(double) * 3 * nv, false);
    c->tris = (int*)pb_alloc(c, sizeof(int) * 3 * nt, false);
    c->qpos = (double*)pb_alloc(c, sizeof(double) * 3 * (nc > 0 ? nc : 1), false);
    c->q = (double*)pb_alloc(c, sizeof(double) * (nc > 0 ? nc : 1), false);
    if (!c->verts || !c->tris || !c->qpos || !c->q) return pb_fail(c, PB_ERR_NOMEM, "mesh_upload: out of memory");
    PB_CUDA(c, cudaMemcpyAsync(c->verts, verts, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaMemcpyAsync(c->tris, tris, sizeof(int) * 3 * nt, cudaMemcpyHostToDevice, c->st));
    if (nc > 0) {
        PB_CUDA(c, cudaMemcpyAsync(c->qpos, qpos, sizeof(double) * 3 * nc, cudaMemcpyHostToDevice, c->st));
        PB_CUDA(c, cudaMemcpyAsync(c->q, q, sizeof(double) * nc, cudaMemcpyHostToDevice, c->st));
    }
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    c->nv = nv;
    c->nt = nt;
    c->nc = nc;
    return PB_OK;
}

extern "C" int pb_set_charges(pb_ctx* c, const double* q, int nc)
{
    PB_ALIVE(c);
    if (!c->verts) return pb_fail(c, PB_ERR_STATE, "set_charges before mesh_upload");
    if (nc != c->nc || (nc > 0 && !q)) return pb_fail(c, PB_ERR_ARG, "set_charges: nc must match the upload");
    for (int k = 0; k < nc; ++k)
        if (!isfinite(q[k])) return pb_fail(c, PB_ERR_MESH, "charge %d not finite", k);
    if (nc > 0) PB_CUDA(c, cudaMemcpyAsync(c->q, q, sizeof(double) * nc, cudaMemcpyHostToDevice, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    return PB_OK;
}

extern "C" int pb_build_tree(pb_ctx* c)
{
    PB_ALIVE(c);
    if (!c->verts) return pb_fail(c, PB_ERR_STATE, "build_tree before mesh_upload");
    pb_free_build(c);
    int rc;
    c->dev_err = (int*)pb_alloc(c, sizeof(int));
    if (!c->dev_err) return pb_fail(c, PB_ERR_NOMEM, "build_tree: out of memory");
    pb_tic(c, PB_T_TREE);
    if ((rc = pb_geometry_and_tree(c))) return rc;
    c->nu = c->prm.basis == PB_BASIS_LINEAR ? c->nv : c->nt;
    if ((rc = pb_regular_setup(c))) return rc;
    pb_toc(c, PB_T_TREE);
    // Everything that reads tree data back to the host is planned first; then the singular
    // integrals run on the first stream while the host prepares the far-field setup. The
    // setup's table kernels (second stream) start when the singular pass ends and run beside
    // the preconditioner's factorisation (first stream), whose block inversions leave most of
    // each SM free; the streams are joined at the end.
    if ((rc = pb_near_setup(c))) return rc;
    if ((rc = pb_near_points_setup(c))) return rc;
    const bool linear = c->prm.basis == PB_BASIS_LINEAR;
    if (!linear && (rc = pb_precond_plan(c))) return rc;
    PB_CUDA(c, cudaEventRecord(c->ev_tree, c->st));
    pb_tic(c, PB_T_SINGULAR);
    if ((rc = pb_touching_and_singular(c))) return rc;
    if ((rc = linear ? pb_p1_setup(c) : pb_regular_corrections(c))) return rc;
    pb_toc(c, PB_T_SINGULAR);
    PB_CUDA(c, cudaEventRecord(c->ev_sing, c->st));
    if ((rc = pb_far_setup(c))) return rc;  // times its table kernels as PB_T_FARSETUP
    pb_tic(c, PB_T_PCBUILD);
    if (!linear && (rc = pb_precond_factor(c))) return rc;
    pb_toc(c, PB_T_PCBUILD);
    PB_CUDA(c, cudaStreamWaitEvent(c->st, c->ev_join, 0));
    size_t n2 = 2 * (size_t)std::max(c->nt, c->nv);  // element or vertex unknowns
    c->xs = (double*)pb_alloc(c, sizeof(double) * n2);
    c->ys = (double*)pb_alloc(c, sizeof(double) * n2);
    c->ws = (double*)pb_alloc(c, sizeof(double) * n2);
    if (!c->xs || !c->ys || !c->ws) return pb_fail(c, PB_ERR_NOMEM, "build_tree: out of memory");
    int ncanon = c->canon_expect;
    if (c->canon_check) PB_CUDA(c, cudaMemcpyAsync(&ncanon, c->canon_check, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    if (ncanon != c->canon_expect)
        return pb_fail(c, PB_ERR_MESH, "touching pairs are not symmetric (%d unordered pairs, %d expected)", ncanon,
                       c->canon_expect);
    c->built = true;
    return PB_OK;
}

// ---------- permutation between element order and tree order ----------
__global__ void k_gather(int n, const int* __restrict__ order, const double* __restrict__ x,
                         double* __restrict__ xs)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    x += 2LL * n * blockIdx.y;  // vector blockIdx.y of a batch
    xs += 2LL * n * blockIdx.y;
    if (k < n) {
        int e = order[k];
        xs[k] = x[e];
        xs[n + k] = x[n + e];
    }
}

__global__ void k_scatter(int n, const int* __restrict__ order, const double* __restrict__ xs,
                          double* __restrict__ x)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    x += 2LL * n * blockIdx.y;
    xs += 2LL * n * blockIdx.y;
    if (k < n) {
        int e = order[k];
        x[e] = xs[k];
        x[n + e] = xs[n + k];
    }
}

int pb_gather(pb_ctx* c, const double* x, double* xs)
{
    if (c->prm.basis == PB_BASIS_LINEAR) {  // vertex vectors keep the uploaded order
        PB_CUDA(c, cudaMemcpyAsync(xs, x, sizeof(double) * 2 * (size_t)c->nv, cudaMemcpyDeviceToDevice, c->st));
        return PB_OK;
    }
    int n = c->nt;
    k_gather<<<(n + 255) / 256, 256, 0, c->st>>>(n, c->order, x, xs);
    PB_LAUNCH(c);
    return PB_OK;
}

int pb_scatter(pb_ctx* c, const double* xs, double* x)
{
    if (c->prm.basis == PB_BASIS_LINEAR) {
        PB_CUDA(c, cudaMemcpyAsync(x, xs, sizeof(double) * 2 * (size_t)c->nv, cudaMemcpyDeviceToDevice, c->st));
        return PB_OK;
    }
    int n = c->nt;
    k_scatter<<<(n + 255) / 256, 256, 0, c->st>>>(n, c->order, xs, x);
    PB_LAUNCH(c);
    return PB_OK;
}

// y = A x in tree order for nr vectors (which: 0 = all, 1 = near field incl. mass and
// corrections, 2 = far field). The far field runs on the context's second stream into its own
// buffer, overlapping the near field; the corrections kernel waits for it and adds it in.
int pb_matvec_reserve(pb_ctx* c, int nr)
{
    int rc;
    if ((rc = pb_far_reserve(c, nr))) return rc;
    if (nr > c->yfar_nr) {
        c->yfar = (double*)pb_alloc(c, sizeof(double) * 2 * (size_t)std::max(c->nt, c->nv) * nr);
        if (!c->yfar) return pb_fail(c, PB_ERR_NOMEM, "matvec: out of memory");
        c->yfar_nr = nr;
    }
    return pb_near_reserve(c, nr);
}

void pb_drop_graphs(pb_ctx* c)
{
    for (cudaGraphExec_t g : c->gb_graphs)
        if (g) cudaGraphExecDestroy(g);
    c->gb_graphs.clear();
    c->gb_graph_n.clear();
    c->gb_graph_key = nullptr;
}

static int matvec_parts(pb_ctx* c, const double* xs, double* ys, int nr, int which)
{
    int rc;
    if (c->q2 > 1 && nr > 1) {  // the regular rule of order > 1 works one vector at a time
        for (int r = 0; r < nr; ++r)
            if ((rc = matvec_parts(c, xs + 2LL * c->nt * r, ys + 2LL * c->nt * r, 1, which))) return rc;
        return PB_OK;
    }
    const bool far = which != 1;
    // every buffer the product touches exists before the fork (and before any capture)
    if ((rc = pb_matvec_reserve(c, nr))) return rc;
    if (far) {
        PB_CUDA(c, cudaEventRecord(c->ev_fork, c->st));
        PB_CUDA(c, cudaStreamWaitEvent(c->st2, c->ev_fork, 0));
        if ((rc = pb_far_apply(c, xs, c->yfar, nr, c->st2))) return rc;
        PB_CUDA(c, cudaEventRecord(c->ev_join, c->st2));
    }
    if (which == 2) {
        PB_CUDA(c, cudaMemsetAsync(ys, 0, sizeof(double) * 2 * c->nt * nr, c->st));
        PB_CUDA(c, cudaStreamWaitEvent(c->st, c->ev_join, 0));
        return pb_corr_apply(c, nullptr, ys, nr, c->yfar);
    }
    pb_tic(c, PB_T_NEAR);
    if ((rc = c->q2 > 1 ? pb_near_q_apply(c, xs, ys)
                        : nr == 1 ? pb_near_apply(c, xs, ys) : pb_near_apply_multi(c, xs, ys, nr)))
        return rc;
    pb_toc(c, PB_T_NEAR);
    if (far) PB_CUDA(c, cudaStreamWaitEvent(c->st, c->ev_join, 0));
    pb_tic(c, PB_T_CORR);
    if ((rc = pb_corr_apply(c, xs, ys, nr, far ? c->yfar : nullptr))) return rc;
    pb_toc(c, PB_T_CORR);
    return PB_OK;
}

int pb_matvec_sorted(pb_ctx* c, const double* xs, double* ys, int which)
{
    if (c->prm.basis == PB_BASIS_LINEAR) return pb_p1_matvec(c, xs, ys);
    return matvec_parts(c, xs, ys, 1, which);
}

// nr products at once: xs and ys hold nr vectors of 2 nt in tree order
int pb_matvec_sorted_multi(pb_ctx* c, const double* xs, double* ys, int nr)
{
    if (c->prm.basis == PB_BASIS_LINEAR) {
        if (nr != 1) return pb_fail(c, PB_ERR_ARG, "piecewise-linear basis: one vector at a time");
        return pb_p1_matvec(c, xs, ys);
    }
    return matvec_parts(c, xs, ys, nr, 0);
}

// tree-ordered work vectors for nr right-hand sides (build lifetime, grown on demand)
static int reserve_multi(pb_ctx* c, int nr)
{
    if (nr <= c->mv_nr) return PB_OK;
    const size_t n = (size_t)nr * 2 * c->nt;
    c->mxs = (double*)pb_alloc(c, sizeof(double) * n);
    c->mys = (double*)pb_alloc(c, sizeof(double) * n);
    if (!c->mxs || !c->mys) return pb_fail(c, PB_ERR_NOMEM, "matvec_multi: out of memory");
    c->mv_nr = nr;
    return PB_OK;
}

extern "C" int pb_matvec_multi(pb_ctx* c, const double* X, double* Y, int nr)
{
    PB_ALIVE(c);
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "matvec before build_tree");
    if (!X || !Y || X == Y || nr < 1 || nr > PB_MAX_RHS) return pb_fail(c, PB_ERR_ARG, "matvec_multi: bad arguments");
    if (c->prm.basis != PB_BASIS_CONSTANT) return pb_fail(c, PB_ERR_ARG, "matvec_multi: piecewise-constant basis only");
    int rc;
    if ((rc = reserve_multi(c, nr))) return rc;
    const int n = c->nt;
    k_gather<<<dim3((n + 255) / 256, nr), 256, 0, c->st>>>(n, c->order, X, c->mxs);
    PB_LAUNCH(c);
    if ((rc = pb_matvec_sorted_multi(c, c->mxs, c->mys, nr))) return rc;
    k_scatter<<<dim3((n + 255) / 256, nr), 256, 0, c->st>>>(n, c->order, c->mys, Y);
    PB_LAUNCH(c);
    return PB_OK;
}

extern "C" int pb_matvec_part(pb_ctx* c, const double* x, double* y, int which)
{
    PB_ALIVE(c);
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "matvec before build_tree");
    if (!x || !y || x == y || which < 0 || which > 2) return pb_fail(c, PB_ERR_ARG, "matvec: bad arguments");
    if (which != 0 && c->prm.basis != PB_BASIS_CONSTANT)
        return pb_fail(c, PB_ERR_ARG, "matvec_part: piecewise-constant basis only");
    int rc;
    if ((rc = pb_gather(c, x, c->xs))) return rc;
    if ((rc = pb_matvec_sorted(c, c->xs, c->ys, which))) return rc;
    return pb_scatter(c, c->ys, y);
}

extern "C" int pb_matvec(pb_ctx* c, const double* x, double* y) { return pb_matvec_part(c, x, y, 0); }

extern "C" int pb_rhs(pb_ctx* c, double* b)
{
    PB_ALIVE(c);
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "rhs before build_tree");
    if (!b) return pb_fail(c, PB_ERR_ARG, "rhs: null output");
    int rc;
    if ((rc = pb_rhs_sorted(c, c->ws))) return rc;
    return pb_scatter(c, c->ws, b);
}

extern "C" int pb_precond_apply(pb_ctx* c, const double* r, double* z)
{
    PB_ALIVE(c);
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "precond before build_tree");
    if (!r || !z || r == z) return pb_fail(c, PB_ERR_ARG, "precond: bad arguments");
    int rc;
    if ((rc = pb_gather(c, r, c->xs))) return rc;
    if ((rc = pb_precond_apply_sorted(c, c->xs, c->ys))) return rc;
    return pb_scatter(c, c->ys, z);
}

extern "C" int pb_gmres_solve(pb_ctx* c, double* x, double tol, int max_iter, int restart,
                              int use_x0, pb_solve_info* info)
{
    PB_ALIVE(c);
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "solve before build_tree");
    if (!x || !(tol > 0) || max_iter < 1 || restart < 1 || restart > 200)
        return pb_fail(c, PB_ERR_ARG, "gmres: bad arguments");
    int rc;
    // b in ws, x0 in xs (both sorted)
    if ((rc = pb_rhs_sorted(c, c->ws))) return rc;
    if (use_x0) {
        if ((rc = pb_gather(c, x, c->xs))) return rc;
    } else {
        PB_CUDA(c, cudaMemsetAsync(c->xs, 0, sizeof(double) * 2 * (size_t)c->nu, c->st));
    }
    pb_solve_info loc;
    // one graph launch with the stopping test on the device; with per-phase timing enabled (or
    // where the graph cannot be built) the host-driven loop, which reads one residual per step
    rc = -1;
    if (!c->timing && !c->dg_failed) {
        rc = pb_gmres_dev(c, c->xs, c->ws, 1, tol, max_iter, restart, use_x0 ? 1 : 0, &loc);
        if (rc == -1) c->dg_failed = true;
    }
    if (rc == -1) rc = pb_gmres_sorted(c, c->xs, c->ws, tol, max_iter, restart, &loc, !use_x0);
    if (rc && rc != PB_ERR_NOT_CONVERGED && rc != PB_ERR_NONFINITE && rc != PB_ERR_TIMEOUT) return rc;
    int rc2 = pb_scatter(c, c->xs, x);
    if (info) *info = loc;
    if (rc2) return rc2;
    if (rc == PB_ERR_NOT_CONVERGED)
        pb_fail(c, rc, "gmres: not converged after %d iterations (relative residual %.3g)", loc.iterations,
                loc.rel_residual);
    else if (rc == PB_ERR_NONFINITE)
        pb_fail(c, rc, "gmres: a residual is not finite");
    return rc;
}

extern "C" int pb_solve_states(pb_ctx* c, const double* q, int nrhs, double* X, double* E, double tol,
                               int max_iter, int restart, int warm, pb_solve_info* infos)
{
    PB_ALIVE(c);
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "solve_states before build_tree");
    if (!q || !X || nrhs < 1 || !(tol > 0) || max_iter < 1 || restart < 1 || restart > 200 || warm < 0 || warm > 2)
        return pb_fail(c, PB_ERR_ARG, "solve_states: bad arguments");
    if (c->prm.basis != PB_BASIS_CONSTANT) return pb_fail(c, PB_ERR_ARG, "solve_states: piecewise-constant basis only");
    for (long long k = 0; k < (long long)nrhs * c->nc; ++k)
        if (!isfinite(q[k])) return pb_fail(c, PB_ERR_MESH, "charge state value %lld not finite", k);
    if (warm == 2 && c->q2 > 1)
        return pb_fail(c, PB_ERR_ARG, "solve_states: batched states need the one-point regular rule");
    const size_t n2 = 2 * (size_t)c->nt;
    int worst = PB_OK;
    // batched: state 0 alone from zero, then the others in lockstep from its solution
    const int nseq = warm == 2 ? 1 : nrhs;
    for (int s = 0; s < nseq; ++s) {
        if (c->nc > 0)
            PB_CUDA(c, cudaMemcpyAsync(c->q, q + (size_t)s * c->nc, sizeof(double) * c->nc, cudaMemcpyHostToDevice,
                                       c->st));
        int rc;
        if ((rc = pb_rhs_sorted(c, c->ws))) return rc;
        if (!(warm && s > 0)) PB_CUDA(c, cudaMemsetAsync(c->xs, 0, sizeof(double) * n2, c->st));
        pb_solve_info loc;
        rc = -1;
        if (!c->timing && !c->dg_failed) {
            rc = pb_gmres_dev(c, c->xs, c->ws, 1, tol, max_iter, restart, (warm && s > 0) ? 1 : 0, &loc);
            if (rc == -1) c->dg_failed = true;
        }
        if (rc == -1) rc = pb_gmres_sorted(c, c->xs, c->ws, tol, max_iter, restart, &loc, !(warm && s > 0));
        if (rc && rc != PB_ERR_NOT_CONVERGED && rc != PB_ERR_NONFINITE && rc != PB_ERR_TIMEOUT) return rc;
        if (rc && worst == PB_OK) worst = rc;
        if (infos) infos[s] = loc;
        if ((rc = pb_scatter(c, c->xs, X + (size_t)s * n2))) return rc;
        if (E) {
            double e = 0.0;
            if ((rc = pb_energy_sorted(c, c->xs, &e))) return rc;
            E[s] = e;
        }
    }
    for (int s0 = nseq; s0 < nrhs; s0 += PB_MAX_RHS) {
        const int nr = std::min(PB_MAX_RHS, nrhs - s0);
        int rc;
        if ((rc = reserve_multi(c, nr))) return rc;
        double *Xs = c->mxs, *Bs = c->mys;
        // the batch's charges on the device, then the right-hand sides 16 states per launch
        // (the pair geometry is shared by the states)
        if (!c->qstates || c->qstates_n < PB_MAX_RHS) {
            c->qstates = (double*)pb_alloc(c, sizeof(double) * ((size_t)PB_MAX_RHS * c->nc + 1));
            if (!c->qstates) return pb_fail(c, PB_ERR_NOMEM, "solve_states: out of memory");
            c->qstates_n = PB_MAX_RHS;
        }
        if (c->nc > 0)
            PB_CUDA(c, cudaMemcpyAsync(c->qstates, q + (size_t)s0 * c->nc, sizeof(double) * c->nc * nr,
                                       cudaMemcpyHostToDevice, c->st));
        for (int g = 0; g < nr; g += 16)
            if ((rc = pb_rhs_states_sorted(c, c->qstates + (size_t)g * c->nc, Bs + g * n2, std::min(16, nr - g))))
                return rc;
        for (int r = 0; r < nr; ++r)
            PB_CUDA(c, cudaMemcpyAsync(Xs + r * n2, c->xs, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->st));
        std::vector<pb_solve_info> loc(nr);
        rc = -1;
        if (!c->timing && !c->dg_failed) {
            rc = pb_gmres_dev(c, Xs, Bs, nr, tol, max_iter, restart, 1, loc.data());
            if (rc == -1) c->dg_failed = true;
        }
        if (rc == -1) rc = pb_gmres_batch_sorted(c, Xs, Bs, nr, tol, max_iter, restart, loc.data());
        if (rc && rc != PB_ERR_NOT_CONVERGED && rc != PB_ERR_NONFINITE && rc != PB_ERR_TIMEOUT) return rc;
        if (rc && worst == PB_OK) worst = rc;
        for (int r = 0; r < nr; ++r) {
            if (infos) infos[s0 + r] = loc[r];
            if ((rc = pb_scatter(c, Xs + r * n2, X + (size_t)(s0 + r) * n2))) return rc;
        }
        if (E)
            for (int g = 0; g < nr; g += 16)
                if ((rc = pb_energy_states_sorted(c, c->qstates + (size_t)g * c->nc, Xs + g * n2,
                                                  std::min(16, nr - g), E + s0 + g)))
                    return rc;
        // the uploaded charges are left as those of the last state
        if (c->nc > 0 && s0 + nr == nrhs)
            PB_CUDA(c, cudaMemcpyAsync(c->q, q + (size_t)(nrhs - 1) * c->nc, sizeof(double) * c->nc,
                                       cudaMemcpyHostToDevice, c->st));
    }
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    return worst;
}

extern "C" int pb_solvation_energy(pb_ctx* c, const double* x, double* E)
{
    PB_ALIVE(c);
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "energy before build_tree");
    if (!x || !E) return pb_fail(c, PB_ERR_ARG, "energy: null argument");
    int rc;
    if ((rc = pb_gather(c, x, c->xs))) return rc;
    return pb_energy_sorted(c, c->xs, E);
}

extern "C" int pb_solvation_energy_treecode(pb_ctx* c, const double* x, double theta, double* E)
{
    PB_ALIVE(c);
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "energy before build_tree");
    if (c->prm.basis != PB_BASIS_CONSTANT) return pb_fail(c, PB_ERR_ARG, "treecode energy: piecewise-constant basis only");
    if (!x || !E || !(theta > 0) || !(theta < 1)) return pb_fail(c, PB_ERR_ARG, "treecode energy: bad argument");
    int rc;
    if ((rc = pb_gather(c, x, c->xs))) return rc;
    return pb_energy_treecode_sorted(c, c->xs, theta, E);
}

extern "C" int pb_get_tree_stats(pb_ctx* c, pb_tree_stats* s)
{
    PB_ALIVE(c);
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "tree stats before build_tree");
    if (!s) return pb_fail(c, PB_ERR_ARG, "null output");
    memset(s, 0, sizeof(*s));
    s->levels = c->L;
    for (int l = 0; l <= c->L; ++l) {
        s->nclusters[l] = c->lev[l].ncl;
        s->nnear[l] = c->lev[l].nnear;
        s->ninter[l] = c->lev[l].ninter;
        s->order[l] = c->lev[l].p;
    }
    s->near_pairs = c->near_pairs;
    s->touching = c->ntouch;
    if (c->touch_class_dev) {
        unsigned long long h[4];
        PB_CUDA(c, cudaMemcpyAsync(h, c->touch_class_dev, sizeof(h), cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
        for (int q = 0; q < 4; ++q) c->touch_class[q] = (long long)h[q];
        c->touch_class_dev = nullptr;
    }
    for (int q = 0; q < 4; ++q) s->touch_class[q] = c->touch_class[q];
    s->max_leaf = c->max_leaf;
    if (c->prm.precond == PB_PRECOND_BLOCK) {
        s->pc_blocks = c->npcblk;
        s->pc_max = c->pc_max;
        s->pc_sum_m3 = c->pc_sum_m3;
    }
    return PB_OK;
}

extern "C" int pb_get_tree(pb_ctx* c, int32_t* order, int32_t* level_begin, int32_t* near_cnt,
                           int32_t* near_idx, int32_t* inter_cnt, int32_t* inter_idx)
{
    PB_ALIVE(c);
    if (!c->built) return pb_fail(c, PB_ERR_STATE, "get_tree before build_tree");
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    if (order) PB_CUDA(c, cudaMemcpy(order, c->order, sizeof(int) * c->nt, cudaMemcpyDeviceToHost));
    size_t cl = 0, nn = 0, ni = 0;
    for (int l = 0; l <= c->L; ++l) {
        const PbLevel& lv = c->lev[l];
        std::vector<int> off(lv.ncl + 1);
        if (level_begin)
            PB_CUDA(c, cudaMemcpy(level_begin + cl, lv.begin, sizeof(int) * lv.ncl, cudaMemcpyDeviceToHost));
        PB_CUDA(c, cudaMemcpy(off.data(), lv.near_off, sizeof(int) * (lv.ncl + 1), cudaMemcpyDeviceToHost));
        if (near_cnt)
            for (int k = 0; k < lv.ncl; ++k) near_cnt[cl + k] = off[k + 1] - off[k];
        if (near_idx && lv.nnear)
            PB_CUDA(c, cudaMemcpy(near_idx + nn, lv.near_idx, sizeof(int) * lv.nnear, cudaMemcpyDeviceToHost));
        PB_CUDA(c, cudaMemcpy(off.data(), lv.int_off, sizeof(int) * (lv.ncl + 1), cudaMemcpyDeviceToHost));
        if (inter_cnt)
            for (int k = 0; k < lv.ncl; ++k) inter_cnt[cl + k] = off[k + 1] - off[k];
        if (inter_idx && lv.ninter)
            PB_CUDA(c, cudaMemcpy(inter_idx + ni, lv.int_idx, sizeof(int) * lv.ninter, cudaMemcpyDeviceToHost));
        cl += lv.ncl;
        nn += lv.nnear;
        ni += lv.ninter;
    }
    return PB_OK;
}

extern "C" int pb_set_timing(pb_ctx* c, int enable)
{
    PB_ALIVE(c);
    if (enable && !c->tev_ready) {
        for (int a = 0; a < 2; ++a)
            for (int s = 0; s < PB_TIMING_SLOTS; ++s)
                for (int k = 0; k < PB_TMAX; ++k) PB_CUDA(c, cudaEventCreate(&c->tev[a][s][k]));
        c->tev_ready = true;
    }
    c->timing = enable != 0;
    for (int s = 0; s < PB_TIMING_SLOTS; ++s) c->tcount[s] = 0;
    return PB_OK;
}

extern "C" int pb_get_timing(pb_ctx* c, double* out)
{
    PB_ALIVE(c);
    if (!out) return pb_fail(c, PB_ERR_ARG, "null output");
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    for (int s = 0; s < PB_TIMING_SLOTS; ++s) {
        double tot = 0.0;
        for (int k = 0; k < c->tcount[s]; ++k) {
            float ms = 0.f;
            PB_CUDA(c, cudaEventElapsedTime(&ms, c->tev[0][s][k], c->tev[1][s][k]));
            tot += ms;
        }
        out[2 * s] = tot;
        out[2 * s + 1] = c->tcount[s];
        c->tcount[s] = 0;
    }
    return PB_OK;
}

extern "C" int pb_get_graph_launches(pb_ctx* c, long long* out)
{
    PB_ALIVE(c);
    if (!out) return pb_fail(c, PB_ERR_ARG, "null output");
    *out = c->graph_launches;
    return PB_OK;
}

extern "C" int pb_get_launch_count(pb_ctx* c, long long* out)
{
    PB_ALIVE(c);
    if (!out) return pb_fail(c, PB_ERR_ARG, "null output");
    *out = c->nlaunch;
    return PB_OK;
}
