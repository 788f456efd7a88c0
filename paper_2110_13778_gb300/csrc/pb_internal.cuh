// Internal declarations shared by the libpb translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pb.h"

#define PB_MAXL 10          // deepest tree level (Morton keys of 3 * 10 bits)
#define PB_PMAX 12          // largest Taylor order
#define PB_PI 3.14159265358979323846
#define PB_TMAX 256         // timed launches remembered per slot

// number of multi-indices with |a| <= p
__host__ __device__ inline int pb_nterms(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// position of multi-index (a, b, c) in the layout: total degree n ascending, then a
// descending, then b descending.
__host__ __device__ inline int pb_midx(int a, int b, int c)
{
    int n = a + b + c;
    int m = n - a;
    return n * (n + 1) * (n + 2) / 6 + m * (m + 1) / 2 + (m - b);
}

struct PbLevel {
    int ncl = 0;             // clusters on this level
    int* begin = nullptr;    // [ncl + 1] first sorted element of each cluster, then N
    int* parent = nullptr;   // [ncl] index of the parent cluster on level - 1
    int* cbeg = nullptr;     // [ncl + 1] first child on level + 1 (children are contiguous)
    double* xc = nullptr;    // [3 * ncl] shrink-box centres
    double* rho = nullptr;   // [ncl] half diagonals
    int* near_off = nullptr; // [ncl + 1] CSR neighbour lists
    int* near_idx = nullptr;
    int* int_off = nullptr;  // [ncl + 1] CSR interaction lists
    int* int_idx = nullptr;
    long long nnear = 0, ninter = 0;
    int p = 0;               // Taylor order on this level
    // far-field expansions, [ncl * nterms(p)] each, of the working precision
    void* sig0 = nullptr;    // moments for G0
    void* sigk = nullptr;    // moments for Gk
    void* lam0 = nullptr;    // local coefficients for G0
    void* lamk = nullptr;    // local coefficients for Gk
    // MtL with precomputed kernel derivatives: each cluster's interaction list padded to a
    // multiple of 32 slots; D^gamma G of slot s stored at ((s / 32) * T + gamma) * 32 + s % 32
    int* slot_off = nullptr; // [ncl + 1]
    int* slot_src = nullptr; // [nslots], -1 for padding
    long long nslots = 0;
    void* D0 = nullptr;      // derivatives of G0, working precision
    void* Dk = nullptr;      // derivatives of Gk
    void* Mg0 = nullptr;     // scaled source moments gathered into the slot layout (per product)
    void* Mgk = nullptr;
    void* Mp0 = nullptr;     // mixed MtL: the sums of the runs that cross a chunk edge, [nr][chunk][2][T]
    void* Mpk = nullptr;
    int* slot_tgt = nullptr; // [nslots] target cluster of each slot (table setup)
    int* slot_mirror = nullptr;  // [nslots] slot of the reversed pair (table setup)
    std::vector<int> h_slot[3];  // host sources of slot_off, slot_src, slot_tgt (kept for the async uploads)
};

struct pb_ctx {
    pb_params prm;
    cudaStream_t st = nullptr;
    cudaStream_t st2 = nullptr;      // far field, concurrent with the near field on st
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_tree = nullptr;
    cudaEvent_t ev_sing = nullptr;  // the singular pass has been queued up to here
    bool tables_ready = false;       // far-field constant tables uploaded
    std::string err = "no error";
    bool dead = false;
    cudaMemPool_t pool = nullptr;    // device memory pool of this context
    std::vector<void*> build_allocs; // freed on a new build or upload
    std::vector<void*> mesh_allocs;  // freed on a new upload
    // mesh
    int nv = 0, nt = 0, nc = 0;
    double* verts = nullptr;  // [3 nv]
    int* tris = nullptr;      // [3 nt]
    double* qpos = nullptr;   // [3 nc]
    double* q = nullptr;      // [nc]
    // per-element geometry, element order
    double* cent = nullptr;   // [3 nt]
    double* area = nullptr;   // [nt]
    double* nrm = nullptr;    // [3 nt]
    // tree
    bool built = false;
    int L = 0;
    PbLevel lev[PB_MAXL + 1];
    int* order = nullptr;     // [nt] sorted position -> element
    int* rank = nullptr;      // [nt] element -> sorted position
    int max_leaf = 0;
    // sorted element data: position (x, y, z, area) and (nx, ny, nz, 0)
    double4_32a* e64p = nullptr;
    double4_32a* e64n = nullptr;
    float4* e32p = nullptr;
    float4* e32n = nullptr;
    float4* e32l = nullptr;   // low parts: centroid - (double)hi, so hi + lo carries ~48 bits
    int* stris = nullptr;     // [3 nt] vertex indices in sorted order
    // mixed-precision near field: target chunks (<= 32 per leaf) and packed source records
    int nchunks = 0;
    int* chunk_leaf = nullptr;
    int* chunk_first = nullptr;
    int p_level[PB_MAXL + 1] = {};  // per-level orders chosen by the autotuner,
    int p_level_L = -1;             // valid for builds of this depth (-1: none)
    int near_nitems = 0;          // work items of the pair-tile near field
    int4* near_items = nullptr;   // (target chunk, first tile, end tile, 0)
    int* near_tiles = nullptr;    // source chunk of each tile
    int near_mitems = 0;          // work items of the several-vector near field (directed tiles)
    int4* near_mitem = nullptr;
    int* near_mtiles = nullptr;
    // the same near field on the points of a regular rule (mixed precision, q2 = 4 or 16)
    int pn_nitems = 0;
    int4* pn_items = nullptr;
    int *pn_tiles = nullptr, *pn_chunk_leaf = nullptr, *pn_chunk_first = nullptr, *pn_begin = nullptr;
    float4 *pn_p32 = nullptr, *pn_l32 = nullptr, *pn_n32 = nullptr, *pn_sp = nullptr, *pn_sn = nullptr;
    double* pn_y = nullptr;
    std::vector<int> h_pn_i[3];
    std::vector<int4> h_pn_i4;
    float4* near_sp = nullptr;  // (x_hi, y_hi, z_hi, A phi)
    float4* near_sn = nullptr;  // (n_x, n_y, n_z, A dphi)
    float2* near_dens = nullptr; // [dens_nr][nt] (A phi, A dphi) for several right-hand sides
    double* yfar = nullptr;      // [yfar_nr][2 nt] far-field part of the product (tree order)
    int yfar_nr = 0;
    int dens_nr = 0;
    // touching pairs (share >= 1 vertex, incl. i == j), CSR by sorted target position
    int* touch_off = nullptr; // [nt + 1]
    int* touch_j = nullptr;   // sorted source position
    double* corr = nullptr;   // [4 * ntouch] exact integral minus one-point rule (I1..I4)
    long long ntouch = 0;
    long long touch_class[4] = {0, 0, 0, 0};  // ordered pairs sharing 0..3 vertices
    unsigned long long* touch_class_dev = nullptr;  // the same on the device, read when reported
    const int* canon_check = nullptr;  // device count of unordered touching pairs, checked at the end of a build
    int canon_expect = 0;
    long long near_pairs = 0;
    // host copies made by the build: the leaf ranges (read back once by the tree build), and
    // the sources of the build's host-to-device uploads, kept until the next build so that
    // those copies need no synchronisation
    std::vector<int> h_leaf_begin, h_near_off, h_near_idx;  // leaf ranges and leaf neighbour lists
    // h_up_i: [0] chunk leaf, [1] chunk first element, [2] preconditioner block ranges, [3] block
    // ids by size class, [4] near-field pair tiles, [5] several-vector directed tiles
    std::vector<int> h_up_i[6];
    std::vector<int4> h_up_i4, h_up_i4m;  // near-field work items: pair tiles, directed tiles
    std::vector<long long> h_up_l;        // preconditioner block offsets
    std::vector<double> h_up_d;           // singular quadrature: Gauss-Legendre nodes and weights
    std::vector<float2> h_up_f2;          // singular quadrature: float-float cube-point table
    // preconditioner: per leaf a dense (2n x 2n) inverse, unknowns [phi of leaf; dphi of leaf]
    int far_nr = 1;               // right-hand sides the far-field work arrays hold
    int npcblk = 0;               // preconditioner blocks
    int pc_max = 0;               // largest block order
    long long pc_total = 0;       // entries of all blocks
    double pc_sum_m3 = 0;         // sum of m^3 over blocks
    int* pc_begin = nullptr;      // [npcblk + 1] first sorted element of each block
    long long* blk_off = nullptr; // [npcblk + 1] offsets into minv
    int* pc_ids = nullptr;        // [npcblk] block indices grouped by size class (order <= 64, 128, 192)
    int pc_cls[4] = {0, 0, 0, 0}; // first position of each class in pc_ids, and the total
    void* minv = nullptr;         // inverse blocks, working precision (float in mixed mode)
    double* dinv = nullptr;       // [4 nt] inverse 2x2 blocks for PB_PRECOND_DIAG
    // work vectors in sorted order
    double* xs = nullptr;
    double* ys = nullptr;
    double* ws = nullptr;
    double* scratch = nullptr;    // reduction partials
    double* escratch = nullptr;   // per-state energy partials (several states at once)
    double* qstates = nullptr;    // device charges of up to PB_MAX_RHS states [PB_MAX_RHS][nc]
    int qstates_n = 0;            // states qstates holds room for (0: PB_MAX_RHS if qstates is set)
    // several right-hand sides: tree-ordered work vectors and the batched GMRES workspace
    double *mxs = nullptr, *mys = nullptr;
    int mv_nr = 0;
    double *gbV = nullptr, *gbW = nullptr, *gbZ = nullptr, *gbB = nullptr, *gbpart = nullptr, *gbsmall = nullptr;
    int gb_nr = 0, gb_m = 0;
    // CUDA graphs of the batched Arnoldi steps (one per step index), valid for one workspace
    std::vector<cudaGraphExec_t> gb_graphs;
    std::vector<long long> gb_graph_n;  // kernel launches each graph holds
    void* gb_graph_key = nullptr;
    int gb_graph_nr = 0;
    bool gb_graph_failed = false;
    long long graph_launches = 0;       // replays of captured Arnoldi steps
    cudaStream_t cap_st = nullptr;      // private stream for capturing
    // device-driven GMRES (one graph per solve with conditional WHILE nodes): the current basis
    // vectors of nr right-hand sides, control blocks (device and pinned host copies), the cached
    // executable graph of a single-context solve with its key and captured launch counts
    double* dgVcur = nullptr;
    float2* dgWf = nullptr;  // mixed precision: float-float work vectors of the device-driven Arnoldi step
    int dg_nr = 0;
    void* dgctl = nullptr;
    void* dgctl_h = nullptr;
    int dg_nctl = 0;
    cudaGraphExec_t dg_exec = nullptr;
    const void* dg_key[6] = {};
    int dg_ikey[3] = {};
    long long dg_cnt[3] = {};
    bool dg_failed = false;           // graphs with conditional nodes cannot be built here
    long long build_gen = 0;          // incremented by every pb_build_tree / pb_mesh_upload
    double* tc_part = nullptr;        // treecode energy: one partial per (charge, level-1 cluster)
    long long tc_nw = 0;
    // regular rule of order q > 1: q2 = q^2 points per element, their records (tree order,
    // element-major), the leaf ranges in points and point work vectors (2 x N q2 each)
    int q2 = 1;
    double4_32a* pts_p = nullptr;
    double4_32a* pts_n = nullptr;
    int* begin_q = nullptr;
    double* xq = nullptr;
    double* yq = nullptr;
    // piecewise-linear basis: unknowns per half (nt, or nv under PB_BASIS_LINEAR); the vertex
    // lists (for each vertex its element corners 3 k + a, sorted), per touching pair the 4 x 3 x
    // 3 blocks exact minus the order-q rule, the exact vertex diagonal (4 per vertex), the 2 x 2
    // inverses of the preconditioner and the near field's work arrays
    int nu = 0;
    int* p1_voff = nullptr;
    int* p1_vlist = nullptr;
    double* p1_corr = nullptr;
    double* p1_diag = nullptr;
    double* p1_pinv = nullptr;
    double* p1_yqn = nullptr;
    double* p1_yl = nullptr;
    double* bE = nullptr;         // energies of the states of a batched multi-molecule solve (device)
    int bE_n = 0;
    double* hscal = nullptr;      // pinned host scalars
    // GMRES workspace (Krylov basis, work vectors, reduction partials, small dense state)
    int gm_m = 0;
    double *gmV = nullptr, *gmw = nullptr, *gmz = nullptr, *gmpart = nullptr, *gmsmall = nullptr;
    float2* gmwf = nullptr;  // mixed precision: float-float work vector of the Arnoldi step
    double* gmvd = nullptr;  // mixed precision: FP64 copy of the current basis vector
    // timing: per slot a ring of (start, stop) event pairs, read back by pb_get_timing
    bool timing = false;
    cudaEvent_t ev[10] = {};
    cudaEvent_t tev[2][PB_TIMING_SLOTS][PB_TMAX] = {};
    int tcount[PB_TIMING_SLOTS] = {};
    bool tev_ready = false;
    long long nlaunch = 0;  // kernels of this library launched on this context
    int* dev_err = nullptr; // set by a kernel whose bounded wait gave up (device, build lifetime)
};

inline void pb_tic(pb_ctx* c, int slot)
{
    if (c->timing && c->tcount[slot] < PB_TMAX) cudaEventRecord(c->tev[0][slot][c->tcount[slot]], c->st);
}
inline void pb_toc(pb_ctx* c, int slot)
{
    if (c->timing && c->tcount[slot] < PB_TMAX) cudaEventRecord(c->tev[1][slot][c->tcount[slot]++], c->st);
}
// the same on another stream of the context
inline void pb_tic_on(pb_ctx* c, int slot, cudaStream_t s)
{
    if (c->timing && c->tcount[slot] < PB_TMAX) cudaEventRecord(c->tev[0][slot][c->tcount[slot]], s);
}
inline void pb_toc_on(pb_ctx* c, int slot, cudaStream_t s)
{
    if (c->timing && c->tcount[slot] < PB_TMAX) cudaEventRecord(c->tev[1][slot][c->tcount[slot]++], s);
}

// error helpers (pb_api.cu)
int pb_fail(pb_ctx* c, int code, const char* fmt, ...);
#define PB_CUDA(c, call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (c)->dead = true;                                                              \
            return pb_fail((c), PB_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                           __FILE__, __LINE__);                                            \
        }                                                                                  \
    } while (0)
#define PB_LAUNCH(c)                          \
    do {                                      \
        ++(c)->nlaunch;                       \
        PB_CUDA(c, cudaGetLastError());       \
    } while (0)

// device allocation owned by the context (zero-filled); nullptr on failure. Build-lifetime
// buffers are freed by the next pb_build_tree or pb_mesh_upload, mesh-lifetime buffers by
// the next pb_mesh_upload.
void* pb_alloc(pb_ctx* c, size_t bytes, bool build_lifetime = true);
void* pb_alloc_on(pb_ctx* c, size_t bytes, cudaStream_t s, bool build_lifetime = true);

// translation-unit entry points
int pb_geometry_and_tree(pb_ctx* c);          // tree.cu
// radix.cu: out[0..n] = exclusive prefix sums of in[0..n) (out[n] the total); stable sort of
// (key, value) pairs by the low `bits` key bits. Both queued on c->st, no read-back.
int pb_scan_exclusive(pb_ctx* c, const int* in, int* out, int n);
int pb_radix_sort_pairs(pb_ctx* c, const unsigned* kin, const int* vin, unsigned* kout, int* vout, int n, int bits);
int pb_touching_and_singular(pb_ctx* c);      // singular.cu
int pb_near_setup(pb_ctx* c);                                      // nearfield.cu
int pb_near_apply(pb_ctx* c, const double* xs, double* ys);        // nearfield.cu (writes ys)
int pb_corr_apply(pb_ctx* c, const double* xs, double* ys, int nr, const double* yfar);  // nearfield.cu (adds)
int pb_near_apply_multi(pb_ctx* c, const double* xs, double* ys, int nr);  // nearfield.cu (writes)
int pb_near_reserve(pb_ctx* c, int nr);
int pb_far_setup(pb_ctx* c);                                       // farfield.cu
int pb_far_apply(pb_ctx* c, const double* xs, double* ys, int nr, cudaStream_t st);  // farfield.cu (sets ys)
int pb_far_reserve(pb_ctx* c, int nr);
int pb_precond_plan(pb_ctx* c);    // precond.cu: block partition (host, synchronises)
int pb_precond_factor(pb_ctx* c);                                   // precond.cu
int pb_precond_apply_sorted(pb_ctx* c, const double* r, double* z);
int pb_precond_apply_multi(pb_ctx* c, const double* r, long long rstr, double* z, long long zstr, int nr);
int pb_matvec_sorted_multi(pb_ctx* c, const double* xs, double* ys, int nr);  // pb_api.cu
int pb_matvec_reserve(pb_ctx* c, int nr);  // pb_api.cu: every buffer a product of nr vectors needs
void pb_drop_graphs(pb_ctx* c);           // pb_api.cu
int pb_gmres_batch_sorted(pb_ctx* c, double* X, const double* B, int nr, double tol, int max_iter, int restart,
                          pb_solve_info* infos);  // krylov.cu
// device-driven GMRES (krylov.cu): returns -1 when its graph cannot be built on this device
// (the caller then takes the host-driven loop); start 0 = from zero, 1 = from X (scaled)
int pb_gmres_dev(pb_ctx* c, double* X, const double* B, int nr, double tol, int max_iter, int restart, int start,
                 pb_solve_info* infos);
void pb_dg_drop(pb_ctx* c);
int pb_energy_treecode_sorted(pb_ctx* c, const double* xs, double theta, double* E);  // farfield.cu
// pieces of the device-driven solve for graphs over several contexts (krylov.cu)
int pb_dg_reserve(pb_ctx* c, int nr, int m, int nctl);
int pb_dg_append(pb_ctx* c, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, double* X, const double* B,
                 int nr, int m, int start, int ictl, std::vector<cudaGraphNode_t>* leaves, long long cnt[3]);
void pb_dg_settings(pb_ctx* c, int ictl, int nr, int m, double tol, int max_iter);
int pb_dg_upload(pb_ctx* c, int nctl);
int pb_dg_download(pb_ctx* c, int nctl);
void pb_dg_results(pb_ctx* c, int ictl, int nr, const long long cnt[3], pb_solve_info* infos, int* worst);
int pb_energy_reserve(pb_ctx* c);
// regular rule of order > 1 (regular.cu)
int pb_regular_setup(pb_ctx* c);        // points (after the tree)
int pb_regular_corrections(pb_ctx* c);  // corrections: exact - order-q rule (after the singular pass)
int pb_near_q_apply(pb_ctx* c, const double* xs, double* ys);
int pb_to_points(pb_ctx* c, const double* xs, double* xq, cudaStream_t st);
// linear.cu: the piecewise-linear basis (set-up after the singular pass; product, preconditioner)
int pb_p1_setup(pb_ctx* c);
// nearfield.cu: the pair-tile near field on the points of the regular rule (mixed precision,
// q2 = 4 or 16): set-up after the points, per-point sums, and the piecewise-constant rows
bool pb_near_points_ok(const pb_ctx* c);
int pb_near_points_setup(pb_ctx* c);
int pb_near_points_apply(pb_ctx* c, const double* xs, const double* xq, double* ypt);
int pb_near_points_elem(pb_ctx* c, const double* xs, double* ys);
void pb_triangle_rule(int q, double* e1, double* e2, double* w);  // regular.cu
int pb_p1_matvec(pb_ctx* c, const double* x, double* y);
int pb_p1_precond(pb_ctx* c, const double* r, double* z);
int pb_p1_to_points(pb_ctx* c, const double* x, double* xq, cudaStream_t st);
int pb_p1_from_points(pb_ctx* c, const double* yq, double* y, int add, cudaStream_t st);
int pb_from_points(pb_ctx* c, const double* yq, double* ys, int add, cudaStream_t st);
int pb_energy_states_queue(pb_ctx* c, const double* Q, const double* X, int nr, double* Edev);  // nr <= 16
int pb_rhs_sorted(pb_ctx* c, double* bs);                          // krylov.cu
int pb_energy_sorted(pb_ctx* c, const double* xs, double* E);      // krylov.cu
int pb_rhs_states_sorted(pb_ctx* c, const double* Q, double* B, int nr);        // krylov.cu, nr <= 16
int pb_energy_states_sorted(pb_ctx* c, const double* Q, const double* X, int nr, double* E);  // nr <= 16
int pb_gmres_sorted(pb_ctx* c, double* xs, const double* bs, double tol, int max_iter,
                    int restart, pb_solve_info* info, bool x_zero);  // krylov.cu (x_zero: xs is zero)
int pb_matvec_sorted(pb_ctx* c, const double* xs, double* ys, int which);  // pb_api.cu
int pb_gather(pb_ctx* c, const double* x, double* xs);   // element -> sorted order
int pb_scatter(pb_ctx* c, const double* xs, double* x);  // sorted -> element order
