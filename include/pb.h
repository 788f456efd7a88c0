/*
 * libpb -- C ABI of the GB300 Galerkin boundary-integral Poisson-Boltzmann solver.
 *
 * The library solves Juffer's derivative boundary integral system (eqbim_3/eqbim_4,
 * Section 2.2) for the surface potential phi and its normal derivative dphi/dn on a
 * triangulated molecular surface, discretised by piecewise-constant Galerkin (Section 2.3),
 * with the matrix-vector product accelerated by the Cartesian FMM of Section 2.4 and solved
 * by right-preconditioned GMRES with the block-diagonal preconditioner of Section 2.6.
 *
 * Conventions for every call:
 *   - Return value: PB_OK (0) or one of the PB_ERR_* codes below; pb_last_error() gives a
 *     one-line reason. A failed call leaves the context usable unless it returns
 *     PB_ERR_CUDA, after which only pb_destroy is allowed.
 *   - Unknowns are ordered x = [phi_1 .. phi_N, dphi_1 .. dphi_N] (def:linsys), element
 *     order as uploaded, FP64.
 *   - "device pointer" arguments point to GPU memory of the current device, allocated and
 *     owned by the caller (for example a torch tensor's data_ptr). "host pointer" arguments
 *     point to CPU memory owned by the caller. The library never frees caller memory and
 *     keeps no caller pointer after a call returns.
 *   - All GPU work is queued on the stream given to pb_create (NULL = legacy default
 *     stream). Calls that return a value on the host synchronise that stream; the others
 *     return with the work queued unless stated otherwise.
 *   - Units: lengths in Angstrom, charges in e, potentials in e/(4 pi Angstrom) (Section 3),
 *     energies in kcal/mol.
 */
#ifndef PB_H
#define PB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PB_OK 0
#define PB_ERR_ARG 1            /* bad argument or parameter */
#define PB_ERR_MESH 2           /* malformed mesh (degenerate triangle, bad index, ...) */
#define PB_ERR_CUDA 3           /* a CUDA call failed; the context is no longer usable */
#define PB_ERR_NOT_CONVERGED 4  /* GMRES hit max_iter before the tolerance */
#define PB_ERR_NONFINITE 5      /* a NaN or Inf appeared in a residual */
#define PB_ERR_STATE 6          /* call out of order (e.g. matvec before pb_build_tree) */
#define PB_ERR_NOMEM 7          /* device allocation failed */
#define PB_ERR_TIMEOUT 8        /* a bounded wait inside a kernel gave up (copy never landed) */

#define PB_FP64 0  /* every step in double precision */
#define PB_MIXED 1 /* near and far field in FP32 with FP64 leaf-sum accumulation; FP64
                      singular integrals, preconditioner, Arnoldi, Givens and energy sum */

#define PB_PRECOND_NONE 0
#define PB_PRECOND_DIAG 1  /* 2x2 blocks of A for each element ("d" in Table 4) */
#define PB_PRECOND_BLOCK 2 /* blocks of A for all element pairs of one leaf ("bd", Sec. 2.6) */

/* Physical and numerical parameters. */
typedef struct pb_params {
    double eps_in;   /* eps_1, dielectric constant inside the surface (Section 2.1) */
    double eps_out;  /* eps_2, dielectric constant outside */
    double kappa;    /* inverse Debye length, 1/Angstrom (eqNPBE, Eq_K1) */
    double eta0;     /* clusters c, c' are neighbours when eta(c,c') > eta0 (def:eta); 0 < eta0 < 1 */
    int leaf_size;   /* s: the tree depth L is the deepest level with mean cluster size >= s */
    int levels;      /* > 0: use this depth L instead (1..10) */
    int p;           /* Taylor order p_L of the finest level (1..10) */
    int adaptive;    /* 1: p_l = p_L + L - l (variable:order), capped at 12; 0: p_l = p_L */
    int qs;          /* Gauss-Legendre points per axis of the 4-cube in the singular
                        (Sauter-Schwab) quadrature, 1..8 */
    int precision;   /* PB_FP64 or PB_MIXED */
    int precond;     /* PB_PRECOND_NONE, PB_PRECOND_DIAG or PB_PRECOND_BLOCK */
    int singular;    /* arithmetic of the Sauter-Schwab integrals: PB_SINGULAR_AUTO (0: float-float
                        under PB_MIXED, FP64 under PB_FP64), PB_SINGULAR_FP64 or PB_SINGULAR_FF */
    int pc_block;    /* PB_PRECOND_BLOCK: most elements in one block (8..96; 0 = 96). Section 2.6
                        takes the clusters of a designated level as blocks; here the leaves, each
                        cut into nearly equal Morton-consecutive parts of at most pc_block
                        elements, so smaller values stand for designated levels below the leaves */
    int qr;          /* order of the regular quadrature rule (Section 3.1, Table 2) for non-touching
                        pairs, the right-hand side and the energy: 0 or 1 = the centroid (one
                        point), 2..4 = q^2 points per element (collapsed Gauss product rule, exact
                        to total degree 2q - 1). Orders above 1 support single right-hand sides
                        (not pb_solve_states mode 2 or pb_batch_solve_states) */
    int basis;       /* PB_BASIS_CONSTANT (0, piecewise constant, one pair of unknowns per element)
                        or PB_BASIS_LINEAR (continuous piecewise-linear hat functions S^1_h of
                        Section 2.3, eqlinearfcn / eqglinearcfcn: one pair per vertex; needs
                        qr 2..4). Under PB_BASIS_LINEAR the vectors of pb_matvec, pb_rhs,
                        pb_precond_apply, pb_gmres_solve and pb_solvation_energy have 2 nv
                        entries [phi at the vertices; dphi/dn at the vertices] in the uploaded
                        vertex order, the preconditioner is the 2 x 2 block diagonal of the vertex
                        system (exact entries), and the several-vector, batched, treecode and
                        learned-start calls are rejected with PB_ERR_ARG */
} pb_params;

#define PB_BASIS_CONSTANT 0
#define PB_BASIS_LINEAR 1

/* Float-float ("double-single", ~1e-13 relative) evaluates every step of the singular
 * quadrature on the FP32 pipe, whose rate on this GPU is 64 times the FP64 rate. */
#define PB_SINGULAR_AUTO 0
#define PB_SINGULAR_FP64 1
#define PB_SINGULAR_FF 2

typedef struct pb_ctx pb_ctx;

typedef struct pb_solve_info {
    int iterations;      /* Arnoldi steps taken (= matrix-vector products after the first) */
    int matvecs;         /* matrix-vector products, including residual evaluations (none for a zero start) */
    double rel_residual; /* final ||b - A x|| / ||b||, recomputed with a true product */
    int status;          /* PB_OK, PB_ERR_NOT_CONVERGED or PB_ERR_NONFINITE */
    double initial_residual; /* ||b - A x0|| / ||b|| of the start (1 for a zero start) */
} pb_solve_info;

/* Tree statistics (for tests and reports). */
typedef struct pb_tree_stats {
    int levels;           /* L */
    int nclusters[11];    /* clusters per level 0..L */
    long long nnear[11];  /* neighbour-list entries per level */
    long long ninter[11]; /* interaction-list entries per level */
    int order[11];        /* p_l per level */
    long long near_pairs; /* element pairs in the near field */
    long long touching;   /* ordered element pairs sharing a vertex (incl. i == j) */
    int max_leaf;         /* largest leaf */
    long long touch_class[4]; /* ordered touching pairs sharing 1, 2, 3 vertices (index 0 unused) */
    int pc_blocks;        /* block-diagonal preconditioner blocks (0 for the other preconditioners) */
    int pc_max;           /* largest block order m = 2 n_c */
    double pc_sum_m3;     /* sum over blocks of m^3 (the Gauss-Jordan inversion takes m^3 FMAs) */
} pb_tree_stats;

/* Create a context. params is copied. stream is a cudaStream_t (may be NULL). */
int pb_create(const pb_params* params, void* stream, pb_ctx** out);

/* Destroy a context and free all library-owned device memory. Accepts NULL. */
int pb_destroy(pb_ctx* ctx);

/* One-line description of the last error on this context (never NULL). */
const char* pb_last_error(const pb_ctx* ctx);

/* Upload a closed surface and its charges (Section 2.3, eqbemesh; source_terms).
 * verts: host pointer, nv x 3 doubles. tris: host pointer, nt x 3 int32 vertex indices,
 * counter-clockwise seen from outside (so the normal (v-u)x(w-u) points out of the solute).
 * qpos: host pointer, nc x 3 doubles; q: host pointer, nc doubles (charge states beyond one
 * are uploaded with pb_set_charges). Replaces any earlier mesh; copies host -> device and
 * synchronises. Rejects nt < 1, indices out of range and zero-area triangles (PB_ERR_MESH). */
int pb_mesh_upload(pb_ctx* ctx, const double* verts, int nv, const int32_t* tris, int nt,
                   const double* qpos, const double* q, int nc);

/* Replace the charge values (same positions). q: host pointer, nc doubles. */
int pb_set_charges(pb_ctx* ctx, const double* q, int nc);

/* Build everything that depends only on the geometry (Sections 2.3-2.6): element geometry,
 * Morton-ordered octree with shrink boxes, neighbour and interaction lists (def:eta),
 * singular Sauter-Schwab integrals of identical and adjacent triangle pairs, and the
 * preconditioner factors. Synchronises (list sizes are read back to size allocations). */
int pb_build_tree(pb_ctx* ctx);

/* y = A x with A of def:linsys/eq_linsysEntry evaluated by the FMM (near field + Taylor
 * far field). x, y: device pointers, 2N doubles each, must not overlap. Queued, no sync. */
int pb_matvec(pb_ctx* ctx, const double* x, double* y);

/* nr products at once, Y_q = A X_q for q < nr (1 <= nr <= PB_MAX_RHS): X and Y are device
 * pointers to nr x 2N doubles (vector q at + 2 N q), element order. The geometry-only work
 * is shared: in mixed precision each near-field pair is evaluated once for up to 16 vectors
 * and every far-field launch covers all nr vectors; FP64 applies the near field per vector.
 * Queues the work. No counterpart in the paper. */
int pb_matvec_multi(pb_ctx* ctx, const double* X, double* Y, int nr);

/* b = [b1; b2] of the Galerkin right-hand side (source_terms) by the one-point rule.
 * b: device pointer, 2N doubles. Queued, no sync. */
int pb_rhs(pb_ctx* ctx, double* b);

/* z = M^-1 r for the configured preconditioner (identity for PB_PRECOND_NONE).
 * r, z: device pointers, 2N doubles. Queued, no sync. */
int pb_precond_apply(pb_ctx* ctx, const double* r, double* z);

/* Solve A x = b for the uploaded charges with right-preconditioned restarted GMRES to
 * ||b - A x|| <= tol ||b|| (Section 2.3, last paragraph; Section 3). x: device pointer,
 * 2N doubles; read as the initial guess when use_x0 != 0 (e.g. a learned warm start), which
 * is first scaled by the factor a >= 0 that minimises ||b - a A x0|| (0 if none is positive);
 * otherwise zero-initialised (the first residual is b, no product); overwritten with the
 * solution. restart: Krylov dimension
 * m (1..200). The Arnoldi process, Givens rotations and updates run on the device in FP64;
 * the host reads one residual estimate per iteration. info may be NULL. */
int pb_gmres_solve(pb_ctx* ctx, double* x, double tol, int max_iter, int restart, int use_x0,
                   pb_solve_info* info);

/* Solve for several charge states of the uploaded charge positions on one built mesh: the
 * geometry (tree, singular integrals, preconditioner, MtL tables) is built once and shared
 * by all states. q: host pointer, nrhs x nc doubles (state s at q + s nc). X: device
 * pointer, nrhs x 2N doubles (state s at X + 2 N s), written with the solutions. E: host
 * pointer, nrhs doubles, written with the solvation energies in kcal/mol (may be NULL).
 * warm = 0: each state from zero, one after the other; 1: each state from the previous
 * state's solution (state 0 from zero); 2: state 0 from zero, then the other states together,
 * in batches of up to PB_MAX_RHS, from state 0's solution: their GMRES iterations run in
 * lockstep, each Arnoldi step applying one batched product (pb_matvec_multi's kernels) to all
 * of them; every state keeps its own Krylov basis, so each result is what its own GMRES would
 * give. infos: host pointer to nrhs records (may be NULL). On return the uploaded charges
 * are those of the last state. Synchronises. */
int pb_solve_states(pb_ctx* ctx, const double* q, int nrhs, double* X, double* E, double tol, int max_iter,
                    int restart, int warm, pb_solve_info* infos);

/* Several molecules, several charge states each, in ONE CUDA-graph launch. A context holds
 * one mesh, so the contexts ctxs[0..nmol) are the meshes of the batch; each must be built, on
 * the current device, appear once and have per-phase timing disabled. q[k]: host pointer,
 * nrhs x nc_k charge values of molecule k (state s at q[k] + s nc_k; positions as uploaded).
 * X[k]: device pointer, nrhs x 2 N_k doubles, written with the solutions (state s at
 * X[k] + 2 N_k s, element order). E: host pointer, nmol x nrhs energies in kcal/mol
 * (molecule-major; may be NULL). infos: host pointer, nmol x nrhs records (may be NULL).
 * The graph has one branch per molecule, run side by side: state 0 by GMRES from zero, then
 * the other states, up to PB_MAX_RHS per batch, by one GMRES over all of them (batched
 * products; each state keeps its own Krylov basis and stopping test) from state 0's solution
 * scaled per state by its least-squares factor, then every state's energy. Every GMRES stops
 * on the device (conditional graph nodes); the host reads nothing until the graph is done.
 * tol, max_iter, restart as pb_gmres_solve; 1 <= nrhs <= 1025. Builds the graph on each call
 * (a few hundred microseconds of host time per molecule). The uploaded charges of each context
 * are left as they were. Synchronises. Returns the first non-OK state status (the others are
 * in infos). No counterpart in the paper, which solves one molecule and one charge state at a
 * time. */
int pb_batch_solve_states(pb_ctx* const* ctxs, int nmol, const double* const* q, int nrhs, double* const* X,
                          double* E, double tol, int max_iter, int restart, pb_solve_info* infos);

/* Electrostatic solvation energy (eqsolengdis) for x = [phi; dphi/dn] in kcal/mol, using
 * the factor 4 pi 332.0716 of Section 3. x: device pointer. E_kcal: host pointer.
 * Synchronises. */
int pb_solvation_energy(pb_ctx* ctx, const double* x, double* E_kcal);

/* The same energy by the Cartesian treecode of Section 2.5 (eqMAC, eqsolengformTree): per
 * charge, clusters from the root down; a cluster with rho_c / |x_n - x_c| <= theta (rho_c the
 * shrink-box half diagonal, tested in FP64) contributes the Taylor series of its far-field
 * moments at the context's per-level orders (the product's P2M and MtM, run on x up to the
 * root), a leaf that fails is summed directly. O(N_c log N) instead of O(N_c N); the error
 * falls with the order and with theta (about 3e-7 relative at p = 8, theta = 0.5 on a
 * 1280-triangle sphere). x: device pointer; 0 < theta < 1; E_kcal: host pointer.
 * Synchronises. */
int pb_solvation_energy_treecode(pb_ctx* ctx, const double* x, double theta, double* E_kcal);

/* Tree statistics after pb_build_tree. out: host pointer. Synchronises. */
int pb_get_tree_stats(pb_ctx* ctx, pb_tree_stats* out);

/* Copy tree data to the host (for parity tests). order: host int32[N], sorted position ->
 * element index; level_begin: host int32[sum_l nclusters[l]] with each level's cluster
 * start offsets, concatenated level by level; near_idx / inter_idx: host int32 arrays
 * sized by pb_tree_stats (sum of nnear / ninter), each level's lists concatenated cluster
 * by cluster in cluster order; near_cnt / inter_cnt: host int32[sum_l nclusters[l]] list
 * lengths. Any pointer may be NULL to skip it. Synchronises. */
int pb_get_tree(pb_ctx* ctx, int32_t* order, int32_t* level_begin, int32_t* near_cnt,
                int32_t* near_idx, int32_t* inter_cnt, int32_t* inter_idx);

/* Split products for parity tests: y = (mass + near field) x, or y = far-field x, with the
 * same conventions as pb_matvec. which: 0 = full, 1 = near field incl. mass and singular
 * corrections, 2 = far field only. */
int pb_matvec_part(pb_ctx* ctx, const double* x, double* y, int which);

/* Per-phase device times measured with CUDA events recorded around each launch (no extra
 * synchronisation) while timing is enabled. pb_get_timing synchronises, writes for each slot
 * s the pair out[2s] = total milliseconds, out[2s+1] = number of timed launches, and resets
 * the counts. out: host double[2 * PB_TIMING_SLOTS]. At most 256 launches per slot are
 * remembered between two reads. */
/* Largest number of right-hand sides of one batched call (pb_matvec_multi, batched solve). */
#define PB_MAX_RHS 64

#define PB_TIMING_SLOTS 13
#define PB_T_NEAR 0       /* near-field kernel (one-point rule + mass terms) */
#define PB_T_CORR 1       /* Sauter-Schwab corrections of touching pairs */
#define PB_T_UP 2         /* leaf moments and MtM */
#define PB_T_M2L 3        /* MtL on all levels */
#define PB_T_DOWN 4       /* LtL and LtP */
#define PB_T_PRECOND 5    /* preconditioner apply */
#define PB_T_ARNOLDI 6    /* orthogonalisation, Givens, update */
#define PB_T_SINGULAR 7   /* singular integrals (setup) */
#define PB_T_TREE 8       /* geometry, octree and lists (setup) */
#define PB_T_PCBUILD 9    /* preconditioner assembly and inversion (setup) */
#define PB_T_ENERGY 10    /* solvation energy */
#define PB_T_RHS 11       /* right-hand side */
#define PB_T_FARSETUP 12  /* MtL derivative table kernels (setup) */
int pb_set_timing(pb_ctx* ctx, int enable);
int pb_get_timing(pb_ctx* ctx, double* out);

/* Number of this library's kernel launches queued on ctx since it was created. */
int pb_get_launch_count(pb_ctx* ctx, long long* out);

/* Number of CUDA-graph replays on ctx: the batched charge-state solve (pb_solve_states mode 2)
 * captures each Arnoldi step of its lockstep GMRES (about 40 launches over the context's two
 * streams) into one graph per step index and replays it; with timing enabled it launches the
 * kernels directly instead. */
int pb_get_graph_launches(pb_ctx* ctx, long long* out);

/* Autotuner (no counterpart in the paper, which sets the leaf size and order by hand): on the
 * uploaded molecule, tries leaf sizes {32, 48, 64, 96, 128} x orders {4, 6, 8} (uniform order,
 * the context's eta0 and precision), timing pb_build_tree and the product with CUDA events and
 * measuring the product's relative L2 error against an order-10 product on a fixed
 * pseudo-random density. The product is timed on nrhs vectors at once (pb_matvec for 1,
 * pb_matvec_multi above; 1 <= nrhs <= PB_MAX_RHS), as the caller will apply it, and
 * matvecs_per_solve counts such products. At each leaf size the orders are tried upwards until
 * one meets tol. Chooses the candidate with the least build_ms + matvecs_per_solve x matvec_ms
 * among those within tol (else the most accurate) and stores its leaf size and order in the
 * context's parameters. Then, from the finest level with a far field upwards, it lowers single
 * levels' orders by 2 (not below 4) while the error stays within tol and the cost falls; these
 * per-level orders (out->order) apply to later builds of the same depth until the next
 * pb_autotune. Leaves the context built with the choice. out: host pointer. Synchronises;
 * takes about 16 + L builds. */
typedef struct pb_tune_result {
    int leaf_size;      /* chosen leaf size s */
    int p;              /* chosen uniform order (before the per-level pass) */
    double matvec_ms;   /* median product time of the choice */
    double build_ms;    /* its pb_build_tree time */
    double rel_err;     /* its product error against the order-10 reference */
    int tried;          /* candidates built */
    int met_tolerance;  /* 1 if rel_err <= tol */
    int order[11];      /* chosen order per level 0..L (0 beyond L) */
} pb_tune_result;
int pb_autotune(pb_ctx* ctx, double tol, int matvecs_per_solve, int nrhs, pb_tune_result* out);

/* Measured FMA throughput of the current device in TFLOP/s (2 flops per FMA): eight
 * independent FMA chains per thread on 8 x (SM count) blocks of 256 threads, timed with CUDA
 * events on stream (cudaStream_t, NULL = default). The roofline denominators of the
 * ALU-bound kernels. Host pointers; synchronises; takes ~15 ms. No counterpart in the paper. */
int pb_measure_alu_peaks(void* stream, double* fp32_tflops, double* fp64_tflops);

/* ---------------- learned warm start for GMRES ----------------
 * The paper starts GMRES from zero (Section 2.6). These calls add a per-element multilayer
 * perceptron that predicts x = [phi; dphi/dn] from local features, so that GMRES can start
 * from the prediction; the converged solution does not depend on the start, only the number
 * of iterations does. The network has nin inputs, depth hidden layers of width units with
 * ReLU, and nout linear outputs; layer l computes z = W_l a + b_l with W_l (out x in,
 * row-major). Forward and backward passes run on the tensor cores with BF16 weights and
 * activations and FP32 accumulation; master weights, gradients and Adam moments are FP32.
 * The loss is the mean squared error over all rows and outputs.
 *
 * Parameter layout (pb_mlp_get_params / set_params / the gradient): every layer's weight
 * matrix in order, then every layer's bias, each in the layer's PADDED shape: inputs rounded
 * up to a multiple of 16 (layer 0 only), outputs of the last layer rounded up to a multiple
 * of 16; padded rows and columns stay zero as long as the caller keeps them zero. */
typedef struct pb_mlp pb_mlp;

/* Create a network with weights drawn uniformly from +-sqrt(6 / (fan_in + fan_out)) by a
 * SplitMix64 sequence of seed, zero biases and zero Adam moments. width: multiple of 16;
 * 1 <= depth <= 7; 1 <= nout <= 64. stream: cudaStream_t for all the network's work.
 * Synchronises. */
int pb_mlp_create(int nin, int width, int depth, int nout, unsigned long long seed, void* stream, pb_mlp** out);
int pb_mlp_destroy(pb_mlp* net);
const char* pb_mlp_last_error(const pb_mlp* net);
/* Number of FP32 parameters in the padded layout above. */
int pb_mlp_param_count(pb_mlp* net, long long* n);
/* Copy all parameters to / from a host array of pb_mlp_param_count floats. Synchronises. */
int pb_mlp_get_params(pb_mlp* net, float* host);
int pb_mlp_set_params(pb_mlp* net, const float* host);
/* Y (device, n x nout FP32, row-major) = network(X) for X (device, n x nin FP32, row-major).
 * Queues the work. */
int pb_mlp_forward(pb_mlp* net, const float* X, int n, float* Y);
/* Loss and gradient of the loss for inputs X and targets T (device, n x nout FP32); loss and
 * grad (pb_mlp_param_count floats) are host pointers and may be NULL. Synchronises. */
int pb_mlp_gradient(pb_mlp* net, const float* X, const float* T, int n, float* loss, float* grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the gradient of the
 * batch (X, T). loss: host pointer or NULL (NULL leaves the step queued, no sync). */
int pb_mlp_train_step(pb_mlp* net, const float* X, const float* T, int n, float lr, float* loss);

/* Per-element features of the learned warm start after pb_build_tree, element order,
 * F (device, nt x 18 FP32). With r the distance from the centroid to charge k: centroid minus
 * the mean charge position over the centroids' radius of gyration (3), unit normal (3),
 * log(area / mean area), 1 - mean normal product with the triangles sharing a vertex,
 * S1 and S2 of eqbim_3/eqbim_4 at the centroid, sum_k |q_k| / (4 pi r), nearest-charge
 * distance / 3 A, sum_k q_k exp(-kappa r) / (4 pi eps_in r), sum_k q_k / (4 pi eps_in
 * sqrt(r^2 + a^2)) for a = 4 and 8 A, sum_k exp(-r^2 / 50) / 10, and -sum_k q_k n . (c - x_k)
 * / (4 pi eps_in (r^2 + a^2)^(3/2)) for a = 4 and 8 A; the eight source columns are divided by
 * their root mean square over the molecule.
 * If x (device, 2 nt FP64, a solution) is given, T (device, nt x 2 FP32) receives the
 * training targets phi_i / s_phi and dphi_i / s_dphi with s_phi = rms S1 * 2 eps_in /
 * (eps_in + eps_out) and s_dphi = rms S2 * 2 eps_out / (eps_in + eps_out) (the flat-interface
 * image-charge values); x and T are both NULL or both set. scales: host double[20] or NULL:
 * [c] the divisor of column c ([0] for columns 0-2, [6] the mean area), [18] s_phi,
 * [19] s_dphi; synchronises when given. */
int pb_features(pb_ctx* ctx, float* F, const double* x, float* T, double* scales);
/* x (device, 2 nt FP64) = the network's prediction for the uploaded molecule, unscaled by
 * s_phi and s_dphi; net must map 18 inputs to 2 outputs. Use as the start of pb_gmres_solve. */
int pb_learned_guess(pb_ctx* ctx, pb_mlp* net, double* x);

/* Solvation energy for callers that cannot allocate device memory.
 *
 * The paper has no counterpart to this call; it exists for callers that must not call
 * cudaMalloc -- a host that gives the library a fixed device-memory budget and forbids
 * allocations after start-up, or code that runs where an allocation is not allowed (an
 * allocation may synchronise the device, or fail when memory is exhausted). It computes the same energy
 * as pb_solvation_energy, without a context, from caller-owned buffers, and allocates
 * nothing: its only scratch (one partial sum per block of 256 triangles) lives in a fixed
 * 64 KiB device array that every GPU loading this library holds until the process exits.
 *
 * verts (nv x 3 doubles), tris (nt x 3 int32), qpos (nc x 3 doubles), q (nc doubles) and
 * x = [phi; dphi/dn] (2 nt doubles, element order): device pointers. E: device pointer to
 * one double, written with the energy in kcal/mol. precision: PB_FP64 or PB_MIXED (FP32
 * kernel evaluation, FP64 sums). stream: cudaStream_t (NULL = default stream); the call
 * only queues work. errbuf/errlen: optional host buffer for a one-line reason on failure.
 * Returns PB_ERR_ARG for nt > 2,097,152 (the fixed scratch limit) or bad arguments, and
 * PB_ERR_CUDA if the launch fails.
 *
 * The first call on a device looks up the scratch array's device address with
 * cudaGetSymbolAddress (with that device current) and keeps it for the life of the process;
 * make that first call before any stream capture. Calls after cudaDeviceReset on that device
 * are not supported (the kept address belongs to the old context). Every call reuses the same
 * array and leaves its partial sums there; calls that may overlap on the GPU (on different
 * streams, or from several threads) race on it and must be serialised by the caller. */
int pb_solvation_energy_noalloc(const double* verts, const int32_t* tris, int nt, const double* qpos,
                                const double* q, int nc, double eps_in, double eps_out, double kappa,
                                int precision, const double* x, double* E, void* stream, char* errbuf,
                                int errlen);

#ifdef __cplusplus
}
#endif

#endif /* PB_H */
