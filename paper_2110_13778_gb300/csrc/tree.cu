// Element geometry, Morton-ordered octree with shrink boxes, neighbour and interaction lists
// (Section 2.4: cluster hierarchy, shrink scheme, def:eta, interaction lists N(c), I(c)).
//
// Every floating-point decision that produces an integer (Morton cell, list membership) is
// made in FP64 with explicitly rounded operations in one fixed order (Morton cell:
// floor((c - origin) * (1024 / side)) clamped to [0, 1023]; neighbour test
// (rho_c + rho_c')^2 > eta0^2 |x_c - x_c'|^2), so that the result is reproducible bit for
// bit on any IEEE machine.

#include <algorithm>
#include <vector>

#include "pb_internal.cuh"

// ---------- per-element geometry (eqparameter): centroid, area, outward unit normal ----------
__global__ void k_geometry(int nt, const double* __restrict__ V, const int* __restrict__ T,
                           double* __restrict__ cent, double* __restrict__ area,
                           double* __restrict__ nrm)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const double* u = V + 3 * T[3 * i];
    const double* v = V + 3 * T[3 * i + 1];
    const double* w = V + 3 * T[3 * i + 2];
    double a[3], b[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = v[k] - u[k];
        b[k] = w[k] - u[k];
        // (u + v + w) / 3, two rounded additions and one rounded division
        cent[3 * i + k] = __ddiv_rn(__dadd_rn(__dadd_rn(u[k], v[k]), w[k]), 3.0);
    }
    double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    area[i] = 0.5 * len;
    for (int k = 0; k < 3; ++k) nrm[3 * i + k] = cr[k] / len;
}

// ---------- bounding box of the vertex array ----------
__global__ void k_bbox(int nv, const double* __restrict__ V, double* __restrict__ part)
{
    __shared__ double s[6][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], V[3 * i + k]);
            hi[k] = fmax(hi[k], V[3 * i + k]);
        }
    for (int k = 0; k < 3; ++k) {
        s[k][threadIdx.x] = lo[k];
        s[3 + k][threadIdx.x] = hi[k];
    }
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < 3; ++k) {
                s[k][threadIdx.x] = fmin(s[k][threadIdx.x], s[k][threadIdx.x + h]);
                s[3 + k][threadIdx.x] = fmax(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + h]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
}

// ---------- Morton keys of the centroids in the level-0 cube ----------
__device__ __forceinline__ unsigned spread3(unsigned x)
{
    // insert two zero bits between the 10 low bits of x
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_morton(int nt, const double* __restrict__ cent, double ox, double oy, double oz,
                         double scale, unsigned* __restrict__ keys, int* __restrict__ idx)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    double o[3] = {ox, oy, oz};
    unsigned cell[3];
    for (int k = 0; k < 3; ++k) {
        double t = floor(__dmul_rn(__dsub_rn(cent[3 * i + k], o[k]), scale));
        t = fmin(fmax(t, 0.0), (double)((1 << PB_MAXL) - 1));
        cell[k] = (unsigned)t;
    }
    keys[i] = (spread3(cell[0]) << 2) | (spread3(cell[1]) << 1) | spread3(cell[2]);
    idx[i] = i;
}

__global__ void k_level_counts(int nt, const unsigned* __restrict__ k, int* __restrict__ cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    for (int l = 0; l <= PB_MAXL; ++l) {
        int sh = 3 * (PB_MAXL - l);
        bool start = (i == 0) || ((k[i] >> sh) != (k[i - 1] >> sh));
        if (start) atomicAdd(&cnt[l], 1);
    }
}

__global__ void k_flags(int nt, const unsigned* __restrict__ k, int sh, int* __restrict__ flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    flag[i] = (i == 0) || ((k[i] >> sh) != (k[i - 1] >> sh));
}

__global__ void k_compact_starts(int nt, const int* __restrict__ flag, const int* __restrict__ pos,
                                 int* __restrict__ begin, int ncl)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nt && flag[i]) begin[pos[i]] = i;
    if (i == 0) begin[ncl] = nt;
}

// parent[c] = index of the cluster on the coarser level whose range contains begin[c]
__global__ void k_parent(int ncl, const int* __restrict__ begin, int npar,
                         const int* __restrict__ pbegin, int* __restrict__ parent)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncl) return;
    int b = begin[c];
    int lo = 0, hi = npar;  // largest j with pbegin[j] <= b
    while (hi - lo > 1) {
        int m = (lo + hi) / 2;
        if (pbegin[m] <= b) lo = m;
        else hi = m;
    }
    parent[c] = lo;
}

// cbeg[c] = first child of c (children are contiguous because parent[] is non-decreasing)
__global__ void k_child_begin(int ncl, int nch, const int* __restrict__ chparent, int* __restrict__ cbeg)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncl) return;
    if (c == ncl) {
        cbeg[c] = nch;
        return;
    }
    int lo = 0, hi = nch;  // first j with chparent[j] >= c
    while (lo < hi) {
        int m = (lo + hi) / 2;
        if (chparent[m] < c) lo = m + 1;
        else hi = m;
    }
    cbeg[c] = lo;
}

__device__ void box_finish(const double* lo, const double* hi, double* xc, double* rho)
{
    double d[3];
    for (int k = 0; k < 3; ++k) {
        xc[k] = __dmul_rn(0.5, __dadd_rn(lo[k], hi[k]));
        d[k] = __dsub_rn(hi[k], lo[k]);
    }
    double s = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
    *rho = __dmul_rn(0.5, __dsqrt_rn(s));
}

// leaf boxes from the vertices of the cluster's triangles; writes lo/hi for the parents
// one warp per leaf: lanes over the leaf's elements, then a shuffle reduction (minimum and
// maximum are exact, so the box does not depend on the order)
__global__ void k_leaf_boxes(int ncl, const int* __restrict__ begin, const int* __restrict__ order,
                             const double* __restrict__ V, const int* __restrict__ T,
                             double* __restrict__ blo, double* __restrict__ bhi,
                             double* __restrict__ xc, double* __restrict__ rho)
{
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= ncl) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int s = begin[c] + lane; s < begin[c + 1]; s += 32) {
        int e = order[s];
        for (int a = 0; a < 3; ++a) {
            const double* p = V + 3 * T[3 * e + a];
            for (int k = 0; k < 3; ++k) {
                lo[k] = fmin(lo[k], p[k]);
                hi[k] = fmax(hi[k], p[k]);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    if (lane == 0) {
        for (int k = 0; k < 3; ++k) {
            blo[3 * c + k] = lo[k];
            bhi[3 * c + k] = hi[k];
        }
        box_finish(lo, hi, xc + 3 * c, rho + c);
    }
}

__global__ void k_parent_boxes(int ncl, const int* __restrict__ cbeg, const double* __restrict__ clo,
                               const double* __restrict__ chi, double* __restrict__ blo,
                               double* __restrict__ bhi, double* __restrict__ xc, double* __restrict__ rho)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncl) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int ch = cbeg[c]; ch < cbeg[c + 1]; ++ch)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], clo[3 * ch + k]);
            hi[k] = fmax(hi[k], chi[3 * ch + k]);
        }
    for (int k = 0; k < 3; ++k) {
        blo[3 * c + k] = lo[k];
        bhi[3 * c + k] = hi[k];
    }
    box_finish(lo, hi, xc + 3 * c, rho + c);
}

// neighbour test of def:eta: (rho_c + rho_c')^2 > eta0^2 |x_c - x_c'|^2
__device__ __forceinline__ bool is_near(const double* xa, double ra, const double* xb, double rb, double e2)
{
    double s = __dadd_rn(ra, rb);
    double dx = __dsub_rn(xa[0], xb[0]), dy = __dsub_rn(xa[1], xb[1]), dz = __dsub_rn(xa[2], xb[2]);
    double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return __dmul_rn(s, s) > __dmul_rn(e2, dd);
}

// candidates of c are the children of the neighbours of its parent; pass 0 counts, pass 1 fills.
// One warp per cluster: lane i takes the i-th neighbour q of the parent (32 at a time) and tests
// q's children (at most 8) into a bit mask; warp scans of the per-lane counts give each lane its
// place, so both lists keep the sequential order (parent's neighbours in list order, children
// in order).
template <int PASS>
__global__ void k_lists(int ncl, const int* __restrict__ parent, const int* __restrict__ pnear_off,
                        const int* __restrict__ pnear_idx, const int* __restrict__ pcbeg,
                        const double* __restrict__ xc, const double* __restrict__ rho, double e2,
                        int* __restrict__ ncnt, int* __restrict__ icnt, const int* __restrict__ noff,
                        const int* __restrict__ ioff, int* __restrict__ nidx, int* __restrict__ iidx)
{
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= ncl) return;
    const int P = parent[c];
    int nb = PASS ? noff[c] : 0, ib = PASS ? ioff[c] : 0;  // running list ends
    const double xa[3] = {xc[3 * c], xc[3 * c + 1], xc[3 * c + 2]};
    const double ra = rho[c];
    int nn = 0, ni = 0;
    for (int t0 = pnear_off[P]; t0 < pnear_off[P + 1]; t0 += 32) {
        const int t = t0 + lane;
        int cb = 0, ce = 0;
        unsigned mask = 0u;  // bit k: child cb + k is near
        if (t < pnear_off[P + 1]) {
            const int q = pnear_idx[t];
            cb = pcbeg[q];
            ce = pcbeg[q + 1];
            for (int c2 = cb; c2 < ce; ++c2)
                if (is_near(xa, ra, xc + 3 * c2, rho[c2], e2)) mask |= 1u << (c2 - cb);
        }
        const int kn = __popc(mask), ki = (ce - cb) - kn;
        // inclusive warp scans of the counts
        int sn = kn, si = ki;
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, sn, o), b = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) {
                sn += a;
                si += b;
            }
        }
        if (PASS) {
            int pn = nb + sn - kn, pi = ib + si - ki;
            for (int c2 = cb; c2 < ce; ++c2) {
                if ((mask >> (c2 - cb)) & 1u) nidx[pn++] = c2;
                else iidx[pi++] = c2;
            }
        }
        const int tn = __shfl_sync(0xffffffffu, sn, 31), ti = __shfl_sync(0xffffffffu, si, 31);
        nb += tn;
        ib += ti;
        nn += tn;
        ni += ti;
    }
    if (!PASS && lane == 0) {
        ncnt[c] = nn;
        icnt[c] = ni;
    }
}

// sorted element records for the field kernels
__global__ void k_sorted_elems(int nt, const int* __restrict__ order, const double* __restrict__ cent,
                               const double* __restrict__ area, const double* __restrict__ nrm,
                               const int* __restrict__ T, double4_32a* __restrict__ e64p,
                               double4_32a* __restrict__ e64n, float4* __restrict__ e32p,
                               float4* __restrict__ e32n, float4* __restrict__ e32l, int* __restrict__ stris,
                               int* __restrict__ rank)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    int e = order[k];
    double4_32a p = make_double4_32a(cent[3 * e], cent[3 * e + 1], cent[3 * e + 2], area[e]);
    double4_32a n = make_double4_32a(nrm[3 * e], nrm[3 * e + 1], nrm[3 * e + 2], 0.0);
    e64p[k] = p;
    e64n[k] = n;
    float hx = (float)p.x, hy = (float)p.y, hz = (float)p.z;
    e32p[k] = make_float4(hx, hy, hz, (float)p.w);
    e32l[k] = make_float4((float)(p.x - (double)hx), (float)(p.y - (double)hy), (float)(p.z - (double)hz), 0.f);
    e32n[k] = make_float4((float)n.x, (float)n.y, (float)n.z, 0.f);
    for (int a = 0; a < 3; ++a) stris[3 * k + a] = T[3 * e + a];
    rank[e] = k;
}

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

// exclusive scan of cnt[0..n) into off[0..n], off[n] = total (queued, no read-back)
static int scan_only(pb_ctx* c, const int* cnt, int* off, int n) { return pb_scan_exclusive(c, cnt, off, n); }

int pb_geometry_and_tree(pb_ctx* c)
{
    const int nt = c->nt, nv = c->nv;
    const int B = 256;
    c->cent = (double*)pb_alloc(c, sizeof(double) * 3 * nt);
    c->area = (double*)pb_alloc(c, sizeof(double) * nt);
    c->nrm = (double*)pb_alloc(c, sizeof(double) * 3 * nt);
    if (!c->cent || !c->area || !c->nrm) return pb_fail(c, PB_ERR_NOMEM, "geometry: out of memory");
    k_geometry<<<nblk(nt, B), B, 0, c->st>>>(nt, c->verts, c->tris, c->cent, c->area, c->nrm);
    PB_LAUNCH(c);

    // level-0 cube: centred on the vertex bounding box, side = longest box edge
    const int nbb = 64;
    double* part = (double*)pb_alloc(c, sizeof(double) * 6 * nbb);
    if (!part) return pb_fail(c, PB_ERR_NOMEM, "bbox: out of memory");
    k_bbox<<<nbb, 256, 0, c->st>>>(nv, c->verts, part);
    PB_LAUNCH(c);
    std::vector<double> hp(6 * nbb);
    PB_CUDA(c, cudaMemcpyAsync(hp.data(), part, sizeof(double) * 6 * nbb, cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nbb; ++b)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], hp[6 * b + k]);
            hi[k] = std::max(hi[k], hp[6 * b + 3 + k]);
        }
    volatile double side = 0.0;
    for (int k = 0; k < 3; ++k) {
        volatile double e = hi[k] - lo[k];
        if (e > side) side = e;
    }
    if (!(side > 0)) return pb_fail(c, PB_ERR_MESH, "mesh has zero extent");
    double origin[3];
    for (int k = 0; k < 3; ++k) {
        volatile double ctr = 0.5 * (lo[k] + hi[k]);
        volatile double hs = 0.5 * side;
        origin[k] = ctr - hs;
    }
    volatile double scale = (double)(1 << PB_MAXL) / side;

    // Morton keys, stable radix sort of (key, element index)
    unsigned *keys = (unsigned*)pb_alloc(c, sizeof(unsigned) * nt), *skeys = (unsigned*)pb_alloc(c, sizeof(unsigned) * nt);
    int* idx = (int*)pb_alloc(c, sizeof(int) * nt);
    c->order = (int*)pb_alloc(c, sizeof(int) * nt);
    c->rank = (int*)pb_alloc(c, sizeof(int) * nt);
    if (!keys || !skeys || !idx || !c->order || !c->rank) return pb_fail(c, PB_ERR_NOMEM, "morton: out of memory");
    k_morton<<<nblk(nt, B), B, 0, c->st>>>(nt, c->cent, origin[0], origin[1], origin[2], scale, keys, idx);
    PB_LAUNCH(c);
    if (int rc = pb_radix_sort_pairs(c, keys, idx, skeys, c->order, nt, 3 * PB_MAXL)) return rc;

    // depth: deepest level whose mean cluster size is >= leaf_size (or the given depth)
    int* cnt = (int*)pb_alloc(c, sizeof(int) * (PB_MAXL + 1));
    if (!cnt) return pb_fail(c, PB_ERR_NOMEM, "levels: out of memory");
    k_level_counts<<<nblk(nt, B), B, 0, c->st>>>(nt, skeys, cnt);
    PB_LAUNCH(c);
    int hc[PB_MAXL + 1];
    PB_CUDA(c, cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, c->st));
    PB_CUDA(c, cudaStreamSynchronize(c->st));
    int L = 0;
    if (c->prm.levels > 0) {
        L = c->prm.levels;
    } else {
        for (int l = 0; l <= PB_MAXL; ++l)
            if ((double)nt / (double)hc[l] >= (double)c->prm.leaf_size) L = l;
    }
    c->L = L;

    // clusters of each level
    // (the cluster counts are known from the level counts, so the scans are not read back
    // one by one: each level's total is kept on the device and all are checked at once)
    int* flag = (int*)pb_alloc(c, sizeof(int) * (nt + 1));
    int* pos = (int*)pb_alloc(c, sizeof(int) * (nt + 1));
    int* tots = (int*)pb_alloc(c, sizeof(int) * (PB_MAXL + 1));
    if (!flag || !pos || !tots) return pb_fail(c, PB_ERR_NOMEM, "levels: out of memory");
    for (int l = 0; l <= L; ++l) {
        PbLevel& lv = c->lev[l];
        lv.ncl = hc[l];
        lv.begin = (int*)pb_alloc(c, sizeof(int) * (lv.ncl + 1));
        lv.parent = (int*)pb_alloc(c, sizeof(int) * lv.ncl);
        lv.cbeg = (int*)pb_alloc(c, sizeof(int) * (lv.ncl + 1));
        lv.xc = (double*)pb_alloc(c, sizeof(double) * 3 * lv.ncl);
        lv.rho = (double*)pb_alloc(c, sizeof(double) * lv.ncl);
        lv.near_off = (int*)pb_alloc(c, sizeof(int) * (lv.ncl + 1));
        lv.int_off = (int*)pb_alloc(c, sizeof(int) * (lv.ncl + 1));
        if (!lv.begin || !lv.parent || !lv.cbeg || !lv.xc || !lv.rho || !lv.near_off || !lv.int_off)
            return pb_fail(c, PB_ERR_NOMEM, "levels: out of memory");
        k_flags<<<nblk(nt, B), B, 0, c->st>>>(nt, skeys, 3 * (PB_MAXL - l), flag);
        PB_LAUNCH(c);
        int rc = scan_only(c, flag, pos, nt);
        if (rc) return rc;
        PB_CUDA(c, cudaMemcpyAsync(tots + l, pos + nt, sizeof(int), cudaMemcpyDeviceToDevice, c->st));
        k_compact_starts<<<nblk(nt, B), B, 0, c->st>>>(nt, flag, pos, lv.begin, lv.ncl);
        PB_LAUNCH(c);
        if (l > 0) {
            k_parent<<<nblk(lv.ncl, B), B, 0, c->st>>>(lv.ncl, lv.begin, c->lev[l - 1].ncl, c->lev[l - 1].begin, lv.parent);
            PB_LAUNCH(c);
        }
    }
    for (int l = 0; l < L; ++l) {
        k_child_begin<<<nblk(c->lev[l].ncl + 1, B), B, 0, c->st>>>(c->lev[l].ncl, c->lev[l + 1].ncl,
                                                                     c->lev[l + 1].parent, c->lev[l].cbeg);
        PB_LAUNCH(c);
    }
    // shrink boxes, finest level first
    std::vector<double*> blo(L + 1), bhi(L + 1);
    for (int l = 0; l <= L; ++l) {
        blo[l] = (double*)pb_alloc(c, sizeof(double) * 3 * c->lev[l].ncl);
        bhi[l] = (double*)pb_alloc(c, sizeof(double) * 3 * c->lev[l].ncl);
        if (!blo[l] || !bhi[l]) return pb_fail(c, PB_ERR_NOMEM, "boxes: out of memory");
    }
    {
        PbLevel& lv = c->lev[L];
        k_leaf_boxes<<<nblk((long long)lv.ncl * 32, 128), 128, 0, c->st>>>(lv.ncl, lv.begin, c->order, c->verts, c->tris,
                                                            blo[L], bhi[L], lv.xc, lv.rho);
        PB_LAUNCH(c);
    }
    for (int l = L - 1; l >= 0; --l) {
        PbLevel& lv = c->lev[l];
        k_parent_boxes<<<nblk(lv.ncl, 128), 128, 0, c->st>>>(lv.ncl, lv.cbeg, blo[l + 1], bhi[l + 1], blo[l],
                                                              bhi[l], lv.xc, lv.rho);
        PB_LAUNCH(c);
    }
    // lists: level 0 holds the root, its own neighbour
    {
        PbLevel& r = c->lev[0];
        int h_off[2] = {0, 1};
        int zero[2] = {0, 0};
        r.near_idx = (int*)pb_alloc(c, sizeof(int));
        r.int_idx = (int*)pb_alloc(c, sizeof(int));
        if (!r.near_idx || !r.int_idx) return pb_fail(c, PB_ERR_NOMEM, "lists: out of memory");
        PB_CUDA(c, cudaMemcpyAsync(r.near_off, h_off, sizeof(h_off), cudaMemcpyHostToDevice, c->st));
        PB_CUDA(c, cudaMemcpyAsync(r.int_off, zero, sizeof(zero), cudaMemcpyHostToDevice, c->st));
        PB_CUDA(c, cudaMemsetAsync(r.near_idx, 0, sizeof(int), c->st));
        r.nnear = 1;
        r.ninter = 0;
        int ht[PB_MAXL + 1];
        PB_CUDA(c, cudaMemcpyAsync(ht, tots, sizeof(int) * (L + 1), cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
        for (int l = 0; l <= L; ++l)
            if (ht[l] != c->lev[l].ncl) return pb_fail(c, PB_ERR_CUDA, "level %d: cluster count mismatch", l);
    }
    volatile double e2 = c->prm.eta0 * c->prm.eta0;
    for (int l = 1; l <= L; ++l) {
        PbLevel& lv = c->lev[l];
        PbLevel& pv = c->lev[l - 1];
        int* ncnt = (int*)pb_alloc(c, sizeof(int) * (lv.ncl + 1));
        int* icnt = (int*)pb_alloc(c, sizeof(int) * (lv.ncl + 1));
        if (!ncnt || !icnt) return pb_fail(c, PB_ERR_NOMEM, "lists: out of memory");
        k_lists<0><<<nblk((long long)lv.ncl * 32, 128), 128, 0, c->st>>>(lv.ncl, lv.parent, pv.near_off, pv.near_idx, pv.cbeg,
                                                          lv.xc, lv.rho, e2, ncnt, icnt, nullptr, nullptr,
                                                          nullptr, nullptr);
        PB_LAUNCH(c);
        int rc = scan_only(c, ncnt, lv.near_off, lv.ncl);
        if (rc) return rc;
        rc = scan_only(c, icnt, lv.int_off, lv.ncl);
        if (rc) return rc;
        // both list lengths with one read-back
        PB_CUDA(c, cudaMemcpyAsync(tots, lv.near_off + lv.ncl, sizeof(int), cudaMemcpyDeviceToDevice, c->st));
        PB_CUDA(c, cudaMemcpyAsync(tots + 1, lv.int_off + lv.ncl, sizeof(int), cudaMemcpyDeviceToDevice, c->st));
        int hn[2];
        PB_CUDA(c, cudaMemcpyAsync(hn, tots, sizeof(hn), cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
        lv.nnear = hn[0];
        lv.ninter = hn[1];
        lv.near_idx = (int*)pb_alloc(c, sizeof(int) * (lv.nnear + 1));
        lv.int_idx = (int*)pb_alloc(c, sizeof(int) * (lv.ninter + 1));
        if (!lv.near_idx || !lv.int_idx) return pb_fail(c, PB_ERR_NOMEM, "lists: out of memory");
        k_lists<1><<<nblk((long long)lv.ncl * 32, 128), 128, 0, c->st>>>(lv.ncl, lv.parent, pv.near_off, pv.near_idx, pv.cbeg,
                                                          lv.xc, lv.rho, e2, nullptr, nullptr, lv.near_off,
                                                          lv.int_off, lv.near_idx, lv.int_idx);
        PB_LAUNCH(c);
    }
    // Taylor orders per level
    for (int l = 0; l <= L; ++l) {
        int p = c->prm.p + (c->prm.adaptive ? (L - l) : 0);
        if (c->p_level_L == L && c->p_level[l] > 0) p = c->p_level[l];  // the autotuner's per-level choice
        c->lev[l].p = p > PB_PMAX ? PB_PMAX : p;
    }
    // sorted element records
    c->e64p = (double4_32a*)pb_alloc(c, sizeof(double4_32a) * nt);
    c->e64n = (double4_32a*)pb_alloc(c, sizeof(double4_32a) * nt);
    c->e32p = (float4*)pb_alloc(c, sizeof(float4) * nt);
    c->e32n = (float4*)pb_alloc(c, sizeof(float4) * nt);
    c->e32l = (float4*)pb_alloc(c, sizeof(float4) * nt);
    c->stris = (int*)pb_alloc(c, sizeof(int) * 3 * nt);
    if (!c->e64p || !c->e64n || !c->e32p || !c->e32n || !c->e32l || !c->stris) return pb_fail(c, PB_ERR_NOMEM, "elements: out of memory");
    k_sorted_elems<<<nblk(nt, B), B, 0, c->st>>>(nt, c->order, c->cent, c->area, c->nrm, c->tris, c->e64p,
                                                 c->e64n, c->e32p, c->e32n, c->e32l, c->stris, c->rank);
    PB_LAUNCH(c);
    // largest leaf and near-field pair count (host, from the leaf ranges and lists)
    {
        PbLevel& lv = c->lev[L];
        std::vector<int> b(lv.ncl + 1), off(lv.ncl + 1), idxh(lv.nnear);
        PB_CUDA(c, cudaMemcpyAsync(b.data(), lv.begin, sizeof(int) * (lv.ncl + 1), cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaMemcpyAsync(off.data(), lv.near_off, sizeof(int) * (lv.ncl + 1), cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaMemcpyAsync(idxh.data(), lv.near_idx, sizeof(int) * lv.nnear, cudaMemcpyDeviceToHost, c->st));
        PB_CUDA(c, cudaStreamSynchronize(c->st));
        int mx = 0;
        long long np = 0;
        for (int k = 0; k < lv.ncl; ++k) {
            mx = std::max(mx, b[k + 1] - b[k]);
            long long s = 0;
            for (int t = off[k]; t < off[k + 1]; ++t) s += b[idxh[t] + 1] - b[idxh[t]];
            np += s * (b[k + 1] - b[k]);
        }
        c->max_leaf = mx;
        c->near_pairs = np;
        c->h_leaf_begin.swap(b);
        c->h_near_off.swap(off);
        c->h_near_idx.swap(idxh);
    }
    return PB_OK;
}
