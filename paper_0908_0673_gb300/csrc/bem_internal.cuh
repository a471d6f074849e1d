// Internal declarations of the GB300 BEM/FMM library: plan layout in HBM,
// error plumbing and small device helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bem.h"

namespace bem {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

// Kernel-launch accounting: every launch site calls count_launch(); while a
// graph is being captured the count goes to that graph's kernel tally, and
// each graph launch adds its tally.
void count_launch(long long n = 1);
extern thread_local long long *tl_capture_count;

#define BEM_CUDA(call)                                                      \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return ::bem::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)
#define BEM_TRY(call)                                                       \
    do {                                                                    \
        int r_ = (call);                                                    \
        if (r_ != BEM_OK) return r_;                                        \
    } while (0)
#define BEM_LAUNCH_CHECK() BEM_CUDA(cudaGetLastError())

constexpr int QBITS = 21;   // Morton bits per axis
constexpr int PMAX = 20;    // largest supported expansion order
constexpr int NQ = 7;       // regular quadrature points per element

// Radon's 7-point degree-5 rule on the reference triangle (Stroud T2:5-1),
// point q in owner order: the centroid with weight 9/80, then two orbits,
// a = (6 - sqrt15)/21, b = (9 + 2 sqrt15)/21 with weight (155 - sqrt15)/2400
// and c = (6 + sqrt15)/21, d = (9 - 2 sqrt15)/21 with weight (155 + sqrt15)/2400
// (weights sum to 1/2).  The one definition both the geometry tables and the
// field evaluator use.
__host__ __device__ inline void radon7(int q, double &s, double &t, double &w) {
    const double r15 = 3.872983346207417;   // sqrt(15), correctly rounded
    const double a = (6.0 - r15) / 21.0, b = (9.0 + 2.0 * r15) / 21.0;
    const double c = (6.0 + r15) / 21.0, d = (9.0 - 2.0 * r15) / 21.0;
    const double wa = (155.0 - r15) / 2400.0, wc = (155.0 + r15) / 2400.0;
    switch (q) {
    case 0: s = 1.0 / 3.0; t = 1.0 / 3.0; w = 9.0 / 80.0; break;
    case 1: s = a; t = a; w = wa; break;
    case 2: s = b; t = a; w = wa; break;
    case 3: s = a; t = b; w = wa; break;
    case 4: s = c; t = c; w = wc; break;
    case 5: s = d; t = c; w = wc; break;
    default: s = c; t = d; w = wc; break;
    }
}

// ---------------------------------------------------------------------------
// device memory of a context, kept for reuse
// ---------------------------------------------------------------------------
// Blocks that the context's plans give back wait here for the next
// allocation of the context (plans are built and destroyed per request in a
// serving loop; cudaMalloc and cudaFree cost tens of microseconds each and
// cudaFree synchronises the device).  A request takes the smallest cached
// block of at least its size and at most twice it.  At most `limit` bytes
// are kept (environment BEM_CACHE_BYTES, default 4 GiB); what would exceed
// it is freed.  A block is given back only when no work can still use it.
struct DevCache {
    std::mutex mu;
    std::multimap<size_t, void *> blocks;   // size -> block
    size_t cached = 0, limit = (size_t)4 << 30;
    void *take(size_t n, size_t *got) {
        std::lock_guard<std::mutex> lock(mu);
        auto it = blocks.lower_bound(n);
        if (it == blocks.end() || it->first > 2 * n) return nullptr;
        void *p = it->second;
        *got = it->first;
        cached -= it->first;
        blocks.erase(it);
        return p;
    }
    void give(void *p, size_t n) {
        std::lock_guard<std::mutex> lock(mu);
        if (cached + n > limit) {
            cudaFree(p);
            return;
        }
        blocks.emplace(n, p);
        cached += n;
    }
    void flush() {
        std::lock_guard<std::mutex> lock(mu);
        for (auto &b : blocks) cudaFree(b.second);
        blocks.clear();
        cached = 0;
    }
    ~DevCache() { flush(); }
};

// ---------------------------------------------------------------------------
// device buffers owned by a plan
// ---------------------------------------------------------------------------
// Sizes are rounded up to 256 bytes.  Allocations may come from two host
// threads of one plan build (the lock keeps the lists consistent).  While a
// build defers, released blocks stay reserved until the build has
// synchronised its streams (end_defer); otherwise a release waits for the
// device, as cudaFree would, before the block goes back to the cache.
struct Arena {
    std::mutex mu;
    std::shared_ptr<DevCache> cache;    // the context's, or none
    std::vector<void *> ptrs;
    std::vector<size_t> sizes;
    std::vector<std::pair<void *, size_t>> pending;
    bool deferring = false;
    size_t bytes = 0;                   // bytes currently held
    size_t peak = 0;                    // most bytes held at any time
    template <class T>
    int alloc(T **p, size_t n) {
        *p = nullptr;
        if (n == 0) n = 1;
        const size_t want = (n * sizeof(T) + 255) & ~(size_t)255;
        std::lock_guard<std::mutex> lock(mu);
        size_t got = want;                // a cached block may be up to twice the request
        void *q = cache ? cache->take(want, &got) : nullptr;
        if (!q) {
            got = want;
            cudaError_t e = cudaMalloc(&q, want);
            if (e != cudaSuccess && cache) {
                cudaGetLastError();
                cudaDeviceSynchronize();
                cache->flush();
                e = cudaMalloc(&q, want);
            }
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
        }
        *p = (T *)q;
        ptrs.push_back(q);
        sizes.push_back(got);
        bytes += got;
        if (bytes > peak) peak = bytes;
        return BEM_OK;
    }
    void release(void *p) {
        std::lock_guard<std::mutex> lock(mu);
        for (size_t i = 0; i < ptrs.size(); i++)
            if (ptrs[i] == p && p) {
                if (deferring) {
                    pending.emplace_back(p, sizes[i]);
                } else if (cache) {
                    cudaDeviceSynchronize();
                    cache->give(p, sizes[i]);
                } else {
                    cudaFree(p);
                }
                ptrs[i] = nullptr;
                bytes -= sizes[i];
            }
    }
    // the build's streams are synchronised: its released blocks are free
    void end_defer() {
        std::lock_guard<std::mutex> lock(mu);
        deferring = false;
        for (auto &b : pending) {
            if (cache) cache->give(b.first, b.second);
            else cudaFree(b.first);
        }
        pending.clear();
    }
    ~Arena() {
        bool any = !pending.empty();
        for (void *p : ptrs) any = any || p;
        if (!any) return;
        if (cache) cudaDeviceSynchronize();
        for (size_t i = 0; i < ptrs.size(); i++)
            if (ptrs[i]) {
                if (cache) cache->give(ptrs[i], sizes[i]);
                else cudaFree(ptrs[i]);
            }
        for (auto &b : pending) {
            if (cache) cache->give(b.first, b.second);
            else cudaFree(b.first);
        }
    }
};

// Multi-index tables for |alpha| <= p, ordered by degree, then m, n descending.
struct MIndex {
    int p = 0, np = 0;
    std::vector<int> m, n, k;
    std::vector<int> deg_off;          // first index of each degree, size p+2
    std::vector<int> idx3;             // [(m*(p+1)+n)*(p+1)+k] -> index or -1
    void init(int p_);
};

// Class-matrix image of the tensor-core M2L (m2l_tc.cu): one block per K-step
// of 8 columns alpha, holding the rows beta that K-step reaches (a prefix of
// the degree-ordered rows, a multiple of 16): block j starts at float ks_off[j]
// of an image plane and has ks_n[j] rows.
constexpr int TC_MAXKS = 64;
struct TcPlan {
    int nks = 0, img_floats = 0;        // K-steps; floats of one image plane (tf32 hi or lo)
    int ks_off[TC_MAXKS], ks_n[TC_MAXKS];
    // an image too large for shared memory is held in two parts, K-steps
    // [0, ks_split) and [ks_split, nks), loaded one after the other per tile
    int ks_split = 0;                   // nks when the image is held whole
    int part_floats[2] = {0, 0};        // floats of each part's plane
};

// Tree and plan state (everything device-resident unless named h_*).
struct Tree {
    int nlev = 0;                       // number of levels (root = level 0)
    std::vector<int> lev_off;           // box range of each level, size nlev+1
    int nbox = 0, nleaf = 0;
    double lo[3] = {0, 0, 0}, side = 0;
    // boxes (level-by-level numbering)
    int *level = nullptr, *ix = nullptr, *iy = nullptr, *iz = nullptr;
    int *parent = nullptr, *child0 = nullptr, *nchild = nullptr;
    int *nb = nullptr, *ne = nullptr;   // node range in Morton order
    int *eb = nullptr, *ee = nullptr;   // element range in owner order
    double *cx = nullptr, *cy = nullptr, *cz = nullptr, *r = nullptr;
    float4 *fbox = nullptr;             // float32 centre and radius of each box (search filters)
    int *leaves = nullptr;              // box ids of the leaves
    int *near_ptr = nullptr, *near_idx = nullptr;
    int *inter_ptr = nullptr, *inter_idx = nullptr;
    int64_t n_near = 0, n_inter = 0;
    // vertices
    unsigned long long *codes = nullptr; // sorted Morton codes
    int *node_perm = nullptr;           // Morton position -> node
    int *node_rank = nullptr;           // node -> Morton position
    int *leaf_of_node = nullptr;        // node -> leaf box
    double *tx = nullptr, *ty = nullptr, *tz = nullptr;  // vertices in Morton order
    // elements, in owner order (sorted by Morton rank of their node 0)
    int *elem_perm = nullptr;           // sorted position -> element
    int *el_phi = nullptr, *el_chi = nullptr;  // [E][npe] indices, sorted order
};

struct Quad {                           // regular 7-point sources, owner order
    double *x = nullptr, *y = nullptr, *z = nullptr;
    double *nx = nullptr, *ny = nullptr, *nz = nullptr, *w = nullptr;
    float *fx = nullptr, *fy = nullptr, *fz = nullptr;   // offsets from the owning leaf centre
    float *fnx = nullptr, *fny = nullptr, *fnz = nullptr, *fw = nullptr;
};

struct Correction {                     // CSR by node (row), special - regular
    int *ptrD = nullptr, *colD = nullptr;
    int *ptrS = nullptr, *colS = nullptr;
    double *valD = nullptr, *valS = nullptr;       // complex pairs for Helmholtz
    float *fvalD = nullptr, *fvalS = nullptr;
    int64_t nnzD = 0, nnzS = 0;
};

}  // namespace bem

struct bem_ctx {
    int device = 0;
    int sm_count = 0;
    std::shared_ptr<bem::DevCache> cache;   // device memory given back by the context's plans
};

struct bem_mesh {
    bem_ctx *ctx = nullptr;
    int64_t n_nodes = 0, n_elems = 0, n_chi = 0;
    int npe = 0, elem_type = 0;
    double edge_angle = 30.0;
    std::vector<double> nodes;          // [n][3]
    std::vector<int32_t> elems;         // [E][npe]
    std::vector<int32_t> chi;           // [E][npe]
    // optional device-resident copy (bem_mesh_upload)
    int dev_device = -1;
    double *d_nodes = nullptr;
    int32_t *d_elems = nullptr, *d_chi = nullptr;
    ~bem_mesh();
};

namespace bem {
// What alloc_fmm builds for one expansion order and free_fmm releases: index
// tables, product buffers and the order-dependent M2L tables.  The plan holds
// one (its own order); during set-up the diagonal's product runs from a
// second one at the diagonal's order (bem_plan::diag_state), so that the
// plan's own can be built while that product runs.  std::swap of the base
// moves a whole state in or out.
struct FmmState {
    bem::MIndex mi;
    // multi-index tables on the device
    int *d_m = nullptr, *d_n = nullptr, *d_k = nullptr, *d_idx3 = nullptr;
    double *d_fact = nullptr;           // [2*PMAX+2]
    // work buffers of one matrix multiplication
    double *f = nullptr;                // quadrature strengths [Q] (x2 for complex)
    double *M = nullptr, *L = nullptr;  // [nbox][np] scaled moments / locals (x2 complex)
    double *ytmp = nullptr;             // [N] far + near regular sums (x2 complex)
    float *fM = nullptr, *fL = nullptr, *ff = nullptr;   // mixed-precision copies
    const void **xptr = nullptr;        // device slot: input vector of the next matvec
    void **yptr = nullptr;              // device slot: output vector
    // M2L on canonical offset classes: the order-dependent part (m2l_tc.cu,
    // m2l_simt.cu); the classes themselves belong to the plan
    int sy_ntile = 0, sy_ldp = 0, sy_nkc = 0;
    int sy_ready = 0;                   // order-dependent tables built for the current order
    int sy_tc = 0;                      // the tensor-core form runs (mixed-precision Laplace)
    int *sy_tile_cls = nullptr, *sy_tile_start = nullptr, *sy_tile_cnt = nullptr;
    int *sy_src = nullptr, *sy_sig = nullptr, *sy_pair = nullptr;   // pairs in class order
    std::vector<int> sy_bt, sy_bb, sy_bu;                 // host: per run, first tile, target and pair (size runs + 1)
    int *sy_ord = nullptr;              // [class][2] source and target order
    double *sy_D = nullptr;             // [class][np][C] derivative tables
    float *sy_fD = nullptr;
    unsigned short *sy_fwd = nullptr;   // [48][np] signed index maps (sign in bit 15)
    unsigned short *sy_fwdq = nullptr;  // [6][np] index maps of the axis permutations (tensor-core form)
    unsigned *sy_sgn = nullptr;         // [48][ldp / 32] sign bits of the canonical-frame moments (tensor-core form)
    float *sy_Mq = nullptr;             // [box][6][ldp] moments under each axis permutation, per product (tensor-core form)
    int *sy_inv = nullptr;              // [48][np] signed index maps (sign in bit 31)
    int *sy_mexp = nullptr;             // [np] exponents m | n << 8 | k << 16 | degree << 24
    double *sy_invf = nullptr;          // [np] 1 / a!
    float *sy_img = nullptr;            // [class][hi, lo][image floats] class-matrix images (tensor-core form)
    void *sy_Lp = nullptr;              // [pair][sy_ldp][C] canonical-frame local contributions
    bem::TcPlan sy_g;
    float *p2m_W = nullptr;             // [Q][np] stored double-layer P2M weights (float32 plans)
    float *xf = nullptr;                // float32 copy of a product's input (correction product)
    std::vector<int> lev_p;             // expansion order of each tree level
    int *d_lev_p = nullptr;
    bool lev_var = false;               // the order varies with the level (p_min > 0 and more than one order)
};
}  // namespace bem

struct bem_plan : bem::FmmState {
    bem_mesh *mesh = nullptr;
    int device = 0, sm_count = 0;
    int green = BEM_LAPLACE;
    double k = 0.0;
    bem_fmm_params prm{};
    int64_t N = 0, E = 0, Q = 0, nchi = 0;
    int npe = 0;
    bem::Arena arena;
    bem::Tree t;
    bem::Quad q;
    bem::Correction corr;
    // device copies of mesh data (original order)
    double *nodes = nullptr;            // [N][3]
    int *elems = nullptr, *chi = nullptr;
    double *C = nullptr;                // diagonal [N]
    int *skip = nullptr;                // device flag: kernels return at once when set
    // graphs
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long graph_kernels[2] = {0, 0};
    cudaStream_t capture_stream = nullptr;
    // M2L on canonical offset classes (m2l_tc.cu: tensor-core form and tables;
    // m2l_simt.cu: SIMT form)
    int sy_ncls = 0;
    // coarsest tree level holding an M2L source (whose moments are used) and an
    // M2L target (whose locals can be nonzero); nlev when there is none
    int m2l_src_lmin = 0, m2l_tgt_lmin = 0;
    double *sy_rho = nullptr;           // [class][3] canonical offsets / h_t
    double *sy_kh = nullptr;            // [class] k h_t (Helmholtz)
    int *sy_dl = nullptr;               // [class] level difference
    int *sy_sig_u = nullptr;            // [pair] symmetry id (permutation * 8 + sign bits)
    std::vector<int> sy_hcls, sy_hsig, sy_hsrc, sy_hip;   // host: per pair class, symmetry, source; list offsets
    std::vector<int> sy_hlev, sy_hdl;                     // host: per canonical class, target level (when keyed) and dl
    int *dev_err = nullptr;             // device word: set when a kernel's bounded wait gave up
    // counters
    double setup_ms[BEM_NSETUP] = {};
    int64_t near_pairs = 0;
    std::vector<void *> deferred;       // set-up temporaries released after the next synchronisation
    double *diag_ones = nullptr;        // phi = 1 of the diagonal's product (set-up only)
    bem::FmmState diag_state;           // the diagonal's order while its product runs (set-up only)
    bool diag_mode = false;             // alloc_fmm for the diagonal's order
    cudaStream_t setup_stream[3] = {nullptr, nullptr, nullptr};
    int2 *near_items[2] = {nullptr, nullptr};   // float32 near-field work items, 64- and 32-target passes
    int near_nitems[2] = {0, 0};
    int last_op = -1;
    // GMRES workspace
    double *V = nullptr, *H = nullptr, *gs = nullptr, *w = nullptr, *xk = nullptr, *bvec = nullptr;
    double *zbuf = nullptr;             // the preconditioned Arnoldi vector M^-1 V_j (the product's input)
    double *npart = nullptr;            // per-block partial sums of |w|^2 [ceil(N / 256)]
    double *dinv = nullptr;             // 1 / C_i: GMRES's right preconditioner M = diag(C) [N]
    double *bc_vec = nullptr, *bc_sc = nullptr;   // BiCGStab vectors (r, rh, p, v, s, t) and scalars
    int *bc_st = nullptr;
    double *scal = nullptr;             // device scalars
    double *hostbuf = nullptr;          // pinned read-back of GMRES scalars
    void **gm_slot = nullptr;           // device pointer slots of the current solve: [0] chi, [1] x
    int *istate = nullptr;              // device ints: [0] converged flag, [1] steps in cycle
    int gm_restart = 0;
    cudaGraphExec_t cycle_graph = nullptr;
    int capture_retries = 0;            // captures invalidated by other host threads
    ~bem_plan();
};

namespace bem {
// stages (each returns BEM_OK or an error code)
int build_tree(bem_plan *P, cudaStream_t s);
int build_geometry(bem_plan *P, cudaStream_t s);
int build_radii_lists(bem_plan *P, cudaStream_t s);
int build_correction(bem_plan *P, cudaStream_t s);
int alloc_fmm(bem_plan *P, cudaStream_t s);
void free_fmm(bem_plan *P);
int build_m2l_classes(bem_plan *P);
int build_translation_tables(bem_plan *P, cudaStream_t s);
void free_translation_tables(bem_plan *P);
void set_translation_attributes();
int build_m2l_sym(bem_plan *P, const std::vector<int> &pair_cls, const std::vector<long long> &kvec,
                  const std::vector<int> &dls, const std::vector<int> &levs, const std::vector<int> &src,
                  const std::vector<int> &ip);
int build_sym_tables(bem_plan *P, cudaStream_t s);
void free_sym_tables(bem_plan *P);
int launch_m2l_tc(bem_plan *P, const float *M, float *L, cudaStream_t s);
void set_tc_attributes();
template <class R, int C>
int launch_m2l_sy(bem_plan *P, const R *M, R *L, cudaStream_t s);
size_t sy_simt_smem_bytes(int prec_float, int C, int np, int p);
void set_sy_attributes();
int launch_m2l_derivs(bem_plan *P, int ncls, const double *rho, const double *kh, double *D, float *fD,
                      cudaStream_t s);
template <class R, int C>
int launch_translations(bem_plan *P, R *M, R *L, cudaStream_t s, cudaEvent_t *ev);
template <class R, int C>
int launch_m2m(bem_plan *P, R *M, cudaStream_t s, int lmin = 0);
int field_moments(bem_plan *P, const void *phi, const void *chi, cudaStream_t s);
int build_near_items(bem_plan *P);
int diagonal_prepare(bem_plan *P, cudaStream_t s);
int diagonal_product(bem_plan *P, cudaStream_t s);
int diagonal_finish(bem_plan *P, cudaStream_t s);
int enqueue_matvec(bem_plan *P, int op, int green, double k, cudaStream_t s);
int set_slots(bem_plan *P, const void *x, void *y, cudaStream_t s);
// Work buffers of one product: quadrature strengths, moments, locals (float32
// or float64 with the plan's precision, complex pairs for Helmholtz) and the
// float64 regular far + near sums.
struct WorkBufs {
    void *f, *M, *L;
    double *ytmp;
};
int enqueue_matvec_raw(bem_plan *P, int op, int green, double k, int with_diag, cudaStream_t s,
                       cudaEvent_t *ev = nullptr, const WorkBufs *wb = nullptr);
int solve(bem_plan *P, const void *chi, void *phi, int nrhs, const bem_solve_params *sp,
          bem_solve_info *info, cudaStream_t s);
int64_t mesh_chi_index(const double *nodes, int64_t nn, const int32_t *elems, int64_t ne, int npe,
                       double angle_deg, int32_t *chi);
// radix sort of (key, value) pairs, stable, ascending in the low `bits` bits of key
int radix_sort_pairs(unsigned long long *keys, int *vals, unsigned long long *tmpk, int *tmpv,
                     int n, int bits, unsigned int *hist, int nblk_cap, cudaStream_t s);
// exclusive scan of n ints, total to *total_dev; blk: device scratch of scan_scratch(n) ints
int scan_exclusive(const int *in, int *out, int n, int *total_dev, int *blk, cudaStream_t s);
size_t scan_scratch(int n);
}  // namespace bem

#ifdef __CUDACC__
// ---------------------------------------------------------------------------
// device helpers: FP64 with explicit rounding (no FMA contraction) where the
// tree, radii and pair classification must follow a fixed operation order
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dist3_rn(double ax, double ay, double az, double bx, double by,
                                           double bz) {
    double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}
#endif
