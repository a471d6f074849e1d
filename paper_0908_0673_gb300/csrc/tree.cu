// Octree over the vertices built on the device (Section 3.1): Morton codes of
// the quantised vertices, a stable radix sort, level-synchronous splitting of
// every box that holds B or more vertices, unique element ownership (the leaf
// of the element's first corner), convergence radii (Section 3.4, Eq. 12) and
// near-field / interaction lists (Section 3.6, Eq. 13).
//
// Every floating-point decision (quantisation, box centres, radii, separation)
// uses FP64 with explicit round-to-nearest operations in a fixed order, so the
// tree and its lists are reproducible bit for bit by any implementation that
// follows the same order.
#include <algorithm>

#include "bem_internal.cuh"

namespace bem {

// ---------------------------------------------------------------------------
// exclusive scan: blocks of SCAN_BLK elements are scanned in shared memory;
// with more than one block, the block totals are scanned by one block and
// added in a third pass.  Integer sums, so the result is exact.
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 512, SCAN_PER = 8, SCAN_BLK = SCAN_T * SCAN_PER;

// exclusive scan of the block's SCAN_BLK elements of sh[] in place; returns the block total
template <class T>
__device__ T block_scan(T *sh, T *warp_tot) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T v[SCAN_PER], s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER; i++) {
        v[i] = sh[tid * SCAN_PER + i];
        s += v[i];
    }
    T x = s;                                   // inclusive scan of the thread sums
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < SCAN_T / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_T / 32) warp_tot[lane] = w;   // inclusive warp offsets
    }
    __syncthreads();
    T run = x - s + (warp > 0 ? warp_tot[warp - 1] : 0);
    const T total = warp_tot[SCAN_T / 32 - 1];
#pragma unroll
    for (int i = 0; i < SCAN_PER; i++) {
        sh[tid * SCAN_PER + i] = run;
        run += v[i];
    }
    __syncthreads();
    return total;
}

// mode 0: block totals only (blk[b]); mode 1: out = scan + blk[b] (blk scanned);
// mode 2: one block scans in[] of n <= SCAN_BLK elements, total to *total
template <class T>
__global__ void __launch_bounds__(SCAN_T) k_scan(const T *__restrict__ in, T *__restrict__ out, int n, T *blk,
                                               T *total, int mode) {
    __shared__ T sh[SCAN_BLK];
    __shared__ T wt[SCAN_T / 32];
    const int b0 = blockIdx.x * SCAN_BLK;
    for (int i = threadIdx.x; i < SCAN_BLK; i += SCAN_T) sh[i] = b0 + i < n ? in[b0 + i] : (T)0;
    __syncthreads();
    if (mode == 0) {
        T s = 0;
#pragma unroll
        for (int i = 0; i < SCAN_PER; i++) s += sh[threadIdx.x * SCAN_PER + i];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) wt[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            T t = 0;
            for (int w = 0; w < SCAN_T / 32; w++) t += wt[w];
            blk[blockIdx.x] = t;
        }
        return;
    }
    const T tot = block_scan<T>(sh, wt);
    const T add = mode == 1 ? blk[blockIdx.x] : (T)0;
    for (int i = threadIdx.x; i < SCAN_BLK; i += SCAN_T)
        if (b0 + i < n) out[b0 + i] = sh[i] + add;
    if (mode == 2 && threadIdx.x == 0 && total) *total = tot;
}

// exclusive scan of n values (in and out may alias); *total_dev = sum;
// blk: device scratch of at least scan_scratch(n) values (the block totals
// of every level: more than SCAN_BLK blocks are scanned the same way)
size_t scan_scratch(int n) {
    size_t t = 1;
    for (int64_t m = n; m > SCAN_BLK;) {
        m = (m + SCAN_BLK - 1) / SCAN_BLK;
        t += (size_t)m;
    }
    return t + 1;
}

template <class T>
static int scan_t(const T *in, T *out, int n, T *total_dev, T *blk, cudaStream_t s) {
    if (n <= 0) return BEM_OK;
    const int nb = (n + SCAN_BLK - 1) / SCAN_BLK;
    if (nb == 1) {
        (k_scan<T><<<1, SCAN_T, 0, s>>>(in, out, n, nullptr, total_dev, 2), ::bem::count_launch());
    } else {
        (k_scan<T><<<nb, SCAN_T, 0, s>>>(in, out, n, blk, nullptr, 0), ::bem::count_launch());
        BEM_TRY(scan_t<T>(blk, blk, nb, total_dev, blk + nb, s));   // the block totals, in place
        (k_scan<T><<<nb, SCAN_T, 0, s>>>(in, out, n, blk, nullptr, 1), ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    return BEM_OK;
}

int scan_exclusive(const int *in, int *out, int n, int *total_dev, int *blk, cudaStream_t s) {
    return scan_t<int>(in, out, n, total_dev, blk, s);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (64-bit key, int value) pairs, 8 bits per pass
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;

__global__ void k_rs_hist(const unsigned long long *__restrict__ keys, int n, int shift,
                          unsigned int *__restrict__ hist, int nblk) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int i = blockIdx.x * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const unsigned long long *__restrict__ keys, const int *__restrict__ vals, int n,
                             int shift, const unsigned int *__restrict__ offs, int nblk,
                             unsigned long long *__restrict__ okeys, int *__restrict__ ovals) {
    __shared__ unsigned int wc[RS_THREADS / 32][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < (RS_THREADS / 32) * 256; t += RS_THREADS) (&wc[0][0])[t] = 0;
    __syncthreads();
    int i = blockIdx.x * RS_THREADS + threadIdx.x;
    unsigned long long key = 0;
    int val = 0;
    unsigned d = 256u;                        // sentinel for lanes past the end
    if (i < n) {
        key = keys[i];
        val = vals[i];
        d = (unsigned)((key >> shift) & 255u);
    }
    unsigned peers = __match_any_sync(0xffffffffu, d);
    unsigned lt = (1u << lane) - 1u;
    int rank = __popc(peers & lt);
    if (d < 256u && rank == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    if (d < 256u) {
        unsigned pos = offs[d * nblk + blockIdx.x] + rank;
        for (int w = 0; w < warp; w++) pos += wc[w][d];
        okeys[pos] = key;
        ovals[pos] = val;
    }
}

// keys/vals are sorted in place (ping-pong through tmp); hist needs
// 256 * ceil(n/256) entries followed by scan_scratch(256 * ceil(n/256)).
int radix_sort_pairs(unsigned long long *keys, int *vals, unsigned long long *tmpk, int *tmpv, int n, int bits,
                     unsigned int *hist, int nblk_cap, cudaStream_t s) {
    if (n <= 1) return BEM_OK;
    const int nblk = (n + RS_THREADS - 1) / RS_THREADS;
    if (nblk > nblk_cap) { set_error("radix sort: histogram too small"); return BEM_EINVAL; }
    const int passes = (bits + 7) / 8;
    unsigned long long *ka = keys, *kb = tmpk;
    int *va = vals, *vb = tmpv;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        (k_rs_hist<<<nblk, RS_THREADS, 0, s>>>(ka, n, shift, hist, nblk), ::bem::count_launch());
        BEM_TRY(scan_t<unsigned int>(hist, hist, 256 * nblk, nullptr, hist + (size_t)256 * nblk_cap, s));
        (k_rs_scatter<<<nblk, RS_THREADS, 0, s>>>(ka, va, n, shift, hist, nblk, kb, vb), ::bem::count_launch());
        BEM_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        BEM_CUDA(cudaMemcpyAsync(keys, ka, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(vals, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    }
    return BEM_OK;
}

// ---------------------------------------------------------------------------
// root cube and Morton codes
// ---------------------------------------------------------------------------
// Bounding box of the vertices: each block reduces a strided share to
// part[block][6] (min x, y, z, max x, y, z; min and max are exact, so the order
// does not matter), then one block combines them and writes root[0..2] lower
// corner, root[3] side, root[4] 2^21 / side.
constexpr int ROOT_T = 256, ROOT_BLOCKS = 304;
__global__ void __launch_bounds__(ROOT_T) k_root_part(const double *__restrict__ nodes, int n, double *part) {
    __shared__ double sh[6][ROOT_T];
    const int tid = threadIdx.x;
    double lo[3] = {nodes[0], nodes[1], nodes[2]}, hi[3] = {nodes[0], nodes[1], nodes[2]};
    for (int i = blockIdx.x * ROOT_T + tid; i < n; i += gridDim.x * ROOT_T)
        for (int c = 0; c < 3; c++) {
            const double v = nodes[3 * (size_t)i + c];
            lo[c] = fmin(lo[c], v);
            hi[c] = fmax(hi[c], v);
        }
    for (int c = 0; c < 3; c++) { sh[c][tid] = lo[c]; sh[3 + c][tid] = hi[c]; }
    __syncthreads();
    for (int off = ROOT_T / 2; off > 0; off >>= 1) {
        if (tid < off)
            for (int c = 0; c < 3; c++) {
                sh[c][tid] = fmin(sh[c][tid], sh[c][tid + off]);
                sh[3 + c][tid] = fmax(sh[3 + c][tid], sh[3 + c][tid + off]);
            }
        __syncthreads();
    }
    if (tid < 6) part[(size_t)blockIdx.x * 6 + tid] = sh[tid][0];
}

__global__ void __launch_bounds__(ROOT_T) k_root(const double *__restrict__ part, int nparts, double *root) {
    __shared__ double sh[6][ROOT_T];
    const int tid = threadIdx.x;
    double v[6];
    for (int c = 0; c < 6; c++) v[c] = part[c];
    for (int b = tid; b < nparts; b += ROOT_T)
        for (int c = 0; c < 6; c++) v[c] = c < 3 ? fmin(v[c], part[6 * b + c]) : fmax(v[c], part[6 * b + c]);
    for (int c = 0; c < 6; c++) sh[c][tid] = v[c];
    __syncthreads();
    for (int off = ROOT_T / 2; off > 0; off >>= 1) {
        if (tid < off)
            for (int c = 0; c < 6; c++)
                sh[c][tid] = c < 3 ? fmin(sh[c][tid], sh[c][tid + off]) : fmax(sh[c][tid], sh[c][tid + off]);
        __syncthreads();
    }
    if (tid == 0) {
        const double mn[3] = {sh[0][0], sh[1][0], sh[2][0]}, mx[3] = {sh[3][0], sh[4][0], sh[5][0]};
        double ext = __dsub_rn(mx[0], mn[0]);
        double ey = __dsub_rn(mx[1], mn[1]), ez = __dsub_rn(mx[2], mn[2]);
        if (ey > ext) ext = ey;
        if (ez > ext) ext = ez;
        double side = __dmul_rn(ext, 1.0 + 0x1p-20);
        for (int c = 0; c < 3; c++)
            root[c] = __dsub_rn(__dmul_rn(__dadd_rn(mn[c], mx[c]), 0.5), __dmul_rn(side, 0.5));
        root[3] = side;
        root[4] = __ddiv_rn(0x1p21, side);
    }
}

__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void k_morton(const double *__restrict__ nodes, int n, const double *__restrict__ root,
                         unsigned long long *__restrict__ codes, int *__restrict__ vals) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long qmax = (1ll << QBITS) - 1;
    unsigned long long q[3];
    for (int c = 0; c < 3; c++) {
        double v = floor(__dmul_rn(__dsub_rn(nodes[3 * i + c], root[c]), root[4]));
        long long iv = (long long)v;
        iv = iv < 0 ? 0 : (iv > qmax ? qmax : iv);
        q[c] = (unsigned long long)iv;
    }
    codes[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    vals[i] = i;
}

// ---------------------------------------------------------------------------
// level-synchronous box splitting
// ---------------------------------------------------------------------------
__device__ __forceinline__ int child_digit(unsigned long long code, int level) {
    return (int)((code >> (3 * (QBITS - 1 - level))) & 7ull);
}

// first position in [b, e) whose child digit (for a box at `level`) is >= d
__device__ int digit_lower_bound(const unsigned long long *codes, int b, int e, int level, int d) {
    while (b < e) {
        int m = (b + e) >> 1;
        if (child_digit(codes[m], level) < d) b = m + 1; else e = m;
    }
    return b;
}

// Splitting a level: eight lanes per box, lane d finding the code range of
// child octant d by two binary searches; a ballot over the group gives the
// number of non-empty octants and each one's place among them.
__global__ void k_count_children(const unsigned long long *__restrict__ codes, const int *__restrict__ nb,
                                 const int *__restrict__ ne, int off, int cnt, int level, int B, int max_level,
                                 int *__restrict__ nch) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, j = tid >> 3, d = tid & 7, lane = threadIdx.x & 31;
    const unsigned gmask = 0xffu << (lane & ~7);
    if (j >= cnt) return;                              // whole groups leave together (cnt * 8 threads)
    const int b = off + j, s = nb[b], e = ne[b];
    bool has = false;
    if (e - s >= B && level < max_level)
        has = digit_lower_bound(codes, s, e, level, d + 1) > digit_lower_bound(codes, s, e, level, d);
    const unsigned m = __ballot_sync(gmask, has) & gmask;
    if (d == 0) nch[j] = __popc(m);
}

__global__ void k_write_children(const unsigned long long *__restrict__ codes, int off, int cnt, int level,
                                 const int *__restrict__ nch, const int *__restrict__ choff, int child_base,
                                 int *nb, int *ne, int *ix, int *iy, int *iz, int *lev, int *parent,
                                 int *child0, int *nchild) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, j = tid >> 3, d = tid & 7, lane = threadIdx.x & 31;
    const unsigned gmask = 0xffu << (lane & ~7);
    if (j >= cnt) return;
    const int b = off + j, n = nch[j];
    if (d == 0) {
        nchild[b] = n;
        child0[b] = n ? child_base + choff[j] : -1;
    }
    if (!n) return;                                    // the whole group
    const int s = nb[b], e = ne[b];
    const int lo = digit_lower_bound(codes, s, e, level, d), hi = digit_lower_bound(codes, s, e, level, d + 1);
    const unsigned m = __ballot_sync(gmask, hi > lo) & gmask;
    if (hi <= lo) return;
    const int w = child_base + choff[j] + __popc(m & ((1u << lane) - 1u) & gmask);
    nb[w] = lo;
    ne[w] = hi;
    ix[w] = 2 * ix[b] + (d & 1);
    iy[w] = 2 * iy[b] + ((d >> 1) & 1);
    iz[w] = 2 * iz[b] + ((d >> 2) & 1);
    lev[w] = level + 1;
    parent[w] = b;
}

__global__ void k_box_geometry(int nbox, const int *__restrict__ lev, const int *__restrict__ ix,
                               const int *__restrict__ iy, const int *__restrict__ iz, const double *__restrict__ root,
                               double *cx, double *cy, double *cz) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    double h = scalbn(root[3], -lev[b]);
    cx[b] = __dadd_rn(root[0], __dmul_rn((double)ix[b] + 0.5, h));
    cy[b] = __dadd_rn(root[1], __dmul_rn((double)iy[b] + 0.5, h));
    cz[b] = __dadd_rn(root[2], __dmul_rn((double)iz[b] + 0.5, h));
}

__global__ void k_leaf_nodes(int nbox, const int *__restrict__ nchild, const int *__restrict__ nb,
                             const int *__restrict__ ne, const int *__restrict__ perm, int *__restrict__ leaf_of_node,
                             int *__restrict__ rank) {
    int b = blockIdx.x;
    if (b >= nbox || nchild[b] != 0) return;
    for (int k = nb[b] + threadIdx.x; k < ne[b]; k += blockDim.x) {
        leaf_of_node[perm[k]] = b;
        rank[perm[k]] = k;
    }
}

__global__ void k_gather_nodes(int n, const int *__restrict__ perm, const double *__restrict__ nodes, double *tx,
                               double *ty, double *tz) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int v = perm[k];
    tx[k] = nodes[3 * v];
    ty[k] = nodes[3 * v + 1];
    tz[k] = nodes[3 * v + 2];
}

__global__ void k_elem_keys(int E, int npe, const int *__restrict__ elems, const int *__restrict__ rank,
                            unsigned long long *keys, int *vals) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    keys[e] = (unsigned long long)rank[elems[(size_t)e * npe]];
    vals[e] = e;
}

__global__ void k_elem_gather(int E, int npe, const int *__restrict__ perm, const int *__restrict__ elems,
                              const int *__restrict__ chi, int *el_phi, int *el_chi) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E) return;
    int e = perm[i];
    for (int a = 0; a < npe; a++) {
        el_phi[(size_t)i * npe + a] = elems[(size_t)e * npe + a];
        el_chi[(size_t)i * npe + a] = chi[(size_t)e * npe + a];
    }
}

__device__ int ull_lower_bound(const unsigned long long *a, int n, unsigned long long v) {
    int b = 0, e = n;
    while (b < e) {
        int m = (b + e) >> 1;
        if (a[m] < v) b = m + 1; else e = m;
    }
    return b;
}

__global__ void k_box_elems(int nbox, int E, const unsigned long long *__restrict__ ekeys, const int *__restrict__ nb,
                            const int *__restrict__ ne, int *eb, int *ee) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    eb[b] = ull_lower_bound(ekeys, E, (unsigned long long)nb[b]);
    ee[b] = ull_lower_bound(ekeys, E, (unsigned long long)ne[b]);
}

template <class T>
static int grow(Arena &A, T **p, size_t &cap, size_t need, size_t used, cudaStream_t s) {
    if (need <= cap) return BEM_OK;
    size_t nc = std::max(need, cap * 2 + 64);
    T *np = nullptr;
    BEM_TRY(A.alloc(&np, nc));
    if (*p && used) BEM_CUDA(cudaMemcpyAsync(np, *p, sizeof(T) * used, cudaMemcpyDeviceToDevice, s));
    if (*p) {
        BEM_CUDA(cudaStreamSynchronize(s));
        A.release(*p);
    }
    *p = np;
    cap = nc;
    return BEM_OK;
}

int build_tree(bem_plan *P, cudaStream_t s) {
    Tree &t = P->t;
    Arena &A = P->arena;
    const int N = (int)P->N, E = (int)P->E, npe = P->npe;
    const int nblk = (std::max(N, E) + RS_THREADS - 1) / RS_THREADS;
    // root cube
    double *root = nullptr;
    BEM_TRY(A.alloc(&root, 8 + 6 * ROOT_BLOCKS));
    {
        const int nparts = std::max(1, std::min(ROOT_BLOCKS, (N + ROOT_T - 1) / ROOT_T));
        (k_root_part<<<nparts, ROOT_T, 0, s>>>(P->nodes, N, root + 8), ::bem::count_launch());
        (k_root<<<1, ROOT_T, 0, s>>>(root + 8, nparts, root), ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    // Morton codes, sorted
    unsigned long long *tmpk = nullptr;
    int *tmpv = nullptr;
    unsigned int *hist = nullptr;
    BEM_TRY(A.alloc(&t.codes, N));
    BEM_TRY(A.alloc(&t.node_perm, N));
    BEM_TRY(A.alloc(&tmpk, std::max(N, E)));
    BEM_TRY(A.alloc(&tmpv, std::max(N, E)));
    BEM_TRY(A.alloc(&hist, (size_t)256 * nblk + scan_scratch(256 * nblk)));
    int *sblk = nullptr;
    BEM_TRY(A.alloc(&sblk, scan_scratch(2 * N + 2)));
    (k_morton<<<(N + 255) / 256, 256, 0, s>>>(P->nodes, N, root, t.codes, t.node_perm), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    BEM_TRY(radix_sort_pairs(t.codes, t.node_perm, tmpk, tmpv, N, 3 * QBITS, hist, nblk, s));
    double hroot[8];
    BEM_CUDA(cudaMemcpyAsync(hroot, root, sizeof(double) * 5, cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    t.lo[0] = hroot[0]; t.lo[1] = hroot[1]; t.lo[2] = hroot[2];
    t.side = hroot[3];

    // boxes, level by level
    size_t cap = 0;
    int *nb = nullptr, *ne = nullptr, *ix = nullptr, *iy = nullptr, *iz = nullptr, *lev = nullptr,
        *par = nullptr, *c0 = nullptr, *nc = nullptr;
    size_t caps[9] = {0};
    auto grow_all = [&](size_t need, size_t used) -> int {
        BEM_TRY(grow(A, &nb, caps[0], need, used, s));
        BEM_TRY(grow(A, &ne, caps[1], need, used, s));
        BEM_TRY(grow(A, &ix, caps[2], need, used, s));
        BEM_TRY(grow(A, &iy, caps[3], need, used, s));
        BEM_TRY(grow(A, &iz, caps[4], need, used, s));
        BEM_TRY(grow(A, &lev, caps[5], need, used, s));
        BEM_TRY(grow(A, &par, caps[6], need, used, s));
        BEM_TRY(grow(A, &c0, caps[7], need, used, s));
        BEM_TRY(grow(A, &nc, caps[8], need, used, s));
        cap = caps[0];
        return BEM_OK;
    };
    BEM_TRY(grow_all(std::max(64, 4 * N / std::max(1, P->prm.leaf_size) + 64), 0));
    {
        int h0[1] = {0}, hN[1] = {N}, hm1[1] = {-1};
        BEM_CUDA(cudaMemcpyAsync(nb, h0, sizeof(int), cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(ne, hN, sizeof(int), cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(ix, h0, sizeof(int), cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(iy, h0, sizeof(int), cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(iz, h0, sizeof(int), cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(lev, h0, sizeof(int), cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(par, hm1, sizeof(int), cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaStreamSynchronize(s));
    }
    int *nch = nullptr, *choff = nullptr, *total = nullptr;
    size_t cap_tmp = 0;
    BEM_TRY(A.alloc(&total, 1));
    t.lev_off.assign(1, 0);
    t.lev_off.push_back(1);
    int level = 0;
    while (true) {
        int off = t.lev_off[level], cnt = t.lev_off[level + 1] - off;
        if (cnt == 0) break;
        size_t c1 = cap_tmp, c2 = cap_tmp;
        BEM_TRY(grow(A, &nch, c1, (size_t)cnt, 0, s));
        BEM_TRY(grow(A, &choff, c2, (size_t)cnt, 0, s));
        cap_tmp = std::min(c1, c2);
        (k_count_children<<<(8 * cnt + 255) / 256, 256, 0, s>>>(t.codes, nb, ne, off, cnt, level, P->prm.leaf_size,
                                                           P->prm.max_level, nch), ::bem::count_launch());
        BEM_LAUNCH_CHECK();
        BEM_TRY(scan_exclusive(nch, choff, cnt, total, sblk, s));
        int htot = 0;
        BEM_CUDA(cudaMemcpyAsync(&htot, total, sizeof(int), cudaMemcpyDeviceToHost, s));
        BEM_CUDA(cudaStreamSynchronize(s));
        int base = t.lev_off[level + 1];
        BEM_TRY(grow_all((size_t)base + htot, (size_t)base));
        (k_write_children<<<(8 * cnt + 255) / 256, 256, 0, s>>>(t.codes, off, cnt, level, nch, choff, base, nb, ne, ix,
                                                           iy, iz, lev, par, c0, nc), ::bem::count_launch());
        BEM_LAUNCH_CHECK();
        t.lev_off.push_back(base + htot);
        level++;
        if (htot == 0) break;
    }
    // the last entry repeats the previous one when the deepest level has no children
    while (t.lev_off.size() >= 2 && t.lev_off[t.lev_off.size() - 1] == t.lev_off[t.lev_off.size() - 2])
        t.lev_off.pop_back();
    t.nlev = (int)t.lev_off.size() - 1;
    t.nbox = t.lev_off.back();
    t.nb = nb; t.ne = ne; t.ix = ix; t.iy = iy; t.iz = iz; t.level = lev; t.parent = par;
    t.child0 = c0; t.nchild = nc;
    (void)cap;

    // box centres
    BEM_TRY(A.alloc(&t.cx, t.nbox));
    BEM_TRY(A.alloc(&t.cy, t.nbox));
    BEM_TRY(A.alloc(&t.cz, t.nbox));
    BEM_TRY(A.alloc(&t.r, t.nbox));
    (k_box_geometry<<<(t.nbox + 255) / 256, 256, 0, s>>>(t.nbox, lev, ix, iy, iz, root, t.cx, t.cy, t.cz), ::bem::count_launch());
    BEM_LAUNCH_CHECK();

    // vertices: leaf, Morton rank, sorted coordinates
    BEM_TRY(A.alloc(&t.leaf_of_node, N));
    BEM_TRY(A.alloc(&t.node_rank, N));
    BEM_TRY(A.alloc(&t.tx, N));
    BEM_TRY(A.alloc(&t.ty, N));
    BEM_TRY(A.alloc(&t.tz, N));
    (k_leaf_nodes<<<t.nbox, 128, 0, s>>>(t.nbox, nc, nb, ne, t.node_perm, t.leaf_of_node, t.node_rank), ::bem::count_launch());
    (k_gather_nodes<<<(N + 255) / 256, 256, 0, s>>>(N, t.node_perm, P->nodes, t.tx, t.ty, t.tz), ::bem::count_launch());
    BEM_LAUNCH_CHECK();

    // leaves in box order
    std::vector<int> hnc(t.nbox);
    BEM_CUDA(cudaMemcpyAsync(hnc.data(), nc, sizeof(int) * t.nbox, cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    std::vector<int> hleaves;
    for (int b = 0; b < t.nbox; b++)
        if (hnc[b] == 0) hleaves.push_back(b);
    t.nleaf = (int)hleaves.size();
    BEM_TRY(A.alloc(&t.leaves, t.nleaf));
    BEM_CUDA(cudaMemcpyAsync(t.leaves, hleaves.data(), sizeof(int) * t.nleaf, cudaMemcpyHostToDevice, s));

    // elements ordered by the Morton rank of their first corner
    unsigned long long *ekeys = nullptr;
    BEM_TRY(A.alloc(&ekeys, E));
    BEM_TRY(A.alloc(&t.elem_perm, E));
    (k_elem_keys<<<(E + 255) / 256, 256, 0, s>>>(E, npe, P->elems, t.node_rank, ekeys, t.elem_perm), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    int rbits = 1;
    while ((1ll << rbits) < N) rbits++;
    BEM_TRY(radix_sort_pairs(ekeys, t.elem_perm, tmpk, tmpv, E, rbits, hist, nblk, s));
    BEM_TRY(A.alloc(&t.el_phi, (size_t)E * npe));
    BEM_TRY(A.alloc(&t.el_chi, (size_t)E * npe));
    (k_elem_gather<<<(E + 255) / 256, 256, 0, s>>>(E, npe, t.elem_perm, P->elems, P->chi, t.el_phi, t.el_chi), ::bem::count_launch());
    BEM_TRY(A.alloc(&t.eb, t.nbox));
    BEM_TRY(A.alloc(&t.ee, t.nbox));
    (k_box_elems<<<(t.nbox + 255) / 256, 256, 0, s>>>(t.nbox, E, ekeys, nb, ne, t.eb, t.ee), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    BEM_CUDA(cudaStreamSynchronize(s));
    A.release(tmpk);
    A.release(tmpv);
    A.release(hist);
    A.release(sblk);
    A.release(ekeys);
    A.release(nch);
    A.release(choff);
    return BEM_OK;
}

// ---------------------------------------------------------------------------
// convergence radii (Section 3.4)
// ---------------------------------------------------------------------------
// leaf: max distance from the centre to its own vertices and to the vertices
// and regular quadrature points of the elements it owns.
__global__ void k_radius_leaf(const int *__restrict__ leaves, int nleaf, const int *__restrict__ nb,
                              const int *__restrict__ ne, const int *__restrict__ eb, const int *__restrict__ ee,
                              const double *__restrict__ cx, const double *__restrict__ cy,
                              const double *__restrict__ cz, const double *__restrict__ tx,
                              const double *__restrict__ ty, const double *__restrict__ tz,
                              const int *__restrict__ el_phi, int npe, const double *__restrict__ nodes,
                              const double *__restrict__ qx, const double *__restrict__ qy,
                              const double *__restrict__ qz, double *r) {
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= nleaf) return;
    int b = leaves[w];
    double c0 = cx[b], c1 = cy[b], c2 = cz[b], m = 0.0;
    for (int k = nb[b] + lane; k < ne[b]; k += 32) m = fmax(m, dist3_rn(c0, c1, c2, tx[k], ty[k], tz[k]));
    for (int i = eb[b] + lane; i < ee[b]; i += 32) {
        for (int a = 0; a < npe; a++) {
            const double *p = nodes + 3 * (size_t)el_phi[(size_t)i * npe + a];
            m = fmax(m, dist3_rn(c0, c1, c2, p[0], p[1], p[2]));
        }
        for (int q = 0; q < NQ; q++) {
            size_t o = (size_t)i * NQ + q;
            m = fmax(m, dist3_rn(c0, c1, c2, qx[o], qy[o], qz[o]));
        }
    }
    for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) r[b] = m;
}

// parent: r_P = max_child r_C + d_C / 2 (Eq. 12), d_C the child diagonal.
__global__ void k_radius_parent(int off, int cnt, const int *__restrict__ child0, const int *__restrict__ nchild,
                                const int *__restrict__ lev, double side, double sqrt3, double *r) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt) return;
    int b = off + j;
    if (nchild[b] == 0) return;
    double m = 0.0;
    for (int c = child0[b]; c < child0[b] + nchild[b]; c++) m = fmax(m, r[c]);
    double hc = scalbn(side, -(lev[b] + 1));
    r[b] = __dadd_rn(m, __dmul_rn(__dmul_rn(sqrt3, hc), 0.5));
}

// ---------------------------------------------------------------------------
// near-field and interaction lists (Section 3.6)
// ---------------------------------------------------------------------------
struct ListArgs {
    const int *parent, *child0, *nchild;
    const double *cx, *cy, *cz, *r;
    const int *pnear_ptr, *pnear_idx;   // lists of the previous levels
    double eta;
    int leaf_descend;
    const float4 *fbox;                 // float32 centres and radii
};

// |c_b - c_n| > eta (r_b + r_n), exactly as in float64 (the oracle's
// operation order).  A float32 estimate decides when it clears the threshold
// by more than its rounding error can move it (1e-5 of the magnitudes
// involved); the float64 test decides the rest.
__device__ __forceinline__ bool separated(const ListArgs &a, int b, int n) {
    const float4 B = a.fbox[b], Nb = a.fbox[n];
    const float dx = B.x - Nb.x, dy = B.y - Nb.y, dz = B.z - Nb.z;
    const float d2 = dx * dx + dy * dy + dz * dz;
    const float T = (float)a.eta * (B.w + Nb.w);
    const float m = 1e-5f * (T + fabsf(B.x) + fabsf(B.y) + fabsf(B.z) + fabsf(Nb.x) + fabsf(Nb.y) + fabsf(Nb.z));
    if (d2 > (T + m) * (T + m)) return true;
    if (T > m && d2 < (T - m) * (T - m)) return false;
    double d = dist3_rn(a.cx[b], a.cy[b], a.cz[b], a.cx[n], a.cy[n], a.cz[n]);
    return d > __dmul_rn(a.eta, __dadd_rn(a.r[b], a.r[n]));
}

__global__ void k_box_floats(int nbox, const double *__restrict__ cx, const double *__restrict__ cy,
                             const double *__restrict__ cz, const double *__restrict__ r, float4 *fbox) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbox) fbox[b] = make_float4((float)cx[b], (float)cy[b], (float)cz[b], (float)r[b]);
}

// Walks the parent's near list for box b; when `write`, stores the entries.
// Returns the (near, interaction) counts.  A small explicit stack opens
// non-leaf entries for a leaf b when leaf_descend is on.
__device__ int2 walk_lists(const ListArgs &a, int b, bool write, int *near_out, int *inter_out, int cap = 1 << 30) {
    int nn = 0, ni = 0;
    int p = a.parent[b];
    bool bleaf = a.nchild[b] == 0;
    int stack[8 * 24];
    for (int t = a.pnear_ptr[p]; t < a.pnear_ptr[p + 1]; t++) {
        int N = a.pnear_idx[t];
        int sp = 0;
        if (a.nchild[N] == 0) {
            stack[sp++] = N;
        } else {
            for (int c = a.child0[N] + a.nchild[N] - 1; c >= a.child0[N]; c--) stack[sp++] = c;
        }
        while (sp > 0) {
            int C = stack[--sp];
            if (separated(a, b, C)) {
                if (write && ni < cap) inter_out[ni] = C;
                ni++;
            } else if (bleaf && a.leaf_descend && a.nchild[C] != 0) {
                for (int c = a.child0[C] + a.nchild[C] - 1; c >= a.child0[C]; c--) stack[sp++] = c;
            } else {
                if (write && nn < cap) near_out[nn] = C;
                nn++;
            }
        }
    }
    return make_int2(nn, ni);
}

// One entry N of the parent's near list, walked as walk_lists does (its
// children, or N itself when a leaf; non-leaf boxes opened for a leaf b when
// leaf_descend is on); entries go to near_out / inter_out from positions
// nbase / ibase on, below cap.  Returns the counts.
__device__ int2 walk_entry(const ListArgs &a, int b, bool bleaf, int N, bool write, int *near_out, int *inter_out,
                           int nbase, int ibase, int cap) {
    int nn = 0, ni = 0;
    int stack[8 * 24];
    int sp = 0;
    if (a.nchild[N] == 0) {
        stack[sp++] = N;
    } else {
        for (int c = a.child0[N] + a.nchild[N] - 1; c >= a.child0[N]; c--) stack[sp++] = c;
    }
    while (sp > 0) {
        int C = stack[--sp];
        if (separated(a, b, C)) {
            if (write && ibase + ni < cap) inter_out[ibase + ni] = C;
            ni++;
        } else if (bleaf && a.leaf_descend && a.nchild[C] != 0) {
            for (int c = a.child0[C] + a.nchild[C] - 1; c >= a.child0[C]; c--) stack[sp++] = c;
        } else {
            if (write && nbase + nn < cap) near_out[nbase + nn] = C;
            nn++;
        }
    }
    return make_int2(nn, ni);
}

// Counts every box's entries and keeps the first `cap` of each list in
// tnear / tinter[j * cap ...]; *overflow is set when a list is longer.  One
// warp per box: lane l walks the parent's near-list entries l, l + 32, ...,
// counting first; a warp prefix sum of the counts places each lane's entries
// where the serial walk would put them, and a second walk writes them.
constexpr int LW_WARPS = 4;
__global__ void __launch_bounds__(32 * LW_WARPS) k_lists_count_w(ListArgs a, int off, int cnt, int *cnear,
                                                                 int *cinter, int *tnear, int *tinter, int cap,
                                                                 int *overflow) {
    const int lane = threadIdx.x & 31, j = blockIdx.x * LW_WARPS + (threadIdx.x >> 5);
    if (j >= cnt) return;
    const int b = off + j, p = a.parent[b];
    const bool bleaf = a.nchild[b] == 0;
    int *no = tnear + (size_t)j * cap, *io = tinter + (size_t)j * cap;
    int nn = 0, ni = 0;
    const int t1 = a.pnear_ptr[p + 1];
    for (int t0 = a.pnear_ptr[p]; t0 < t1; t0 += 32) {
        const int t = t0 + lane;
        const int N = t < t1 ? a.pnear_idx[t] : -1;
        int2 c = N >= 0 ? walk_entry(a, b, bleaf, N, false, nullptr, nullptr, 0, 0, cap) : make_int2(0, 0);
        int pn = c.x, pi = c.y;                          // inclusive prefix sums over the lanes
        for (int o = 1; o < 32; o <<= 1) {
            const int yn = __shfl_up_sync(0xffffffffu, pn, o), yi = __shfl_up_sync(0xffffffffu, pi, o);
            if (lane >= o) { pn += yn; pi += yi; }
        }
        if (N >= 0) walk_entry(a, b, bleaf, N, true, no, io, nn + pn - c.x, ni + pi - c.y, cap);
        nn += __shfl_sync(0xffffffffu, pn, 31);
        ni += __shfl_sync(0xffffffffu, pi, 31);
    }
    if (lane == 0) {
        cnear[j] = nn;
        cinter[j] = ni;
        if (nn > cap || ni > cap) atomicOr(overflow, 1);
    }
}

// the kept lists into place, with their pointers
__global__ void k_lists_copy(int off, int cnt, const int *__restrict__ onear, const int *__restrict__ ointer,
                             const int *__restrict__ cnear, const int *__restrict__ cinter, const int *__restrict__ tnear,
                             const int *__restrict__ tinter, int cap, int near_base, int inter_base, int *near_ptr,
                             int *near_idx, int *inter_ptr, int *inter_idx) {
    const int j = blockIdx.x;
    if (threadIdx.x == 0) {
        near_ptr[off + j] = near_base + onear[j];
        inter_ptr[off + j] = inter_base + ointer[j];
    }
    for (int i = threadIdx.x; i < cnear[j]; i += blockDim.x)
        near_idx[near_base + onear[j] + i] = tnear[(size_t)j * cap + i];
    for (int i = threadIdx.x; i < cinter[j]; i += blockDim.x)
        inter_idx[inter_base + ointer[j] + i] = tinter[(size_t)j * cap + i];
}

__global__ void k_lists_write(ListArgs a, int off, int cnt, const int *__restrict__ onear, const int *__restrict__ ointer,
                              int near_base, int inter_base, int *near_ptr, int *near_idx, int *inter_ptr,
                              int *inter_idx) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt) return;
    int b = off + j;
    near_ptr[b] = near_base + onear[j];
    inter_ptr[b] = inter_base + ointer[j];
    walk_lists(a, b, true, near_idx + near_base + onear[j], inter_idx + inter_base + ointer[j]);
}

__global__ void k_set_root_lists(int *near_ptr, int *near_idx, int *inter_ptr) {
    near_ptr[0] = 0;
    near_idx[0] = 0;
    inter_ptr[0] = 0;
}

__global__ void k_close_ptr(int *ptr, int at, int value) { ptr[at] = value; }

int build_radii_lists(bem_plan *P, cudaStream_t s) {
    Tree &t = P->t;
    Arena &A = P->arena;
    const int npe = P->npe;
    // radii
    (k_radius_leaf<<<(t.nleaf * 32 + 255) / 256, 256, 0, s>>>(t.leaves, t.nleaf, t.nb, t.ne, t.eb, t.ee, t.cx, t.cy,
                                                              t.cz, t.tx, t.ty, t.tz, t.el_phi, npe, P->nodes,
                                                              P->q.x, P->q.y, P->q.z, t.r), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    const double sqrt3 = std::sqrt(3.0);
    for (int l = t.nlev - 2; l >= 0; l--) {
        int off = t.lev_off[l], cnt = t.lev_off[l + 1] - off;
        (k_radius_parent<<<(cnt + 255) / 256, 256, 0, s>>>(off, cnt, t.child0, t.nchild, t.level, t.side, sqrt3, t.r), ::bem::count_launch());
        BEM_LAUNCH_CHECK();
    }
    BEM_TRY(A.alloc(&t.fbox, t.nbox));
    (k_box_floats<<<(t.nbox + 255) / 256, 256, 0, s>>>(t.nbox, t.cx, t.cy, t.cz, t.r, t.fbox), ::bem::count_launch());
    // lists, level by level; level-l lists only read level < l lists
    BEM_TRY(A.alloc(&t.near_ptr, t.nbox + 1));
    BEM_TRY(A.alloc(&t.inter_ptr, t.nbox + 1));
    size_t capn = 1024, capi = 1024;
    int *near_idx = nullptr, *inter_idx = nullptr;
    BEM_TRY(A.alloc(&near_idx, capn));
    BEM_TRY(A.alloc(&inter_idx, capi));
    (k_set_root_lists<<<1, 1, 0, s>>>(t.near_ptr, near_idx, t.inter_ptr), ::bem::count_launch());
    int nnear = 1, ninter = 0;
    int *cn = nullptr, *ci = nullptr, *on = nullptr, *oi = nullptr, *tot = nullptr;
    int maxcnt = 1;
    for (int l = 1; l < t.nlev; l++) maxcnt = std::max(maxcnt, t.lev_off[l + 1] - t.lev_off[l]);
    BEM_TRY(A.alloc(&cn, maxcnt));
    BEM_TRY(A.alloc(&ci, maxcnt));
    BEM_TRY(A.alloc(&on, maxcnt));
    BEM_TRY(A.alloc(&oi, maxcnt));
    BEM_TRY(A.alloc(&tot, 3));
    int *sblk = nullptr;
    BEM_TRY(A.alloc(&sblk, scan_scratch(maxcnt)));
    // one walk per level: up to LIST_CAP entries of each list are kept by the
    // counting walk and copied into place; a longer list makes the level walk again
    constexpr int LIST_CAP = 1024;
    int *tn = nullptr, *ti = nullptr;
    BEM_TRY(A.alloc(&tn, (size_t)maxcnt * LIST_CAP));
    BEM_TRY(A.alloc(&ti, (size_t)maxcnt * LIST_CAP));
    for (int l = 1; l < t.nlev; l++) {
        int off = t.lev_off[l], cnt = t.lev_off[l + 1] - off;
        ListArgs a{t.parent, t.child0, t.nchild, t.cx, t.cy, t.cz, t.r, t.near_ptr, near_idx, P->prm.eta,
                   P->prm.leaf_descend, t.fbox};
        // level l-1 pointers must be closed for the walk: ptr[off] = running total
        (k_close_ptr<<<1, 1, 0, s>>>(t.near_ptr, off, nnear), ::bem::count_launch());
        (k_close_ptr<<<1, 1, 0, s>>>(t.inter_ptr, off, ninter), ::bem::count_launch());
        BEM_CUDA(cudaMemsetAsync(tot + 2, 0, sizeof(int), s));
        (k_lists_count_w<<<(cnt + LW_WARPS - 1) / LW_WARPS, 32 * LW_WARPS, 0, s>>>(a, off, cnt, cn, ci, tn, ti,
                                                                                 LIST_CAP, tot + 2),
         ::bem::count_launch());
        BEM_LAUNCH_CHECK();
        BEM_TRY(scan_exclusive(cn, on, cnt, tot, sblk, s));
        BEM_TRY(scan_exclusive(ci, oi, cnt, tot + 1, sblk, s));
        int h[3];
        BEM_CUDA(cudaMemcpyAsync(h, tot, sizeof(int) * 3, cudaMemcpyDeviceToHost, s));
        BEM_CUDA(cudaStreamSynchronize(s));
        BEM_TRY(grow(A, &near_idx, capn, (size_t)nnear + h[0], (size_t)nnear, s));
        BEM_TRY(grow(A, &inter_idx, capi, (size_t)ninter + h[1], (size_t)ninter, s));
        a.pnear_idx = near_idx;
        if (h[2])
            (k_lists_write<<<(cnt + 127) / 128, 128, 0, s>>>(a, off, cnt, on, oi, nnear, ninter, t.near_ptr, near_idx,
                                                            t.inter_ptr, inter_idx), ::bem::count_launch());
        else
            (k_lists_copy<<<cnt, 64, 0, s>>>(off, cnt, on, oi, cn, ci, tn, ti, LIST_CAP, nnear, ninter, t.near_ptr,
                                             near_idx, t.inter_ptr, inter_idx), ::bem::count_launch());
        BEM_LAUNCH_CHECK();
        nnear += h[0];
        ninter += h[1];
    }
    (k_close_ptr<<<1, 1, 0, s>>>(t.near_ptr, t.nbox, nnear), ::bem::count_launch());
    (k_close_ptr<<<1, 1, 0, s>>>(t.inter_ptr, t.nbox, ninter), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    t.near_idx = near_idx;
    t.inter_idx = inter_idx;
    t.n_near = nnear;
    t.n_inter = ninter;
    BEM_CUDA(cudaStreamSynchronize(s));
    A.release(cn);
    A.release(ci);
    A.release(on);
    A.release(oi);
    A.release(sblk);
    A.release(tn);
    A.release(ti);
    return BEM_OK;
}

}  // namespace bem
