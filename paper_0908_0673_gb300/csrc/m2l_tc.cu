// M2L (Eq. 7) of the mixed-precision Laplace product on the tensor cores.
//
// Symmetry reduction.  The Laplace kernel is radial, so for a signed axis
// permutation Q (r_i = s_i rhat_pi(i)) the derivatives obey
//     D_mu(r) = sign_s(mu) D_{mu o pi^-1}(rhat),   sign_s(mu) = prod_i s_i^mu_i,
// and the factorial / sign / level-scale factors of the contraction depend on
// |alpha| and alpha! only.  Every interaction pair therefore maps to a
// canonical offset rhat (|components| sorted in decreasing order) and one of
// 48 symmetries: with Mhat_ahat = sign(a) M_a (a = ahat o pi) the canonical
// contraction Lhat = T(rhat) Mhat gives L_b = sign(b) Lhat_{b o pi^-1}.  The
// offset classes of a box tree collapse from thousands to a few hundred, each
// shared by hundreds to thousands of pairs.
//
// Contraction.  For a tile of up to 128 pairs of one canonical class the
// product is a dense GEMM  D[pair][b] = sum_a Mom[pair][a] T[b][a]  with
// T[b][a] = Dhat[a + b] / b! (zero where |a| + |b| > p), issued as tcgen05
// kind::tf32 MMAs: M = 128 pairs (TMEM lanes), N = rows b in degree bands
// whose K extent (the largest number of columns a any row of the band needs)
// shrinks with the degree, so most of the zero triangle is skipped.  Each
// float32 operand is split into tf32 hi + lo and the product accumulated as
// hi*hi + hi*lo + lo*hi in float32 (about 2^-21 relative per product).  The
// moments are gathered, sign-permuted and scaled into shared memory in K
// chunks of 32 (double-buffered against the MMAs); the class matrix is built
// in shared memory once per run of tiles of one class.  Each pair's row of
// Lhat is written out; a gather kernel sums every target's rows in list
// order, undoing the permutation: deterministic, no atomics.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bem_internal.cuh"
#include "tc_ptx.cuh"

namespace bem {

namespace {

constexpr int TC_T = 512;           // threads per block (16 warps)
constexpr int TC_M = 128;           // pairs per tile (MMA M, TMEM lanes)
constexpr int TC_KC = 32;           // K chunk of the moment operand
constexpr int TC_MOM_BYTES = TC_M * TC_KC * 4;   // one tf32 plane of a chunk
constexpr int TC_PAD = 1024;        // slack after the last operand
constexpr int TC_MAXE = 192;        // MMA schedule entries
constexpr long long TC_WAIT = 4000000000ll;      // clock cycles before a wait gives up
constexpr int TC_SMEM_MAX = 220 * 1024;

// the six axis permutations; PERMS[q][i] = canonical position of axis i
constexpr int PERMS[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

struct TcArgs {
    TcGroups g;
    int np, ntile, nkc, nsched;
    const int *tile_cls, *tile_start, *tile_cnt;
    const int *src, *sig, *pair;
    const int *dl, *tidx;
    const unsigned short *fwd;
    const float *tfac, *fD, *M;
    const uint4 *sched;                 // MMA schedule: {T offset, sbo, idesc, dcol | ks << 16 | acc << 31}
    const int *sched_ptr;               // [nkc + 1] schedule entries of each chunk
    float *Lp;                          // rows of this run's pairs, row u - u0
    int ldp, u0;
    int *err;
    const int *skip;
};

struct SchedEntry {                     // one tf32 MMA triple, descriptors resolved in shared memory
    uint64_t bh, bl;
    uint32_t idesc, meta;
};

__device__ __forceinline__ uint32_t mom_off(int r, int k) {   // byte offset in a chunk plane
    return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// shared-memory layout of the tensor-core M2L block
struct TcLayout {
    size_t mom, fwd, d, sched, bars, total;
};
__host__ __device__ inline TcLayout tc_layout(const TcGroups &g, int ldp) {
    TcLayout L;
    L.mom = ((2 * (size_t)g.tsize * 4 + 1023) / 1024) * 1024;
    L.fwd = L.mom + 4 * (size_t)TC_MOM_BYTES;
    L.d = L.fwd + ((48 * (size_t)ldp * 2 + 15) / 16) * 16;
    L.sched = L.d + (size_t)ldp * 4;
    L.bars = L.sched + (size_t)TC_MAXE * sizeof(SchedEntry);
    L.total = L.bars + 8 * 8 + 16 + TC_PAD;
    return L;
}

// bounded wait that also gives up as soon as another role has given up
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > TC_WAIT) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// Roles: warp 0 lane 0 issues the MMAs; warps 0-3 read the accumulator back
// (warp w owns TMEM lanes 32 w .. 32 w + 31, i.e. pairs); warps 4-15 gather
// the moments into the two chunk buffers and rebuild the class matrix when
// the class changes.  Handshakes: full[b] (12 producer warps) -> MMA;
// empty[b] (MMA commit) -> producers; tfull (commit after a tile's last
// chunk) -> epilogue and producers; tempty (4 epilogue warps) -> MMA.
__global__ void __launch_bounds__(TC_T, 1) k_m2l_tc(const __grid_constant__ TcArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcGroups &G = a.g;
    const TcLayout LY = tc_layout(G, a.ldp);
    const int np = a.np, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *sTh = (float *)smem, *sTl = sTh + G.tsize;                 // class matrix, tf32 hi / lo
    unsigned char *sMom = smem + LY.mom;                                // [2 buffers][hi, lo] chunk planes
    unsigned short *sFwd = (unsigned short *)(smem + LY.fwd);          // [48][ldp] signed index maps
    SchedEntry *sSched = (SchedEntry *)(smem + LY.sched);
    uint64_t *full = (uint64_t *)(smem + LY.bars), *empty = full + 2, *tfull = full + 4, *tempty = full + 5,
             *fin = full + 6;
    uint32_t *sTmem = (uint32_t *)(full + 8);
    volatile int *sAbort = (volatile int *)(sTmem + 1);

    if (tid == 0) {
        tc::mbar_init(&full[0], 12);
        tc::mbar_init(&full[1], 12);
        tc::mbar_init(&empty[0], 1);
        tc::mbar_init(&empty[1], 1);
        tc::mbar_init(tfull, 1);
        tc::mbar_init(tempty, 4);
        tc::mbar_init(fin, 1);
        *sAbort = 0;
        tc::mbar_fence_init();
    }
    for (int i = tid; i < 48 * a.ldp; i += TC_T) {
        const int sg = i / a.ldp, h = i - sg * a.ldp;
        sFwd[i] = h < np ? a.fwd[(size_t)sg * np + h] : 0;
    }
    if (warp == 0) tc::tmem_alloc(sTmem, 512);
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *sTmem;
    {   // schedule with resolved descriptors (class matrix addresses are fixed)
        const uint32_t th = tc::smem_u32(sTh), tl = tc::smem_u32(sTl);
        for (int i = tid; i < a.nsched; i += TC_T) {
            const uint4 e = a.sched[i];
            sSched[i].bh = tc::smem_desc(th + e.x, 128, e.y);
            sSched[i].bl = tc::smem_desc(tl + e.x, 128, e.y);
            sSched[i].idesc = e.z;
            sSched[i].meta = e.w;
        }
    }
    __syncthreads();

    const int t_begin = (int)((long long)a.ntile * blockIdx.x / gridDim.x);
    const int t_end = (int)((long long)a.ntile * (blockIdx.x + 1) / gridDim.x);

    if (warp < 4) {
        // ---- MMA issue (warp 0 lane 0) and accumulator read-back (warps 0-3) ----
        int it = 0;                                       // running chunk counter
        for (int tile = t_begin; tile < t_end; tile++) {
            const int k = tile - t_begin;
            if (warp == 0) {
                bool ok = true;
                if (lane == 0) {
                    if (k > 0) ok = wait_or_abort(tempty, (uint32_t)((k - 1) & 1), sAbort);
                    tc::tc_fence_after_sync();
                    const uint32_t mb = tc::smem_u32(sMom);
                    for (int kc = 0; kc < a.nkc && ok; kc++, it++) {
                        const int b = it & 1;
                        ok = wait_or_abort(&full[b], (uint32_t)((it >> 1) & 1), sAbort);
                        if (!ok) break;
                        tc::tc_fence_after_sync();
                        const uint64_t ah0 = tc::smem_desc(mb + (uint32_t)b * 2 * TC_MOM_BYTES, 128, 1024);
                        const uint64_t al0 = tc::smem_desc(mb + (uint32_t)b * 2 * TC_MOM_BYTES + TC_MOM_BYTES, 128, 1024);
                        for (int e = a.sched_ptr[kc]; e < a.sched_ptr[kc + 1]; e++) {
                            const SchedEntry &S = sSched[e];
                            const uint32_t d = tmem + (S.meta & 0xffffu);
                            const uint64_t ks16 = (uint64_t)((S.meta >> 16) & 3u) * 16u;   // 256 B steps
                            const bool acc = (S.meta >> 31) != 0;
                            tc::mma_tf32(d, ah0 + ks16, S.bh, S.idesc, acc);
                            tc::mma_tf32(d, ah0 + ks16, S.bl, S.idesc, true);
                            tc::mma_tf32(d, al0 + ks16, S.bh, S.idesc, true);
                        }
                        tc::mma_commit(&empty[b]);
                    }
                    if (ok) tc::mma_commit(tfull);
                }
                __syncwarp();
            }
            // read-back of this tile's accumulator
            bool ok = wait_or_abort(tfull, (uint32_t)(k & 1), sAbort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc::tc_fence_after_sync();
            const int r = 32 * warp + lane;
            const int cnt = a.tile_cnt[tile];
            const int u = r < cnt ? a.pair[a.tile_start[tile] + r] : -1;
            const int nch = G.ncols / 32;
            for (int c = 0; c < nch; c++) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * c), v);
                if (u >= 0) {
                    float4 *dst = (float4 *)(a.Lp + (size_t)(u - a.u0) * a.ldp + 32 * c);
#pragma unroll
                    for (int i = 0; i < 8; i++) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
            }
            tc::tc_fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty);
            if (__any_sync(0xffffffffu, *sAbort != 0)) break;
        }
    } else {
        // ---- producers: warps 4-15 ----
        const int pt = tid - 128;                         // 0 .. 383
        constexpr int NE = (TC_M * TC_KC + 383) / 384;    // elements per thread per chunk (11)
        int it = 0, prev_cls = -1;
        for (int tile = t_begin; tile < t_end; tile++) {
            const int k = tile - t_begin;
            const int cls = a.tile_cls[tile], st = a.tile_start[tile], cnt = a.tile_cnt[tile];
            // this thread's elements: e = pt + 384 i -> row r = 8 rg + lane / 4, column 4 kq + lane % 4
            int srow[NE], sgo[NE], col[NE];
#pragma unroll
            for (int i = 0; i < NE; i++) {
                const int e = pt + 384 * i, gi = e >> 5;
                const int r = (gi >> 3) * 8 + (lane >> 2);
                col[i] = (gi & 7) * 4 + (lane & 3);
                const bool v = e < TC_M * TC_KC && r < cnt;
                srow[i] = v ? a.src[st + r] : -1;
                sgo[i] = v ? a.sig[st + r] * a.ldp : 0;
            }
            if (cls != prev_cls) {
                // the class matrix may only change once the previous tile's MMAs
                // are done: T[b][a] = Dhat[a+b] (-1)^|a| 2^(dl |a|) / (a! b!)
                if (k > 0 && !__all_sync(0xffffffffu, wait_or_abort(tfull, (uint32_t)((k - 1) & 1), sAbort))) break;
                const int dl = a.dl[cls];
                const float *Dc = a.fD + (size_t)cls * np;
                for (int e0 = pt; e0 < G.tsize; e0 += 4 * 384) {
                    int gi[4];
                    float fc[4], dv[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int e = e0 + q * 384;
                        gi[q] = e < G.tsize ? __ldg(a.tidx + e) : -1;
                        fc[q] = e < G.tsize ? __ldg(a.tfac + e) : 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < 4; q++) dv[q] = gi[q] >= 0 ? __ldg(Dc + (gi[q] & 0xffff)) : 0.f;
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int e = e0 + q * 384;
                        if (e < G.tsize) {
                            const float v = gi[q] >= 0 ? ldexpf(dv[q] * fc[q], dl * (gi[q] >> 16)) : 0.f;
                            const float hi = tc::to_tf32(v);
                            sTh[e] = hi;
                            sTl[e] = tc::to_tf32(v - hi);
                        }
                    }
                }
                prev_cls = cls;
            }
            float raw[NE];
            auto fetch = [&](int kc) {
#pragma unroll
                for (int i = 0; i < NE; i++) {
                    const int al = kc * TC_KC + col[i];
                    float x = 0.f;
                    if (srow[i] >= 0 && al < np) {
                        const unsigned f = sFwd[sgo[i] + al];
                        x = __int_as_float(__float_as_int(__ldg(a.M + (size_t)srow[i] * np + (f & 0x7fffu))) ^
                                           (int)((f & 0x8000u) << 16));
                    }
                    raw[i] = x;
                }
            };
            fetch(0);
            bool ok = true;
            for (int kc = 0; kc < a.nkc; kc++, it++) {
                const int b = it & 1, n = it >> 1;
                if (n > 0) {
                    ok = __all_sync(0xffffffffu, wait_or_abort(&empty[b], (uint32_t)((n - 1) & 1), sAbort));
                    if (!ok) break;
                }
                unsigned char *hi = sMom + (size_t)b * 2 * TC_MOM_BYTES, *lo = hi + TC_MOM_BYTES;
#pragma unroll
                for (int i = 0; i < NE; i++) {
                    const int e = pt + 384 * i;
                    if (e < TC_M * TC_KC) {
                        const int gi = e >> 5, r = (gi >> 3) * 8 + (lane >> 2);
                        const uint32_t o = mom_off(r, col[i]);
                        const float h = tc::to_tf32(raw[i]);
                        *(float *)(hi + o) = h;
                        *(float *)(lo + o) = tc::to_tf32(raw[i] - h);
                    }
                }
                if (kc + 1 < a.nkc) fetch(kc + 1);       // in flight while the chunk is consumed
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[b]);
            }
            if (!ok) break;
        }
    }
    // every MMA issued has completed before the accumulator is released
    __syncthreads();
    if (tid == 0) {
        tc::mma_commit(fin);
        if (!tc::mbar_wait_bounded(fin, 0, TC_WAIT)) *sAbort = 1;
        if (*sAbort) atomicExch(a.err, 1);
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// L_t[b] = (1 / h_t) sum over t's interaction list, in list order, of
// sign * Lhat_u[b o pi_u^-1]; one thread per row b, eight rows of Lhat in flight
constexpr int GA_LIST = 512;            // list entries staged per pass
__global__ void __launch_bounds__(512) k_m2l_gather_sym(int t0, int nbox, const int *__restrict__ level, double side,
                                                        const int *__restrict__ inter_ptr, int u0r, int np, int ldp,
                                                        const int *__restrict__ sig_u, const int *__restrict__ inv,
                                                        const float *__restrict__ Lp, float *__restrict__ L,
                                                        const int *__restrict__ skip) {
    if (skip && *skip) return;
    __shared__ int sOff[GA_LIST];          // sig * np of every staged pair
    const int t = t0 + blockIdx.x, b = threadIdx.x;
    if (t >= nbox) return;
    const float sc = (float)(1.0 / scalbn(side, -level[t]));
    const int u0 = inter_ptr[t], u1 = inter_ptr[t + 1];
    float sum = 0.f;
    for (int base = u0; base < u1; base += GA_LIST) {
        const int n = min(GA_LIST, u1 - base);
        __syncthreads();
        for (int i = b; i < n; i += blockDim.x) sOff[i] = sig_u[base + i] * np;
        __syncthreads();
        if (b < np) {
            int i = 0;
            for (; i + 8 <= n; i += 8) {
                int f[8];
                float v[8];
#pragma unroll
                for (int q = 0; q < 8; q++) f[q] = __ldg(inv + sOff[i + q] + b);
#pragma unroll
                for (int q = 0; q < 8; q++) v[q] = Lp[(size_t)(base + i + q - u0r) * ldp + (f[q] & 0x7fffffff)];
#pragma unroll
                for (int q = 0; q < 8; q++) sum += f[q] < 0 ? -v[q] : v[q];
            }
            for (; i < n; i++) {
                const int f = __ldg(inv + sOff[i] + b);
                const float v = Lp[(size_t)(base + i - u0r) * ldp + (f & 0x7fffffff)];
                sum += f < 0 ? -v : v;
            }
        }
    }
    if (b < np) L[(size_t)t * np + b] = sum * sc;
}

}  // namespace

// ---------------------------------------------------------------------------
// host: canonical classes of the interaction pairs (order independent), from
// the exact offset classes (integer offset vector, level difference)
// ---------------------------------------------------------------------------
int build_m2l_sym(bem_plan *P, const std::vector<int> &pair_cls, const std::vector<long long> &kvec,
                  const std::vector<int> &dls, const std::vector<int> &levs, const std::vector<int> &src,
                  const std::vector<int> &ip) {
    const int64_t npair = P->t.n_inter;
    const int nfull = (int)dls.size();
    // every exact offset class maps to one canonical class and one symmetry
    // key: level difference, target level (Helmholtz: the derivatives depend
    // on k h_t; zero for Laplace), sorted absolute offset components
    struct Key {
        long long v[5];
        bool operator<(const Key &o) const {
            for (int i = 0; i < 5; i++)
                if (v[i] != o.v[i]) return v[i] < o.v[i];
            return false;
        }
    };
    std::vector<Key> fkey(nfull);
    std::vector<int> fsig(nfull);
    for (int c = 0; c < nfull; c++) {
        const long long *K = &kvec[3 * (size_t)c];
        int order[3] = {0, 1, 2};
        std::stable_sort(order, order + 3, [&](int x, int y) { return std::llabs(K[x]) > std::llabs(K[y]); });
        int pi[3];
        for (int j = 0; j < 3; j++) pi[order[j]] = j;
        int q = 0;
        while (!(PERMS[q][0] == pi[0] && PERMS[q][1] == pi[1] && PERMS[q][2] == pi[2])) q++;
        fsig[c] = q * 8 + ((K[0] < 0 ? 1 : 0) | (K[1] < 0 ? 2 : 0) | (K[2] < 0 ? 4 : 0));
        fkey[c] = Key{{(long long)dls[c], (long long)levs[c], std::llabs(K[order[0]]), std::llabs(K[order[1]]),
                       std::llabs(K[order[2]])}};
    }
    std::vector<int> fidx(nfull);
    for (int c = 0; c < nfull; c++) fidx[c] = c;
    std::sort(fidx.begin(), fidx.end(), [&](int x, int y) { return fkey[x] < fkey[y] || (!(fkey[y] < fkey[x]) && x < y); });
    std::vector<int> fcan(nfull), dlc;
    std::vector<double> rho, khc;
    P->sy_hlev.clear();
    const bool helm = P->green == BEM_HELMHOLTZ;
    int nc = 0;
    for (int i = 0; i < nfull; i++) {
        const Key &k = fkey[fidx[i]];
        if (i == 0 || fkey[fidx[i - 1]] < k) {
            const int dl = (int)k.v[0], e = std::max(0, -dl);
            const double sc = std::ldexp(1.0, -(e + 1));
            rho.push_back(k.v[2] * sc);
            rho.push_back(k.v[3] * sc);
            rho.push_back(k.v[4] * sc);
            khc.push_back(helm ? P->k * std::ldexp(P->t.side, -(int)k.v[1]) : 0.0);
            dlc.push_back(dl);
            P->sy_hlev.push_back((int)k.v[1]);
            nc++;
        }
        fcan[fidx[i]] = nc - 1;
    }
    // per pair (list order): canonical class, symmetry, source box; the tiles
    // are cut per order (build_sym_tables), when the row size is known
    P->sy_hcls.assign(npair, 0);
    P->sy_hsig.assign(npair, 0);
    P->sy_hsrc.assign(src.begin(), src.begin() + npair);
    P->sy_hip = ip;
    for (int64_t u = 0; u < npair; u++) {
        P->sy_hcls[u] = fcan[pair_cls[u]];
        P->sy_hsig[u] = fsig[pair_cls[u]];
    }
    P->sy_ncls = nc;
    Arena &A = P->arena;
    auto up = [&](auto **d, const auto &h) -> int {
        using T = std::decay_t<decltype(h[0])>;
        BEM_TRY(A.alloc((T **)d, std::max<size_t>(1, h.size())));
        if (!h.empty()) BEM_CUDA(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
        return BEM_OK;
    };
    BEM_TRY(up(&P->sy_rho, rho));
    BEM_TRY(up(&P->sy_kh, khc));
    BEM_TRY(up(&P->sy_dl, dlc));
    P->sy_hdl = dlc;
    BEM_TRY(up(&P->sy_sig_u, P->sy_hsig));
    return BEM_OK;
}

// Batches and tiles for rows of row_bytes: the targets are cut into runs whose
// interaction lists hold at most SY_LP_BYTES of rows together (a run holds at
// least one whole list), and within a run the pairs are sorted by canonical
// class (counting sort, stable in list order) and cut into tiles of up to
// 128 pairs of one class.  Each run's rows are computed into the same buffer
// and gathered before the next run starts, so the buffer is bounded however
// large the mesh, and every target's sum keeps its list order.
constexpr size_t SY_LP_BYTES = (size_t)128 << 20;

static int build_sym_tiles(bem_plan *P, size_t row_bytes, int64_t &max_rows) {
    const int nbox = P->t.nbox, nc = P->sy_ncls;
    const std::vector<int> &ip = P->sy_hip;
    const int64_t npair = P->t.n_inter;
    int64_t longest = 0;
    for (int b = 0; b < nbox; b++) longest = std::max<int64_t>(longest, ip[b + 1] - ip[b]);
    const int64_t cap = std::max<int64_t>(std::max<int64_t>(1, longest), (int64_t)(SY_LP_BYTES / row_bytes));
    std::vector<int> psrc(std::max<int64_t>(1, npair)), psig(std::max<int64_t>(1, npair)),
        pu(std::max<int64_t>(1, npair)), tcls, tst, tcnt, cnt(nc + 1);
    P->sy_bt.assign(1, 0);
    P->sy_bb.assign(1, 0);
    P->sy_bu.assign(1, 0);
    max_rows = 0;
    for (int t0 = 0; t0 < nbox;) {
        int t1 = t0 + 1;
        while (t1 < nbox && ip[t1 + 1] - ip[t0] <= cap) t1++;
        const int u0 = ip[t0], u1 = ip[t1];
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int u = u0; u < u1; u++) cnt[P->sy_hcls[u] + 1]++;
        for (int c = 0; c < nc; c++) cnt[c + 1] += cnt[c];
        for (int c = 0; c < nc; c++)
            for (int k = cnt[c]; k < cnt[c + 1]; k += TC_M) {
                tcls.push_back(c);
                tst.push_back(u0 + k);
                tcnt.push_back(std::min(TC_M, cnt[c + 1] - k));
            }
        for (int u = u0; u < u1; u++) {
            const int i = u0 + cnt[P->sy_hcls[u]]++;
            psrc[i] = P->sy_hsrc[u];
            psig[i] = P->sy_hsig[u];
            pu[i] = u;
        }
        P->sy_bt.push_back((int)tcls.size());
        P->sy_bb.push_back(t1);
        P->sy_bu.push_back(u1);
        max_rows = std::max<int64_t>(max_rows, u1 - u0);
        t0 = t1;
    }
    P->sy_ntile = (int)tcls.size();
    Arena &A = P->arena;
    auto up = [&](auto **d, const auto &h) -> int {
        using T = std::decay_t<decltype(h[0])>;
        BEM_TRY(A.alloc((T **)d, std::max<size_t>(1, h.size())));
        if (!h.empty()) BEM_CUDA(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
        return BEM_OK;
    };
    BEM_TRY(up(&P->sy_tile_cls, tcls));
    BEM_TRY(up(&P->sy_tile_start, tst));
    BEM_TRY(up(&P->sy_tile_cnt, tcnt));
    BEM_TRY(up(&P->sy_src, psrc));
    BEM_TRY(up(&P->sy_sig, psig));
    BEM_TRY(up(&P->sy_pair, pu));
    return BEM_OK;
}

// ---------------------------------------------------------------------------
// host: order-dependent tables (symmetry maps, class-matrix layout, derivative
// tables of the canonical classes); decides whether the tensor-core form runs
// ---------------------------------------------------------------------------
size_t tc_smem_bytes(const TcGroups &g, int ldp) { return tc_layout(g, ldp).total; }

// The TC tables of the current order, when the tensor-core form applies:
// degree bands of the class matrix, its gather table in shared-memory layout
// order, the MMA schedule.  Returns false (nothing allocated) when the order
// does not fit the fixed band table, the schedule or shared memory.
static bool tc_plan(const MIndex &mi, const std::vector<int> &deg, TcGroups &g, int &ldp, int &nkc,
                    std::vector<uint4> &sched, std::vector<int> &sptr) {
    const int p = mi.p, np = mi.np;
    // degree bands of rows b: K extent = columns a with |a| <= p - |b|, i.e.
    // the count of multi-indices of degree <= p - |b|
    auto cum = [](int d) { return d <= 0 ? 0 : d * (d + 1) * (d + 2) / 6; };
    g = TcGroups{};
    const int ncols = (np + 15) / 16 * 16;
    std::vector<int> bk;
    for (int b0 = 0; b0 < ncols; b0 += 16) {
        int K = 8;
        for (int b = b0; b < b0 + 16 && b < np; b++) K = std::max(K, cum(p - deg[b] + 1));
        bk.push_back((K + 7) / 8 * 8);
    }
    g.ng = 0;
    for (size_t i = 0; i < bk.size();) {
        size_t j = i;
        while (j < bk.size() && bk[j] == bk[i] && (int)(j - i + 1) * 16 <= 256) j++;
        if (g.ng >= TC_MAXG) return false;        // does not fit the fixed group table
        g.b0[g.ng] = (int)i * 16;
        g.n[g.ng] = (int)(j - i) * 16;
        g.k[g.ng] = bk[i];
        g.ng++;
        i = j;
    }
    g.tsize = 0;
    for (int q = 0; q < g.ng; q++) {
        g.off[q] = g.tsize;
        g.tsize += g.n[q] * g.k[q];
    }
    ldp = (ncols + 31) / 32 * 32;                 // TMEM columns read back, 32 at a time
    g.ncols = ldp;
    const int kmax = (g.k[0] + TC_KC - 1) / TC_KC * TC_KC;
    nkc = kmax / TC_KC;
    // MMA schedule: per chunk, every band whose K extent reaches into it,
    // 8 columns (one tf32 MMA) at a time
    sched.clear();
    sptr.assign(nkc + 1, 0);
    for (int kc = 0; kc < nkc; kc++) {
        sptr[kc] = (int)sched.size();
        for (int q = 0; q < g.ng; q++) {
            const int kext = g.k[q] - kc * TC_KC;
            for (int ks = 0; ks < std::min(4, kext / 8); ks++) {
                const int j = kc * 4 + ks;
                sched.push_back(make_uint4((unsigned)(g.off[q] * 4 + j * 256), (unsigned)(g.k[q] / 4 * 128),
                                           tc::idesc_tf32(TC_M, g.n[q]),
                                           (unsigned)g.b0[q] | ((unsigned)ks << 16) | (j > 0 ? 0x80000000u : 0u)));
            }
        }
    }
    sptr[nkc] = (int)sched.size();
    if ((int)sched.size() > TC_MAXE) return false;
    return tc_smem_bytes(g, ldp) <= (size_t)TC_SMEM_MAX && ldp <= 512;
}

// Order-dependent tables of the M2L on canonical classes: symmetry maps,
// exponent and factorial tables, derivative tables of the canonical classes,
// the per-pair row buffer, and the tensor-core tables when that form applies
// (mixed-precision Laplace at an order whose tables fit); else the SIMT form runs.
int build_sym_tables(bem_plan *P, cudaStream_t s) {
    P->sy_tc = 0;
    P->sy_ready = 0;
    const MIndex &mi = P->mi;
    const int p = mi.p, np = mi.np, P1 = p + 1;
    const int C = P->green == BEM_HELMHOLTZ ? 2 : 1;
    const bool mx = P->prm.precision == BEM_MIXED;
    auto idx = [&](int m, int n, int k) { return mi.idx3[((size_t)m * P1 + n) * P1 + k]; };
    std::vector<int> deg(np), mexp(np);
    std::vector<double> fact(2 * PMAX + 2), invf(np);
    fact[0] = 1.0;
    for (int i = 1; i < (int)fact.size(); i++) fact[i] = fact[i - 1] * i;
    for (int a = 0; a < np; a++) {
        deg[a] = mi.m[a] + mi.n[a] + mi.k[a];
        mexp[a] = mi.m[a] | (mi.n[a] << 8) | (mi.k[a] << 16) | (deg[a] << 24);
        invf[a] = 1.0 / (fact[mi.m[a]] * fact[mi.n[a]] * fact[mi.k[a]]);
    }
    // symmetry maps: fwd[sig][ahat] = a = ahat o pi (with sign_s(a)),
    // inv[sig][b] = bhat = b o pi^-1 (with sign_s(b)); sign in bit 15 / 31
    std::vector<unsigned short> fwd(48 * (size_t)np);
    std::vector<int> inv(48 * (size_t)np);
    for (int q = 0; q < 6; q++)
        for (int sb = 0; sb < 8; sb++) {
            const int sig = q * 8 + sb;
            const int *pi = PERMS[q];
            int pinv[3];
            for (int i = 0; i < 3; i++) pinv[pi[i]] = i;
            for (int h = 0; h < np; h++) {
                const int c[3] = {mi.m[h], mi.n[h], mi.k[h]};
                int av[3], bv[3];
                for (int i = 0; i < 3; i++) av[i] = c[pi[i]];        // (c o pi)_i = c_pi(i)
                for (int j = 0; j < 3; j++) bv[j] = c[pinv[j]];      // (c o pi^-1)_j = c_pi^-1(j)
                const int sa = ((sb & 1) ? av[0] : 0) + ((sb & 2) ? av[1] : 0) + ((sb & 4) ? av[2] : 0);
                const int sbb = ((sb & 1) ? c[0] : 0) + ((sb & 2) ? c[1] : 0) + ((sb & 4) ? c[2] : 0);
                fwd[(size_t)sig * np + h] = (unsigned short)(idx(av[0], av[1], av[2]) | ((sa & 1) ? 0x8000 : 0));
                inv[(size_t)sig * np + h] = idx(bv[0], bv[1], bv[2]) | ((sbb & 1) ? (int)0x80000000 : 0);
            }
        }
    Arena &A = P->arena;
    auto up = [&](auto **d, const auto &h) -> int {
        using T = std::decay_t<decltype(h[0])>;
        BEM_TRY(A.alloc((T **)d, std::max<size_t>(1, h.size())));
        if (!h.empty()) BEM_CUDA(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
        return BEM_OK;
    };
    BEM_TRY(up(&P->sy_fwd, fwd));
    BEM_TRY(up(&P->sy_inv, inv));
    BEM_TRY(up(&P->sy_mexp, mexp));
    BEM_TRY(up(&P->sy_invf, invf));
    const int ncls = P->sy_ncls;
    BEM_TRY(A.alloc(&P->sy_D, std::max<size_t>(1, (size_t)ncls * np * C)));
    if (mx) BEM_TRY(A.alloc(&P->sy_fD, std::max<size_t>(1, (size_t)ncls * np * C)));
    BEM_TRY(launch_m2l_derivs(P, ncls, P->sy_rho, C == 2 ? P->sy_kh : nullptr, P->sy_D, mx ? P->sy_fD : nullptr, s));
    TcGroups g{};
    int ldp = 0, nkc = 0;
    std::vector<uint4> sched;
    std::vector<int> sptr;
    const bool tc = C == 1 && mx && ncls > 0 && !P->lev_var && tc_plan(mi, deg, g, ldp, nkc, sched, sptr);
    // source and target order of every canonical class (one order unless it varies with the level;
    // the class key then holds the target level)
    {
        std::vector<int> ord(2 * (size_t)std::max(1, ncls), p);
        if (P->lev_var)
            for (int c = 0; c < ncls; c++) {
                const int lt = P->sy_hlev[c], ls = lt - P->sy_hdl[c];
                auto at = [&](int l) { return l >= 0 && l < (int)P->lev_p.size() ? P->lev_p[l] : p; };
                ord[2 * c] = at(ls);
                ord[2 * c + 1] = at(lt);
            }
        BEM_TRY(up(&P->sy_ord, ord));
    }
    if (tc) {
        // class-matrix gather table in shared-memory layout order
        std::vector<int> tidx(g.tsize, -1);
        std::vector<float> tfac(g.tsize, 0.f);
        for (int q = 0; q < g.ng; q++)
            for (int bl = 0; bl < g.n[q]; bl++)
                for (int al = 0; al < g.k[q]; al++) {
                    const int b = g.b0[q] + bl, e = g.off[q] + (bl >> 3) * (g.k[q] / 4) * 32 + (al >> 2) * 32 +
                                                    (bl & 7) * 4 + (al & 3);
                    if (b < np && al < np && deg[b] + deg[al] <= p) {
                        tidx[e] = idx(mi.m[al] + mi.m[b], mi.n[al] + mi.n[b], mi.k[al] + mi.k[b]) | (deg[al] << 16);
                        tfac[e] = (float)(((deg[al] & 1) ? -1.0 : 1.0) * invf[al] * invf[b]);
                    }
                }
        BEM_TRY(up(&P->sy_tidx, tidx));
        BEM_TRY(up(&P->sy_tfac, tfac));
        BEM_TRY(up(&P->sy_sched, sched));
        BEM_TRY(up(&P->sy_sched_ptr, sptr));
        P->sy_g = g;
        P->sy_nkc = nkc;
        P->sy_nsched = (int)sched.size();
    } else {
        ldp = (np + 3) / 4 * 4;
        if (sy_simt_smem_bytes(mx, C, np, p) > (size_t)200 * 1024) {
            set_error("M2L: order %d needs more shared memory than a block has", p);
            return BEM_EINVAL;
        }
    }
    int64_t max_rows = 0;
    BEM_TRY(build_sym_tiles(P, (size_t)ldp * C * (mx ? sizeof(float) : sizeof(double)), max_rows));
    const size_t nLp = std::max<size_t>(1, (size_t)max_rows * ldp * C);
    if (mx) BEM_TRY(A.alloc((float **)&P->sy_Lp, nLp));
    else BEM_TRY(A.alloc((double **)&P->sy_Lp, nLp));
    P->sy_ldp = ldp;
    P->sy_tc = tc ? 1 : 0;
    P->sy_ready = 1;
    return BEM_OK;
}

void free_sym_tables(bem_plan *P) {
    Arena &A = P->arena;
    for (void *q : {(void *)P->sy_tidx, (void *)P->sy_tfac, (void *)P->sy_fwd, (void *)P->sy_inv, (void *)P->sy_D,
                    (void *)P->sy_fD, (void *)P->sy_Lp, (void *)P->sy_sched, (void *)P->sy_sched_ptr,
                    (void *)P->sy_mexp, (void *)P->sy_invf, (void *)P->sy_ord, (void *)P->sy_tile_cls, (void *)P->sy_tile_start,
                    (void *)P->sy_tile_cnt, (void *)P->sy_src, (void *)P->sy_sig, (void *)P->sy_pair})
        A.release(q);
    P->sy_tile_cls = P->sy_tile_start = P->sy_tile_cnt = P->sy_src = P->sy_sig = P->sy_pair = nullptr;
    P->sy_ord = nullptr;
    P->sy_ntile = 0;
    P->sy_tidx = P->sy_inv = P->sy_mexp = nullptr;
    P->sy_fwd = nullptr;
    P->sy_sched = nullptr;
    P->sy_sched_ptr = nullptr;
    P->sy_tfac = P->sy_fD = nullptr;
    P->sy_Lp = nullptr;
    P->sy_D = P->sy_invf = nullptr;
    P->sy_tc = 0;
    P->sy_ready = 0;
}

int launch_m2l_tc(bem_plan *P, const float *M, float *L, cudaStream_t s) {
    const Tree &t = P->t;
    TcArgs a{};
    a.g = P->sy_g;
    a.np = P->mi.np;
    a.nkc = P->sy_nkc;
    a.nsched = P->sy_nsched;
    a.sched = P->sy_sched;
    a.sched_ptr = P->sy_sched_ptr;
    a.src = P->sy_src;
    a.sig = P->sy_sig;
    a.pair = P->sy_pair;
    a.dl = P->sy_dl;
    a.fwd = P->sy_fwd;
    a.tidx = P->sy_tidx;
    a.tfac = P->sy_tfac;
    a.fD = P->sy_fD;
    a.M = M;
    a.Lp = (float *)P->sy_Lp;
    a.ldp = P->sy_ldp;
    a.err = P->dev_err;
    a.skip = P->skip;
    const size_t sm = tc_smem_bytes(a.g, a.ldp);
    // one run of targets at a time: its tiles, then the gather of its targets
    for (size_t r = 0; r + 1 < P->sy_bt.size(); r++) {
        const int bt0 = P->sy_bt[r], nt = P->sy_bt[r + 1] - bt0, tg0 = P->sy_bb[r], ntg = P->sy_bb[r + 1] - tg0;
        a.ntile = nt;
        a.tile_cls = P->sy_tile_cls + bt0;
        a.tile_start = P->sy_tile_start + bt0;
        a.tile_cnt = P->sy_tile_cnt + bt0;
        a.u0 = P->sy_bu[r];
        if (nt > 0) (k_m2l_tc<<<std::min(nt, std::max(1, P->sm_count)), TC_T, sm, s>>>(a), ::bem::count_launch());
        if (ntg > 0)
            (k_m2l_gather_sym<<<ntg, a.ldp, 0, s>>>(tg0, t.nbox, t.level, t.side, t.inter_ptr, a.u0, a.np, a.ldp,
                                                    P->sy_sig_u, P->sy_inv, (const float *)P->sy_Lp, L, P->skip),
             ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    return BEM_OK;
}

void set_tc_attributes() {
    cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_MAX);
}

}  // namespace bem
