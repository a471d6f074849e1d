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
// kind::tf32 MMAs: M = 128 pairs (TMEM lanes), K = 8 columns a per MMA, and N
// = the rows b that K-step reaches (|b| <= p - min |a| of the step: a prefix of
// the degree-ordered rows), so the zero triangle is mostly skipped with one
// MMA per K-step (two when N exceeds 256).  Each float32 operand is split into
// tf32 hi + lo and the product accumulated as hi*hi + hi*lo + lo*hi in float32
// (about 2^-21 relative per product).  The class matrices are built once per
// plan as shared-memory images (one block per K-step) and brought in by one
// bulk copy when the class changes.  The moments are gathered, permuted and
// sign-flipped by 11 producer warps through 4-byte cp.async copies into a
// three-stage ring of 32-column K chunks, converted to hi/lo in place by the
// thread that copied them; one thread of a fifth warp issues the MMAs, four
// warps read the accumulator back.  Each pair's row of Lhat is written out; a
// gather kernel sums every target's rows in list order, undoing the
// permutation: deterministic, no atomics.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bem_internal.cuh"
#include "tc_ptx.cuh"

namespace bem {

namespace {

constexpr int TC_T = 512;           // threads per block (16 warps)
constexpr int TC_M = 128;           // pairs per tile (MMA M, TMEM lanes)
constexpr int TC_KC = 32;           // K chunk of the moment operand (4 K-steps of 8)
constexpr int TC_NS = 3;            // moment chunks in flight
constexpr int TC_PLANE = TC_M * TC_KC * 4;       // one tf32 plane of a chunk
constexpr int TC_EPI = 4;           // epilogue warps 0-3 (TMEM lane quadrants)
constexpr int TC_MMA_WARP = 4;      // one thread of warp 4 issues the MMAs
constexpr int TC_PROD0 = 5;         // producer warps 5-15
constexpr int TC_NPROD = TC_T / 32 - TC_PROD0;
constexpr long long TC_WAIT = 4000000000ll;      // clock cycles before a wait gives up
constexpr int TC_SMEM_MAX = 227 * 1024;

// the six axis permutations; PERMS[q][i] = canonical position of axis i
constexpr int PERMS[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

struct TcArgs {
    TcPlan g;
    int np, ldp, ntile, nkc;
    const int *tile_cls, *tile_start, *tile_cnt;
    const int *src, *sig, *pair;
    const float *img;                   // [class][part][hi, lo][g.part_floats[part]]
    const unsigned *sgn;                // [48][ldp / 32] sign bit of every canonical-frame moment
    const float *Mq;                    // [box][6][ldp] moments permuted by each axis permutation
    float *Lp;                          // rows of this run's pairs, row u - u0
    int u0;
    int *err;
    const int *skip;
};

__device__ __forceinline__ uint32_t mom_off(int r, int k) {   // byte offset in a chunk plane
    return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// shared-memory layout of the tensor-core M2L block
constexpr int TC_XLD = 36;              // row stride (floats) of the epilogue's transpose buffer
constexpr int TC_XPOSE = 32 * TC_XLD;   // floats of one epilogue warp's transpose buffer
struct TcLayout {
    size_t img, stage, sgn, xpose, bars, total;
};
__host__ __device__ inline TcLayout tc_layout(const TcPlan &g, int ldp) {
    TcLayout L;
    L.img = 0;
    const int pf = g.part_floats[0] > g.part_floats[1] ? g.part_floats[0] : g.part_floats[1];
    L.stage = ((2 * (size_t)pf * 4 + 1023) / 1024) * 1024;
    L.sgn = L.stage + (size_t)TC_NS * 2 * TC_PLANE;
    L.xpose = L.sgn + ((48 * (size_t)(ldp / 32) * 4 + 15) / 16) * 16;
    L.bars = L.xpose + (size_t)TC_EPI * TC_XPOSE * 4;
    L.total = L.bars + 16 * 8 + 16 + 1024;
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

// Roles: warps 0-3 read the accumulator back (warp w owns TMEM lanes
// 32 w .. 32 w + 31, i.e. pairs); warp 4 lane 0 loads the class image and
// issues the MMAs; warps 5-15 gather the moments into the chunk ring.
// Handshakes: full[s] (11 producer warps) -> MMA; empty[s] (MMA commit) ->
// producers; tfull (commit after a tile's last chunk) -> epilogue; tovl
// (4 epilogue warps) -> MMA; bfull (bulk copy of a class image) -> MMA.
// Two accumulators: even tiles use TMEM columns [0, ldp), odd tiles
// [512 - ldp, 512).  Where the two share columns (ldp > 256), the epilogue
// reads the shared ones first and then arrives on tovl, so the MMAs of the
// next tile run while it reads the rest of the previous one.
__global__ void __launch_bounds__(TC_T, 1) k_m2l_tc(const __grid_constant__ TcArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcPlan &G = a.g;
    const TcLayout LY = tc_layout(G, a.ldp);
    const int ldp = a.ldp, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *sImg = (float *)(smem + LY.img);                             // class image: hi plane, lo plane
    unsigned char *sStage = smem + LY.stage;                            // [TC_NS][hi, lo] chunk planes
    unsigned *sSgn = (unsigned *)(smem + LY.sgn);                       // [48][ldp / 32]
    float *sX = (float *)(smem + LY.xpose);                             // [TC_EPI][32][33]
    uint64_t *full = (uint64_t *)(smem + LY.bars), *empty = full + TC_NS, *tfull = full + 2 * TC_NS,
             *tovl = tfull + 1, *bfull = tfull + 2, *fin = tfull + 3, *imgfree = tfull + 4;
    uint32_t *sTmem = (uint32_t *)(imgfree + 1);
    volatile int *sAbort = (volatile int *)(sTmem + 1);
    const int nw = ldp / 32;
    const int colB = 512 - ldp;                         // first column of the second accumulator
    const int gs = colB < ldp ? colB / 32 : 0;          // first group of the first one that the second shares
    const int novl = colB < ldp ? nw - gs : 0;          // groups the two accumulators share

    if (tid == 0) {
        for (int s = 0; s < TC_NS; s++) {
            tc::mbar_init(&full[s], TC_NPROD);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(tfull, 1);
        tc::mbar_init(tovl, TC_EPI);
        tc::mbar_init(bfull, 1);
        tc::mbar_init(fin, 1);
        tc::mbar_init(imgfree, 1);
        *sAbort = 0;
        tc::mbar_fence_init();
    }
    for (int i = tid; i < 48 * nw; i += TC_T) sSgn[i] = a.sgn[i];
    if (warp == 0) tc::tmem_alloc(sTmem, 512);
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *sTmem;

    const int t_begin = (int)((long long)a.ntile * blockIdx.x / gridDim.x);
    const int t_end = (int)((long long)a.ntile * (blockIdx.x + 1) / gridDim.x);
    bool bulk_pending = false;                        // MMA thread: a class image copy not yet observed complete
    uint32_t nbulk = 0;

    if (warp < TC_EPI) {
        // ---- accumulator read-back: TMEM lane 32 w + lane = pair row ----
        const uint64_t pol = tc::policy_evict_last();    // the gather reads these rows next
        const int r = 32 * warp + lane;
        for (int tile = t_begin; tile < t_end; tile++) {
            const int k = tile - t_begin;
            const int cnt = a.tile_cnt[tile];
            const int u = r < cnt ? a.pair[a.tile_start[tile] + r] : -1;
            bool ok = wait_or_abort(tfull, (uint32_t)(k & 1), sAbort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc::tc_fence_after_sync();
            // 32 x 32 blocks through shared memory: lane l holds row l after
            // the TMEM load; after the transpose a store of 32 lanes writes 16
            // bytes each, 128 contiguous bytes of four rows
            float *xb = sX + warp * TC_XPOSE;
            const int ur = u >= 0 ? u - a.u0 : -1;
            const int rq = lane >> 3, cg = lane & 7;
            // odd tiles use the second accumulator; the first accumulator's
            // shared groups go first, so that the next tile can start
            const bool second = (k & 1) != 0;
            const int start = second ? 0 : gs;
            const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + (second ? (uint32_t)colB : 0u);
            bool sig = false;
            auto release = [&]() {
                tc::tc_fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(tovl);
                sig = true;
            };
            if (novl == 0) release();
            for (int q = 0; q < nw; q += 2) {
                const int g0 = (start + q) % nw, g1 = (start + q + 1) % nw;
                const bool two = q + 1 < nw;
                uint32_t v0[32], v1[32];
                tc::tmem_ld32_nowait(base + (uint32_t)(32 * g0), v0);
                if (two) tc::tmem_ld32_nowait(base + (uint32_t)(32 * g1), v1);
                tc::tmem_wait_ld2(v0, v1);
                if (!sig && q + 2 >= novl) release();
                for (int h = 0; h < 2 && (h == 0 || two); h++) {
                    const int col = 32 * (h ? g1 : g0);
                    __syncwarp();
#pragma unroll
                    for (int k4 = 0; k4 < 8; k4++) {
                        const uint32_t *v = h ? v1 : v0;
                        *(float4 *)(xb + lane * TC_XLD + 4 * k4) = make_float4(
                            __uint_as_float(v[4 * k4]), __uint_as_float(v[4 * k4 + 1]),
                            __uint_as_float(v[4 * k4 + 2]), __uint_as_float(v[4 * k4 + 3]));
                    }
                    __syncwarp();
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int row = 4 * i + rq;
                        const int uq = __shfl_sync(0xffffffffu, ur, row);
                        const float4 x = *(const float4 *)(xb + row * TC_XLD + 4 * cg);
                        if (uq >= 0) tc::st_v4_hint(a.Lp + (size_t)uq * ldp + col + 4 * cg, x.x, x.y, x.z, x.w, pol);
                    }
                }
            }
            if (!sig) release();
            if (__any_sync(0xffffffffu, *sAbort != 0)) break;
        }
    } else if (warp == TC_MMA_WARP) {
        // ---- class images and MMA issue (one thread) ----
        if (lane == 0) {
            const bool split = G.ks_split < G.nks;
            const uint32_t pb0 = (uint32_t)G.part_floats[0] * 4u, pb1 = (uint32_t)G.part_floats[1] * 4u;
            const uint32_t ih = tc::smem_u32(sImg), st0 = tc::smem_u32(sStage);
            int it = 0, cur_cls = -1, cur_part = -1;
            uint32_t nfree = 0;
            bool ok = true;
            // one part of a class image into shared memory (hi plane, then lo)
            auto load_part = [&](int cls, int part) {
                const float *src = a.img + (size_t)cls * 2 * G.img_floats + (part ? 2 * (size_t)G.part_floats[0] : 0);
                const uint32_t bytes = 2u * (part ? pb1 : pb0);
                tc::mbar_arrive_expect_tx(bfull, bytes);
                tc::bulk_g2s(sImg, src, bytes, bfull);
                bulk_pending = true;
                if (!wait_or_abort(bfull, nbulk & 1u, sAbort)) return false;
                bulk_pending = false;
                nbulk++;
                cur_cls = cls;
                cur_part = part;
                return true;
            };
            for (int tile = t_begin; tile < t_end && ok; tile++) {
                const int k = tile - t_begin, cls = a.tile_cls[tile];
                // this tile's accumulator is free once the epilogue has read the
                // columns it shares with the previous tile's (which it does after
                // every MMA of that tile has completed, so the image is free too)
                if (k > 0) ok = wait_or_abort(tovl, (uint32_t)((k - 1) & 1), sAbort);
                if (!ok) break;
                if (cls != cur_cls || cur_part != 0) {
                    ok = load_part(cls, 0);
                    if (!ok) break;
                }
                tc::tc_fence_after_sync();
                const uint32_t dacc = tmem + ((k & 1) ? (uint32_t)colB : 0u);
                for (int kc = 0; kc < a.nkc && ok; kc++, it++) {
                    const int s = it % TC_NS;
                    ok = wait_or_abort(&full[s], (uint32_t)((it / TC_NS) & 1), sAbort);
                    if (!ok) break;
                    tc::tc_fence_after_sync();
                    const uint32_t ab = st0 + (uint32_t)s * 2u * TC_PLANE;
                    const uint64_t ah0 = tc::smem_desc(ab, 128, 1024), al0 = tc::smem_desc(ab + TC_PLANE, 128, 1024);
                    for (int ks = 0; ks < 4; ks++) {
                        const int j = kc * 4 + ks;
                        if (j >= G.nks) break;
                        if (split && j == G.ks_split) {
                            // every MMA so far reads the first part: once they have
                            // completed, the second part replaces it
                            tc::mma_commit(imgfree);
                            ok = wait_or_abort(imgfree, nfree & 1u, sAbort);
                            nfree++;
                            if (!ok) break;
                            ok = load_part(cls, 1);
                            if (!ok) break;
                            tc::tc_fence_after_sync();
                        }
                        const int pbase = cur_part ? G.part_floats[0] : 0;   // == ks_off[ks_split]
                        const uint32_t il = ih + (cur_part ? pb1 : pb0);
                        const uint32_t boff = (uint32_t)(G.ks_off[j] - pbase) * 4u;
                        const int n = G.ks_n[j];
                        for (int part = 0; part < n; part += 256) {
                            const int nn = min(256, n - part);
                            const uint32_t po = boff + (uint32_t)(part / 8) * 256u;
                            const uint64_t bh = tc::smem_desc(ih + po, 128, 256), bl = tc::smem_desc(il + po, 128, 256);
                            const uint32_t id = tc::idesc_tf32(TC_M, nn), d = dacc + (uint32_t)part;
                            const uint64_t ao = (uint64_t)ks * 16u;   // 256 B per K-step
                            tc::mma_tf32(d, ah0 + ao, bh, id, j > 0);
                            tc::mma_tf32(d, ah0 + ao, bl, id, true);
                            tc::mma_tf32(d, al0 + ao, bh, id, true);
                        }
                    }
                    if (!ok) break;
                    tc::mma_commit(&empty[s]);
                }
                if (ok) tc::mma_commit(tfull);
            }
            if (bulk_pending) {
                // a copy in flight when a wait gave up: let it land before exit
                if (!tc::mbar_wait_bounded(bfull, nbulk & 1u, TC_WAIT)) *sAbort = 1;
            }
        }
        __syncwarp();
    } else {
        // ---- producers: warps 5-15, 16-byte asynchronous copies ----
        // A chunk is 128 rows x 8 groups of 4 columns, in 32 slots of 32 lanes:
        // slot sl holds rows 8 (sl / 2) + lane % 8 and groups 4 (sl % 2) +
        // lane / 8 (64 contiguous bytes per row in global memory, 4 shared-
        // memory wavefronts per slot).  This thread's slots: pw + 11 i.
        constexpr int NI = (32 + TC_NPROD - 1) / TC_NPROD;       // 3
        const int pw = warp - TC_PROD0;
        size_t srow[NI];                              // Mq row of the pair (box, permutation), or ~0 if none
        unsigned pvm = 0u;                            // items of the pending chunk that were copied
        int it = 0;
        bool ok = true, pend = false;
        auto item = [&](int i, int &r, int &g) {
            const int sl = pw + TC_NPROD * i;
            r = (sl >> 1) * 8 + (lane & 7);
            g = (sl & 1) * 4 + (lane >> 3);
            return sl < 32;
        };
        int psig[NI];                                 // symmetry of each item of the pending chunk
        // sign flips and hi/lo split of chunk `c` in place, zeros where nothing was copied
        auto convert = [&](int c, unsigned vm) {
            unsigned char *hi = sStage + (size_t)(c % TC_NS) * 2 * TC_PLANE, *lo = hi + TC_PLANE;
            const int kc = c % a.nkc;
#pragma unroll
            for (int i = 0; i < NI; i++) {
                int r, g;
                if (!item(i, r, g)) continue;
                const uint32_t o = mom_off(r, 4 * g);
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if ((vm >> i) & 1u) {
                    x = *(const float4 *)(hi + o);
                    const unsigned sb = (sSgn[psig[i] * nw + kc] >> (4 * g)) & 15u;
                    x.x = (sb & 1u) ? -x.x : x.x;
                    x.y = (sb & 2u) ? -x.y : x.y;
                    x.z = (sb & 4u) ? -x.z : x.z;
                    x.w = (sb & 8u) ? -x.w : x.w;
                }
                float4 h, l;
                h.x = tc::to_tf32(x.x); l.x = tc::to_tf32(x.x - h.x);
                h.y = tc::to_tf32(x.y); l.y = tc::to_tf32(x.y - h.y);
                h.z = tc::to_tf32(x.z); l.z = tc::to_tf32(x.z - h.z);
                h.w = tc::to_tf32(x.w); l.w = tc::to_tf32(x.w - h.w);
                *(float4 *)(hi + o) = h;
                *(float4 *)(lo + o) = l;
            }
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[c % TC_NS]);
        };
        int csig[NI];
        for (int tile = t_begin; tile < t_end && ok; tile++) {
            const int st = a.tile_start[tile], cnt = a.tile_cnt[tile];
#pragma unroll
            for (int i = 0; i < NI; i++) {
                int r, g;
                const bool v = item(i, r, g) && r < cnt;
                const int sg = v ? a.sig[st + r] : 0;
                srow[i] = v ? ((size_t)a.src[st + r] * 6 + (size_t)(sg >> 3)) * ldp : ~(size_t)0;
                csig[i] = sg;
            }
            for (int kc = 0; kc < a.nkc; kc++, it++) {
                const int s = it % TC_NS, n = it / TC_NS;
                if (n > 0) {
                    ok = __all_sync(0xffffffffu, wait_or_abort(&empty[s], (uint32_t)((n - 1) & 1), sAbort));
                    if (!ok) break;
                }
                unsigned char *hi = sStage + (size_t)s * 2 * TC_PLANE;
                unsigned vm = 0u;
#pragma unroll
                for (int i = 0; i < NI; i++) {
                    int r, g;
                    item(i, r, g);
                    if (srow[i] != ~(size_t)0) {
                        tc::cp_async16(hi + mom_off(r, 4 * g), a.Mq + srow[i] + kc * TC_KC + 4 * g);
                        vm |= 1u << i;
                    }
                }
                tc::cp_async_commit();
                if (pend) {                               // the previous chunk has landed: convert it
                    tc::cp_async_wait<1>();
                    convert(it - 1, pvm);
                }
#pragma unroll
                for (int i = 0; i < NI; i++) psig[i] = csig[i];
                pvm = vm;
                pend = true;
            }
        }
        tc::cp_async_wait<0>();
        if (pend && ok) convert(it - 1, pvm);
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

// Class-matrix images of every canonical class: element e of a plane (in the
// K-step block layout) is T[b][a] = Dhat[a+b] (-1)^|a| 2^(dl |a|) / (a! b!),
// tidx[e] = index of a + b | |a| << 16 (-1 outside the triangle), tfac[e] the
// factorial and sign factor; split into tf32 hi and lo planes.
__global__ void k_tc_images(int img_floats, int part0, int np, const int *__restrict__ tidx,
                            const float *__restrict__ tfac, const float *__restrict__ fD, const int *__restrict__ dl,
                            float *__restrict__ img) {
    const int cls = blockIdx.y;
    float *ci = img + (size_t)cls * 2 * img_floats;   // part 0: hi, lo; part 1: hi, lo
    const float *Dc = fD + (size_t)cls * np;
    const int d = dl[cls];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < img_floats; e += gridDim.x * blockDim.x) {
        const int gi = tidx[e];
        const float v = gi >= 0 ? ldexpf(Dc[gi & 0xffff] * tfac[e], d * (gi >> 16)) : 0.f;
        const float h = tc::to_tf32(v);
        const bool second = e >= part0;
        const int pn = second ? img_floats - part0 : part0, eo = second ? e - part0 : e;
        float *hi = ci + (second ? 2 * (size_t)part0 : 0);
        hi[eo] = h;
        hi[pn + eo] = tc::to_tf32(v - h);
    }
}

// Moments of every box under each of the six axis permutations, rows of ldp
// floats (zero beyond np): Mq[box][q][h] = M[box][a], a = h o pi_q, so that a
// tile's producers copy contiguous row segments.
__global__ void k_m2l_permute(int nbox, int np, int ldp, const unsigned short *__restrict__ fwdq,
                              const float *__restrict__ M, float *__restrict__ Mq, const int *__restrict__ skip) {
    if (skip && *skip) return;
    const int64_t n = (int64_t)nbox * 6 * ldp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int h = (int)(i % ldp);
        const int64_t rq = i / ldp;
        const int q = (int)(rq % 6);
        const int64_t box = rq / 6;
        Mq[i] = h < np ? M[box * np + fwdq[q * np + h]] : 0.f;
    }
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
        // axes by decreasing |K|, ties in axis order (a stable insertion sort of
        // three: std::stable_sort would take a heap buffer per class)
        int order[3] = {0, 1, 2};
        for (int x = 1; x < 3; x++)
            for (int y = x; y > 0 && std::llabs(K[order[y]]) > std::llabs(K[order[y - 1]]); y--)
                std::swap(order[y], order[y - 1]);
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
    // the keys as one 64-bit word when every field fits (level difference
    // + 64 in 7 bits, level in 6, the sorted offset magnitudes in 17 each):
    // the same order, one integer compare
    bool packs = true;
    for (int c = 0; c < nfull && packs; c++) {
        const long long *v = fkey[c].v;
        packs = v[0] > -64 && v[0] < 64 && v[1] >= 0 && v[1] < 64 && v[2] < (1 << 17) && v[3] < (1 << 17) && v[4] < (1 << 17);
    }
    if (packs) {
        std::vector<std::pair<unsigned long long, int>> kp(nfull);
        for (int c = 0; c < nfull; c++) {
            const long long *v = fkey[c].v;
            kp[c] = {((unsigned long long)(v[0] + 64) << 57) | ((unsigned long long)v[1] << 51) |
                         ((unsigned long long)v[2] << 34) | ((unsigned long long)v[3] << 17) | (unsigned long long)v[4],
                     c};
        }
        std::sort(kp.begin(), kp.end());
        for (int c = 0; c < nfull; c++) fidx[c] = kp[c].second;
    } else {
        std::sort(fidx.begin(), fidx.end(), [&](int x, int y) { return fkey[x] < fkey[y] || (!(fkey[y] < fkey[x]) && x < y); });
    }
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

static int build_sym_tiles(bem_plan *P, size_t row_bytes, int64_t &max_rows, cudaStream_t s) {
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
        // (pageable source: staged before the call returns, so h may go)
        if (!h.empty()) BEM_CUDA(cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
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
size_t tc_smem_bytes(const TcPlan &g, int ldp) { return tc_layout(g, ldp).total; }

// The class-matrix image layout of the current order, when the tensor-core
// form applies: K-step j (columns a in [8j, 8j + 8)) reaches the rows b with
// |b| <= p - min |a| of the step, the first cum(p - min|a| + 1) rows in degree
// order, rounded up to 16 (MMA N).  Returns false when the order does not fit
// the K-step table, TMEM or shared memory.
static bool tc_plan(const MIndex &mi, const std::vector<int> &deg, TcPlan &g, int &ldp, int &nkc) {
    const int p = mi.p, np = mi.np;
    auto cum = [](int d) { return d <= 0 ? 0 : d * (d + 1) * (d + 2) / 6; };
    g = TcPlan{};
    g.nks = (np + 7) / 8;
    if (g.nks > TC_MAXKS) return false;
    int off = 0;
    for (int j = 0; j < g.nks; j++) {
        int dmin = p;
        for (int al = 8 * j; al < std::min(np, 8 * j + 8); al++) dmin = std::min(dmin, deg[al]);
        g.ks_off[j] = off;
        g.ks_n[j] = (cum(p - dmin + 1) + 15) / 16 * 16;
        off += g.ks_n[j] * 8;
    }
    g.img_floats = off;
    ldp = (g.ks_n[0] + 31) / 32 * 32;             // TMEM columns read back, 32 at a time
    nkc = (g.nks + 3) / 4;
    if (ldp > 512) return false;
    g.ks_split = g.nks;
    g.part_floats[0] = off;
    g.part_floats[1] = 0;
    if (tc_smem_bytes(g, ldp) <= (size_t)TC_SMEM_MAX) return true;
    // two parts of about equal size
    int best = 1;
    for (int j = 1; j < g.nks; j++)
        if (std::max(g.ks_off[j], off - g.ks_off[j]) < std::max(g.ks_off[best], off - g.ks_off[best])) best = j;
    g.ks_split = best;
    g.part_floats[0] = g.ks_off[best];
    g.part_floats[1] = off - g.ks_off[best];
    return tc_smem_bytes(g, ldp) <= (size_t)TC_SMEM_MAX;
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
        // (pageable source: staged before the call returns, so h may go)
        if (!h.empty()) BEM_CUDA(cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
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
    TcPlan g{};
    int ldp = 0, nkc = 0;
    const bool tc = C == 1 && mx && ncls > 0 && !P->lev_var && tc_plan(mi, deg, g, ldp, nkc);
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
        // class-matrix images of every canonical class, built once: gather
        // table (index of a + b and |a|) and factors in image layout order
        std::vector<int> tidx(g.img_floats, -1);
        std::vector<float> tfac(g.img_floats, 0.f);
        for (int j = 0; j < g.nks; j++)
            for (int b = 0; b < g.ks_n[j]; b++)
                for (int kk = 0; kk < 8; kk++) {
                    const int al = 8 * j + kk, e = g.ks_off[j] + (b >> 3) * 64 + (kk >> 2) * 32 + (b & 7) * 4 + (kk & 3);
                    if (b < np && al < np && deg[b] + deg[al] <= p) {
                        tidx[e] = idx(mi.m[al] + mi.m[b], mi.n[al] + mi.n[b], mi.k[al] + mi.k[b]) | (deg[al] << 16);
                        tfac[e] = (float)(((deg[al] & 1) ? -1.0 : 1.0) * invf[al] * invf[b]);
                    }
                }
        int *d_tidx = nullptr;
        float *d_tfac = nullptr;
        BEM_TRY(up(&d_tidx, tidx));
        BEM_TRY(up(&d_tfac, tfac));
        BEM_TRY(A.alloc(&P->sy_img, (size_t)ncls * 2 * g.img_floats));
        (k_tc_images<<<dim3((g.img_floats + 255) / 256, ncls), 256, 0, s>>>(g.img_floats, g.part_floats[0], np, d_tidx, d_tfac, P->sy_fD,
                                                                            P->sy_dl, P->sy_img),
         ::bem::count_launch());
        BEM_LAUNCH_CHECK();
        P->deferred.push_back(d_tidx);
        P->deferred.push_back(d_tfac);
        // permutation maps without the sign, and the sign bits per symmetry
        // in words of 32 canonical-frame columns (one word per K chunk)
        std::vector<unsigned short> fq(6 * (size_t)np);
        for (int q = 0; q < 6; q++)
            for (int h = 0; h < np; h++) fq[(size_t)q * np + h] = fwd[(size_t)(q * 8) * np + h] & 0x7fff;
        BEM_TRY(up(&P->sy_fwdq, fq));
        const int nw = ldp / 32;
    const int colB = 512 - ldp;                         // first column of the second accumulator
    const int gs = colB < ldp ? colB / 32 : 0;          // first group of the first one that the second shares
    const int novl = colB < ldp ? nw - gs : 0;          // groups the two accumulators share
        std::vector<unsigned> sg(48 * (size_t)nw, 0u);
        for (int sig = 0; sig < 48; sig++)
            for (int h = 0; h < np; h++)
                if (fwd[(size_t)sig * np + h] & 0x8000) sg[(size_t)sig * nw + h / 32] |= 1u << (h % 32);
        BEM_TRY(up(&P->sy_sgn, sg));
        BEM_TRY(A.alloc(&P->sy_Mq, (size_t)P->t.nbox * 6 * ldp));
        P->sy_g = g;
        P->sy_nkc = nkc;
    } else {
        ldp = (np + 3) / 4 * 4;
        if (sy_simt_smem_bytes(mx, C, np, p) > (size_t)200 * 1024) {
            set_error("M2L: order %d needs more shared memory than a block has", p);
            return BEM_EINVAL;
        }
    }
    int64_t max_rows = 0;
    BEM_TRY(build_sym_tiles(P, (size_t)ldp * C * (mx ? sizeof(float) : sizeof(double)), max_rows, s));
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
    for (void *q : {(void *)P->sy_img, (void *)P->sy_fwdq, (void *)P->sy_sgn, (void *)P->sy_Mq, (void *)P->sy_fwd, (void *)P->sy_inv, (void *)P->sy_D,
                    (void *)P->sy_fD, (void *)P->sy_Lp, (void *)P->sy_mexp, (void *)P->sy_invf, (void *)P->sy_ord,
                    (void *)P->sy_tile_cls, (void *)P->sy_tile_start, (void *)P->sy_tile_cnt, (void *)P->sy_src,
                    (void *)P->sy_sig, (void *)P->sy_pair})
        A.release(q);
    P->sy_tile_cls = P->sy_tile_start = P->sy_tile_cnt = P->sy_src = P->sy_sig = P->sy_pair = nullptr;
    P->sy_ord = nullptr;
    P->sy_ntile = 0;
    P->sy_inv = P->sy_mexp = nullptr;
    P->sy_fwd = P->sy_fwdq = nullptr;
    P->sy_sgn = nullptr;
    P->sy_Mq = nullptr;
    P->sy_img = P->sy_fD = nullptr;
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
    a.ldp = P->sy_ldp;
    a.nkc = P->sy_nkc;
    a.src = P->sy_src;
    a.sig = P->sy_sig;
    a.pair = P->sy_pair;
    a.img = P->sy_img;
    a.sgn = P->sy_sgn;
    a.Mq = P->sy_Mq;
    a.Lp = (float *)P->sy_Lp;
    a.err = P->dev_err;
    a.skip = P->skip;
    const size_t sm = tc_smem_bytes(a.g, a.ldp);
    {
        const int64_t n = (int64_t)t.nbox * 6 * a.ldp;
        const int grid = (int)std::min<int64_t>((n + 255) / 256, 8 * std::max(1, P->sm_count));
        (k_m2l_permute<<<grid, 256, 0, s>>>(t.nbox, a.np, a.ldp, P->sy_fwdq, M, P->sy_Mq, P->skip),
         ::bem::count_launch());
    }
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
