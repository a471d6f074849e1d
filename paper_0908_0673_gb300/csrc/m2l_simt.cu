// M2L (Eq. 7) on the canonical offset classes, SIMT form: every product the
// tensor-core form does not take (float32 Helmholtz, float64 of either
// Green's function, and orders beyond the tensor-core tables, such as the
// order p + 2 of the mixed plan's diagonal product).
//
// The pairs, tiles, symmetry maps and canonical derivative tables are those
// of the tensor-core form (m2l_tc.cu): a tile holds up to 128 pairs of one
// canonical class, and the block computes
//     Lhat[pair][b] = sum_a T[b][a] Mhat[pair][a],
//     T[b][a] = Dhat[a + b] (-1)^|a| 2^(dl |a|) / (a! b!)   (|a| + |b| <= p),
// with Mhat the sign-permuted moments of the pair's source box, as a
// register-blocked GEMM: rows b in chunks of BB (ordered by degree, so a chunk
// needs only the columns a with |a| <= p - |b0|), columns a in chunks of 16
// staged with the moments in shared memory, and each thread holding RB rows x
// 8 pairs of accumulators.  Complex values (Helmholtz) are kept as real and
// imaginary planes in shared memory and multiplied out in registers.  Every
// row of Lhat is computed by one thread in a fixed order and the gather sums
// each target's rows in list order: deterministic, no atomics.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bem_internal.cuh"

namespace bem {

namespace {

constexpr int SY_T = 256;           // threads: 16 row groups x 16 pair groups
constexpr int SY_M = 128;           // pairs per tile
constexpr int SY_KA = 16;           // columns a per staged chunk
constexpr int SY_MS = SY_M + 4;     // row stride of the staged moments (16-byte rows, 2-way store conflicts)

template <class R, int C> struct SyShape;   // rows per thread
template <> struct SyShape<float, 1> { static constexpr int RB = 8; };
template <> struct SyShape<float, 2> { static constexpr int RB = 4; };
template <> struct SyShape<double, 1> { static constexpr int RB = 4; };
template <> struct SyShape<double, 2> { static constexpr int RB = 2; };

struct SyArgs {
    int p, np, ldp, ntile, u0;          // rows of this run's pairs: row u - u0
    const int *tile_cls, *tile_start, *tile_cnt;
    const int *src, *sig, *pair, *dl;
    const int *ord;                     // [class][2] source and target order
    const unsigned short *fwd;          // [48][np] signed index maps (sign in bit 15)
    const int *mexp;                    // [np] exponents m | n << 8 | k << 16 | degree << 24
    const int *idx3;                    // [(p+1)^3] multi-index -> index
    const double *invf;                 // [np] 1 / a!
    const void *D;                      // [class][np][C] canonical derivatives (R)
    const void *M;                      // [box][np][C] moments (R)
    void *Lp;                           // [pair][ldp][C] canonical-frame rows (R)
    const int *skip;
};

// shared-memory layout (bytes), R arrays first so that every array is aligned
struct SyLayout {
    size_t T, Mo, D, Fa, Fb, Exp, Idx, Src, Sig, Pair, total;
};
template <class R, int C>
__host__ __device__ inline SyLayout sy_layout(int np, int p) {
    constexpr int BB = 16 * SyShape<R, C>::RB;
    SyLayout L;
    L.T = 0;
    L.Mo = L.T + sizeof(R) * C * SY_KA * BB;
    L.D = L.Mo + sizeof(R) * C * SY_KA * SY_MS;
    L.Fa = L.D + sizeof(R) * C * np;
    L.Fb = L.Fa + sizeof(R) * np;
    L.Exp = ((L.Fb + sizeof(R) * np + 15) / 16) * 16;
    L.Idx = L.Exp + sizeof(int) * np;
    L.Src = ((L.Idx + sizeof(short) * (p + 1) * (p + 1) * (p + 1) + 15) / 16) * 16;
    L.Sig = L.Src + sizeof(int) * SY_M;
    L.Pair = L.Sig + sizeof(int) * SY_M;
    L.total = L.Pair + sizeof(int) * SY_M;
    return L;
}

template <class R, int N>
__device__ __forceinline__ void lds_vec(const R *p, R (&v)[N]) {
    if constexpr (sizeof(R) == 4 && N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N / 4; i++) {
            const float4 x = reinterpret_cast<const float4 *>(p)[i];
            v[4 * i] = x.x; v[4 * i + 1] = x.y; v[4 * i + 2] = x.z; v[4 * i + 3] = x.w;
        }
    } else if constexpr (sizeof(R) == 8 && N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N / 2; i++) {
            const double2 x = reinterpret_cast<const double2 *>(p)[i];
            v[2 * i] = x.x; v[2 * i + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; i++) v[i] = p[i];
    }
}

// number of multi-indices of degree <= q
__device__ __forceinline__ int n_upto(int q) { return q < 0 ? 0 : (q + 1) * (q + 2) * (q + 3) / 6; }

template <class R, int C>
__global__ void __launch_bounds__(SY_T) k_m2l_sy(const __grid_constant__ SyArgs a) {
    if (a.skip && *a.skip) return;
    constexpr int RB = SyShape<R, C>::RB, BB = 16 * RB;
    extern __shared__ __align__(16) unsigned char smem[];
    const int np = a.np, p = a.p, P1 = p + 1, tid = threadIdx.x;
    const int tp = tid & 15, tb = tid >> 4;
    const SyLayout LY = sy_layout<R, C>(np, p);
    R *sT = (R *)(smem + LY.T);          // [C][SY_KA][BB]
    R *sMo = (R *)(smem + LY.Mo);        // [C][SY_KA][SY_MS]
    R *sD = (R *)(smem + LY.D);          // [np][C]
    R *sFa = (R *)(smem + LY.Fa);        // [np] (-1)^|a| 2^(dl |a|) / a!
    R *sFb = (R *)(smem + LY.Fb);        // [np] 1 / b!
    int *sExp = (int *)(smem + LY.Exp);
    short *sIdx = (short *)(smem + LY.Idx);
    int *sSrc = (int *)(smem + LY.Src), *sSig = (int *)(smem + LY.Sig), *sPair = (int *)(smem + LY.Pair);
    const R *Dg = (const R *)a.D, *Mg = (const R *)a.M;
    R *Lp = (R *)a.Lp;
    for (int i = tid; i < np; i += SY_T) {
        sExp[i] = a.mexp[i];
        sFb[i] = (R)a.invf[i];
    }
    for (int i = tid; i < P1 * P1 * P1; i += SY_T) sIdx[i] = (short)a.idx3[i];
    // contiguous runs of tiles (tiles are in class order), so the class tables
    // are reloaded only when the class changes
    const int t_begin = (int)((long long)a.ntile * blockIdx.x / gridDim.x);
    const int t_end = (int)((long long)a.ntile * (blockIdx.x + 1) / gridDim.x);
    int prev_cls = -1, prev_dl = 1 << 30;
    for (int tile = t_begin; tile < t_end; tile++) {
        const int cls = a.tile_cls[tile], st = a.tile_start[tile], cnt = a.tile_cnt[tile];
        __syncthreads();                                  // the previous tile is done with the tables
        if (tid < SY_M) {
            const bool v = tid < cnt;
            sSrc[tid] = v ? a.src[st + tid] : -1;
            sSig[tid] = v ? a.sig[st + tid] * np : 0;
            sPair[tid] = v ? a.pair[st + tid] : -1;
        }
        if (cls != prev_cls) {
            for (int i = tid; i < np * C; i += SY_T) sD[i] = Dg[(size_t)cls * np * C + i];
            const int dl = a.dl[cls];
            if (dl != prev_dl)
                for (int i = tid; i < np; i += SY_T) {
                    const int dg = a.mexp[i] >> 24;
                    sFa[i] = (R)(((dg & 1) ? -1.0 : 1.0) * ldexp(a.invf[i], dl * dg));
                }
            prev_cls = cls;
            prev_dl = dl;
        }
        __syncthreads();
        // orders of the class: moments |a| <= ps, locals |b| <= pt, |a| + |b| <= max(ps, pt)
        const int ps = a.ord[2 * cls], pt = a.ord[2 * cls + 1], pm = max(ps, pt);
        const int nps = n_upto(ps), npt = n_upto(pt);
        for (int b0 = 0; b0 < npt; b0 += BB) {
            // columns needed by the chunk (its first row has the lowest degree)
            // and by this thread's rows; products beyond them are zero
            const int kext = min(nps, n_upto(pm - (sExp[b0] >> 24)));
            const int kthr = b0 + tb * RB < npt ? min(nps, n_upto(pm - (sExp[b0 + tb * RB] >> 24))) : 0;
            R acc[RB][8][C];
#pragma unroll
            for (int r = 0; r < RB; r++)
#pragma unroll
                for (int q = 0; q < 8; q++)
#pragma unroll
                    for (int c = 0; c < C; c++) acc[r][q][c] = (R)0;
            // moment chunks are gathered one chunk ahead into registers, so
            // their loads are in flight while the previous chunk is multiplied:
            // element i of this thread is pair j = tid / SY_KA + 16 i, column
            // k = tid % SY_KA of the chunk; Mhat[k][j] = sign * M[src_j][a o pi_j]
            constexpr int NG = SY_KA * SY_M / SY_T;   // 8
            R pre[NG][C];
            auto gather = [&](int k0g) {
                const int k = tid % SY_KA, ai = k0g + k;
#pragma unroll
                for (int i = 0; i < NG; i++) {
                    const int j = tid / SY_KA + (SY_T / SY_KA) * i, s = sSrc[j];
#pragma unroll
                    for (int c = 0; c < C; c++) pre[i][c] = (R)0;
                    if (s >= 0 && ai < kext) {
                        const unsigned f = __ldg(a.fwd + sSig[j] + ai);
                        const R *src = Mg + ((size_t)s * np + (f & 0x7fffu)) * C;
#pragma unroll
                        for (int c = 0; c < C; c++) pre[i][c] = (f & 0x8000u) ? -__ldg(src + c) : __ldg(src + c);
                    }
                }
            };
            gather(0);
            for (int k0 = 0; k0 < kext; k0 += SY_KA) {
                __syncthreads();                          // the previous chunk is consumed
                // class matrix chunk: T[k][bl] = Dhat[a + b] fa fb
                for (int e = tid; e < SY_KA * BB; e += SY_T) {
                    const int k = e / BB, bl = e - k * BB, ai = k0 + k, b = b0 + bl;
                    R v[C];
#pragma unroll
                    for (int c = 0; c < C; c++) v[c] = (R)0;
                    if (ai < kext && b < npt) {
                        const int ea = sExp[ai], eb = sExp[b];
                        if ((ea >> 24) + (eb >> 24) <= pm) {
                            const int m = (ea & 0xff) + (eb & 0xff), n = ((ea >> 8) & 0xff) + ((eb >> 8) & 0xff),
                                      kk = ((ea >> 16) & 0xff) + ((eb >> 16) & 0xff);
                            const int g = sIdx[(m * P1 + n) * P1 + kk];
                            const R f = sFa[ai] * sFb[b];
#pragma unroll
                            for (int c = 0; c < C; c++) v[c] = sD[g * C + c] * f;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < C; c++) sT[(c * SY_KA + k) * BB + bl] = v[c];
                }
                {
                    const int k = tid % SY_KA;
#pragma unroll
                    for (int i = 0; i < NG; i++) {
                        const int j = tid / SY_KA + (SY_T / SY_KA) * i;
#pragma unroll
                        for (int c = 0; c < C; c++) sMo[(c * SY_KA + k) * SY_MS + j] = pre[i][c];
                    }
                }
                if (k0 + SY_KA < kext) gather(k0 + SY_KA);
                __syncthreads();
                const int kn = min(SY_KA, kthr - k0);
                for (int k = 0; k < kn; k++) {
                    R t[C][RB], m[C][8];
#pragma unroll
                    for (int c = 0; c < C; c++) {
                        lds_vec<R, RB>(sT + (c * SY_KA + k) * BB + tb * RB, t[c]);
                        R lo[4], hi[4];
                        lds_vec<R, 4>(sMo + (c * SY_KA + k) * SY_MS + tp * 4, lo);
                        lds_vec<R, 4>(sMo + (c * SY_KA + k) * SY_MS + 64 + tp * 4, hi);
#pragma unroll
                        for (int i = 0; i < 4; i++) { m[c][i] = lo[i]; m[c][4 + i] = hi[i]; }
                    }
#pragma unroll
                    for (int r = 0; r < RB; r++)
#pragma unroll
                        for (int q = 0; q < 8; q++) {
                            if (C == 1) {
                                acc[r][q][0] += t[0][r] * m[0][q];
                            } else {
                                acc[r][q][0] += t[0][r] * m[0][q];
                                acc[r][q][0] -= t[C - 1][r] * m[C - 1][q];
                                acc[r][q][C - 1] += t[0][r] * m[C - 1][q];
                                acc[r][q][C - 1] += t[C - 1][r] * m[0][q];
                            }
                        }
                }
            }
            // rows of this chunk, pair by pair
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int j = tp * 4 + 64 * (q >> 2) + (q & 3);
                const int u = sPair[j];
                if (u < 0) continue;
                R *row = Lp + ((size_t)(u - a.u0) * a.ldp + b0 + tb * RB) * C;
#pragma unroll
                for (int r = 0; r < RB; r++)
                    if (b0 + tb * RB + r < npt)
#pragma unroll
                        for (int c = 0; c < C; c++) row[r * C + c] = acc[r][q][c];
            }
        }
    }
}

// L_t[b] = (1 / h_t) sum over t's interaction list, in list order, of
// sign * Lhat_u[b o pi_u^-1]
constexpr int SG_LIST = 256;
template <class R, int C>
__global__ void __launch_bounds__(256) k_m2l_gather_sy(int t0, int nbox, const int *__restrict__ level, double side,
                                                       const int *__restrict__ lev_p, const int *__restrict__ inter_ptr,
                                                       int u0r, int np, int ldp,
                                                       const int *__restrict__ sig_u, const int *__restrict__ inv,
                                                       const R *__restrict__ Lp, R *__restrict__ L,
                                                       const int *__restrict__ skip) {
    if (skip && *skip) return;
    __shared__ int sOff[SG_LIST];
    const int t = t0 + blockIdx.x;
    if (t >= nbox) return;
    const R sc = (R)(1.0 / scalbn(side, -level[t]));
    const int u0 = inter_ptr[t], u1 = inter_ptr[t + 1];
    const int npt = lev_p ? n_upto(lev_p[level[t]]) : np;   // the target's own coefficients
    for (int b0 = 0; b0 < npt; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        R sum[C];
#pragma unroll
        for (int c = 0; c < C; c++) sum[c] = (R)0;
        for (int base = u0; base < u1; base += SG_LIST) {
            const int n = min(SG_LIST, u1 - base);
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) sOff[i] = sig_u[base + i] * np;
            __syncthreads();
            if (b < npt) {
                int i = 0;
                for (; i + 4 <= n; i += 4) {
                    int f[4];
                    R v[4][C];
#pragma unroll
                    for (int q = 0; q < 4; q++) f[q] = __ldg(inv + sOff[i + q] + b);
#pragma unroll
                    for (int q = 0; q < 4; q++)
#pragma unroll
                        for (int c = 0; c < C; c++)
                            v[q][c] = Lp[((size_t)(base + i + q - u0r) * ldp + (f[q] & 0x7fffffff)) * C + c];
#pragma unroll
                    for (int q = 0; q < 4; q++)
#pragma unroll
                        for (int c = 0; c < C; c++) sum[c] += f[q] < 0 ? -v[q][c] : v[q][c];
                }
                for (; i < n; i++) {
                    const int f = __ldg(inv + sOff[i] + b);
#pragma unroll
                    for (int c = 0; c < C; c++) {
                        const R v = Lp[((size_t)(base + i - u0r) * ldp + (f & 0x7fffffff)) * C + c];
                        sum[c] += f < 0 ? -v : v;
                    }
                }
            }
        }
        if (b < npt)
#pragma unroll
            for (int c = 0; c < C; c++) L[((size_t)t * np + b) * C + c] = sum[c] * sc;
    }
}


}  // namespace

size_t sy_simt_smem_bytes(int prec_float, int C, int np, int p) {
    if (prec_float) return C == 1 ? sy_layout<float, 1>(np, p).total : sy_layout<float, 2>(np, p).total;
    return C == 1 ? sy_layout<double, 1>(np, p).total : sy_layout<double, 2>(np, p).total;
}

template <class R, int C>
int launch_m2l_sy(bem_plan *P, const R *M, R *L, cudaStream_t s) {
    const Tree &t = P->t;
    SyArgs a{};
    a.p = P->mi.p;
    a.np = P->mi.np;
    a.ldp = P->sy_ldp;
    a.src = P->sy_src;
    a.sig = P->sy_sig;
    a.pair = P->sy_pair;
    a.dl = P->sy_dl;
    a.ord = P->sy_ord;
    a.fwd = P->sy_fwd;
    a.mexp = P->sy_mexp;
    a.idx3 = P->d_idx3;
    a.invf = P->sy_invf;
    a.D = sizeof(R) == 4 ? (const void *)P->sy_fD : (const void *)P->sy_D;
    a.M = M;
    a.Lp = P->sy_Lp;
    a.skip = P->skip;
    const size_t sm = sy_layout<R, C>(a.np, a.p).total;
    // one run of targets at a time: its tiles, then the gather of its targets;
    // enough blocks to fill the device twice over, each on a contiguous run of tiles
    for (size_t r = 0; r + 1 < P->sy_bt.size(); r++) {
        const int bt0 = P->sy_bt[r], nt = P->sy_bt[r + 1] - bt0, tg0 = P->sy_bb[r], ntg = P->sy_bb[r + 1] - tg0;
        a.ntile = nt;
        a.tile_cls = P->sy_tile_cls + bt0;
        a.tile_start = P->sy_tile_start + bt0;
        a.tile_cnt = P->sy_tile_cnt + bt0;
        a.u0 = P->sy_bu[r];
        if (nt > 0)
            (k_m2l_sy<R, C><<<std::min(nt, 2 * std::max(1, P->sm_count)), SY_T, sm, s>>>(a), ::bem::count_launch());
        if (ntg > 0)
            (k_m2l_gather_sy<R, C><<<ntg, 256, 0, s>>>(tg0, t.nbox, t.level, t.side, P->lev_var ? P->d_lev_p : nullptr,
                                                       t.inter_ptr, a.u0, a.np, a.ldp,
                                                       P->sy_sig_u, P->sy_inv, (const R *)P->sy_Lp, L, P->skip),
             ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    return BEM_OK;
}

void set_sy_attributes() {
    const int big = 200 * 1024;
    cudaFuncSetAttribute(k_m2l_sy<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_sy<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_sy<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_sy<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

template int launch_m2l_sy<float, 1>(bem_plan *, const float *, float *, cudaStream_t);
template int launch_m2l_sy<float, 2>(bem_plan *, const float *, float *, cudaStream_t);
template int launch_m2l_sy<double, 1>(bem_plan *, const double *, double *, cudaStream_t);
template int launch_m2l_sy<double, 2>(bem_plan *, const double *, double *, cudaStream_t);

}  // namespace bem
