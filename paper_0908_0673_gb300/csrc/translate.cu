// Translation operators of the fast method:
//
//   M2M  coefficient shift (Eq. 8):  Ms'_a = sum_{b<=a} C(a,b) s^b 2^-(|a|+|b|) Ms_{a-b}
//   L2L  expansion shift (Eq. 9):    Ls'_b += sum_g C(b+g,b) s^g 2^-(2|g|+|b|) Ls_{b+g}
//   M2L  local expansion (Eq. 7):    Ls_t[b] = 1/(h_t b!) sum_a D[a+b] (-1)^|a| (h_s/h_t)^|a| Ms_s[a] / a!
//
// Moments / locals are scaled by the box edge (Ms = I / h^|a|, Ls = F h^|b|),
// so a child's offset from its parent is +-1/4 of the parent edge per axis and
// every shift coefficient is a product of per-axis binomials and powers of
// two; the octant only flips signs.
//
// M2L: the derivatives D[g] = d^g Ghat(rho) (Tausch's recursions, Section
// 3.3) depend only on rho = (c_t - c_s) / h_t, the level difference and, for
// Helmholtz, k h_t.  Boxes sit on dyadic lattices, so every interaction pair
// falls into one of a small number of exact offset classes; one FP64 table of
// derivatives per class is built at set-up, and the per-pair work is the
// contraction alone, walked through a precomputed (a, a+b) list per b.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <map>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "bem_internal.cuh"

namespace bem {

constexpr int TT = 128;                   // threads per block of the translation kernels
constexpr int TSLOTS = (969 + TT - 1) / TT;

template <class R, int C>
__device__ __forceinline__ void cmac(R *acc, R cf, const R *v) {
#pragma unroll
    for (int c = 0; c < C; c++) acc[c] += cf * v[c];
}

// ---------------------------------------------------------------------------
// Shifts as three one-dimensional passes.  With box-scaled expansions every
// shift coefficient is a product of per-axis factors,
//   M2M  M'_a = 2^-|a| sum_{g <= a} prod_i binom(a_i, g_i) 2^-g_i s_i^g_i  M_{a-g},
//   L2L  L'_b = 2^-|b| sum_{|b|+|g| <= p} prod_i binom(b_i+g_i, b_i) 4^-g_i s_i^g_i  L_{b+g},
// (s_i = -1 where the child lies on the low side of axis i), so each shift is
// done axis by axis: an output of one pass sums at most p + 1 terms, and the
// degree bound |.| <= p carries through the passes unchanged.  Multi-index
// table and per-axis factors sit in shared memory.  M2M: every child of the
// parent at once, children then added in a fixed order; L2L: one child per
// block.  Deterministic.
// ---------------------------------------------------------------------------
constexpr int MM_T = 512;

template <class R>
__device__ __forceinline__ void shift_tables(int p, const int *__restrict__ idx3, const double *__restrict__ binom,
                                             bool m2m, short *sIdx, R *sG) {
    const int P1 = p + 1;
    for (int i = threadIdx.x; i < P1 * P1 * P1; i += blockDim.x) sIdx[i] = (short)idx3[i];
    for (int i = threadIdx.x; i < P1 * P1; i += blockDim.x) {
        const int a = i / P1, g = i - a * P1;
        // M2M: binom(a, g) 2^-g (g <= a);  L2L: binom(a + g, a) 4^-g (a + g <= p)
        double v = 0.0;
        if (m2m && g <= a) v = ldexp(binom[a * (PMAX + 1) + g], -g);
        if (!m2m && a + g <= p) v = ldexp(binom[(a + g) * (PMAX + 1) + a], -2 * g);
        sG[i] = (R)v;
    }
}

// one axis pass over nv vectors: out[v][a] = sum_g G[a_ax][g] s_v^g in[v][a -/+ g e_ax]
template <class R, int C, bool DOWN>
__device__ __forceinline__ void shift_pass(int ax, int nv, int p, int np, const int *__restrict__ tm,
                                           const int *__restrict__ tn, const int *__restrict__ tk, const short *sIdx,
                                           const R *sG, const int *smask, const R *in, R *out) {
    const int P1 = p + 1;
    for (int t = threadIdx.x; t < nv * np; t += blockDim.x) {
        const int v = t / np, a = t - v * np;
        int c3[3] = {tm[a], tn[a], tk[a]};
        const int e = c3[ax], rest = p - (c3[0] + c3[1] + c3[2]);
        const R sg = (smask[v] >> ax) & 1 ? (R)-1 : (R)1;
        const R *iv = in + (size_t)v * np * C;
        R acc[C];
#pragma unroll
        for (int c = 0; c < C; c++) acc[c] = (R)0;
        R gs = (R)1;
        const int ng = DOWN ? e : rest;          // M2M: g <= a_ax;  L2L: |a| + g <= p
        for (int g = 0; g <= ng; g++, gs *= sg) {
            c3[ax] = DOWN ? e - g : e + g;
            const int src = sIdx[(c3[0] * P1 + c3[1]) * P1 + c3[2]];
            cmac<R, C>(acc, gs * sG[e * P1 + g], iv + src * C);
        }
#pragma unroll
        for (int c = 0; c < C; c++) out[((size_t)v * np + a) * C + c] = acc[c];
    }
}

template <class R, int C>
__global__ void __launch_bounds__(MM_T) k_m2m_sep(int off, int cnt, const int *__restrict__ child0,
                                                  const int *__restrict__ nchild, const int *__restrict__ ix,
                                                  const int *__restrict__ iy, const int *__restrict__ iz, int p, int np,
                                                  int grp, const int *__restrict__ tm, const int *__restrict__ tn,
                                                  const int *__restrict__ tk, const int *__restrict__ idx3,
                                                  const double *__restrict__ binom, R *__restrict__ M,
                                                  const int *__restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    const int P1 = p + 1;
    R *sA = (R *)smem_raw;                                  // [grp][np][C]
    R *sB = sA + (size_t)grp * np * C;                       // [grp][np][C]
    R *sS = sB + (size_t)grp * np * C;                       // [np][C] sum over children
    R *sG = sS + (size_t)np * C;                             // [P1][P1]
    short *sIdx = (short *)(sG + P1 * P1);                   // [P1^3]
    __shared__ int smask[8];
    if (blockIdx.x >= cnt) return;
    const int b = off + blockIdx.x, nch = nchild[b];
    if (nch == 0) return;
    const int c0 = child0[b], tid = threadIdx.x;
    shift_tables<R>(p, idx3, binom, true, sIdx, sG);
    for (int g0 = 0; g0 < nch; g0 += grp) {
        const int ng = min(grp, nch - g0);
        __syncthreads();
        for (int t = tid; t < ng * np * C; t += MM_T) sA[t] = M[(size_t)(c0 + g0) * np * C + t];   // consecutive
        // a child on the low side of an axis has offset -1/4 of the parent edge
        if (tid < ng) {
            const int c = c0 + g0 + tid;
            smask[tid] = ((ix[c] & 1) ? 0 : 1) | ((iy[c] & 1) ? 0 : 2) | ((iz[c] & 1) ? 0 : 4);
        }
        __syncthreads();
        shift_pass<R, C, true>(0, ng, p, np, tm, tn, tk, sIdx, sG, smask, sA, sB);
        __syncthreads();
        shift_pass<R, C, true>(1, ng, p, np, tm, tn, tk, sIdx, sG, smask, sB, sA);
        __syncthreads();
        shift_pass<R, C, true>(2, ng, p, np, tm, tn, tk, sIdx, sG, smask, sA, sB);
        __syncthreads();
        for (int t = tid; t < np * C; t += MM_T) {
            R sum = g0 == 0 ? (R)0 : sS[t];
            for (int j = 0; j < ng; j++) sum += sB[(size_t)j * np * C + t];
            sS[t] = sum;
        }
    }
    __syncthreads();
    for (int a = tid; a < np; a += MM_T) {
        const R sc = (R)ldexp(1.0, -(tm[a] + tn[a] + tk[a]));
#pragma unroll
        for (int c = 0; c < C; c++) M[((size_t)b * np + a) * C + c] = sS[(size_t)a * C + c] * sc;
    }
}

template <class R, int C>
__global__ void __launch_bounds__(MM_T) k_l2l_sep(int off, int cnt, const int *__restrict__ parent,
                                                  const int *__restrict__ ix, const int *__restrict__ iy,
                                                  const int *__restrict__ iz, int p, int np, const int *__restrict__ tm,
                                                  const int *__restrict__ tn, const int *__restrict__ tk,
                                                  const int *__restrict__ idx3, const double *__restrict__ binom,
                                                  R *__restrict__ L, const int *__restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    const int P1 = p + 1;
    R *sA = (R *)smem_raw;                                  // [np][C]
    R *sB = sA + (size_t)np * C;                             // [np][C]
    R *sG = sB + (size_t)np * C;                             // [P1][P1]
    short *sIdx = (short *)(sG + P1 * P1);                   // [P1^3]
    __shared__ int smask[1];
    if (blockIdx.x >= cnt) return;
    const int b = off + blockIdx.x, pa = parent[b], tid = threadIdx.x;
    for (int t = tid; t < np * C; t += MM_T) sA[t] = L[(size_t)pa * np * C + t];
    shift_tables<R>(p, idx3, binom, false, sIdx, sG);
    if (tid == 0) smask[0] = ((ix[b] & 1) ? 0 : 1) | ((iy[b] & 1) ? 0 : 2) | ((iz[b] & 1) ? 0 : 4);
    __syncthreads();
    shift_pass<R, C, false>(2, 1, p, np, tm, tn, tk, sIdx, sG, smask, sA, sB);
    __syncthreads();
    shift_pass<R, C, false>(1, 1, p, np, tm, tn, tk, sIdx, sG, smask, sB, sA);
    __syncthreads();
    shift_pass<R, C, false>(0, 1, p, np, tm, tn, tk, sIdx, sG, smask, sA, sB);
    __syncthreads();
    for (int a = tid; a < np; a += MM_T) {
        const R sc = (R)ldexp(1.0, -(tm[a] + tn[a] + tk[a]));
#pragma unroll
        for (int c = 0; c < C; c++) L[((size_t)b * np + a) * C + c] += sB[(size_t)a * C + c] * sc;
    }
}

// ---------------------------------------------------------------------------
// M2L derivative tables, one block per offset class (FP64)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TT) k_m2l_tables(int ncls, int p, int np, int C, const int *__restrict__ tm,
                                                   const int *__restrict__ tn, const int *__restrict__ tk,
                                                   const int *__restrict__ idx3, const double *__restrict__ rho,
                                                   const double *__restrict__ kh, double *__restrict__ D,
                                                   float *__restrict__ Df) {
    extern __shared__ unsigned char smem_raw[];
    const int cls = blockIdx.x, tid = threadIdx.x, P1 = p + 1;
    if (cls >= ncls) return;
    double *Gh = (double *)smem_raw;             // [(p+2)][2]
    double *up = Gh + 2 * (p + 2), *cur = up + 2 * np;
    const double rx = rho[3 * cls], ry = rho[3 * cls + 1], rz = rho[3 * cls + 2];
    if (tid == 0) {
        // G^(h) = (R^-1 d/dR)^h Ghat at |rho|; Laplace: G^(h+1) = -(2h+1) G^(h) / R^2;
        // Helmholtz adds -khat^2 G^(h-1) / R^2 with G^(-1) = -j e^{j khat R} / (4 pi khat)
        const double r2 = rx * rx + ry * ry + rz * rz, r1 = sqrt(r2), inv4pi = 0.25 / M_PI;
        if (C == 1) {
            double g = inv4pi / r1;
            for (int h = 0; h <= p; h++) {
                Gh[2 * h] = g;
                Gh[2 * h + 1] = 0.0;
                g = -(2.0 * h + 1.0) * g / r2;
            }
        } else {
            const double k = kh[cls];
            double sn, cs;
            sincos(k * r1, &sn, &cs);
            double pr = sn * inv4pi / k, pi = -cs * inv4pi / k, cr = cs * inv4pi / r1, ci = sn * inv4pi / r1;
            for (int h = 0; h <= p; h++) {
                Gh[2 * h] = cr;
                Gh[2 * h + 1] = ci;
                const double nr = -((2.0 * h + 1.0) * cr + k * k * pr) / r2;
                const double ni = -((2.0 * h + 1.0) * ci + k * k * pi) / r2;
                pr = cr; pi = ci; cr = nr; ci = ni;
            }
        }
        up[0] = Gh[2 * p];
        up[1] = Gh[2 * p + 1];
    }
    __syncthreads();
    const double rr[3] = {rx, ry, rz};
    for (int h = p - 1; h >= 0; h--) {
        const int top = p - h, n = (top + 1) * (top + 2) * (top + 3) / 6;
        for (int u = tid; u < n; u += TT) {
            const int m = tm[u], nn = tn[u], k = tk[u];
            double v0, v1;
            if (m + nn + k == 0) {
                v0 = Gh[2 * h];
                v1 = Gh[2 * h + 1];
            } else {
                const int ax = m > 0 ? 0 : (nn > 0 ? 1 : 2);
                const int g = ax == 0 ? m : (ax == 1 ? nn : k);
                const int m1 = m - (ax == 0), n1 = nn - (ax == 1), k1 = k - (ax == 2);
                const int i1 = idx3[(m1 * P1 + n1) * P1 + k1];
                v0 = rr[ax] * up[2 * i1];
                v1 = rr[ax] * up[2 * i1 + 1];
                if (g > 1) {
                    const int i2 = idx3[((m1 - (ax == 0)) * P1 + (n1 - (ax == 1))) * P1 + (k1 - (ax == 2))];
                    v0 += (g - 1) * up[2 * i2];
                    v1 += (g - 1) * up[2 * i2 + 1];
                }
            }
            cur[2 * u] = v0;
            cur[2 * u + 1] = v1;
        }
        __syncthreads();
        double *sw = up; up = cur; cur = sw;
        __syncthreads();
    }
    for (int u = tid; u < np; u += TT)
        for (int c = 0; c < C; c++) {
            const double v = up[2 * u + c];
            D[((size_t)cls * np + u) * C + c] = v;
            if (Df) Df[((size_t)cls * np + u) * C + c] = (float)v;
        }
}

// ---------------------------------------------------------------------------
// M2L contraction: one block per target box
// ---------------------------------------------------------------------------
template <class R, int C>
__device__ __forceinline__ void cmul_add(R *acc, const R *d, const R *m) {
    if (C == 1) {
        acc[0] += d[0] * m[0];
    } else {
        acc[0] += d[0] * m[0] - d[1] * m[1];
        acc[C - 1] += d[0] * m[1] + d[1] * m[0];
    }
}

template <class R, int C>
__global__ void __launch_bounds__(TT) k_m2l_tab(int nbox, const int *__restrict__ level, double side,
                                                const int *__restrict__ inter_ptr, const int *__restrict__ inter_idx,
                                                const int *__restrict__ cls, const int *__restrict__ cls_dl, int np,
                                                const int *__restrict__ deg, const double *__restrict__ sgn_fact,
                                                const double *__restrict__ inv_fact, const int *__restrict__ cptr,
                                                const int *__restrict__ cag, const int *__restrict__ beta_of,
                                                const R *__restrict__ D, const R *__restrict__ M, R *__restrict__ L,
                                                const int *__restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    const int t = blockIdx.x, tid = threadIdx.x;
    if (t >= nbox) return;
    R *sD = (R *)smem_raw, *sm = sD + np * C;
    int bs[TSLOTS];
#pragma unroll
    for (int s = 0; s < TSLOTS; s++) bs[s] = beta_of[tid * TSLOTS + s];
    R acc[TSLOTS][C];
#pragma unroll
    for (int s = 0; s < TSLOTS; s++)
#pragma unroll
        for (int c = 0; c < C; c++) acc[s][c] = (R)0;
    for (int it = inter_ptr[t]; it < inter_ptr[t + 1]; it++) {
        const int src = inter_idx[it], cl = cls[it], dl = cls_dl[cl];
        __syncthreads();
        for (int u = tid; u < np * C; u += TT) sD[u] = D[(size_t)cl * np * C + u];
        for (int u = tid; u < np; u += TT) {
            const R f = (R)(sgn_fact[u] * scalbn(1.0, dl * deg[u]));
#pragma unroll
            for (int c = 0; c < C; c++) sm[u * C + c] = f * M[((size_t)src * np + u) * C + c];
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < TSLOTS; s++) {
            const int b = bs[s];
            if (b < 0) continue;
            for (int k = cptr[b]; k < cptr[b + 1]; k++) {
                const int ag = cag[k];
                cmul_add<R, C>(acc[s], sD + (ag >> 16) * C, sm + (ag & 0xffff) * C);
            }
        }
    }
    const double ht = scalbn(side, -level[t]);
#pragma unroll
    for (int s = 0; s < TSLOTS; s++) {
        const int b = bs[s];
        if (b < 0) continue;
        const R sc = (R)(inv_fact[b] / ht);
#pragma unroll
        for (int c = 0; c < C; c++) L[((size_t)t * np + b) * C + c] = acc[s][c] * sc;
    }
}


// ---------------------------------------------------------------------------
// M2L, float32 class-major form.  Interaction pairs are grouped by offset
// class (a class holds ~36 pairs on average; the radius-based separation
// makes the classes many and small).  A tile = up to CM_N pairs of one class.
// The block expands the class's derivative table into the matrix
// A[b][a] = D[a+b] (-1)^|a| 2^(dl|a|) / (a! b!) (zero where |a| + |b| > p),
// stored as equal 4 x 8 units (degree-sorted rows b and columns a) through a
// precomputed index table, multiplies it by the tile's source moments (one
// unit per thread, accumulators in registers), and writes one row per pair
// in target-major pair order.  k_m2l_gather then sums each target's rows in
// list order and scales by 1 / h_t: no atomics, deterministic.
// ---------------------------------------------------------------------------
constexpr int CM_N = 16, CM_T = 512, CM_UR = 4, CM_UA = 8;

__global__ void __launch_bounds__(CM_T) k_m2l_cm(int ntile, const int *__restrict__ tile_cls,
                                                 const int *__restrict__ tile_start, const int *__restrict__ tile_cnt,
                                                 const int *__restrict__ order, const int *__restrict__ inter_idx,
                                                 const int *__restrict__ cls_dl, int np, int nunits, int nrt,
                                                 const int *__restrict__ ur0, const int *__restrict__ ua0,
                                                 const int *__restrict__ rt_ptr, const int *__restrict__ gidx,
                                                 const int *__restrict__ deg, const double *__restrict__ sgnf,
                                                 const double *__restrict__ invf, const float *__restrict__ fD,
                                                 const float *__restrict__ M, float *__restrict__ Lp,
                                                 const int *__restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    const int npad = ((np + CM_UA - 1) / CM_UA) * CM_UA, NE = nunits * CM_UR * CM_UA;
    // float arrays first: sB (read as float4) starts the buffer, 16-byte aligned,
    // and every float array before an int table has a length divisible by 4
    float *sB = (float *)smem_raw;                              // [npad][CM_N]
    float *sOut = sB + (size_t)npad * CM_N;                     // [nunits][4][CM_N]
    float *sA = sOut + (size_t)nunits * CM_UR * CM_N;           // [NE]
    float *sD = sA + NE;                                        // [npad]
    float *sCol = sD + npad;                                    // [npad]
    float *sRow = sCol + npad;                                  // [npad] 1 / b!
    int *tG = (int *)(sRow + npad);                             // [NE] derivative index of every unit entry
    int *tA0 = tG + NE, *tR0 = tA0 + nunits, *tRT = tR0 + nunits;   // [nunits], [nunits], [nrt+1]
    int *tSrc = tRT + (nrt + 1);                                // [CM_N] sources of the current tile
    int *tDeg = tSrc + CM_N;                                    // [npad]
    const int tid = threadIdx.x;
    for (int i = tid; i < NE; i += CM_T) tG[i] = gidx[i];
    for (int i = tid; i < nunits; i += CM_T) { tA0[i] = ua0[i]; tR0[i] = ur0[i]; }
    for (int i = tid; i <= nrt; i += CM_T) tRT[i] = rt_ptr[i];
    for (int i = tid; i < npad; i += CM_T) {
        tDeg[i] = i < np ? deg[i] : 0;
        sRow[i] = i < np ? (float)invf[i] : 0.f;
    }
    for (int i = tid; i < npad * CM_N; i += CM_T) sB[i] = 0.f;     // rows >= np stay zero
    // each block takes a contiguous run of tiles (tiles are ordered by class),
    // so consecutive tiles of one class reuse the class matrix in shared memory
    const int t_begin = (int)((long long)ntile * blockIdx.x / gridDim.x);
    const int t_end = (int)((long long)ntile * (blockIdx.x + 1) / gridDim.x);
    int prev_cls = -1;
    for (int tile = t_begin; tile < t_end; tile++) {
        const int cl = tile_cls[tile], st = tile_start[tile], cnt = tile_cnt[tile], dl = cls_dl[cl];
        const bool same = cl == prev_cls;
        prev_cls = cl;
        __syncthreads();
        if (tid < CM_N) tSrc[tid] = tid < cnt ? inter_idx[order[st + tid]] : -1;
        if (!same)
            for (int i = tid; i < npad; i += CM_T) {
                sD[i] = i < np ? fD[(size_t)cl * np + i] : 0.f;
                sCol[i] = i < np ? ldexpf((float)sgnf[i], dl * tDeg[i]) : 0.f;   // exact power of two
            }
        __syncthreads();
        for (int a = tid; a < np; a += CM_T) {
            float v[CM_N];
#pragma unroll
            for (int j = 0; j < CM_N; j++) v[j] = tSrc[j] >= 0 ? M[(size_t)tSrc[j] * np + a] : 0.f;
#pragma unroll
            for (int j = 0; j < CM_N; j++) sB[a * CM_N + j] = v[j];
        }
        if (!same)
            for (int e = tid; e < NE; e += CM_T) {
                const int g = tG[e];
                float v = 0.f;
                if (g >= 0) {
                    const int uu = e / (CM_UR * CM_UA), rc = e - uu * (CM_UR * CM_UA);
                    const int r = rc / CM_UA, cc = rc - r * CM_UA;
                    v = sD[g] * sCol[tA0[uu] + cc] * sRow[tR0[uu] + r];
                }
                sA[e] = v;
            }
        __syncthreads();
        const int u = tid;
        if (u < nunits) {
            float acc[CM_UR][CM_N];
#pragma unroll
            for (int r = 0; r < CM_UR; r++)
#pragma unroll
                for (int j = 0; j < CM_N; j++) acc[r][j] = 0.f;
            const int a0 = tA0[u];
            const float *Au = sA + (size_t)u * CM_UR * CM_UA;
#pragma unroll
            for (int c = 0; c < CM_UA; c++) {
                const float4 *bp = (const float4 *)(sB + (size_t)(a0 + c) * CM_N);
                float bv[CM_N];
#pragma unroll
                for (int q = 0; q < CM_N / 4; q++) {
                    const float4 x = bp[q];
                    bv[4 * q] = x.x; bv[4 * q + 1] = x.y; bv[4 * q + 2] = x.z; bv[4 * q + 3] = x.w;
                }
#pragma unroll
                for (int r = 0; r < CM_UR; r++) {
                    const float av = Au[r * CM_UA + c];
#pragma unroll
                    for (int j = 0; j < CM_N; j++) acc[r][j] = fmaf(av, bv[j], acc[r][j]);
                }
            }
#pragma unroll
            for (int r = 0; r < CM_UR; r++)
#pragma unroll
                for (int j = 0; j < CM_N; j++) sOut[((size_t)u * CM_UR + r) * CM_N + j] = acc[r][j];
        }
        __syncthreads();
        // per pair row b: fixed-order sum over the column units of its row tile
        for (int b = tid; b < np; b += CM_T) {
            const int rt = b / CM_UR, r = b - rt * CM_UR, u0 = tRT[rt], u1 = tRT[rt + 1];
            for (int j = 0; j < cnt; j++) {
                float sum = 0.f;
                for (int uu = u0; uu < u1; uu++) sum += sOut[((size_t)uu * CM_UR + r) * CM_N + j];
                Lp[(size_t)order[st + j] * np + b] = sum;
            }
        }
    }
}

// Ls_t[b] = (1 / h_t) sum over the interaction list of t, in list order
__global__ void k_m2l_gather(int nbox, const int *__restrict__ level, double side, const int *__restrict__ inter_ptr,
                             int np, const float *__restrict__ Lp, float *__restrict__ L, const int *__restrict__ skip) {
    if (skip && *skip) return;
    const int t = blockIdx.x;
    if (t >= nbox) return;
    const float sc = (float)(1.0 / scalbn(side, -level[t]));
    for (int b = threadIdx.x; b < np; b += blockDim.x) {
        float sum = 0.f;
        for (int u = inter_ptr[t]; u < inter_ptr[t + 1]; u++) sum += Lp[(size_t)u * np + b];
        L[(size_t)t * np + b] = sum * sc;
    }
}

// ---------------------------------------------------------------------------
// host: tables
// ---------------------------------------------------------------------------

// Offset classes of the interaction pairs (independent of the order p).
int build_m2l_classes(bem_plan *P) {
    const Tree &t = P->t;
    std::vector<int> lev(t.nbox), ix(t.nbox), iy(t.nbox), iz(t.nbox), ip(t.nbox + 1), ii(t.n_inter);
    BEM_CUDA(cudaMemcpy(lev.data(), t.level, sizeof(int) * t.nbox, cudaMemcpyDeviceToHost));
    BEM_CUDA(cudaMemcpy(ix.data(), t.ix, sizeof(int) * t.nbox, cudaMemcpyDeviceToHost));
    BEM_CUDA(cudaMemcpy(iy.data(), t.iy, sizeof(int) * t.nbox, cudaMemcpyDeviceToHost));
    BEM_CUDA(cudaMemcpy(iz.data(), t.iz, sizeof(int) * t.nbox, cudaMemcpyDeviceToHost));
    BEM_CUDA(cudaMemcpy(ip.data(), t.inter_ptr, sizeof(int) * (t.nbox + 1), cudaMemcpyDeviceToHost));
    if (t.n_inter) BEM_CUDA(cudaMemcpy(ii.data(), t.inter_idx, sizeof(int) * t.n_inter, cudaMemcpyDeviceToHost));
    const bool helm = P->green == BEM_HELMHOLTZ;
    // Class key: (dl, level for Helmholtz, K).  Offsets of interacting boxes
    // are small integers, so the key packs into 64 bits (17 bits per K
    // component, biased) and goes into a flat open-addressing table; a key
    // that does not fit the packing uses an ordered map.
    const int KB = 17;
    const long long KMAX = (1ll << (KB - 1)) - 1;
    std::vector<unsigned long long> tkey;
    std::vector<int> tval;
    size_t tmask = 1;
    while (tmask < 2 * (size_t)t.n_inter + 1024) tmask <<= 1;     // more slots than keys: probing ends
    tkey.assign(tmask, 0ull);
    tval.assign(tmask, -1);
    tmask -= 1;
    std::map<std::tuple<int, int, long long, long long, long long>, int> wide;
    std::vector<int> pair_cls(std::max<int64_t>(1, t.n_inter));
    std::vector<double> rho, kh;
    std::vector<int> dls;
    std::vector<long long> kvec;        // integer offset vector of every class
    auto new_class = [&](int b, int dl, int e, long long kx, long long ky, long long kz) {
        const int c = (int)dls.size();
        const double sc = std::ldexp(1.0, -(e + 1));
        rho.push_back(kx * sc);
        rho.push_back(ky * sc);
        rho.push_back(kz * sc);
        kh.push_back(helm ? P->k * std::ldexp(t.side, -lev[b]) : 0.0);
        dls.push_back(dl);
        kvec.push_back(kx);
        kvec.push_back(ky);
        kvec.push_back(kz);
        return c;
    };
    for (int b = 0; b < t.nbox; b++)
        for (int u = ip[b]; u < ip[b + 1]; u++) {
            const int s = ii[u], dl = lev[b] - lev[s], e = std::max(0, -dl);
            // 2 rho 2^e = (2 i_t + 1) 2^e - (2 i_s + 1) 2^(dl + e), an integer vector
            auto K = [&](int it_, int is_) {
                return (long long)(2 * it_ + 1) * (1ll << e) - (long long)(2 * is_ + 1) * (1ll << (dl + e));
            };
            const long long kx = K(ix[b], ix[s]), ky = K(iy[b], iy[s]), kz = K(iz[b], iz[s]);
            const int lv = helm ? lev[b] : 0;
            int c;
            if (std::llabs(kx) <= KMAX && std::llabs(ky) <= KMAX && std::llabs(kz) <= KMAX && dl > -64 && dl < 64) {
                const unsigned long long key =
                    1ull + (((unsigned long long)(kx + KMAX)) | ((unsigned long long)(ky + KMAX) << KB) |
                            ((unsigned long long)(kz + KMAX) << (2 * KB)) |
                            ((unsigned long long)(dl + 64) << (3 * KB)) | ((unsigned long long)lv << (3 * KB + 7)));
                size_t h = (size_t)((key * 0x9E3779B97F4A7C15ull) >> 20) & tmask;
                while (tkey[h] != 0ull && tkey[h] != key) h = (h + 1) & tmask;
                if (tkey[h] == 0ull) {
                    tkey[h] = key;
                    tval[h] = new_class(b, dl, e, kx, ky, kz);
                }
                c = tval[h];
            } else {
                auto wk = std::make_tuple(dl, lv, kx, ky, kz);
                auto it = wide.find(wk);
                if (it == wide.end()) it = wide.emplace(wk, new_class(b, dl, e, kx, ky, kz)).first;
                c = it->second;
            }
            pair_cls[u] = c;
        }
    P->m2l_ncls = (int)dls.size();
    // class-major tiles for the float32 M2L: pairs ordered by class (stable),
    // cut into tiles of at most CM_N pairs of one class
    {
        const int nc = (int)dls.size();
        std::vector<int> cstart(nc + 1, 0), order(std::max<int64_t>(1, t.n_inter));
        for (int64_t u = 0; u < t.n_inter; u++) cstart[pair_cls[u] + 1]++;
        for (int c = 0; c < nc; c++) cstart[c + 1] += cstart[c];
        std::vector<int> fill(cstart.begin(), cstart.end() - 1);
        for (int64_t u = 0; u < t.n_inter; u++) order[fill[pair_cls[u]]++] = (int)u;
        std::vector<int> tcls, tst, tcnt;
        for (int c = 0; c < nc; c++)
            for (int k = cstart[c]; k < cstart[c + 1]; k += CM_N) {
                tcls.push_back(c);
                tst.push_back(k);
                tcnt.push_back(std::min(CM_N, cstart[c + 1] - k));
            }
        P->cm_ntile = (int)tcls.size();
        auto up = [&](int **d, const std::vector<int> &h) -> int {
            BEM_TRY(P->arena.alloc(d, std::max<size_t>(1, h.size())));
            if (!h.empty()) BEM_CUDA(cudaMemcpy(*d, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice));
            return BEM_OK;
        };
        BEM_TRY(up(&P->cm_order, order));
        BEM_TRY(up(&P->cm_tile_cls, tcls));
        BEM_TRY(up(&P->cm_tile_start, tst));
        BEM_TRY(up(&P->cm_tile_cnt, tcnt));
    }
    const int nc = std::max(1, P->m2l_ncls);
    BEM_TRY(P->arena.alloc(&P->m2l_cls, pair_cls.size()));
    BEM_TRY(P->arena.alloc(&P->cls_rho, 3 * nc));
    BEM_TRY(P->arena.alloc(&P->cls_kh, nc));
    BEM_TRY(P->arena.alloc(&P->cls_dl, nc));
    BEM_CUDA(cudaMemcpy(P->m2l_cls, pair_cls.data(), sizeof(int) * pair_cls.size(), cudaMemcpyHostToDevice));
    if (P->m2l_ncls) {
        BEM_CUDA(cudaMemcpy(P->cls_rho, rho.data(), sizeof(double) * rho.size(), cudaMemcpyHostToDevice));
        BEM_CUDA(cudaMemcpy(P->cls_kh, kh.data(), sizeof(double) * kh.size(), cudaMemcpyHostToDevice));
        BEM_CUDA(cudaMemcpy(P->cls_dl, dls.data(), sizeof(int) * dls.size(), cudaMemcpyHostToDevice));
    }
    return build_m2l_sym(P, pair_cls, kvec, dls, ii);
}

// derivative tables of ncls offset classes (rho: [class][3]; kh: [class], Helmholtz only)
int launch_m2l_derivs(bem_plan *P, int ncls, const double *rho, const double *kh, double *D, float *fD,
                      cudaStream_t s) {
    if (ncls <= 0) return BEM_OK;
    const int p = P->mi.p, np = P->mi.np, C = P->green == BEM_HELMHOLTZ ? 2 : 1;
    const size_t sm = sizeof(double) * (2 * (p + 2) + 4 * (size_t)np) + 64;
    (k_m2l_tables<<<ncls, TT, sm, s>>>(ncls, p, np, C, P->d_m, P->d_n, P->d_k, P->d_idx3, rho, kh, D, fD),
     ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    return BEM_OK;
}

// Coefficient lists and M2L tables for the current order (called by alloc_fmm).
int build_translation_tables(bem_plan *P, cudaStream_t s) {
    Arena &A = P->arena;
    const MIndex &mi = P->mi;
    const int p = mi.p, np = mi.np, P1 = p + 1;
    auto idx = [&](int m, int n, int k) { return mi.idx3[((size_t)m * P1 + n) * P1 + k]; };
    std::vector<double> fact(2 * PMAX + 2);
    fact[0] = 1.0;
    for (int i = 1; i < (int)fact.size(); i++) fact[i] = fact[i - 1] * i;
    // contraction lists: for every b, the (a, a+b) pairs with |a| + |b| <= p
    std::vector<int> cptr(np + 1, 0), cag, deg(np);
    std::vector<double> sgnf(np), invf(np);
    for (int b = 0; b < np; b++) {
        const int bm = mi.m[b], bn = mi.n[b], bk = mi.k[b], db = bm + bn + bk;
        deg[b] = db;
        const double fb = fact[bm] * fact[bn] * fact[bk];
        sgnf[b] = ((db & 1) ? -1.0 : 1.0) / fb;
        invf[b] = 1.0 / fb;
        for (int a = 0; a < np; a++) {
            if (mi.m[a] + mi.n[a] + mi.k[a] + db > p) continue;
            cag.push_back(a | (idx(mi.m[a] + bm, mi.n[a] + bn, mi.k[a] + bk) << 16));
        }
        cptr[b + 1] = (int)cag.size();
    }
    // longest-first assignment of b to threads, at most TSLOTS per thread
    std::vector<int> order(np), load(TT, 0), nslot(TT, 0), beta_of(TT * TSLOTS, -1);
    for (int b = 0; b < np; b++) order[b] = b;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        return cptr[x + 1] - cptr[x] > cptr[y + 1] - cptr[y];
    });
    for (int b : order) {
        int best = -1;
        for (int th = 0; th < TT; th++)
            if (nslot[th] < TSLOTS && (best < 0 || load[th] < load[best])) best = th;
        beta_of[best * TSLOTS + nslot[best]++] = b;
        load[best] += cptr[b + 1] - cptr[b];
    }
    auto up = [&](auto **d, const auto &h) -> int {
        using T = std::decay_t<decltype(h[0])>;
        BEM_TRY(A.alloc((T **)d, h.size()));
        BEM_CUDA(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
        return BEM_OK;
    };
    BEM_TRY(up(&P->ctr_ptr, cptr)); BEM_TRY(up(&P->ctr_ag, cag)); BEM_TRY(up(&P->ctr_beta, beta_of));
    BEM_TRY(up(&P->m_deg, deg)); BEM_TRY(up(&P->m_sgnf, sgnf)); BEM_TRY(up(&P->m_invf, invf));
    // the tensor-core form (mixed-precision Laplace) replaces the per-class tables
    BEM_TRY(build_tc_tables(P, s));
    if (P->sy_on) return BEM_OK;
    // derivative tables of every offset class
    const int C = P->green == BEM_HELMHOLTZ ? 2 : 1;
    // units of the float32 class-major M2L (real kernels, one unit per thread)
    P->cm_nunits = 0;
    std::vector<int> ur0, ua0, rtp, gidx;
    {
        const int nrt = (np + CM_UR - 1) / CM_UR, nac = (np + CM_UA - 1) / CM_UA;
        rtp.assign(nrt + 1, 0);
        for (int rt = 0; rt < nrt; rt++) {
            for (int ac = 0; ac < nac; ac++)
                if (deg[rt * CM_UR] + deg[ac * CM_UA] <= p) {
                    ur0.push_back(rt * CM_UR);
                    ua0.push_back(ac * CM_UA);
                }
            rtp[rt + 1] = (int)ur0.size();
        }
        for (size_t uu = 0; uu < ur0.size(); uu++)
            for (int r = 0; r < CM_UR; r++)
                for (int c = 0; c < CM_UA; c++) {
                    const int b = ur0[uu] + r, a = ua0[uu] + c;
                    int g = -1;
                    if (b < np && a < np && deg[a] + deg[b] <= p)
                        g = idx(mi.m[a] + mi.m[b], mi.n[a] + mi.n[b], mi.k[a] + mi.k[b]);
                    gidx.push_back(g);
                }
    }
    const bool use_cm = P->prm.precision == BEM_MIXED && C == 1 && (int)ur0.size() <= CM_T && P->m2l_ncls > 0;
    if (use_cm) {
        P->cm_nunits = (int)ur0.size();
        BEM_TRY(up(&P->cm_ur0, ur0)); BEM_TRY(up(&P->cm_ua0, ua0)); BEM_TRY(up(&P->cm_rtp, rtp));
        BEM_TRY(up(&P->cm_gidx, gidx));
        BEM_TRY(A.alloc(&P->cm_Lp, std::max<size_t>(1, (size_t)P->t.n_inter * np)));
    }
    const int nc = std::max(1, P->m2l_ncls);
    BEM_TRY(A.alloc(&P->m2l_D, (size_t)nc * np * C));
    if (P->prm.precision == BEM_MIXED) BEM_TRY(A.alloc(&P->m2l_fD, (size_t)nc * np * C));
    return launch_m2l_derivs(P, P->m2l_ncls, P->cls_rho, P->cls_kh, P->m2l_D, P->m2l_fD, s);
}

void free_translation_tables(bem_plan *P) {
    free_tc_tables(P);
    Arena &A = P->arena;
    for (void *q : {(void *)P->ctr_ptr, (void *)P->ctr_ag, (void *)P->ctr_beta, (void *)P->m_deg, (void *)P->m_sgnf,
                    (void *)P->m_invf, (void *)P->m2l_D, (void *)P->m2l_fD, (void *)P->cm_ur0, (void *)P->cm_ua0,
                    (void *)P->cm_rtp, (void *)P->cm_gidx, (void *)P->cm_Lp})
        A.release(q);
    P->cm_ur0 = P->cm_ua0 = P->cm_rtp = P->cm_gidx = nullptr;
    P->cm_Lp = nullptr;
    P->cm_nunits = 0;
    P->ctr_ptr = P->ctr_ag = P->ctr_beta = P->m_deg = nullptr;
    P->m_sgnf = P->m_invf = P->m2l_D = nullptr;
    P->m2l_fD = nullptr;
}

// ---------------------------------------------------------------------------
// host: launchers
// ---------------------------------------------------------------------------
// upward pass: moments of every parent from its children, level by level
template <class R, int C>
int launch_m2m(bem_plan *P, R *M, cudaStream_t s) {
    const Tree &t = P->t;
    const int np = P->mi.np;
    const int *sk = P->skip;
    const int P1 = P->mi.p + 1;
    const size_t tab_sm = sizeof(R) * P1 * P1 + sizeof(short) * P1 * P1 * P1 + 16;
    int grp = 8;                                 // children shifted together (shared memory permitting)
    while (grp > 1 && sizeof(R) * (2 * grp + 1) * np * C + tab_sm > 220 * 1024) grp /= 2;
    const size_t m2m_sm = sizeof(R) * (2 * grp + 1) * np * C + tab_sm;
    for (int l = t.nlev - 2; l >= 0; l--) {
        const int off = t.lev_off[l], cnt = t.lev_off[l + 1] - off;
        (k_m2m_sep<R, C><<<cnt, MM_T, m2m_sm, s>>>(off, cnt, t.child0, t.nchild, t.ix, t.iy, t.iz, P->mi.p, np, grp,
                                                   P->d_m, P->d_n, P->d_k, P->d_idx3, P->d_binom, M, sk),
         ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    return BEM_OK;
}

template <class R, int C>
int launch_translations(bem_plan *P, R *M, R *L, cudaStream_t s, cudaEvent_t *ev) {
    const Tree &t = P->t;
    const int np = P->mi.np;
    const int *sk = P->skip;
    const int P1 = P->mi.p + 1;
    const size_t tab_sm = sizeof(R) * P1 * P1 + sizeof(short) * P1 * P1 * P1 + 16;
    BEM_TRY((launch_m2m<R, C>(P, M, s)));
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[3], s));
    const R *D = sizeof(R) == sizeof(double) ? (const R *)P->m2l_D : (const R *)P->m2l_fD;
    if (std::is_same<R, float>::value && C == 1 && P->sy_on) {
        BEM_TRY(launch_m2l_tc(P, (const float *)M, (float *)L, s));
    } else if (std::is_same<R, float>::value && C == 1 && P->cm_nunits > 0) {
        const size_t npad = ((size_t)np + CM_UA - 1) / CM_UA * CM_UA, nu = P->cm_nunits, NE = nu * CM_UR * CM_UA;
        const size_t nrt = ((size_t)np + CM_UR - 1) / CM_UR;
        const size_t sm = sizeof(int) * (NE + 2 * nu + nrt + 1 + CM_N + npad) +
                          sizeof(float) * (4 * npad + NE + npad * CM_N + nu * CM_UR * CM_N);
        const int grid = std::min(P->cm_ntile, std::max(1, P->sm_count));
        if (P->cm_ntile > 0)
            (k_m2l_cm<<<grid, CM_T, sm, s>>>(P->cm_ntile, P->cm_tile_cls, P->cm_tile_start, P->cm_tile_cnt,
                                             P->cm_order, t.inter_idx, P->cls_dl, np, P->cm_nunits, (int)nrt,
                                             P->cm_ur0, P->cm_ua0, P->cm_rtp, P->cm_gidx, P->m_deg, P->m_sgnf,
                                             P->m_invf, P->m2l_fD, (const float *)M, P->cm_Lp, sk),
             ::bem::count_launch());
        (k_m2l_gather<<<t.nbox, 128, 0, s>>>(t.nbox, t.level, t.side, t.inter_ptr, np, P->cm_Lp, (float *)L, sk),
         ::bem::count_launch());
    } else {
        (k_m2l_tab<R, C><<<t.nbox, TT, sizeof(R) * 2 * np * C, s>>>(t.nbox, t.level, t.side, t.inter_ptr, t.inter_idx,
                                                                    P->m2l_cls, P->cls_dl, np, P->m_deg, P->m_sgnf,
                                                                    P->m_invf, P->ctr_ptr, P->ctr_ag, P->ctr_beta, D, M,
                                                                    L, sk), ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[4], s));
    for (int l = 1; l < t.nlev; l++) {
        const int off = t.lev_off[l], cnt = t.lev_off[l + 1] - off;
        (k_l2l_sep<R, C><<<cnt, MM_T, sizeof(R) * 2 * np * C + tab_sm, s>>>(off, cnt, t.parent, t.ix, t.iy, t.iz,
                                                                       P->mi.p, np, P->d_m, P->d_n, P->d_k, P->d_idx3,
                                                                       P->d_binom, L, sk),
         ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[5], s));
    return BEM_OK;
}

// large dynamic shared memory for every instantiation (outside any capture)
void set_translation_attributes() {
    const int big = 220 * 1024;
    cudaFuncSetAttribute(k_m2l_tab<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_tab<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_tab<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_tab<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_tables, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_sep<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_sep<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_sep<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_sep<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_sep<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_sep<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_sep<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_sep<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_cm, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    set_tc_attributes();
}

template int launch_m2m<double, 1>(bem_plan *, double *, cudaStream_t);
template int launch_m2m<double, 2>(bem_plan *, double *, cudaStream_t);
template int launch_m2m<float, 1>(bem_plan *, float *, cudaStream_t);
template int launch_m2m<float, 2>(bem_plan *, float *, cudaStream_t);
template int launch_translations<double, 1>(bem_plan *, double *, double *, cudaStream_t, cudaEvent_t *);
template int launch_translations<double, 2>(bem_plan *, double *, double *, cudaStream_t, cudaEvent_t *);
template int launch_translations<float, 1>(bem_plan *, float *, float *, cudaStream_t, cudaEvent_t *);
template int launch_translations<float, 2>(bem_plan *, float *, float *, cudaStream_t, cudaEvent_t *);

}  // namespace bem
