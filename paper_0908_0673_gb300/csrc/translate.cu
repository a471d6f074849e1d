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
// falls into one of a small number of exact offset classes, and these reduce
// further to canonical classes under the signed axis permutations
// (m2l_tc.cu).  This file builds the exact classes and the FP64 derivative
// tables; the contraction runs on the tensor cores (m2l_tc.cu) or as a SIMT
// GEMM (m2l_simt.cu).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <map>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "bem_internal.cuh"

namespace bem {

constexpr int TT = 128;                   // threads per block of the translation kernels

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

// Shift tables in shared memory, built from the multi-indices alone: the np
// coefficients' (m, n, k) packed as m | n << 8 | k << 16, the index of every
// multi-index of degree <= p (the only ones a pass looks up) at
// (m (p + 1) + n) (p + 1) + k, and the per-axis factors from exact integer
// binomials.  One round of global loads (tm, tn, tk) per block.
__device__ __forceinline__ int binom_int(int n, int k) {
    int b = 1;                                  // C(n - k + i, i) after step i: exact
    for (int i = 1; i <= k; i++) b = b * (n - k + i) / i;
    return b;
}
template <class R>
__device__ __forceinline__ void shift_tables(int p, int np, const int *__restrict__ tm, const int *__restrict__ tn,
                                             const int *__restrict__ tk, bool m2m, short *sIdx, R *sG, int *sMNK) {
    const int P1 = p + 1;
    for (int a = threadIdx.x; a < np; a += blockDim.x) {
        const int m = tm[a], n = tn[a], k = tk[a];
        sMNK[a] = m | n << 8 | k << 16;
        sIdx[(m * P1 + n) * P1 + k] = (short)a;
    }
    for (int i = threadIdx.x; i < P1 * P1; i += blockDim.x) {
        const int a = i / P1, g = i - a * P1;
        // M2M: binom(a, g) 2^-g (g <= a);  L2L: binom(a + g, a) 4^-g (a + g <= p)
        R v = (R)0, sc = (R)1;
        for (int j = 0; j < g; j++) sc *= m2m ? (R)0.5 : (R)0.25;
        if (m2m && g <= a) v = (R)binom_int(a, g) * sc;
        if (!m2m && a + g <= p) v = (R)binom_int(a + g, a) * sc;
        sG[i] = v;
    }
}

// shared-memory bytes of the shift tables at order p (sG, sIdx, sMNK)
template <class R>
__host__ __device__ inline size_t shift_tab_bytes(int p, int np) {
    const int P1 = p + 1;
    return (((size_t)sizeof(R) * P1 * P1 + sizeof(short) * P1 * P1 * P1 + 15) / 16) * 16 + 4 * (size_t)np + 16;
}

// one axis pass over nv vectors: out[v][a] = sum_g G[a_ax][g] s_v^g in[v][a -/+ g e_ax]
template <class R, int C, bool DOWN>
__device__ __forceinline__ void shift_pass(int ax, int nv, int p, int np, const int *sMNK, const short *sIdx,
                                           const R *sG, const int *smask, const R *in, R *out) {
    const int P1 = p + 1;
    for (int t = threadIdx.x; t < nv * np; t += blockDim.x) {
        const int v = t / np, a = t - v * np;
        const int mnk = sMNK[a];
        int c3[3] = {mnk & 255, (mnk >> 8) & 255, mnk >> 16};
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

// 2^-|a| of the coefficient with packed multi-index mnk
template <class R>
__device__ __forceinline__ R deg_scale(int mnk) {
    const int d = (mnk & 255) + ((mnk >> 8) & 255) + (mnk >> 16);
    if constexpr (sizeof(R) == sizeof(float)) return ldexpf(1.f, -d);
    else return ldexp(1.0, -d);
}

template <class R, int C>
__global__ void __launch_bounds__(MM_T) k_m2m_sep(int off, int cnt, const int *__restrict__ child0,
                                                  const int *__restrict__ nchild, const int *__restrict__ ix,
                                                  const int *__restrict__ iy, const int *__restrict__ iz, int p, int np,
                                                  int nps, int npc, int grp, const int *__restrict__ tm,
                                                  const int *__restrict__ tn, const int *__restrict__ tk,
                                                  R *__restrict__ M, const int *__restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    const int P1 = p + 1;
    R *sA = (R *)smem_raw;                                  // [grp][np][C]
    R *sB = sA + (size_t)grp * np * C;                       // [grp][np][C]
    R *sS = sB + (size_t)grp * np * C;                       // [np][C] sum over children
    R *sG = sS + (size_t)np * C;                             // [P1][P1]
    short *sIdx = (short *)(sG + P1 * P1);                   // [P1^3]
    int *sMNK = (int *)((unsigned char *)sG + (shift_tab_bytes<R>(p, np) - 4 * (size_t)np - 16));   // [np]
    __shared__ int smask[8];
    if (blockIdx.x >= cnt) return;
    const int b = off + blockIdx.x, nch = nchild[b], c0 = child0[b], tid = threadIdx.x;
    if (nch == 0) return;
    // children (consecutive boxes, row stride nps) hold npc coefficients; the
    // rest enter as zero.  U values per thread are loaded before any is
    // stored, so their latencies overlap (and the first ones the tables')
    constexpr int U = 6 * C;
    R v[U];
    auto load = [&](int g0, int nt, int t0) {
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = t0 + u * MM_T;
            const int j = t / (np * C), r = t - j * np * C, a = r / C;
            v[u] = t < nt && a < npc ? M[((size_t)(c0 + g0 + j) * nps) * C + r] : (R)0;
        }
    };
    auto store = [&](int nt, int t0) {
#pragma unroll
        for (int u = 0; u < U; u++)
            if (t0 + u * MM_T < nt) sA[t0 + u * MM_T] = v[u];
    };
    load(0, min(grp, nch) * np * C, tid);
    shift_tables<R>(p, np, tm, tn, tk, true, sIdx, sG, sMNK);
    for (int g0 = 0; g0 < nch; g0 += grp) {
        const int ng = min(grp, nch - g0), nt = ng * np * C;
        __syncthreads();
        if (g0 > 0) load(g0, nt, tid);
        store(nt, tid);
        for (int t0 = tid + U * MM_T; t0 < nt; t0 += U * MM_T) {
            load(g0, nt, t0);
            store(nt, t0);
        }
        // a child on the low side of an axis has offset -1/4 of the parent edge
        if (tid < ng) {
            const int c = c0 + g0 + tid;
            smask[tid] = ((ix[c] & 1) ? 0 : 1) | ((iy[c] & 1) ? 0 : 2) | ((iz[c] & 1) ? 0 : 4);
        }
        __syncthreads();
        shift_pass<R, C, true>(0, ng, p, np, sMNK, sIdx, sG, smask, sA, sB);
        __syncthreads();
        shift_pass<R, C, true>(1, ng, p, np, sMNK, sIdx, sG, smask, sB, sA);
        __syncthreads();
        shift_pass<R, C, true>(2, ng, p, np, sMNK, sIdx, sG, smask, sA, sB);
        __syncthreads();
        for (int t = tid; t < np * C; t += MM_T) {
            R sum = g0 == 0 ? (R)0 : sS[t];
            for (int j = 0; j < ng; j++) sum += sB[(size_t)j * np * C + t];
            sS[t] = sum;
        }
    }
    __syncthreads();
    for (int a = tid; a < np; a += MM_T) {
        const R sc = deg_scale<R>(sMNK[a]);
#pragma unroll
        for (int c = 0; c < C; c++) M[((size_t)b * nps + a) * C + c] = sS[(size_t)a * C + c] * sc;
    }
}

template <class R, int C>
__global__ void __launch_bounds__(MM_T) k_l2l_sep(int off, int cnt, const int *__restrict__ parent,
                                                  const int *__restrict__ ix, const int *__restrict__ iy,
                                                  const int *__restrict__ iz, int p, int np, int nps, int npo,
                                                  const int *__restrict__ tm, const int *__restrict__ tn,
                                                  const int *__restrict__ tk, R *__restrict__ L,
                                                  const int *__restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    const int P1 = p + 1;
    R *sA = (R *)smem_raw;                                  // [np][C]
    R *sB = sA + (size_t)np * C;                             // [np][C]
    R *sG = sB + (size_t)np * C;                             // [P1][P1]
    short *sIdx = (short *)(sG + P1 * P1);                   // [P1^3]
    int *sMNK = (int *)((unsigned char *)sG + (shift_tab_bytes<R>(p, np) - 4 * (size_t)np - 16));   // [np]
    __shared__ int smask[1];
    if (blockIdx.x >= cnt) return;
    const int b = off + blockIdx.x, pa = parent[b], tid = threadIdx.x;
    // the parent's np coefficients, all of a thread's in flight before the tables
    constexpr int U = 2 * C;
    const int nt = np * C;
    R v[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int t = tid + u * MM_T;
        v[u] = t < nt ? L[(size_t)pa * nps * C + t] : (R)0;
    }
    if (tid == 0) smask[0] = ((ix[b] & 1) ? 0 : 1) | ((iy[b] & 1) ? 0 : 2) | ((iz[b] & 1) ? 0 : 4);
    shift_tables<R>(p, np, tm, tn, tk, false, sIdx, sG, sMNK);
#pragma unroll
    for (int u = 0; u < U; u++)
        if (tid + u * MM_T < nt) sA[tid + u * MM_T] = v[u];
    for (int t = tid + U * MM_T; t < nt; t += MM_T) sA[t] = L[(size_t)pa * nps * C + t];
    __syncthreads();
    shift_pass<R, C, false>(2, 1, p, np, sMNK, sIdx, sG, smask, sA, sB);
    __syncthreads();
    shift_pass<R, C, false>(1, 1, p, np, sMNK, sIdx, sG, smask, sB, sA);
    __syncthreads();
    shift_pass<R, C, false>(0, 1, p, np, sMNK, sIdx, sG, smask, sA, sB);
    __syncthreads();
    for (int a = tid; a < npo; a += MM_T) {         // the child keeps its own order's npo coefficients (npo <= np)
        const R sc = deg_scale<R>(sMNK[a]);
#pragma unroll
        for (int c = 0; c < C; c++) L[((size_t)b * nps + a) * C + c] += sB[(size_t)a * C + c] * sc;
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
// host: tables
// ---------------------------------------------------------------------------

// Offset classes: key (dl, level for Helmholtz, K).  Offsets of interacting
// boxes are small integers, so the key packs into 64 bits (17 bits per K
// component, biased) and goes into a flat open-addressing table (Fibonacci
// hashing: the product's top bits depend on every bit of the key; the table
// starts small and doubles at half load, so it stays in cache); a key that
// does not pack goes to an ordered map.  Per class its offset vector, level
// difference and key level, in order of first appearance.
struct ClassSet {
    std::vector<unsigned long long> tkey = std::vector<unsigned long long>(4096, 0ull);
    std::vector<int> tval = std::vector<int>(4096, -1);
    size_t tmask = 4095, tused = 0;
    int tbits = 12;
    std::map<std::tuple<int, int, long long, long long, long long>, int> wide;
    std::vector<int> dls, levs;
    std::vector<long long> kvec;
    int find_or_add(long long kx, long long ky, long long kz, int dl, int lv) {
        constexpr int KB = 17;
        constexpr long long KMAX = (1ll << (KB - 1)) - 1;
        if (std::llabs(kx) <= KMAX && std::llabs(ky) <= KMAX && std::llabs(kz) <= KMAX && dl > -64 && dl < 64) {
            const unsigned long long key =
                1ull + (((unsigned long long)(kx + KMAX)) | ((unsigned long long)(ky + KMAX) << KB) |
                        ((unsigned long long)(kz + KMAX) << (2 * KB)) | ((unsigned long long)(dl + 64) << (3 * KB)) |
                        ((unsigned long long)lv << (3 * KB + 7)));
            unsigned long long *tk = tkey.data();
            size_t h = (size_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - tbits));
            while (tk[h] != 0ull && tk[h] != key) h = (h + 1) & tmask;
            if (tk[h] == key) return tval[h];
            if (2 * (tused + 1) > tmask + 1) {
                grow();
                tk = tkey.data();
                h = (size_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - tbits));
                while (tk[h] != 0ull) h = (h + 1) & tmask;
            }
            tk[h] = key;
            tused++;
            return tval[h] = add(kx, ky, kz, dl, lv);
        }
        auto wk = std::make_tuple(dl, lv, kx, ky, kz);
        auto it = wide.find(wk);
        if (it == wide.end()) it = wide.emplace(wk, add(kx, ky, kz, dl, lv)).first;
        return it->second;
    }
    int add(long long kx, long long ky, long long kz, int dl, int lv) {
        dls.push_back(dl);
        levs.push_back(lv);
        kvec.push_back(kx);
        kvec.push_back(ky);
        kvec.push_back(kz);
        return (int)dls.size() - 1;
    }
    void grow() {
        std::vector<unsigned long long> ok;
        std::vector<int> ov;
        ok.swap(tkey);
        ov.swap(tval);
        tmask = 2 * (tmask + 1) - 1;
        tbits++;
        tkey.assign(tmask + 1, 0ull);
        tval.assign(tmask + 1, -1);
        for (size_t i = 0; i < ok.size(); i++)
            if (ok[i]) {
                size_t h = (size_t)((ok[i] * 0x9E3779B97F4A7C15ull) >> (64 - tbits));
                while (tkey[h] != 0ull) h = (h + 1) & tmask;
                tkey[h] = ok[i];
                tval[h] = ov[i];
            }
    }
};

// the classes of the pairs of boxes [b0, b1), in a set of their own
static void number_classes(int b0, int b1, bool by_level, const int *lev, const int *ix, const int *iy, const int *iz,
                           const int *ip, const int *ii, int *pair_cls, ClassSet &S) {
    for (int b = b0; b < b1; b++) {
        const int lb = lev[b], xb = ix[b], yb = iy[b], zb = iz[b], lv = by_level ? lb : 0;
        for (int u = ip[b]; u < ip[b + 1]; u++) {
            const int s = ii[u], dl = lb - lev[s], e = std::max(0, -dl);
            // 2 rho 2^e = (2 i_t + 1) 2^e - (2 i_s + 1) 2^(dl + e), an integer vector
            const long long ft = 1ll << e, fs = 1ll << (dl + e);
            pair_cls[u] = S.find_or_add((2ll * xb + 1) * ft - (2ll * ix[s] + 1) * fs, (2ll * yb + 1) * ft - (2ll * iy[s] + 1) * fs,
                                        (2ll * zb + 1) * ft - (2ll * iz[s] + 1) * fs, dl, lv);
        }
    }
}

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
    const bool by_level = helm || P->prm.p_min > 0;   // the target level enters the key
    // Classes are numbered in order of first appearance over the pairs in list
    // order.  The boxes are cut into up to three ranges of about equal pair
    // counts, numbered on threads of their own (number_classes); the ranges'
    // classes are then numbered together in range order, which is the
    // numbering of one pass over all pairs.
    const int64_t npair = t.n_inter;
    const int nth = (int)std::max<int64_t>(1, std::min<int64_t>(3, npair / 32768));
    std::vector<int> bcut(nth + 1, t.nbox);
    bcut[0] = 0;
    for (int k = 1, b = 0; k < nth; k++) {
        while (b < t.nbox && (int64_t)ip[b] * nth < npair * k) b++;
        bcut[k] = b;
    }
    std::vector<int> pair_cls(std::max<int64_t>(1, npair));
    std::vector<ClassSet> sets(nth);
    {
        std::vector<std::thread> th;
        for (int k = 1; k < nth; k++)
            th.emplace_back(number_classes, bcut[k], bcut[k + 1], by_level, lev.data(), ix.data(), iy.data(),
                            iz.data(), ip.data(), ii.data(), pair_cls.data(), std::ref(sets[k]));
        number_classes(bcut[0], bcut[1], by_level, lev.data(), ix.data(), iy.data(), iz.data(), ip.data(), ii.data(),
                       pair_cls.data(), sets[0]);
        for (auto &x : th) x.join();
    }
    // the first range's numbers are already global; later ranges' are mapped
    ClassSet &all = sets[0];
    for (int k = 1; k < nth; k++) {
        const ClassSet &R = sets[k];
        std::vector<int> to(R.dls.size());
        for (size_t c = 0; c < R.dls.size(); c++)
            to[c] = all.find_or_add(R.kvec[3 * c], R.kvec[3 * c + 1], R.kvec[3 * c + 2], R.dls[c], R.levs[c]);
        for (int u = ip[bcut[k]]; u < ip[bcut[k + 1]]; u++) pair_cls[u] = to[pair_cls[u]];
    }
    const std::vector<int> &dls = all.dls, &levs = all.levs;
    const std::vector<long long> &kvec = all.kvec;
    P->m2l_src_lmin = P->m2l_tgt_lmin = t.nlev;
    for (int b = 0; b < t.nbox; b++)
        if (ip[b + 1] > ip[b]) P->m2l_tgt_lmin = std::min(P->m2l_tgt_lmin, lev[b]);
    for (int64_t u = 0; u < t.n_inter; u++) P->m2l_src_lmin = std::min(P->m2l_src_lmin, lev[ii[u]]);
    return build_m2l_sym(P, pair_cls, kvec, dls, levs, ii, ip);
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

// M2L tables for the current order (called by alloc_fmm).
int build_translation_tables(bem_plan *P, cudaStream_t s) { return build_sym_tables(P, s); }

void free_translation_tables(bem_plan *P) { free_sym_tables(P); }

// ---------------------------------------------------------------------------
// host: launchers
// ---------------------------------------------------------------------------
static int np_host(int q) { return (q + 1) * (q + 2) * (q + 3) / 6; }
static int level_order(const bem_plan *P, int l) {
    return l < (int)P->lev_p.size() ? P->lev_p[l] : P->mi.p;
}

// upward pass: moments of every parent from its children, level by level,
// up to level lmin (coarser moments are not formed)
template <class R, int C>
int launch_m2m(bem_plan *P, R *M, cudaStream_t s, int lmin) {
    const Tree &t = P->t;
    const int nps = P->mi.np;
    const int *sk = P->skip;
    for (int l = t.nlev - 2; l >= std::max(0, lmin); l--) {
        const int off = t.lev_off[l], cnt = t.lev_off[l + 1] - off;
        const int p = level_order(P, l), np = np_host(p), npc = np_host(level_order(P, l + 1));
        const size_t tab_sm = shift_tab_bytes<R>(p, np);
        int grp = 8;                             // children shifted together (shared memory permitting)
        while (grp > 1 && sizeof(R) * (2 * grp + 1) * np * C + tab_sm > 220 * 1024) grp /= 2;
        const size_t m2m_sm = sizeof(R) * (2 * grp + 1) * np * C + tab_sm;
        (k_m2m_sep<R, C><<<cnt, MM_T, m2m_sm, s>>>(off, cnt, t.child0, t.nchild, t.ix, t.iy, t.iz, p, np, nps, npc, grp,
                                                   P->d_m, P->d_n, P->d_k, M, sk),
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
    // M2L reads moments at levels >= m2l_src_lmin only, and every local
    // coarser than m2l_tgt_lmin is zero (the gathers write each box's local),
    // so the upward pass stops at the first and the downward one starts below
    // the second
    BEM_TRY((launch_m2m<R, C>(P, M, s, P->m2l_src_lmin)));
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[3], s));
    if (std::is_same<R, float>::value && C == 1 && P->sy_tc) {
        BEM_TRY(launch_m2l_tc(P, (const float *)M, (float *)L, s));
    } else {
        BEM_TRY((launch_m2l_sy<R, C>(P, M, L, s)));
    }
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[4], s));
    for (int l = std::max(1, P->m2l_tgt_lmin + 1); l < t.nlev; l++) {
        // the shift runs at the parent's order; the child keeps its own order's terms
        const int off = t.lev_off[l], cnt = t.lev_off[l + 1] - off;
        const int p = level_order(P, l - 1), pnp = np_host(p), npo = np_host(level_order(P, l));
        const size_t tab_sm = shift_tab_bytes<R>(p, pnp);
        (k_l2l_sep<R, C><<<cnt, MM_T, sizeof(R) * 2 * pnp * C + tab_sm, s>>>(off, cnt, t.parent, t.ix, t.iy, t.iz, p,
                                                                           pnp, np, npo, P->d_m, P->d_n, P->d_k, L,
                                                                           sk),
         ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[5], s));
    return BEM_OK;
}

// large dynamic shared memory for every instantiation (outside any capture)
void set_translation_attributes() {
    const int big = 220 * 1024;
    cudaFuncSetAttribute(k_m2l_tables, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_sep<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_sep<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_sep<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_sep<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_sep<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_sep<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_sep<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_sep<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    set_tc_attributes();
    set_sy_attributes();
}

template int launch_m2m<double, 1>(bem_plan *, double *, cudaStream_t, int);
template int launch_m2m<double, 2>(bem_plan *, double *, cudaStream_t, int);
template int launch_m2m<float, 1>(bem_plan *, float *, cudaStream_t, int);
template int launch_m2m<float, 2>(bem_plan *, float *, cudaStream_t, int);
template int launch_translations<double, 1>(bem_plan *, double *, double *, cudaStream_t, cudaEvent_t *);
template int launch_translations<double, 2>(bem_plan *, double *, double *, cudaStream_t, cudaEvent_t *);
template int launch_translations<float, 1>(bem_plan *, float *, float *, cudaStream_t, cudaEvent_t *);
template int launch_translations<float, 2>(bem_plan *, float *, float *, cudaStream_t, cudaEvent_t *);

}  // namespace bem
