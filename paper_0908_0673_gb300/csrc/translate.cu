// Translation operators of the fast method with precomputed tables:
//
//   M2M  coefficient shift (Eq. 8):  Ms'_a = sum_{b<=a} C(a,b) s^b 2^-(|a|+|b|) Ms_{a-b}
//   L2L  expansion shift (Eq. 9):    Ls'_b += sum_g C(b+g,b) s^g 2^-(2|g|+|b|) Ls_{b+g}
//   M2L  local expansion (Eq. 7):    Ls_t[b] = 1/(h_t b!) sum_a D[a+b] (-1)^|a| (h_s/h_t)^|a| Ms_s[a] / a!
//
// Moments / locals are scaled by the box edge (Ms = I / h^|a|, Ls = F h^|b|),
// so a child's offset from its parent is +-1/4 of the parent edge per axis and
// every shift coefficient is a binomial times a power of two; the octant only
// flips signs.  The coefficient lists (source index, coefficient, parity of
// the shift exponent per axis) are built once per expansion order.
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
// M2M for the parents of one level: one block per parent, all children staged
// ---------------------------------------------------------------------------
template <class R, int C>
__global__ void __launch_bounds__(TT) k_m2m_tab(int off, int cnt, const int *__restrict__ child0,
                                                const int *__restrict__ nchild, const int *__restrict__ ix,
                                                const int *__restrict__ iy, const int *__restrict__ iz, int np,
                                                const int *__restrict__ ptr, const int *__restrict__ src,
                                                const double *__restrict__ coef, const unsigned char *__restrict__ par,
                                                R *__restrict__ M, const int *__restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    R *sM = (R *)smem_raw;                       // [8][np][C]
    __shared__ int smask[8];
    const int b = off + blockIdx.x;
    if (blockIdx.x >= cnt) return;
    const int nch = nchild[b];
    if (nch == 0) return;
    const int c0 = child0[b], tid = threadIdx.x;
    for (int j = 0; j < nch; j++)
        for (int t = tid; t < np * C; t += TT) sM[j * np * C + t] = M[(size_t)(c0 + j) * np * C + t];
    if (tid < nch) {
        const int c = c0 + tid;
        // a child on the low side of an axis has offset -1/4 of the parent edge
        smask[tid] = ((ix[c] & 1) ? 0 : 1) | ((iy[c] & 1) ? 0 : 2) | ((iz[c] & 1) ? 0 : 4);
    }
    __syncthreads();
    for (int a = tid; a < np; a += TT) {
        R acc[C];
#pragma unroll
        for (int c = 0; c < C; c++) acc[c] = (R)0;
        for (int k = ptr[a]; k < ptr[a + 1]; k++) {
            const R cf = (R)coef[k];
            const int sidx = src[k], pr = par[k];
            for (int j = 0; j < nch; j++) {
                const R sg = (__popc(pr & smask[j]) & 1) ? -cf : cf;
                cmac<R, C>(acc, sg, sM + (j * np + sidx) * C);
            }
        }
#pragma unroll
        for (int c = 0; c < C; c++) M[((size_t)b * np + a) * C + c] = acc[c];
    }
}

// ---------------------------------------------------------------------------
// L2L for the boxes of one level: one block per child, parent staged
// ---------------------------------------------------------------------------
template <class R, int C>
__global__ void __launch_bounds__(TT) k_l2l_tab(int off, int cnt, const int *__restrict__ parent,
                                                const int *__restrict__ ix, const int *__restrict__ iy,
                                                const int *__restrict__ iz, int np, const int *__restrict__ ptr,
                                                const int *__restrict__ src, const double *__restrict__ coef,
                                                const unsigned char *__restrict__ par, R *__restrict__ L,
                                                const int *__restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    R *sL = (R *)smem_raw;
    if (blockIdx.x >= cnt) return;
    const int b = off + blockIdx.x, pa = parent[b], tid = threadIdx.x;
    for (int t = tid; t < np * C; t += TT) sL[t] = L[(size_t)pa * np * C + t];
    const int mask = ((ix[b] & 1) ? 0 : 1) | ((iy[b] & 1) ? 0 : 2) | ((iz[b] & 1) ? 0 : 4);
    __syncthreads();
    for (int a = tid; a < np; a += TT) {
        R acc[C];
#pragma unroll
        for (int c = 0; c < C; c++) acc[c] = (R)0;
        for (int k = ptr[a]; k < ptr[a + 1]; k++) {
            const R cf = (R)coef[k];
            cmac<R, C>(acc, (__popc(par[k] & mask) & 1) ? -cf : cf, sL + src[k] * C);
        }
#pragma unroll
        for (int c = 0; c < C; c++) L[((size_t)b * np + a) * C + c] += acc[c];
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
    std::map<std::tuple<int, int, long long, long long, long long>, int> id;
    std::vector<int> pair_cls(std::max<int64_t>(1, t.n_inter));
    std::vector<double> rho, kh;
    std::vector<int> dls;
    for (int b = 0; b < t.nbox; b++)
        for (int u = ip[b]; u < ip[b + 1]; u++) {
            const int s = ii[u], dl = lev[b] - lev[s], e = std::max(0, -dl);
            // 2 rho 2^e = (2 i_t + 1) 2^e - (2 i_s + 1) 2^(dl + e), an integer vector
            auto K = [&](int it_, int is_) {
                return (long long)(2 * it_ + 1) * (1ll << e) - (long long)(2 * is_ + 1) * (1ll << (dl + e));
            };
            const long long kx = K(ix[b], ix[s]), ky = K(iy[b], iy[s]), kz = K(iz[b], iz[s]);
            auto key = std::make_tuple(dl, helm ? lev[b] : 0, kx, ky, kz);
            auto it = id.find(key);
            int c;
            if (it == id.end()) {
                c = (int)dls.size();
                id.emplace(key, c);
                const double sc = std::ldexp(1.0, -(e + 1));
                rho.push_back(kx * sc);
                rho.push_back(ky * sc);
                rho.push_back(kz * sc);
                kh.push_back(helm ? P->k * std::ldexp(t.side, -lev[b]) : 0.0);
                dls.push_back(dl);
            } else {
                c = it->second;
            }
            pair_cls[u] = c;
        }
    P->m2l_ncls = (int)dls.size();
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
    auto binom = [&](int a, int b) { return std::round(fact[a] / (fact[b] * fact[a - b])); };
    std::vector<int> mptr(np + 1, 0), msrc, lptr(np + 1, 0), lsrc;
    std::vector<double> mcoef, lcoef;
    std::vector<unsigned char> mpar, lpar;
    for (int a = 0; a < np; a++) {
        const int m = mi.m[a], n = mi.n[a], k = mi.k[a], da = m + n + k;
        for (int q = 0; q <= m; q++)
            for (int r = 0; r <= n; r++)
                for (int t = 0; t <= k; t++) {
                    msrc.push_back(idx(m - q, n - r, k - t));
                    mcoef.push_back(std::ldexp(binom(m, q) * binom(n, r) * binom(k, t), -(da + q + r + t)));
                    mpar.push_back((unsigned char)((q & 1) | ((r & 1) << 1) | ((t & 1) << 2)));
                }
        mptr[a + 1] = (int)msrc.size();
        for (int q = 0; q + da <= p; q++)
            for (int r = 0; q + r + da <= p; r++)
                for (int t = 0; q + r + t + da <= p; t++) {
                    lsrc.push_back(idx(m + q, n + r, k + t));
                    lcoef.push_back(std::ldexp(binom(m + q, m) * binom(n + r, n) * binom(k + t, k), -(2 * (q + r + t) + da)));
                    lpar.push_back((unsigned char)((q & 1) | ((r & 1) << 1) | ((t & 1) << 2)));
                }
        lptr[a + 1] = (int)lsrc.size();
    }
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
    BEM_TRY(up(&P->sh_m2m_ptr, mptr)); BEM_TRY(up(&P->sh_m2m_src, msrc));
    BEM_TRY(up(&P->sh_m2m_coef, mcoef)); BEM_TRY(up(&P->sh_m2m_par, mpar));
    BEM_TRY(up(&P->sh_l2l_ptr, lptr)); BEM_TRY(up(&P->sh_l2l_src, lsrc));
    BEM_TRY(up(&P->sh_l2l_coef, lcoef)); BEM_TRY(up(&P->sh_l2l_par, lpar));
    BEM_TRY(up(&P->ctr_ptr, cptr)); BEM_TRY(up(&P->ctr_ag, cag)); BEM_TRY(up(&P->ctr_beta, beta_of));
    BEM_TRY(up(&P->m_deg, deg)); BEM_TRY(up(&P->m_sgnf, sgnf)); BEM_TRY(up(&P->m_invf, invf));
    // derivative tables of every offset class
    const int C = P->green == BEM_HELMHOLTZ ? 2 : 1;
    const int nc = std::max(1, P->m2l_ncls);
    BEM_TRY(A.alloc(&P->m2l_D, (size_t)nc * np * C));
    if (P->prm.precision == BEM_MIXED) BEM_TRY(A.alloc(&P->m2l_fD, (size_t)nc * np * C));
    if (P->m2l_ncls) {
        const size_t sm = sizeof(double) * (2 * (p + 2) + 4 * (size_t)np) + 64;
        (k_m2l_tables<<<P->m2l_ncls, TT, sm, s>>>(P->m2l_ncls, p, np, C, P->d_m, P->d_n, P->d_k, P->d_idx3,
                                                  P->cls_rho, P->cls_kh, P->m2l_D, P->m2l_fD), ::bem::count_launch());
        BEM_LAUNCH_CHECK();
    }
    return BEM_OK;
}

void free_translation_tables(bem_plan *P) {
    Arena &A = P->arena;
    for (void *q : {(void *)P->sh_m2m_ptr, (void *)P->sh_m2m_src, (void *)P->sh_m2m_coef, (void *)P->sh_m2m_par,
                    (void *)P->sh_l2l_ptr, (void *)P->sh_l2l_src, (void *)P->sh_l2l_coef, (void *)P->sh_l2l_par,
                    (void *)P->ctr_ptr, (void *)P->ctr_ag, (void *)P->ctr_beta, (void *)P->m_deg, (void *)P->m_sgnf,
                    (void *)P->m_invf, (void *)P->m2l_D, (void *)P->m2l_fD})
        A.release(q);
    P->sh_m2m_ptr = P->sh_m2m_src = P->sh_l2l_ptr = P->sh_l2l_src = nullptr;
    P->sh_m2m_coef = P->sh_l2l_coef = nullptr;
    P->sh_m2m_par = P->sh_l2l_par = nullptr;
    P->ctr_ptr = P->ctr_ag = P->ctr_beta = P->m_deg = nullptr;
    P->m_sgnf = P->m_invf = P->m2l_D = nullptr;
    P->m2l_fD = nullptr;
}

// ---------------------------------------------------------------------------
// host: launchers
// ---------------------------------------------------------------------------
template <class R, int C>
int launch_translations(bem_plan *P, R *M, R *L, cudaStream_t s, cudaEvent_t *ev) {
    const Tree &t = P->t;
    const int np = P->mi.np;
    const int *sk = P->skip;
    for (int l = t.nlev - 2; l >= 0; l--) {
        const int off = t.lev_off[l], cnt = t.lev_off[l + 1] - off;
        (k_m2m_tab<R, C><<<cnt, TT, sizeof(R) * 8 * np * C, s>>>(off, cnt, t.child0, t.nchild, t.ix, t.iy, t.iz, np,
                                                                 P->sh_m2m_ptr, P->sh_m2m_src, P->sh_m2m_coef,
                                                                 P->sh_m2m_par, M, sk), ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[3], s));
    const R *D = sizeof(R) == sizeof(double) ? (const R *)P->m2l_D : (const R *)P->m2l_fD;
    (k_m2l_tab<R, C><<<t.nbox, TT, sizeof(R) * 2 * np * C, s>>>(t.nbox, t.level, t.side, t.inter_ptr, t.inter_idx,
                                                                P->m2l_cls, P->cls_dl, np, P->m_deg, P->m_sgnf,
                                                                P->m_invf, P->ctr_ptr, P->ctr_ag, P->ctr_beta, D, M, L,
                                                                sk), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[4], s));
    for (int l = 1; l < t.nlev; l++) {
        const int off = t.lev_off[l], cnt = t.lev_off[l + 1] - off;
        (k_l2l_tab<R, C><<<cnt, TT, sizeof(R) * np * C, s>>>(off, cnt, t.parent, t.ix, t.iy, t.iz, np, P->sh_l2l_ptr,
                                                             P->sh_l2l_src, P->sh_l2l_coef, P->sh_l2l_par, L, sk),
         ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[5], s));
    return BEM_OK;
}

// large dynamic shared memory for every instantiation (outside any capture)
void set_translation_attributes() {
    const int big = 200 * 1024;
    cudaFuncSetAttribute(k_m2m_tab<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_tab<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_tab<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2m_tab<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_tab<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_tab<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_tab<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_l2l_tab<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_tab<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_tab<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_tab<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_tab<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_m2l_tables, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

template int launch_translations<double, 1>(bem_plan *, double *, double *, cudaStream_t, cudaEvent_t *);
template int launch_translations<double, 2>(bem_plan *, double *, double *, cudaStream_t, cudaEvent_t *);
template int launch_translations<float, 1>(bem_plan *, float *, float *, cudaStream_t, cudaEvent_t *);
template int launch_translations<float, 2>(bem_plan *, float *, float *, cudaStream_t, cudaEvent_t *);

}  // namespace bem
