// One fast matrix multiplication (Section 3.6, steps 1-4) on the device:
//
//   P2Q  quadrature-point strengths f_q = w_q J_q sum_a L_a(xi_q) x_idx(e,a)
//   P2M  leaf moments I_alpha = sum_q f_q (x_q - c)^alpha            (Eq. 6, monopoles)
//        or sum_q f_q n_q . grad (x_q - c)^alpha                       (dipoles)
//   M2M  coefficient shift child -> parent                            (Eq. 8)
//   M2L  local expansion from the interaction list                     (Eq. 7)
//   L2L  expansion shift parent -> child, with binomials               (Eq. 9)
//   L2P  local expansion at every vertex of a leaf, fused with
//   P2P  the regular-rule sum over the elements of the near-field boxes
//   then the stored special-pair correction and the diagonal C.
//
// Moments and locals are stored scaled by powers of the box edge h:
// Ms_alpha = I_alpha / h^|alpha|, Ls_beta = F_beta h^|beta|, so that every
// shift factor is an exact power of two and float32 storage stays in range.
// Green's-function derivatives come from Tausch's recursions (Section 3.3)
// evaluated per interaction pair at r / h_t.
//
// Templates: R = double (BEM_F64) or float (BEM_MIXED); C = 1 (real, Laplace)
// or 2 (complex, Helmholtz); DL selects dipole (op A) or monopole (op B)
// sources.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "bem_internal.cuh"

namespace bem {

__constant__ double c_Lq[2][NQ][6];   // shape values at the 7 rule points (tri3, tri6)

struct Tabs {
    const int *m, *n, *k, *idx3;
    const double *fact;
    int p, np;                          // largest order, and the coefficient count (array stride)
    const int *lev_p;                   // order of each tree level (nullptr: p everywhere)
};

// number of multi-indices of degree <= q (the coefficients of order q)
__host__ __device__ __forceinline__ int np_of(int q) { return (q + 1) * (q + 2) * (q + 3) / 6; }
__device__ __forceinline__ int order_of(const Tabs &tb, int level) { return tb.lev_p ? tb.lev_p[level] : tb.p; }

struct TreeView {
    const int *level, *ix, *iy, *iz, *parent, *child0, *nchild, *nb, *ne, *eb, *ee, *leaves;
    const int *near_ptr, *near_idx, *inter_ptr, *inter_idx, *node_perm;
    const double *cx, *cy, *cz, *tx, *ty, *tz;
    double side;
};

struct QuadView {
    const double *x, *y, *z, *nx, *ny, *nz, *w;
    const float *fx, *fy, *fz, *fnx, *fny, *fnz, *fw;
};

template <class R> struct Vec { R v[2]; };

__device__ __forceinline__ int deg_of(int m, int n, int k) { return m + n + k; }

// ---------------------------------------------------------------------------
// P2Q
// ---------------------------------------------------------------------------
template <class R, int C>
__global__ void k_p2q(int Q, int npe, const int *__restrict__ el_idx, const double *__restrict__ w,
                      const void *const *__restrict__ xslot, R *__restrict__ f, const int *__restrict__ skip) {
    if (skip && *skip) return;
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= Q) return;
    const double *x = (const double *)*xslot;
    int i = o / NQ, q = o - i * NQ, t6 = npe == 6;
    double acc[C];
#pragma unroll
    for (int c = 0; c < C; c++) acc[c] = 0.0;
    for (int a = 0; a < npe; a++) {
        double L = c_Lq[t6][q][a];
        int j = el_idx[(size_t)i * npe + a];
#pragma unroll
        for (int c = 0; c < C; c++) acc[c] += L * x[(size_t)j * C + c];
    }
    double ww = w[o];
#pragma unroll
    for (int c = 0; c < C; c++) f[(size_t)o * C + c] = (R)(ww * acc[c]);
}

// ---------------------------------------------------------------------------
// P2M: one block per leaf, threads over multi-indices, sources in batches of 32
// ---------------------------------------------------------------------------
constexpr int P2M_T = 128, P2M_B = 32;
// index slots per thread (NS >= ceil(n_p / P2M_T)): instantiated for orders
// up to 11 (3), 16 (8) and 20 (14)
constexpr int p2m_slots(int np) { return np <= 3 * P2M_T ? 3 : np <= 8 * P2M_T ? 8 : 14; }

// WEIGHTS: instead of the moments, write each point's row of P2M weights
// W[o][a] (the value that multiplies f[o] in moment a) for the stored form.
//
// Per batch of points, shared memory holds for every point and axis the pairs
// (d^e, e n d^(e-1) / h) (d = offset / h, n the normal's component), so a
// monopole coefficient is Px Py Pz and a double-layer one, the normal
// derivative of the monomial, (Qx Py + Px Qy) Pz + Px Py Qz: three paired
// loads and no branches per (point, coefficient).
template <class R, int C, bool DL, bool WEIGHTS, int NS>
__global__ void __launch_bounds__(P2M_T) k_p2m(int nleaf, Tabs tb, TreeView tv, QuadView qv, const R *__restrict__ f,
                                               R *__restrict__ M, const int *__restrict__ skip, R *__restrict__ W = nullptr) {
    using R2 = typename std::conditional<sizeof(R) == sizeof(float), float2, double2>::type;
    if (skip && *skip) return;
    const int li = blockIdx.x;
    if (li >= nleaf) return;
    const int b = tv.leaves[li];
    const int np = tb.np, tid = threadIdx.x;
    const int p = order_of(tb, tv.level[b]), npl = np_of(p);   // this leaf's order; np is the stride
    __shared__ R2 pq[3][P2M_B][PMAX + 1];            // [axis][point][power]: (d^e, e n d^(e-1) / h)
    __shared__ R sf[P2M_B][C];
    const double h = scalbn(tv.side, -tv.level[b]);
    const R hinv = (R)(1.0 / h);
    const double c0 = tv.cx[b], c1 = tv.cy[b], c2 = tv.cz[b];
    int am[NS], an[NS], ak[NS];
    R acc[NS][C];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        int a = tid + s * P2M_T;
        am[s] = a < npl ? tb.m[a] : 0;
        an[s] = a < npl ? tb.n[a] : 0;
        ak[s] = a < npl ? tb.k[a] : 0;
#pragma unroll
        for (int c = 0; c < C; c++) acc[s][c] = (R)0;
    }
    const int q0 = tv.eb[b] * NQ, q1 = tv.ee[b] * NQ;
    for (int base = q0; base < q1; base += P2M_B) {
        const int nb = min(P2M_B, q1 - base);
        __syncthreads();
        if (tid < 3 * P2M_B) {
            int pt = tid % P2M_B, ax = tid / P2M_B;
            R d = (R)0, nd = (R)0;
            if (pt < nb) {
                int o = base + pt;
                if constexpr (sizeof(R) == sizeof(double)) {
                    double xx = ax == 0 ? qv.x[o] - c0 : (ax == 1 ? qv.y[o] - c1 : qv.z[o] - c2);
                    d = (R)(xx / h);
                    if (DL) nd = (R)(ax == 0 ? qv.nx[o] : (ax == 1 ? qv.ny[o] : qv.nz[o]));
                } else {
                    // float path: offsets from the owning leaf (this box) centre
                    R xx = ax == 0 ? (R)qv.fx[o] : (ax == 1 ? (R)qv.fy[o] : (R)qv.fz[o]);
                    d = xx * hinv;
                    if (DL) nd = (R)(ax == 0 ? qv.fnx[o] : (ax == 1 ? qv.fny[o] : qv.fnz[o]));
                }
            }
            nd *= hinv;
            R v = (R)1, vm = (R)0;                    // d^e, d^(e-1)
            for (int e = 0; e <= p; e++) {
                R2 t;
                t.x = v;
                t.y = DL ? (R)e * nd * vm : (R)0;
                pq[ax][pt][e] = t;
                vm = v;
                v *= d;
            }
        } else if (!WEIGHTS && tid < 3 * P2M_B + P2M_B) {
            int pt = tid - 3 * P2M_B;
            int o = base + pt;
#pragma unroll
            for (int c = 0; c < C; c++) sf[pt][c] = pt < nb ? f[(size_t)o * C + c] : (R)0;
        }
        __syncthreads();
        for (int pt = 0; pt < nb; pt++) {
#pragma unroll
            for (int s = 0; s < NS; s++) {
                if (tid + s * P2M_T >= npl) break;
                const R2 X = pq[0][pt][am[s]], Y = pq[1][pt][an[s]], Z = pq[2][pt][ak[s]];
                const R xy = X.x * Y.x;
                R val;
                if (!DL) val = xy * Z.x;
                else val = xy * Z.y + (X.y * Y.x + X.x * Y.y) * Z.x;
                if (WEIGHTS) {
                    W[(size_t)(base + pt) * np + tid + s * P2M_T] = val;
                } else {
#pragma unroll
                    for (int c = 0; c < C; c++) acc[s][c] += val * sf[pt][c];
                }
            }
        }
    }
    if (WEIGHTS) return;
#pragma unroll
    for (int s = 0; s < NS; s++) {
        int a = tid + s * P2M_T;
        if (a < npl)
#pragma unroll
            for (int c = 0; c < C; c++) M[((size_t)b * np + a) * C + c] = acc[s][c];
    }
}

// ---------------------------------------------------------------------------
// P2M from stored weights (float32 double-layer moments): M[a] = sum over the
// leaf's points of W[o][a] f[o] with W the values the on-the-fly form builds;
// each product only streams the weight rows (coalesced across the indices a),
// two halves of the block taking alternate chunks of points to keep more
// loads in flight.
// ---------------------------------------------------------------------------
constexpr int P2S_T = 2 * P2M_T, P2S_U = 8;           // two halves of P2M_T threads; points per chunk

template <int C, int NS>
__global__ void __launch_bounds__(P2S_T) k_p2m_stored(int nleaf, int np, TreeView tv, const float *__restrict__ W,
                                                      const float *__restrict__ f, float *__restrict__ M,
                                                      const int *__restrict__ skip) {
    if (skip && *skip) return;
    const int li = blockIdx.x;
    if (li >= nleaf) return;
    __shared__ float part[NS][C][P2M_T];
    const int b = tv.leaves[li], half = threadIdx.x / P2M_T, tid = threadIdx.x % P2M_T;
    const int q0 = tv.eb[b] * NQ, q1 = tv.ee[b] * NQ;
    float acc[NS][C];
#pragma unroll
    for (int s = 0; s < NS; s++)
#pragma unroll
        for (int c = 0; c < C; c++) acc[s][c] = 0.f;
    // chunks of P2S_U points alternate between the halves; within a half the
    // points are summed in order, then half 1's sums are added to half 0's
    for (int o0 = q0 + half * P2S_U; o0 < q1; o0 += 2 * P2S_U) {
        const int n = min(P2S_U, q1 - o0);
        float w[P2S_U][NS], fv[P2S_U][C];
#pragma unroll
        for (int u = 0; u < P2S_U; u++) {
            const bool on = u < n;
#pragma unroll
            for (int c = 0; c < C; c++) fv[u][c] = on ? __ldg(f + (size_t)(o0 + u) * C + c) : 0.f;
#pragma unroll
            for (int s = 0; s < NS; s++) {
                const int a = tid + s * P2M_T;
                w[u][s] = on && a < np ? __ldg(W + (size_t)(o0 + u) * np + a) : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < P2S_U; u++)
#pragma unroll
            for (int s = 0; s < NS; s++)
#pragma unroll
                for (int c = 0; c < C; c++) acc[s][c] += w[u][s] * fv[u][c];
    }
    if (half == 1)
#pragma unroll
        for (int s = 0; s < NS; s++)
#pragma unroll
            for (int c = 0; c < C; c++) part[s][c][tid] = acc[s][c];
    __syncthreads();
    if (half == 0)
#pragma unroll
        for (int s = 0; s < NS; s++) {
            const int a = tid + s * P2M_T;
            if (a < np)
#pragma unroll
                for (int c = 0; c < C; c++) M[((size_t)b * np + a) * C + c] = acc[s][c] + part[s][c][tid];
        }
}


// P2M launches with the slot count of the plan's largest order
template <class R, int C, bool DL, bool WEIGHTS = false>
static void launch_p2m(int nleaf, const Tabs &tb, const TreeView &tv, const QuadView &qv, const R *f, R *M,
                       const int *skip, cudaStream_t s, R *W = nullptr) {
    const int ns = p2m_slots(tb.np);
    if (ns == 3) (k_p2m<R, C, DL, WEIGHTS, 3><<<nleaf, P2M_T, 0, s>>>(nleaf, tb, tv, qv, f, M, skip, W), ::bem::count_launch());
    else if (ns == 8) (k_p2m<R, C, DL, WEIGHTS, 8><<<nleaf, P2M_T, 0, s>>>(nleaf, tb, tv, qv, f, M, skip, W), ::bem::count_launch());
    else (k_p2m<R, C, DL, WEIGHTS, 14><<<nleaf, P2M_T, 0, s>>>(nleaf, tb, tv, qv, f, M, skip, W), ::bem::count_launch());
}

template <int C>
static void launch_p2m_stored(int nleaf, int np, const TreeView &tv, const float *W, const float *f, float *M,
                              const int *skip, cudaStream_t s) {
    const int ns = p2m_slots(np);
    if (ns == 3) (k_p2m_stored<C, 3><<<nleaf, P2S_T, 0, s>>>(nleaf, np, tv, W, f, M, skip), ::bem::count_launch());
    else if (ns == 8) (k_p2m_stored<C, 8><<<nleaf, P2S_T, 0, s>>>(nleaf, np, tv, W, f, M, skip), ::bem::count_launch());
    else (k_p2m_stored<C, 14><<<nleaf, P2S_T, 0, s>>>(nleaf, np, tv, W, f, M, skip), ::bem::count_launch());
}

// ---------------------------------------------------------------------------
// near field (regular rule over the near-list boxes) fused with L2P
// ---------------------------------------------------------------------------
constexpr int NF_T = 256, NF_TGT = 64, NF_SL = NF_T / NF_TGT, NF_TILE = 256;

template <class R, int C, bool DL>
__device__ __forceinline__ void pair_kernel(R rx, R ry, R rz, R nx, R ny, R nz, const R *fv, R kw, R *acc) {
    const R r2 = rx * rx + ry * ry + rz * rz;
    R inv;
    if constexpr (sizeof(R) == sizeof(double)) inv = (R)rsqrt((double)r2);
    else inv = (R)rsqrtf((float)r2);
    if (C == 1) {
        if (DL) acc[0] += fv[0] * (rx * nx + ry * ny + rz * nz) * inv * inv * inv;
        else acc[0] += fv[0] * inv;
    } else {
        const R R1 = r2 * inv;
        R sn, cs;
        if constexpr (sizeof(R) == sizeof(double)) sincos((double)(kw * R1), (double *)&sn, (double *)&cs);
        else sincosf((float)(kw * R1), (float *)&sn, (float *)&cs);
        R gr, gi;
        if (DL) {
            const R kr = kw * R1, rn = (rx * nx + ry * ny + rz * nz) * inv * inv * inv;
            gr = (cs + kr * sn) * rn;
            gi = (sn - kr * cs) * rn;
        } else {
            gr = cs * inv;
            gi = sn * inv;
        }
        acc[0] += gr * fv[0] - gi * fv[1];
        acc[1] += gr * fv[1] + gi * fv[0];
    }
}

template <class R, int C, bool DL>
__global__ void __launch_bounds__(NF_T) k_near(int nleaf, Tabs tb, TreeView tv, QuadView qv, double kwave,
                                               const R *__restrict__ f, const R *__restrict__ L,
                                               double *__restrict__ ytmp, const int *__restrict__ skip) {
    if (skip && *skip) return;
    const int li = blockIdx.x;
    if (li >= nleaf) return;
    const int b = tv.leaves[li];
    const int tid = threadIdx.x, tt = tid % NF_TGT, sl = tid / NF_TGT;
    const int np = tb.np, p = order_of(tb, tv.level[b]), npl = np_of(p);   // the leaf's order; np the stride
    __shared__ R sx[NF_TILE], sy[NF_TILE], sz[NF_TILE], snx[NF_TILE], sny[NF_TILE], snz[NF_TILE];
    __shared__ R sf[NF_TILE][C];
    __shared__ double red[NF_T][C];
    const double cbx = tv.cx[b], cby = tv.cy[b], cbz = tv.cz[b];
    const double h = scalbn(tv.side, -tv.level[b]);
    const R kw = (R)kwave;
    for (int t0 = tv.nb[b]; t0 < tv.ne[b]; t0 += NF_TGT) {
        const int tk = t0 + tt;
        const bool active = tk < tv.ne[b];
        // target position: absolute (F64) or offset from this leaf's centre (F32)
        double txd = active ? tv.tx[tk] : cbx, tyd = active ? tv.ty[tk] : cby, tzd = active ? tv.tz[tk] : cbz;
        double acc[C];
#pragma unroll
        for (int c = 0; c < C; c++) acc[c] = 0.0;
        for (int u = tv.near_ptr[b]; u < tv.near_ptr[b + 1]; u++) {
            const int s = tv.near_idx[u];
            const int q0 = tv.eb[s] * NQ, q1 = tv.ee[s] * NQ;
            R tx, ty, tz;
            if constexpr (sizeof(R) == sizeof(double)) {
                tx = (R)txd; ty = (R)tyd; tz = (R)tzd;
            } else {
                // r = (c_b - c_s) + (t - c_b) - (q - c_s), each part small
                tx = (R)(cbx - tv.cx[s]) + (R)(txd - cbx);
                ty = (R)(cby - tv.cy[s]) + (R)(tyd - cby);
                tz = (R)(cbz - tv.cz[s]) + (R)(tzd - cbz);
            }
            R part[C];
#pragma unroll
            for (int c = 0; c < C; c++) part[c] = (R)0;
            for (int base = q0; base < q1; base += NF_TILE) {
                const int nt = min(NF_TILE, q1 - base);
                __syncthreads();
                if (tid < nt) {
                    const int o = base + tid;
                    if constexpr (sizeof(R) == sizeof(double)) {
                        sx[tid] = (R)qv.x[o]; sy[tid] = (R)qv.y[o]; sz[tid] = (R)qv.z[o];
                        if (DL) { snx[tid] = (R)qv.nx[o]; sny[tid] = (R)qv.ny[o]; snz[tid] = (R)qv.nz[o]; }
                    } else {
                        sx[tid] = (R)qv.fx[o]; sy[tid] = (R)qv.fy[o]; sz[tid] = (R)qv.fz[o];
                        if (DL) { snx[tid] = (R)qv.fnx[o]; sny[tid] = (R)qv.fny[o]; snz[tid] = (R)qv.fnz[o]; }
                    }
#pragma unroll
                    for (int c = 0; c < C; c++) sf[tid][c] = f[(size_t)o * C + c];
                }
                __syncthreads();
                if (active)
                    for (int j = sl; j < nt; j += NF_SL)
                        pair_kernel<R, C, DL>(tx - sx[j], ty - sy[j], tz - sz[j], DL ? snx[j] : (R)0,
                                              DL ? sny[j] : (R)0, DL ? snz[j] : (R)0, sf[j], kw, part);
            }
#pragma unroll
            for (int c = 0; c < C; c++) acc[c] += (double)part[c];
        }
        // local expansion at the target: sum_b Ls_b ((x - c)/h)^b, slices split b
        double loc[C];
#pragma unroll
        for (int c = 0; c < C; c++) loc[c] = 0.0;
        if (active) {
            const R dx = (R)((txd - cbx) / h), dy = (R)((tyd - cby) / h), dz = (R)((tzd - cbz) / h);
            R px[PMAX + 1], py[PMAX + 1], pz[PMAX + 1];
            px[0] = py[0] = pz[0] = (R)1;
            for (int e = 1; e <= p; e++) {
                px[e] = px[e - 1] * dx;
                py[e] = py[e - 1] * dy;
                pz[e] = pz[e - 1] * dz;
            }
            for (int a = sl; a < npl; a += NF_SL) {
                const R mono = px[tb.m[a]] * py[tb.n[a]] * pz[tb.k[a]];
#pragma unroll
                for (int c = 0; c < C; c++) loc[c] += (double)(mono * L[((size_t)b * np + a) * C + c]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; c++) red[tid][c] = acc[c] * (0.25 / M_PI) + loc[c];
        __syncthreads();
        if (sl == 0 && active) {
            double s[C];
#pragma unroll
            for (int c = 0; c < C; c++) s[c] = red[tid][c];
            for (int u = 1; u < NF_SL; u++)
#pragma unroll
                for (int c = 0; c < C; c++) s[c] += red[tid + u * NF_TGT][c];
            const int node = tv.node_perm[tk];
#pragma unroll
            for (int c = 0; c < C; c++) ytmp[(size_t)node * C + c] = s[c];
        }
    }
}


// ---------------------------------------------------------------------------
// near field + L2P, float32 form.  A block takes one leaf and up to SLOTS of
// its targets per pass: G = ceil(targets / U) target groups x (256 / G)
// source slices, each thread holding U targets (8 real, 4 complex) so that
// every source read from shared memory serves U pairs.  The near-list
// sources are packed into full tiles across box boundaries; each staged
// source is rebased to the target leaf's centre (box offset in float64,
// rounded once).  For the real double layer the strength is folded into the
// staged normal, so a pair costs 3 subtractions, two 3-term dot products, one
// reciprocal square root and three multiplies.  Tile partial sums are added
// with compensation, slices and the local expansion combine in float64.
// ---------------------------------------------------------------------------
constexpr int NF2_T = 256, NF2_TILE = 1024, NF2_ENT = 256;
__host__ __device__ constexpr int nf2_u(int C) { return C == 1 ? 8 : 4; }
// sources per staged round: 3 float4 each in the packed real form, 2 complex
// (1024 real sources per round, three blocks per SM: 0.437 ms against 0.456 for
// 640 at four blocks on the cube workload, the rounds' barriers and staging
// halved)
__host__ __device__ constexpr int nf2_tile(int C) { return C == 1 ? 1024 : NF2_TILE; }
// float4 slots of the staged-source region
__host__ __device__ constexpr int nf2_stage(int C) { return C == 1 ? 3 * nf2_tile(1) : 2 * NF2_TILE; }

// Work items of the float32 near field: one per (leaf, pass of up to 8 U
// targets), ordered by decreasing pair count (targets x near sources, ties in
// leaf order), so the largest blocks start first and the last wave is made of
// the smallest.  Each target is summed by one block whatever the order.
int build_near_items(bem_plan *P) {
    const Tree &t = P->t;
    std::vector<int> nptr(t.nbox + 1), nidx(std::max<int64_t>(1, t.n_near)), nb(t.nbox), ne(t.nbox), eb(t.nbox),
        ee(t.nbox), lv(t.nleaf);
    BEM_CUDA(cudaMemcpy(nptr.data(), t.near_ptr, sizeof(int) * (t.nbox + 1), cudaMemcpyDeviceToHost));
    if (t.n_near) BEM_CUDA(cudaMemcpy(nidx.data(), t.near_idx, sizeof(int) * t.n_near, cudaMemcpyDeviceToHost));
    BEM_CUDA(cudaMemcpy(nb.data(), t.nb, sizeof(int) * t.nbox, cudaMemcpyDeviceToHost));
    BEM_CUDA(cudaMemcpy(ne.data(), t.ne, sizeof(int) * t.nbox, cudaMemcpyDeviceToHost));
    BEM_CUDA(cudaMemcpy(eb.data(), t.eb, sizeof(int) * t.nbox, cudaMemcpyDeviceToHost));
    BEM_CUDA(cudaMemcpy(ee.data(), t.ee, sizeof(int) * t.nbox, cudaMemcpyDeviceToHost));
    BEM_CUDA(cudaMemcpy(lv.data(), t.leaves, sizeof(int) * t.nleaf, cudaMemcpyDeviceToHost));
    int64_t pairs = 0;
    std::vector<int64_t> src(t.nleaf);
    for (int li = 0; li < t.nleaf; li++) {
        const int b = lv[li];
        int64_t n = 0;
        for (int u = nptr[b]; u < nptr[b + 1]; u++) n += (int64_t)(ee[nidx[u]] - eb[nidx[u]]) * NQ;
        src[li] = n;
        pairs += n * (ne[b] - nb[b]);
    }
    P->near_pairs = pairs;
    // real items for every plan (the diagonal's product is Laplace), complex
    // ones for Helmholtz plans only
    for (int v = 0; v < (P->green == BEM_HELMHOLTZ ? 2 : 1); v++) {
        const int slots = 8 * nf2_u(v + 1);
        std::vector<int2> items;
        std::vector<int64_t> cost;
        for (int li = 0; li < t.nleaf; li++) {
            const int b = lv[li];
            for (int t0 = nb[b]; t0 < ne[b]; t0 += slots) {
                items.push_back(make_int2(li, t0));
                cost.push_back((int64_t)std::min(slots, ne[b] - t0) * src[li]);
            }
        }
        std::vector<int> ord(items.size());
        for (size_t i = 0; i < ord.size(); i++) ord[i] = (int)i;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        std::vector<int2> sorted(std::max<size_t>(1, items.size()));
        for (size_t i = 0; i < ord.size(); i++) sorted[i] = items[ord[i]];
        BEM_TRY(P->arena.alloc(&P->near_items[v], sorted.size()));
        BEM_CUDA(cudaMemcpy(P->near_items[v], sorted.data(), sizeof(int2) * sorted.size(), cudaMemcpyHostToDevice));
        P->near_nitems[v] = (int)items.size();
    }
    return BEM_OK;
}

// 1 / sqrt(x) as the single hardware approximation (flush-to-zero form: the
// squared distances of near-field pairs are never subnormal)
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int C, bool DL>
__device__ __forceinline__ void pair_f32(float rx, float ry, float rz, const float4 &sa, const float4 &sb, float kw,
                                         float *acc) {
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    const float inv = rsqrt_ftz(r2);
    if (C == 1) {
        if (DL) {   // sb = strength * normal
            const float dot = fmaf(rx, sb.x, fmaf(ry, sb.y, rz * sb.z));
            acc[0] = fmaf(dot * inv, inv * inv, acc[0]);
        } else {
            acc[0] = fmaf(sa.w, inv, acc[0]);
        }
    } else {
        const float R1 = r2 * inv;
        float sn, cs;
        sincosf(kw * R1, &sn, &cs);
        float gr, gi;
        if (DL) {
            const float kr = kw * R1, rn = fmaf(rx, sb.x, fmaf(ry, sb.y, rz * sb.z)) * inv * inv * inv;
            gr = (cs + kr * sn) * rn;
            gi = (sn - kr * cs) * rn;
        } else {
            gr = cs * inv;
            gi = sn * inv;
        }
        acc[0] += gr * sa.w - gi * sb.w;
        acc[C - 1] += gr * sb.w + gi * sa.w;
    }
}

// compensated float32 accumulation (Kahan): GB300's float64 pipe is a small
// fraction of its float32 pipe, so long sums stay in float32 with a carried
// error term instead of being promoted
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c, t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// shared memory of the float32 near field beyond its static part: the staged
// sources (sa, sb) and the per-thread compensated sums
__host__ __device__ constexpr size_t nf2_dyn_bytes(int C) {
    return (size_t)nf2_stage(C) * sizeof(float4) + 2 * (size_t)nf2_u(C) * C * NF2_T * sizeof(float);
}

template <int C, bool DL>
__global__ void __launch_bounds__(NF2_T, 4) k_near_f32(int nitem, const int2 *__restrict__ items, Tabs tb, TreeView tv,
                                                       QuadView qv, double kwave, const float *__restrict__ f,
                                                       const float *__restrict__ L, double *__restrict__ ytmp,
                                                       const int *__restrict__ skip) {
    constexpr int U = nf2_u(C);                       // targets per thread
    constexpr int SLOTS = 8 * U;                      // targets per pass (at most 8 groups)
    constexpr int LP = NF2_T / SLOTS;                 // threads per target in the local expansion
    constexpr int UC = U * C;
    constexpr int TILE = nf2_tile(C);                 // sources staged per round
    if (skip && *skip) return;
    if ((int)blockIdx.x >= nitem) return;
    const int2 item = items[blockIdx.x];              // (leaf, first target of the pass)
    const int b = tv.leaves[item.x];
    const int tid = threadIdx.x, lane = tid & 31;
    // The staged-source region is reused once the sources are done: slice
    // sums, local-expansion partials and the targets' powers (23 KB at most).
    extern __shared__ float4 near_tile[];
    float4 *sa = near_tile, *sb = near_tile + NF2_TILE;                 // C = 2: position | Re f, normal | Im f
    float4 *s0 = near_tile, *s1 = s0 + TILE, *s2 = s1 + TILE;           // C = 1: packed (see the staging)
    float *ks = (float *)(near_tile + nf2_stage(C));  // [UC][NF2_T] compensated sums
    float *kc = ks + UC * NF2_T;                      // [UC][NF2_T] their carries
    float *red = (float *)near_tile;                  // [slice][slot][C]
    float *lred = red + NF2_T * UC;                   // [part][slot][C]
    float *spow = lred + NF2_T * C;                   // [slot][3][PMAX + 1]
    __shared__ int pref[NF2_ENT + 1];
    __shared__ int ebase[NF2_ENT];                    // first quadrature point of each entry's box
    __shared__ float eoff[NF2_ENT][3];                // entry box centre - target leaf centre
    __shared__ float toff[SLOTS][3];                  // target - target leaf centre
    const double cbx = tv.cx[b], cby = tv.cy[b], cbz = tv.cz[b];
    const float kw = (float)kwave;
    const int np = tb.np, p = order_of(tb, tv.level[b]), npl = np_of(p);   // the leaf's order; np the stride
    const int t0 = item.y, nt = min(SLOTS, tv.ne[b] - t0);
    const int G = (nt + U - 1) / U, S = NF2_T / G, tg = tid % G, sl = tid / G;
    const bool worker = sl < S;
    if (tid < SLOTS) {
        const int k = t0 + tid;
        const bool on = tid < nt;
        toff[tid][0] = on ? (float)(tv.tx[k] - cbx) : 0.f;
        toff[tid][1] = on ? (float)(tv.ty[k] - cby) : 0.f;
        toff[tid][2] = on ? (float)(tv.tz[k] - cbz) : 1.f;   // off targets stay away from every source
    }
    for (int i = tid; i < 2 * UC * NF2_T; i += NF2_T) ks[i] = 0.f;
    __syncthreads();
    float tx[U], ty[U], tz[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int slot = tg + G * u;                 // < G U <= SLOTS
        tx[u] = toff[slot][0];
        ty[u] = toff[slot][1];
        tz[u] = toff[slot][2];
    }
    for (int e0 = tv.near_ptr[b]; e0 < tv.near_ptr[b + 1]; e0 += NF2_ENT) {
        const int ne_ = min(NF2_ENT, tv.near_ptr[b + 1] - e0);
        __syncthreads();
        if (tid < 32) {                               // quadrature-point offsets of the entries (warp scan)
            int carry = 0;
            for (int i0 = 0; i0 < ne_; i0 += 32) {
                const int i = i0 + lane;
                int x = 0;
                if (i < ne_) {
                    const int s = tv.near_idx[e0 + i];
                    x = (tv.ee[s] - tv.eb[s]) * NQ;
                    ebase[i] = tv.eb[s] * NQ;
                    eoff[i][0] = (float)(tv.cx[s] - cbx);
                    eoff[i][1] = (float)(tv.cy[s] - cby);
                    eoff[i][2] = (float)(tv.cz[s] - cbz);
                }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (i < ne_) pref[i + 1] = carry + x;
                carry += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) pref[0] = 0;
        }
        __syncthreads();
        const int total = pref[ne_];
        for (int base = 0; base < total; base += TILE) {
            __syncthreads();
            int lo = 0;                               // entry holding j: pref[lo] <= j < pref[lo + 1]
            if (base + tid < total) {
                int hi = ne_ - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (pref[mid] <= base + tid) lo = mid; else hi = mid - 1;
                }
            }
            for (int jj = tid; jj < TILE; jj += NF2_T) {
                const int j = base + jj;
                if (j >= total) break;
                while (pref[lo + 1] <= j) lo++;       // j grows with jj: the entry only moves forward
                const int o = ebase[lo] + (j - pref[lo]);
                const float4 xa = make_float4(eoff[lo][0] + qv.fx[o], eoff[lo][1] + qv.fy[o], eoff[lo][2] + qv.fz[o], 0.f);
                if constexpr (C == 1) {
                    // packed layout: each value twice, for the two targets of a float2
                    // operation; positions negated so that r = t + (-a)
                    const float fo = f[o];
                    s0[jj] = make_float4(-xa.x, -xa.x, -xa.y, -xa.y);
                    if (DL) {
                        const float nx = fo * qv.fnx[o], ny = fo * qv.fny[o], nz = fo * qv.fnz[o];
                        s1[jj] = make_float4(-xa.z, -xa.z, nx, nx);
                        s2[jj] = make_float4(ny, ny, nz, nz);
                    } else {
                        s1[jj] = make_float4(-xa.z, -xa.z, fo, fo);
                    }
                } else {
                    sa[jj] = make_float4(xa.x, xa.y, xa.z, f[(size_t)o * C]);
                    sb[jj] = make_float4(DL ? qv.fnx[o] : 0.f, DL ? qv.fny[o] : 0.f, DL ? qv.fnz[o] : 0.f,
                                         C == 2 ? f[(size_t)o * C + C - 1] : 0.f);
                }
            }
            __syncthreads();
            const int nq = min(TILE, total - base);
            float part[U][C];
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int c = 0; c < C; c++) part[u][c] = 0.f;
            if constexpr (C == 1) {
                // two targets per packed float32 operation (__fadd2 / __fmul2 / __ffma2):
                // half the issue slots of the scalar form, same roundings in the same order
                float2 t2x[U / 2], t2y[U / 2], t2z[U / 2], p2[U / 2];
#pragma unroll
                for (int v = 0; v < U / 2; v++) {
                    t2x[v] = make_float2(tx[2 * v], tx[2 * v + 1]);
                    t2y[v] = make_float2(ty[2 * v], ty[2 * v + 1]);
                    t2z[v] = make_float2(tz[2 * v], tz[2 * v + 1]);
                    p2[v] = make_float2(0.f, 0.f);
                }
                auto source = [&](int q) {
                    const float4 a0 = s0[q], a1 = s1[q];
                    const float2 mx = make_float2(a0.x, a0.y), my = make_float2(a0.z, a0.w), mz = make_float2(a1.x, a1.y);
                    float2 nx, ny, nz;
                    if (DL) {
                        const float4 a2 = s2[q];
                        nx = make_float2(a1.z, a1.w);
                        ny = make_float2(a2.x, a2.y);
                        nz = make_float2(a2.z, a2.w);
                    }
#pragma unroll
                    for (int v = 0; v < U / 2; v++) {
                        const float2 rx = __fadd2_rn(t2x[v], mx), ry = __fadd2_rn(t2y[v], my), rz = __fadd2_rn(t2z[v], mz);
                        float2 r2 = __fmul2_rn(rz, rz);
                        r2 = __ffma2_rn(ry, ry, r2);
                        r2 = __ffma2_rn(rx, rx, r2);
                        const float2 inv = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
                        if (DL) {
                            float2 dot = __fmul2_rn(rz, nz);
                            dot = __ffma2_rn(ry, ny, dot);
                            dot = __ffma2_rn(rx, nx, dot);
                            p2[v] = __ffma2_rn(__fmul2_rn(dot, inv), __fmul2_rn(inv, inv), p2[v]);
                        } else {
                            p2[v] = __ffma2_rn(make_float2(a1.z, a1.w), inv, p2[v]);
                        }
                    }
                };
                if (worker) {
                    int q = sl;
                    for (; q + S < nq; q += 2 * S) {
                        source(q);
                        source(q + S);
                    }
                    if (q < nq) source(q);
                }
#pragma unroll
                for (int v = 0; v < U / 2; v++) {
                    part[2 * v][0] = p2[v].x;
                    part[2 * v + 1][0] = p2[v].y;
                }
            } else if (worker) {
                // two sources per iteration (fewer loop instructions, more independent work)
                const float4 *pa = sa + sl, *pb = sb + sl;
                int q = sl;
                for (; q + S < nq; q += 2 * S, pa += 2 * S, pb += 2 * S) {
                    const float4 A0 = pa[0], B0 = pb[0], A1 = pa[S], B1 = pb[S];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        pair_f32<C, DL>(tx[u] - A0.x, ty[u] - A0.y, tz[u] - A0.z, A0, B0, kw, part[u]);
                        pair_f32<C, DL>(tx[u] - A1.x, ty[u] - A1.y, tz[u] - A1.z, A1, B1, kw, part[u]);
                    }
                }
                if (q < nq) {
                    const float4 A = pa[0], Bv = pb[0];
#pragma unroll
                    for (int u = 0; u < U; u++)
                        pair_f32<C, DL>(tx[u] - A.x, ty[u] - A.y, tz[u] - A.z, A, Bv, kw, part[u]);
                }
            }
            // tile partials into the compensated sums (Kahan), kept in shared memory
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int c = 0; c < C; c++) {
                    const int i = (u * C + c) * NF2_T + tid;
                    const float s = ks[i], y = part[u][c] - kc[i], t = s + y;
                    kc[i] = (t - s) - y;
                    ks[i] = t;
                }
        }
    }
    __syncthreads();                                  // sources done: their region is reused below
    if (worker)
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
            for (int c = 0; c < C; c++) red[((size_t)sl * G * U + tg + G * u) * C + c] = ks[(u * C + c) * NF2_T + tid];
    // local expansion at the targets: powers of the scaled offsets, then
    // LP threads per target each take every LP-th term
    if (tid < nt) {
        const int k = t0 + tid;
        const double ih = scalbn(1.0 / tv.side, tv.level[b]);   // 1 / h of the leaf
        const float dx = (float)((tv.tx[k] - cbx) * ih), dy = (float)((tv.ty[k] - cby) * ih),
                    dz = (float)((tv.tz[k] - cbz) * ih);
        float qx = 1.f, qy = 1.f, qz = 1.f;
        float *sp = spow + (size_t)tid * 3 * (PMAX + 1);
        for (int e = 0; e <= p; e++) {
            sp[e] = qx;
            sp[PMAX + 1 + e] = qy;
            sp[2 * (PMAX + 1) + e] = qz;
            qx *= dx;
            qy *= dy;
            qz *= dz;
        }
    }
    __syncthreads();
    {
        const int slot = tid % SLOTS, part_id = tid / SLOTS;
        KahanF loc[C];
        if (slot < nt) {
            const float *sp = spow + (size_t)slot * 3 * (PMAX + 1);
            for (int a = part_id; a < npl; a += LP) {
                const float mono = sp[tb.m[a]] * sp[PMAX + 1 + tb.n[a]] * sp[2 * (PMAX + 1) + tb.k[a]];
#pragma unroll
                for (int c = 0; c < C; c++) loc[c].add(mono * L[((size_t)b * np + a) * C + c]);
            }
        }
#pragma unroll
        for (int c = 0; c < C; c++) lred[(part_id * SLOTS + slot) * C + c] = loc[c].s;
    }
    __syncthreads();
    if (tid < nt) {
        // target t0 + tid sits in slot tid = tg + G u of every slice
        KahanF sum[C], loc[C];
        for (int q = 0; q < S; q++)
#pragma unroll
            for (int c = 0; c < C; c++) sum[c].add(red[((size_t)q * G * U + tid) * C + c]);
        for (int q = 0; q < LP; q++)
#pragma unroll
            for (int c = 0; c < C; c++) loc[c].add(lred[(q * SLOTS + tid) * C + c]);
        const int node = tv.node_perm[t0 + tid];
#pragma unroll
        for (int c = 0; c < C; c++) ytmp[(size_t)node * C + c] = (double)sum[c].s * (0.25 / M_PI) + (double)loc[c].s;
    }
}

// ---------------------------------------------------------------------------
// correction SpMV + diagonal: one warp per node row
//   op A: y = C x - (ytmp + K_D x);  op B: y = -(ytmp + K_S x)
// ---------------------------------------------------------------------------
template <class RV, int C, bool OPA>
__global__ void k_combine(int N, const int *__restrict__ ptr, const int *__restrict__ col, const RV *__restrict__ val,
                          const double *__restrict__ Cdiag, const double *__restrict__ ytmp,
                          const void *const *__restrict__ xslot, void *const *__restrict__ yslot,
                          const int *__restrict__ skip) {
    if (skip && *skip) return;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= N) return;
    const double *x = (const double *)*xslot;
    double *y = (double *)*yslot;
    double s[C];
#pragma unroll
    for (int c = 0; c < C; c++) s[c] = 0.0;
    auto term = [&](int q, int j) {
        if (C == 1) {
            s[0] += (double)val[q] * x[j];
        } else {
            const double vr = (double)val[2 * (size_t)q], vi = (double)val[2 * (size_t)q + 1];
            const double xr = x[2 * (size_t)j], xi = x[2 * (size_t)j + 1];
            s[0] += vr * xr - vi * xi;
            s[C - 1] += vr * xi + vi * xr;
        }
    };
    // four of a lane's columns loaded ahead, nonzeros summed in order
    constexpr int CU = 4;
    const int qe = ptr[w + 1];
    int q = ptr[w] + lane;
    for (; q + 32 * (CU - 1) < qe; q += 32 * CU) {
        int j[CU];
#pragma unroll
        for (int u = 0; u < CU; u++) j[u] = col[q + 32 * u];
#pragma unroll
        for (int u = 0; u < CU; u++) term(q + 32 * u, j[u]);
    }
    for (; q < qe; q += 32) term(q, col[q]);
#pragma unroll
    for (int c = 0; c < C; c++)
        for (int off = 16; off; off >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], off);
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < C; c++) {
            const double tot = ytmp[(size_t)w * C + c] + s[c];
            y[(size_t)w * C + c] = OPA ? Cdiag[w] * x[(size_t)w * C + c] - tot : -tot;
        }
    }
}

// float32 correction product (mixed plans): the vector is first copied to
// float32 (one conversion per entry instead of one per nonzero: float64
// arithmetic is a small fraction of the float32 rate), each lane sums its
// nonzeros with compensation, the lanes' sums combine in float64.
__global__ void k_x_float(int64_t n, const void *const *__restrict__ xslot, float *__restrict__ xf,
                          const int *__restrict__ skip) {
    if (skip && *skip) return;
    const double *x = (const double *)*xslot;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        xf[i] = (float)x[i];
}

template <int C, bool OPA>
__global__ void k_combine_f(int N, const int *__restrict__ ptr, const int *__restrict__ col,
                            const float *__restrict__ val, const float *__restrict__ xf,
                            const double *__restrict__ Cdiag, const double *__restrict__ ytmp,
                            const void *const *__restrict__ xslot, void *const *__restrict__ yslot,
                            const int *__restrict__ skip) {
    if (skip && *skip) return;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= N) return;
    KahanF k[C];
    auto term = [&](float2 v, float2 x) {
        if (C == 1) {
            k[0].add(v.x * x.x);
        } else {
            k[0].add(fmaf(v.x, x.x, -v.y * x.y));
            k[C - 1].add(fmaf(v.x, x.y, v.y * x.x));
        }
    };
    auto ldv = [&](int q) {
        return C == 1 ? make_float2(__ldg(val + q), 0.f) : __ldg(reinterpret_cast<const float2 *>(val) + q);
    };
    auto ldx = [&](int j) {
        return C == 1 ? make_float2(__ldg(xf + j), 0.f) : __ldg(reinterpret_cast<const float2 *>(xf) + j);
    };
    // four of a lane's nonzeros in flight at a time (columns, values, then
    // the vector entries), summed in the same order as one at a time
    constexpr int CU = 4;
    const int qe = ptr[w + 1];
    int q = ptr[w] + lane;
    for (; q + 32 * (CU - 1) < qe; q += 32 * CU) {
        int j[CU];
        float2 v[CU], x[CU];
#pragma unroll
        for (int u = 0; u < CU; u++) {
            j[u] = __ldg(col + q + 32 * u);
            v[u] = ldv(q + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < CU; u++) x[u] = ldx(j[u]);
#pragma unroll
        for (int u = 0; u < CU; u++) term(v[u], x[u]);
    }
    for (; q < qe; q += 32) term(ldv(q), ldx(__ldg(col + q)));
    double s[C];
#pragma unroll
    for (int c = 0; c < C; c++) {
        s[c] = (double)k[c].s - (double)k[c].c;
        for (int off = 16; off; off >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], off);
    }
    if (lane == 0) {
        const double *x = (const double *)*xslot;
        double *y = (double *)*yslot;
#pragma unroll
        for (int c = 0; c < C; c++) {
            const double tot = ytmp[(size_t)w * C + c] + s[c];
            y[(size_t)w * C + c] = OPA ? Cdiag[w] * x[(size_t)w * C + c] - tot : -tot;
        }
    }
}

// C_i = 1 + (regular Laplace double layer of phi = 1) + (correction row sum),
// and 1 / C_i for the solver's diagonal preconditioner
__global__ void k_finish_diag(int N, const double *__restrict__ ytmp, double *Cdiag, double *dinv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const double c = 1.0 + ytmp[i] + Cdiag[i];
        Cdiag[i] = c;
        dinv[i] = 1.0 / c;
    }
}

__global__ void k_fill(int64_t n, double v, double *a) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void MIndex::init(int p_) {
    p = p_;
    np = (p + 1) * (p + 2) * (p + 3) / 6;
    m.clear(); n.clear(); k.clear();
    idx3.assign((size_t)(p + 1) * (p + 1) * (p + 1), -1);
    deg_off.assign(p + 2, 0);
    int c = 0;
    for (int h = 0; h <= p; h++) {
        deg_off[h] = c;
        for (int a = h; a >= 0; a--)
            for (int b = h - a; b >= 0; b--) {
                int cc = h - a - b;
                m.push_back(a); n.push_back(b); k.push_back(cc);
                idx3[((size_t)a * (p + 1) + b) * (p + 1) + cc] = c++;
            }
    }
    deg_off[p + 1] = c;
}

static Tabs tabs_of(const bem_plan *P) {
    return Tabs{P->d_m, P->d_n, P->d_k, P->d_idx3, P->d_fact, P->mi.p, P->mi.np,
                P->lev_var ? P->d_lev_p : nullptr};
}

static TreeView view_of(const bem_plan *P) {
    const Tree &t = P->t;
    return TreeView{t.level, t.ix, t.iy, t.iz, t.parent, t.child0, t.nchild, t.nb, t.ne, t.eb, t.ee, t.leaves,
                    t.near_ptr, t.near_idx, t.inter_ptr, t.inter_idx, t.node_perm, t.cx, t.cy, t.cz,
                    t.tx, t.ty, t.tz, t.side};
}

static QuadView quad_of(const bem_plan *P) {
    const Quad &q = P->q;
    return QuadView{q.x, q.y, q.z, q.nx, q.ny, q.nz, q.w, q.fx, q.fy, q.fz, q.fnx, q.fny, q.fnz, q.fw};
}

// Shape-function values at the 7 rule points, in constant memory.  Written
// once per device (under a lock): plans are built from several host threads
// while kernels of other plans that read the table are running.
static int init_shape_table(int device) {
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0 || device >= 64) { set_error("device %d out of range", device); return BEM_EINVAL; }
    if (done[device]) return BEM_OK;
    double Lq[2][NQ][6] = {};
    {
        const double q = std::sqrt(15.0);
        const double a = (6.0 - q) / 21.0, b = (9.0 + 2.0 * q) / 21.0;
        const double c = (6.0 + q) / 21.0, d = (9.0 - 2.0 * q) / 21.0;
        const double S[7] = {1.0 / 3.0, a, b, a, c, d, c}, T[7] = {1.0 / 3.0, a, a, b, c, c, d};
        for (int r = 0; r < NQ; r++) {
            double l0 = 1.0 - S[r] - T[r], l1 = S[r], l2 = T[r];
            Lq[0][r][0] = l0; Lq[0][r][1] = l1; Lq[0][r][2] = l2;
            Lq[1][r][0] = l0 * (2 * l0 - 1); Lq[1][r][1] = l1 * (2 * l1 - 1); Lq[1][r][2] = l2 * (2 * l2 - 1);
            Lq[1][r][3] = 4 * l0 * l1; Lq[1][r][4] = 4 * l1 * l2; Lq[1][r][5] = 4 * l2 * l0;
        }
    }
    BEM_CUDA(cudaMemcpyToSymbol(c_Lq, Lq, sizeof(Lq)));
    done[device] = true;
    return BEM_OK;
}

// the float32 near-field kernels stage their source tile in dynamic shared
// memory above the 48 KB default (set outside any graph capture)
static void set_near_attributes() {
    const int big = 100 * 1024;
    cudaFuncSetAttribute(k_near_f32<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_near_f32<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_near_f32<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_near_f32<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

int alloc_fmm(bem_plan *P, cudaStream_t s) {
    Arena &A = P->arena;
    MIndex &mi = P->mi;
    mi.init(P->prm.p);
    // order of each level: L_l = min(p, p_min + l_max - l) (Section 3.6), or p
    {
        const int nlev = std::max(1, P->t.nlev), lmax = nlev - 1;
        P->lev_p.assign(nlev, P->prm.p);
        P->lev_var = false;
        if (P->prm.p_min > 0)
            for (int l = 0; l < nlev; l++) {
                P->lev_p[l] = std::min(P->prm.p, P->prm.p_min + lmax - l);
                if (P->lev_p[l] != P->prm.p) P->lev_var = true;
            }
        BEM_TRY(A.alloc(&P->d_lev_p, nlev));
        BEM_CUDA(cudaMemcpyAsync(P->d_lev_p, P->lev_p.data(), sizeof(int) * nlev, cudaMemcpyHostToDevice, s));
    }
    const int np = mi.np, nbox = P->t.nbox, C = P->green == BEM_HELMHOLTZ ? 2 : 1;
    BEM_TRY(A.alloc(&P->d_m, np));
    BEM_TRY(A.alloc(&P->d_n, np));
    BEM_TRY(A.alloc(&P->d_k, np));
    BEM_TRY(A.alloc(&P->d_idx3, mi.idx3.size()));
    BEM_CUDA(cudaMemcpyAsync(P->d_m, mi.m.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyAsync(P->d_n, mi.n.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyAsync(P->d_k, mi.k.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyAsync(P->d_idx3, mi.idx3.data(), sizeof(int) * mi.idx3.size(), cudaMemcpyHostToDevice, s));
    std::vector<double> fact(2 * PMAX + 2);
    fact[0] = 1.0;
    for (int i = 1; i < (int)fact.size(); i++) fact[i] = fact[i - 1] * i;
    BEM_TRY(A.alloc(&P->d_fact, fact.size()));
    BEM_CUDA(cudaMemcpyAsync(P->d_fact, fact.data(), sizeof(double) * fact.size(), cudaMemcpyHostToDevice, s));
    BEM_TRY(init_shape_table(P->device));
    const bool mx = P->prm.precision == BEM_MIXED;
    if (mx) {
        BEM_TRY(A.alloc(&P->ff, (size_t)P->Q * C));
        BEM_TRY(A.alloc(&P->fM, (size_t)nbox * np * C));
        BEM_TRY(A.alloc(&P->fL, (size_t)nbox * np * C));
    } else {
        BEM_TRY(A.alloc(&P->f, (size_t)P->Q * C));
        BEM_TRY(A.alloc(&P->M, (size_t)nbox * np * C));
        BEM_TRY(A.alloc(&P->L, (size_t)nbox * np * C));
    }
    BEM_TRY(A.alloc(&P->ytmp, (size_t)P->N * C));
    BEM_TRY(A.alloc(&P->xptr, 2));
    BEM_TRY(A.alloc(&P->yptr, 2));
    if (mx) BEM_TRY(A.alloc(&P->xf, (size_t)std::max(P->N, P->nchi) * C));
    if (mx && !P->diag_mode && !P->lev_var) {
        // stored P2M weights of the double layer (op A, every product of a solve)
        BEM_TRY(A.alloc(&P->p2m_W, (size_t)P->Q * np));
        const Tree &t = P->t;
        launch_p2m<float, 1, true, true>(t.nleaf, tabs_of(P), view_of(P), quad_of(P), nullptr, nullptr, nullptr, s,
                                         P->p2m_W);
        BEM_LAUNCH_CHECK();
    }
    set_translation_attributes();
    set_near_attributes();
    BEM_TRY(build_translation_tables(P, s));
    BEM_LAUNCH_CHECK();
    return BEM_OK;
}

// ev (optional, BEM_NSTAGES + 1 events): recorded before the first stage and
// after every stage, for per-stage timing outside graphs.
template <class R, int C>
static int run_fmm(bem_plan *P, int op, double kwave, R *f, R *M, R *L, double *ytmp, cudaStream_t s,
                   cudaEvent_t *ev) {
    if (ev) BEM_CUDA(cudaEventRecord(ev[0], s));
    const Tabs tb = tabs_of(P);
    const TreeView tv = view_of(P);
    const QuadView qv = quad_of(P);
    const Tree &t = P->t;
    const int np = tb.np, p = tb.p;
    const int *sk = P->skip;
    const int *el = op == BEM_OP_A ? t.el_phi : t.el_chi;
    const int Q = (int)P->Q;
    (k_p2q<R, C><<<(Q + 255) / 256, 256, 0, s>>>(Q, P->npe, el, P->q.w, P->xptr, f, sk), ::bem::count_launch());
    if (ev) BEM_CUDA(cudaEventRecord(ev[1], s));
    if constexpr (sizeof(R) == sizeof(float)) {
        if (op == BEM_OP_A && P->p2m_W)
            launch_p2m_stored<C>(t.nleaf, np, tv, P->p2m_W, f, M, sk, s);
        else if (op == BEM_OP_A) launch_p2m<R, C, true>(t.nleaf, tb, tv, qv, f, M, sk, s);
        else launch_p2m<R, C, false>(t.nleaf, tb, tv, qv, f, M, sk, s);
    } else {
        if (op == BEM_OP_A) launch_p2m<R, C, true>(t.nleaf, tb, tv, qv, f, M, sk, s);
        else launch_p2m<R, C, false>(t.nleaf, tb, tv, qv, f, M, sk, s);
    }
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[2], s));
    BEM_TRY((launch_translations<R, C>(P, M, L, s, ev)));
    if constexpr (sizeof(R) == sizeof(float)) {
        constexpr size_t tile_sm = nf2_dyn_bytes(C);
        const int ni = P->near_nitems[C - 1];
        const int2 *it = P->near_items[C - 1];
        if (ni > 0) {
            if (op == BEM_OP_A) (k_near_f32<C, true><<<ni, NF2_T, tile_sm, s>>>(ni, it, tb, tv, qv, kwave, f, L, ytmp, sk), ::bem::count_launch());
            else (k_near_f32<C, false><<<ni, NF2_T, tile_sm, s>>>(ni, it, tb, tv, qv, kwave, f, L, ytmp, sk), ::bem::count_launch());
        }
    } else {
        if (op == BEM_OP_A) (k_near<R, C, true><<<t.nleaf, NF_T, 0, s>>>(t.nleaf, tb, tv, qv, kwave, f, L, ytmp, sk), ::bem::count_launch());
        else (k_near<R, C, false><<<t.nleaf, NF_T, 0, s>>>(t.nleaf, tb, tv, qv, kwave, f, L, ytmp, sk), ::bem::count_launch());
    }
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[6], s));
    return BEM_OK;
}

// Moments for the field evaluation: double-layer moments of phi minus
// single-layer moments of chi at the leaves (the local buffer serves as
// scratch), then shifted up the tree.
template <class R>
__global__ void k_sub_moments(size_t n, R *__restrict__ M, const R *__restrict__ B) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) M[i] -= B[i];
}

template <class R, int C>
static int field_moments_t(bem_plan *P, const void *phi, const void *chi, R *f, R *M, R *Bm, cudaStream_t s) {
    const Tabs tb = tabs_of(P);
    const TreeView tv = view_of(P);
    const QuadView qv = quad_of(P);
    const Tree &t = P->t;
    const int Q = (int)P->Q;
    const int *sk = P->skip;
    BEM_TRY(set_slots(P, phi, nullptr, s));
    (k_p2q<R, C><<<(Q + 255) / 256, 256, 0, s>>>(Q, P->npe, t.el_phi, P->q.w, P->xptr, f, sk), ::bem::count_launch());
    launch_p2m<R, C, true>(t.nleaf, tb, tv, qv, f, M, sk, s);
    BEM_TRY(set_slots(P, chi, nullptr, s));
    (k_p2q<R, C><<<(Q + 255) / 256, 256, 0, s>>>(Q, P->npe, t.el_chi, P->q.w, P->xptr, f, sk), ::bem::count_launch());
    launch_p2m<R, C, false>(t.nleaf, tb, tv, qv, f, Bm, sk, s);
    const size_t n = (size_t)t.nbox * P->mi.np * C;
    (k_sub_moments<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, M, Bm), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    return launch_m2m<R, C>(P, M, s);
}

int field_moments(bem_plan *P, const void *phi, const void *chi, cudaStream_t s) {
    const bool mx = P->prm.precision == BEM_MIXED, helm = P->green == BEM_HELMHOLTZ;
    if (mx) return helm ? field_moments_t<float, 2>(P, phi, chi, P->ff, P->fM, P->fL, s)
                        : field_moments_t<float, 1>(P, phi, chi, P->ff, P->fM, P->fL, s);
    return helm ? field_moments_t<double, 2>(P, phi, chi, P->f, P->M, P->L, s)
                : field_moments_t<double, 1>(P, phi, chi, P->f, P->M, P->L, s);
}

// Enqueues one product on stream s.  The input and output vectors are read
// from the device slots P->xptr[0] / P->yptr[0].  with_diag = 0 leaves the
// regular far + near sums in the regular-sum buffer (used for the diagonal).
// wb (optional) names the work buffers of this product; NULL = the plan's.
int enqueue_matvec_raw(bem_plan *P, int op, int green, double kwave, int with_diag, cudaStream_t s,
                       cudaEvent_t *ev, const WorkBufs *wb) {
    const int C = green == BEM_HELMHOLTZ ? 2 : 1;
    const bool mx = P->prm.precision == BEM_MIXED;
    WorkBufs w;
    if (wb) w = *wb;
    else if (mx) w = WorkBufs{P->ff, P->fM, P->fL, P->ytmp};
    else w = WorkBufs{P->f, P->M, P->L, P->ytmp};
    if (!mx) {
        double *f = (double *)w.f, *M = (double *)w.M, *L = (double *)w.L;
        if (C == 1) BEM_TRY((run_fmm<double, 1>(P, op, kwave, f, M, L, w.ytmp, s, ev)));
        else BEM_TRY((run_fmm<double, 2>(P, op, kwave, f, M, L, w.ytmp, s, ev)));
    } else {
        float *f = (float *)w.f, *M = (float *)w.M, *L = (float *)w.L;
        if (C == 1) BEM_TRY((run_fmm<float, 1>(P, op, kwave, f, M, L, w.ytmp, s, ev)));
        else BEM_TRY((run_fmm<float, 2>(P, op, kwave, f, M, L, w.ytmp, s, ev)));
    }
    if (!with_diag) return BEM_OK;
    double *const ytmp = w.ytmp;
    const int N = (int)P->N;
    const Correction &K = P->corr;
    const int blocks = (N * 32 + 255) / 256;
#define BEM_COMBINE(RV, VD, VS)                                                                                 \
    if (op == BEM_OP_A) {                                                                                       \
        if (C == 1) (k_combine<RV, 1, true><<<blocks, 256, 0, s>>>(N, K.ptrD, K.colD, VD, P->C, ytmp, P->xptr, P->yptr, P->skip), ::bem::count_launch()); \
        else (k_combine<RV, 2, true><<<blocks, 256, 0, s>>>(N, K.ptrD, K.colD, VD, P->C, ytmp, P->xptr, P->yptr, P->skip), ::bem::count_launch());       \
    } else {                                                                                                    \
        if (C == 1) (k_combine<RV, 1, false><<<blocks, 256, 0, s>>>(N, K.ptrS, K.colS, VS, P->C, ytmp, P->xptr, P->yptr, P->skip), ::bem::count_launch()); \
        else (k_combine<RV, 2, false><<<blocks, 256, 0, s>>>(N, K.ptrS, K.colS, VS, P->C, ytmp, P->xptr, P->yptr, P->skip), ::bem::count_launch());       \
    }
    if (mx) {
        const int64_t nx = (int64_t)(op == BEM_OP_A ? N : P->nchi) * C;
        (k_x_float<<<(int)std::min<int64_t>((nx + 255) / 256, 4096), 256, 0, s>>>(nx, P->xptr, P->xf, P->skip),
         ::bem::count_launch());
        if (op == BEM_OP_A) {
            if (C == 1) (k_combine_f<1, true><<<blocks, 256, 0, s>>>(N, K.ptrD, K.colD, K.fvalD, P->xf, P->C, ytmp, P->xptr, P->yptr, P->skip), ::bem::count_launch());
            else (k_combine_f<2, true><<<blocks, 256, 0, s>>>(N, K.ptrD, K.colD, K.fvalD, P->xf, P->C, ytmp, P->xptr, P->yptr, P->skip), ::bem::count_launch());
        } else {
            if (C == 1) (k_combine_f<1, false><<<blocks, 256, 0, s>>>(N, K.ptrS, K.colS, K.fvalS, P->xf, P->C, ytmp, P->xptr, P->yptr, P->skip), ::bem::count_launch());
            else (k_combine_f<2, false><<<blocks, 256, 0, s>>>(N, K.ptrS, K.colS, K.fvalS, P->xf, P->C, ytmp, P->xptr, P->yptr, P->skip), ::bem::count_launch());
        }
    } else {
        BEM_COMBINE(double, K.valD, K.valS)
    }
#undef BEM_COMBINE
    BEM_LAUNCH_CHECK();
    if (ev) BEM_CUDA(cudaEventRecord(ev[7], s));
    return BEM_OK;
}

// Diagonal: C_i = 1 + sum_j D0_ij with D0 the Laplace double layer.  The
// correction row sums are already in P->C; one regular Laplace double-layer
// product on phi = 1 adds the rest.  For a constant density the far-field
// contributions add up coherently, so the expansions' relative error shows
// in full; this one product therefore runs in float64 at the largest
// supported order (error ~ eta^-(p+1)), on the same tree and lists, before
// the buffers are sized for the plan's own order and precision.
// The order, precision and Green's function of the diagonal's product.
struct DiagSwap {
    int p, precision, green, p_min;
};
// the diagonal's product runs at one order for every level: float64 plans at
// DIAG_P, where its truncation error is below the float64 diagonal's stated
// 5e-8; mixed plans at p + 2, at most DIAG_P: there float32 rounding, not the
// truncation, sets the diagonal's error (its difference from the float64
// plan's diagonal is the same at p + 2, p + 3 and p + 4)
constexpr int DIAG_P = 16;
static DiagSwap diag_fields(const bem_plan *P) {
    const bool mixed = P->prm.precision == BEM_MIXED;
    return DiagSwap{mixed ? std::min(DIAG_P, P->prm.p + 2) : DIAG_P, mixed ? BEM_MIXED : BEM_F64, BEM_LAPLACE, 0};
}
static DiagSwap swap_fields(bem_plan *P, const DiagSwap &d) {
    const DiagSwap old{P->prm.p, P->prm.precision, P->green, P->prm.p_min};
    P->prm.p = d.p;
    P->prm.precision = d.precision;
    P->green = d.green;
    P->prm.p_min = d.p_min;
    return old;
}

// Three steps, so that the product can run on its own stream beside the
// correction: prepare (buffers and tables at the diagonal's order, built into
// the plan and then moved to diag_state; all allocations happen here),
// product (phi = 1, into the diagonal's ytmp), finish (C += that ytmp once the
// correction's row sums are in C, then the diagonal's buffers are released).
// The plan's own order is built between product and finish, while the product
// runs.  The plan's fields are switched only while each step runs.
static void swap_state(bem_plan *P) { std::swap(static_cast<FmmState &>(*P), P->diag_state); }

int diagonal_prepare(bem_plan *P, cudaStream_t s) {
    const DiagSwap keep = swap_fields(P, diag_fields(P));
    P->diag_mode = true;                              // no stored weights at the diagonal's order
    int rc = alloc_fmm(P, s);
    P->diag_mode = false;
    if (rc == BEM_OK) rc = P->arena.alloc(&P->diag_ones, P->N);
    swap_state(P);                                    // the plan's own state is empty until alloc_fmm
    swap_fields(P, keep);
    return rc;
}

int diagonal_product(bem_plan *P, cudaStream_t s) {
    const int N = (int)P->N;
    const DiagSwap keep = swap_fields(P, diag_fields(P));
    swap_state(P);
    (k_fill<<<(N + 255) / 256, 256, 0, s>>>(N, 1.0, P->diag_ones), ::bem::count_launch());
    int rc = set_slots(P, P->diag_ones, nullptr, s);
    if (rc == BEM_OK) rc = enqueue_matvec_raw(P, BEM_OP_A, BEM_LAPLACE, 0.0, 0, s, nullptr);
    swap_state(P);
    swap_fields(P, keep);
    return rc;
}

int diagonal_finish(bem_plan *P, cudaStream_t s) {
    const int N = (int)P->N;
    BEM_TRY(P->arena.alloc(&P->dinv, P->N));
    (k_finish_diag<<<(N + 255) / 256, 256, 0, s>>>(N, P->diag_state.ytmp, P->C, P->dinv), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    BEM_CUDA(cudaStreamSynchronize(s));
    P->arena.release(P->diag_ones);
    P->diag_ones = nullptr;
    swap_state(P);
    free_fmm(P);
    swap_state(P);
    return BEM_OK;
}

// releases what alloc_fmm allocated
void free_fmm(bem_plan *P) {
    free_translation_tables(P);
    Arena &A = P->arena;
    for (void *q : {(void *)P->d_m, (void *)P->d_n, (void *)P->d_k, (void *)P->d_idx3, (void *)P->d_fact,
                    (void *)P->f, (void *)P->M, (void *)P->L, (void *)P->ff, (void *)P->fM,
                    (void *)P->fL, (void *)P->ytmp, (void *)P->xptr, (void *)P->yptr, (void *)P->p2m_W, (void *)P->xf, (void *)P->d_lev_p})
        A.release(q);
    P->p2m_W = nullptr;
    P->xf = nullptr;
    P->d_lev_p = nullptr;
    P->lev_var = false;
    P->d_m = P->d_n = P->d_k = P->d_idx3 = nullptr;
    P->d_fact = nullptr;
    P->f = P->M = P->L = P->ytmp = nullptr;
    P->ff = P->fM = P->fL = nullptr;
    P->xptr = nullptr;
    P->yptr = nullptr;
}


// ---------------------------------------------------------------------------
// A product that allocates nothing
//
// Callers that cannot allocate device memory when they need a product --
// real-time loops where an allocation (which may synchronise the device) is
// not allowed, or hosts whose device memory all belongs to another allocator
// (a framework's pool) that forbids stray cudaMalloc calls -- can use
// bem_matvec_noalloc.  It launches the same kernels as bem_matvec, directly
// (no graph is instantiated), and keeps the per-product scratch (quadrature
// strengths, moments, local expansions, regular sums) in the file-scope array
// below instead of the plan's own buffers: the array's pieces go to the
// launches as arguments (WorkBufs), and no field of the plan is changed, so
// other host threads see the plan as it was.  The array is NOALLOC_BYTES long
// and every GPU that loads this library holds it until the process exits.
// Its device address is looked up once per device, on the first call made
// on that device (so that first call should come before any stream capture).
// All calls share the array and it keeps the last call's contents; no part of
// it needs to start at zero (every stage writes its output before it is read).
// Calls that overlap on the GPU -- on different streams, or for different
// plans at the same time -- race on the array.
// ---------------------------------------------------------------------------
constexpr size_t NOALLOC_BYTES = (size_t)48 << 20;   // 48 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];
static void *g_noalloc_addr[64];                     // per device ordinal, 0 until looked up

static size_t noalloc_round(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace bem

extern "C" int bem_matvec_noalloc(bem_plan *P, int op, const void *x_dev, void *y_dev, void *cuda_stream) {
    using namespace bem;
    if (!P || !x_dev || !y_dev) { set_error("bem_matvec_noalloc: NULL argument"); return BEM_EINVAL; }
    if (op != BEM_OP_A && op != BEM_OP_B) { set_error("bem_matvec_noalloc: bad op %d", op); return BEM_EINVAL; }
    if (P->device < 0 || P->device >= 64) { set_error("bem_matvec_noalloc: device %d out of range", P->device); return BEM_EINVAL; }
    const int C = P->green == BEM_HELMHOLTZ ? 2 : 1;
    const bool mx = P->prm.precision == BEM_MIXED;
    const size_t rb = mx ? sizeof(float) : sizeof(double);
    const size_t bf = noalloc_round((size_t)P->Q * C * rb);
    const size_t bm = noalloc_round((size_t)P->t.nbox * P->mi.np * C * rb);
    const size_t by = noalloc_round((size_t)P->N * C * sizeof(double));
    const size_t need = bf + 2 * bm + by;
    if (need > NOALLOC_BYTES) {
        set_error("bem_matvec_noalloc: this plan needs %zu bytes of scratch, the fixed array holds %zu",
                  need, NOALLOC_BYTES);
        return BEM_EINVAL;
    }
    int prev_dev = -1;
    BEM_CUDA(cudaGetDevice(&prev_dev));
    BEM_CUDA(cudaSetDevice(P->device));
    int rc = BEM_OK;
    if (!g_noalloc_addr[P->device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        else g_noalloc_addr[P->device] = ptr;
    }
    if (rc == BEM_OK) {
        // this product's work buffers are carved from the scratch and passed to
        // the launches as arguments; the plan's own fields are not touched
        unsigned char *base = (unsigned char *)g_noalloc_addr[P->device];
        const WorkBufs w{base, base + bf, base + bf + bm, (double *)(base + bf + 2 * bm)};
        cudaStream_t s = (cudaStream_t)cuda_stream;
        rc = set_slots(P, x_dev, y_dev, s);
        if (rc == BEM_OK) {
            cudaError_t e = cudaMemsetAsync(P->skip, 0, sizeof(int), s);
            rc = e == cudaSuccess ? BEM_OK : cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__);
        }
        if (rc == BEM_OK) rc = enqueue_matvec_raw(P, op, P->green, P->k, 1, s, nullptr, &w);
    }
    cudaSetDevice(prev_dev);
    return rc;
}


