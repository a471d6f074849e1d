// Element geometry at the regular quadrature points and the stored
// near-field correction of singular and near-singular pairs.
//
// Geometry (Section 2.2): isoparametric 3- and 6-node triangles, position,
// outward unit normal t1 x t2 / |t1 x t2| and Jacobian at each point of
// Radon's 7-point degree-5 rule, in owner order.  Positions follow a fixed
// FP64 operation order because the convergence radii are taken over them.
//
// Correction (Section 3.6: the near field is precomputed and stored as a
// sparse matrix): for every collocation node i and element e that is
//   singular       node i is a node of e, or
//   near-singular  |x_i - X_e(1/3,1/3)| < tau h_e  (h_e longest corner chord),
// the matrix stores (special rule - regular rule) integrals of L_a G and
// L_a dG/dn1, so that the fast method, which sums every pair with the regular
// rule, becomes exact on these pairs.  Special rules: Duffy-collapsed
// Gauss-Legendre product rule at the singular node (split at mid-side nodes);
// recursive 4-way subdivision until each piece is tau times its size away.
#include <cmath>
#include <vector>

#include "bem_internal.cuh"

namespace bem {

struct Rule7 {
    double s[7], t[7], w[7];
};

// Radon's rule (Stroud T2:5-1): centroid weight 9/80, two orbits with
// a = (6 - sqrt15)/21, b = (9 + 2 sqrt15)/21, weight (155 - sqrt15)/2400 and
// c = (6 + sqrt15)/21, d = (9 - 2 sqrt15)/21, weight (155 + sqrt15)/2400.
static Rule7 make_rule7() {
    Rule7 r;
    const double q = std::sqrt(15.0);
    const double a = (6.0 - q) / 21.0, b = (9.0 + 2.0 * q) / 21.0;
    const double c = (6.0 + q) / 21.0, d = (9.0 - 2.0 * q) / 21.0;
    const double wa = (155.0 - q) / 2400.0, wc = (155.0 + q) / 2400.0;
    const double S[7] = {1.0 / 3.0, a, b, a, c, d, c};
    const double T[7] = {1.0 / 3.0, a, a, b, c, c, d};
    const double W[7] = {9.0 / 80.0, wa, wa, wa, wc, wc, wc};
    for (int i = 0; i < 7; i++) { r.s[i] = S[i]; r.t[i] = T[i]; r.w[i] = W[i]; }
    return r;
}

// Gauss-Legendre nodes on [-1, 1] by Newton's method on P_n (three-term
// recurrence), weights 2 / ((1 - x^2) P_n'(x)^2).
static void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; i++) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

__constant__ Rule7 c_rule;
__constant__ double c_glx[64], c_glw[64];

// Shape functions in the fixed operation order that the radii and the pair
// classification rely on.  L0 = (1 - s) - t, L1 = s, L2 = t.
__device__ __forceinline__ void shape_rn(int npe, double s, double t, double N[6]) {
    double L0 = __dsub_rn(__dsub_rn(1.0, s), t), L1 = s, L2 = t;
    if (npe == 3) {
        N[0] = L0; N[1] = L1; N[2] = L2;
        return;
    }
    N[0] = __dmul_rn(L0, __dsub_rn(__dmul_rn(2.0, L0), 1.0));
    N[1] = __dmul_rn(L1, __dsub_rn(__dmul_rn(2.0, L1), 1.0));
    N[2] = __dmul_rn(L2, __dsub_rn(__dmul_rn(2.0, L2), 1.0));
    N[3] = __dmul_rn(__dmul_rn(4.0, L0), L1);
    N[4] = __dmul_rn(__dmul_rn(4.0, L1), L2);
    N[5] = __dmul_rn(__dmul_rn(4.0, L2), L0);
}

__device__ __forceinline__ void dshape(int npe, double s, double t, double Ns[6], double Nt[6]) {
    if (npe == 3) {
        Ns[0] = -1.0; Ns[1] = 1.0; Ns[2] = 0.0;
        Nt[0] = -1.0; Nt[1] = 0.0; Nt[2] = 1.0;
        return;
    }
    double L0 = 1.0 - s - t;
    Ns[0] = 1.0 - 4.0 * L0; Ns[1] = 4.0 * s - 1.0; Ns[2] = 0.0;
    Ns[3] = 4.0 * (L0 - s); Ns[4] = 4.0 * t; Ns[5] = -4.0 * t;
    Nt[0] = 1.0 - 4.0 * L0; Nt[1] = 0.0; Nt[2] = 4.0 * t - 1.0;
    Nt[3] = -4.0 * s; Nt[4] = 4.0 * s; Nt[5] = 4.0 * (L0 - t);
}

// x = sum_a N_a X_a, summed in node order with separate roundings.
__device__ __forceinline__ void map_rn(int npe, const double N[6], const double X[18], double x[3]) {
    x[0] = 0.0; x[1] = 0.0; x[2] = 0.0;
    for (int a = 0; a < npe; a++) {
        x[0] = __dadd_rn(x[0], __dmul_rn(N[a], X[3 * a]));
        x[1] = __dadd_rn(x[1], __dmul_rn(N[a], X[3 * a + 1]));
        x[2] = __dadd_rn(x[2], __dmul_rn(N[a], X[3 * a + 2]));
    }
}

__device__ __forceinline__ void load_elem(const double *__restrict__ nodes, const int *__restrict__ el, int npe,
                                          double X[18]) {
    for (int a = 0; a < npe; a++) {
        const double *p = nodes + 3 * (size_t)el[a];
        X[3 * a] = p[0]; X[3 * a + 1] = p[1]; X[3 * a + 2] = p[2];
    }
}

// normal (unit, outward) and Jacobian at (s, t)
__device__ __forceinline__ void normal_jac(int npe, double s, double t, const double X[18], double n[3], double &J) {
    double Ns[6], Nt[6], u[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    dshape(npe, s, t, Ns, Nt);
    for (int a = 0; a < npe; a++)
        for (int c = 0; c < 3; c++) {
            u[c] += Ns[a] * X[3 * a + c];
            v[c] += Nt[a] * X[3 * a + c];
        }
    n[0] = u[1] * v[2] - u[2] * v[1];
    n[1] = u[2] * v[0] - u[0] * v[2];
    n[2] = u[0] * v[1] - u[1] * v[0];
    J = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] /= J; n[1] /= J; n[2] /= J;
}

// ---------------------------------------------------------------------------
// regular quadrature points (owner order) and per-element centroid / size
// ---------------------------------------------------------------------------
__global__ void k_geometry(int E, int npe, const int *__restrict__ el_phi, const double *__restrict__ nodes,
                           const int *__restrict__ leaf_of_node, const double *__restrict__ cx,
                           const double *__restrict__ cy, const double *__restrict__ cz, double *qx, double *qy,
                           double *qz, double *qnx, double *qny, double *qnz, double *qw, float *fx, float *fy,
                           float *fz, float *fnx, float *fny, float *fnz, float *fw) {
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= E * NQ) return;
    int i = o / NQ, q = o % NQ;
    double X[18], N[6], x[3], n[3], J;
    load_elem(nodes, el_phi + (size_t)i * npe, npe, X);
    shape_rn(npe, c_rule.s[q], c_rule.t[q], N);
    map_rn(npe, N, X, x);
    normal_jac(npe, c_rule.s[q], c_rule.t[q], X, n, J);
    double w = c_rule.w[q] * J;
    qx[o] = x[0]; qy[o] = x[1]; qz[o] = x[2];
    qnx[o] = n[0]; qny[o] = n[1]; qnz[o] = n[2];
    qw[o] = w;
    int leaf = leaf_of_node[el_phi[(size_t)i * npe]];
    fx[o] = (float)(x[0] - cx[leaf]);
    fy[o] = (float)(x[1] - cy[leaf]);
    fz[o] = (float)(x[2] - cz[leaf]);
    fnx[o] = (float)n[0]; fny[o] = (float)n[1]; fnz[o] = (float)n[2];
    fw[o] = (float)w;
}

__global__ void k_elem_centroid(int E, int npe, const int *__restrict__ el_phi, const double *__restrict__ nodes,
                                double *ecx, double *ecy, double *ecz, double *eh) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E) return;
    double X[18], N[6], x[3];
    load_elem(nodes, el_phi + (size_t)i * npe, npe, X);
    shape_rn(npe, 1.0 / 3.0, 1.0 / 3.0, N);
    map_rn(npe, N, X, x);
    double h01 = dist3_rn(X[0], X[1], X[2], X[3], X[4], X[5]);
    double h12 = dist3_rn(X[3], X[4], X[5], X[6], X[7], X[8]);
    double h20 = dist3_rn(X[6], X[7], X[8], X[0], X[1], X[2]);
    double m = h01;
    if (h12 > m) m = h12;
    if (h20 > m) m = h20;
    ecx[i] = x[0]; ecy[i] = x[1]; ecz[i] = x[2]; eh[i] = m;
}

int build_geometry(bem_plan *P, cudaStream_t s) {
    Tree &t = P->t;
    Arena &A = P->arena;
    static bool consts = false;
    (void)consts;
    Rule7 r = make_rule7();
    BEM_CUDA(cudaMemcpyToSymbolAsync(c_rule, &r, sizeof(r), 0, cudaMemcpyHostToDevice, s));
    const int nd = P->prm.n_duffy;
    double gx[64], gw[64];
    gauss_legendre(nd, gx, gw);
    BEM_CUDA(cudaMemcpyToSymbolAsync(c_glx, gx, sizeof(double) * nd, 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyToSymbolAsync(c_glw, gw, sizeof(double) * nd, 0, cudaMemcpyHostToDevice, s));
    const int64_t Q = P->Q;
    Quad &q = P->q;
    BEM_TRY(A.alloc(&q.x, Q)); BEM_TRY(A.alloc(&q.y, Q)); BEM_TRY(A.alloc(&q.z, Q));
    BEM_TRY(A.alloc(&q.nx, Q)); BEM_TRY(A.alloc(&q.ny, Q)); BEM_TRY(A.alloc(&q.nz, Q));
    BEM_TRY(A.alloc(&q.w, Q));
    BEM_TRY(A.alloc(&q.fx, Q)); BEM_TRY(A.alloc(&q.fy, Q)); BEM_TRY(A.alloc(&q.fz, Q));
    BEM_TRY(A.alloc(&q.fnx, Q)); BEM_TRY(A.alloc(&q.fny, Q)); BEM_TRY(A.alloc(&q.fnz, Q));
    BEM_TRY(A.alloc(&q.fw, Q));
    (k_geometry<<<(int)((Q + 255) / 256), 256, 0, s>>>((int)P->E, P->npe, t.el_phi, P->nodes, t.leaf_of_node, t.cx,
                                                       t.cy, t.cz, q.x, q.y, q.z, q.nx, q.ny, q.nz, q.w, q.fx, q.fy,
                                                       q.fz, q.fnx, q.fny, q.fnz, q.fw), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    return BEM_OK;
}

// ---------------------------------------------------------------------------
// stored correction
// ---------------------------------------------------------------------------
struct CorrArgs {
    int N, E, npe, green, nd, maxdepth;
    double k, tau;
    const double *nodes;
    const int *el_phi, *el_chi;
    const double *ecx, *ecy, *ecz, *eh;   // per element centroid image and size
    const double *bcx, *bcy, *bcz, *brho; // per box centre and search radius
    const int *child0, *nchild, *eb, *ee;
};

// Per box: radius of a ball around the centre that holds every point a
// special pair can involve: max over the subtree's elements of
// max(|c_e - c| + tau h_e, max_a |X_a - c|), inflated by 1e-12.
__global__ void k_box_search_radius(CorrArgs a, int nbox, double *rho) {
    int b = blockIdx.x;
    if (b >= nbox) return;
    double m = 0.0;
    for (int i = a.eb[b] + threadIdx.x; i < a.ee[b]; i += blockDim.x) {
        double d = dist3_rn(a.ecx[i], a.ecy[i], a.ecz[i], a.bcx[b], a.bcy[b], a.bcz[b]) + a.tau * a.eh[i];
        for (int v = 0; v < a.npe; v++) {
            const double *p = a.nodes + 3 * (size_t)a.el_phi[(size_t)i * a.npe + v];
            d = fmax(d, dist3_rn(p[0], p[1], p[2], a.bcx[b], a.bcy[b], a.bcz[b]));
        }
        m = fmax(m, d);
    }
    __shared__ double red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int off = blockDim.x / 2; off; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x == 0) rho[b] = red[0] * (1.0 + 1e-12);
}

// 0 regular, 1 singular (*a_sing = local node), 2 near-singular
__device__ __forceinline__ int classify_pair(const CorrArgs &a, int node, const double xi[3], int e, int *a_sing) {
    const int *el = a.el_phi + (size_t)e * a.npe;
    for (int v = 0; v < a.npe; v++)
        if (el[v] == node) { *a_sing = v; return 1; }
    double d = dist3_rn(xi[0], xi[1], xi[2], a.ecx[e], a.ecy[e], a.ecz[e]);
    return d < __dmul_rn(a.tau, a.eh[e]) ? 2 : 0;
}

// Visits, for collocation node `node`, every element of a leaf whose search
// ball holds the node; writes special (element, kind) pairs when `out`.
__device__ int find_special(const CorrArgs &a, int node, int *out_e) {
    double xi[3] = {a.nodes[3 * (size_t)node], a.nodes[3 * (size_t)node + 1], a.nodes[3 * (size_t)node + 2]};
    int stack[8 * 24], sp = 0, cnt = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        int b = stack[--sp];
        double d = dist3_rn(xi[0], xi[1], xi[2], a.bcx[b], a.bcy[b], a.bcz[b]);
        if (d > a.brho[b]) continue;
        if (a.nchild[b] != 0) {
            for (int c = a.child0[b] + a.nchild[b] - 1; c >= a.child0[b]; c--) stack[sp++] = c;
            continue;
        }
        for (int e = a.eb[b]; e < a.ee[b]; e++) {
            int as;
            if (classify_pair(a, node, xi, e, &as)) {
                if (out_e) out_e[cnt] = e;
                cnt++;
            }
        }
    }
    return cnt;
}

__global__ void k_special_count(CorrArgs a, int *cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    cnt[i] = find_special(a, i, nullptr);
}

__global__ void k_special_write(CorrArgs a, const int *__restrict__ off, int *pair_e) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    find_special(a, i, pair_e + off[i]);
}

struct Acc {
    double Sre[6], Sim[6], Dre[6], Dim[6], D0[6];
};

// One quadrature point with reference-space weight wref.
// G = exp(jkR)/(4 pi R); dG/dn1 = exp(jkR)(1 - jkR) ((x - x1).n1)/(4 pi R^3).
__device__ __forceinline__ void acc_point(const CorrArgs &a, const double X[18], const double xi[3], double s,
                                          double t, double wref, Acc &A) {
    double N[6], x[3], n[3], J;
    shape_rn(a.npe, s, t, N);
    map_rn(a.npe, N, X, x);
    normal_jac(a.npe, s, t, X, n, J);
    double r0 = xi[0] - x[0], r1 = xi[1] - x[1], r2 = xi[2] - x[2];
    double R = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
    double rn = r0 * n[0] + r1 * n[1] + r2 * n[2];
    double w = wref * J;
    const double inv4pi = 0.25 / M_PI;
    double G0 = inv4pi / R, dG0 = inv4pi * rn / (R * R * R);
    double Gre = G0, Gim = 0.0, dre = dG0, dim = 0.0;
    if (a.green == BEM_HELMHOLTZ) {
        double sn, cs;
        sincos(a.k * R, &sn, &cs);
        Gre = cs * G0; Gim = sn * G0;
        // (cs + j sn)(1 - j kR) = cs + kR sn + j (sn - kR cs)
        double kr = a.k * R;
        dre = (cs + kr * sn) * dG0;
        dim = (sn - kr * cs) * dG0;
    }
    for (int v = 0; v < a.npe; v++) {
        double wn = w * N[v];
        A.Sre[v] += wn * Gre; A.Sim[v] += wn * Gim;
        A.Dre[v] += wn * dre; A.Dim[v] += wn * dim;
        A.D0[v] += wn * dG0;
    }
}

__device__ void integrate_duffy(const CorrArgs &a, const double X[18], const double xi[3], const double P[2],
                                const double Q1[2], const double Q2[2], Acc &A) {
    double det = fabs((Q1[0] - P[0]) * (Q2[1] - P[1]) - (Q1[1] - P[1]) * (Q2[0] - P[0]));
    for (int iu = 0; iu < a.nd; iu++) {
        double u = 0.5 * (1.0 + c_glx[iu]), wu = 0.5 * c_glw[iu];
        for (int iv = 0; iv < a.nd; iv++) {
            double v = 0.5 * (1.0 + c_glx[iv]), wv = 0.5 * c_glw[iv];
            double s = P[0] + u * (Q1[0] - P[0]) + u * v * (Q2[0] - Q1[0]);
            double t = P[1] + u * (Q1[1] - P[1]) + u * v * (Q2[1] - Q1[1]);
            acc_point(a, X, xi, s, t, wu * wv * u * det, A);
        }
    }
}

__device__ void integrate_singular(const CorrArgs &a, const double X[18], const double xi[3], int as, Acc &A) {
    const double c0[2] = {0.0, 0.0}, c1[2] = {1.0, 0.0}, c2[2] = {0.0, 1.0};
    const double m3[2] = {0.5, 0.0}, m4[2] = {0.5, 0.5}, m5[2] = {0.0, 0.5};
    switch (as) {
    case 0: integrate_duffy(a, X, xi, c0, c1, c2, A); break;
    case 1: integrate_duffy(a, X, xi, c1, c2, c0, A); break;
    case 2: integrate_duffy(a, X, xi, c2, c0, c1, A); break;
    case 3: integrate_duffy(a, X, xi, m3, c1, c2, A); integrate_duffy(a, X, xi, m3, c2, c0, A); break;
    case 4: integrate_duffy(a, X, xi, m4, c2, c0, A); integrate_duffy(a, X, xi, m4, c0, c1, A); break;
    default: integrate_duffy(a, X, xi, m5, c0, c1, A); integrate_duffy(a, X, xi, m5, c1, c2, A); break;
    }
}

// Recursive 4-way split with an explicit stack (pieces processed depth first,
// children in the order (a,ab,ca), (ab,b,bc), (ca,bc,c), (ab,bc,ca)).
__device__ void integrate_subdivided(const CorrArgs &a, const double X[18], const double xi[3], Acc &A) {
    struct Piece { double a0, a1, b0, b1, c0, c1; int depth; };
    Piece st[4 * 8 + 4];
    int sp = 0;
    st[sp++] = {0.0, 0.0, 1.0, 0.0, 0.0, 1.0, 0};
    while (sp > 0) {
        Piece P = st[--sp];
        double N[6], xa[3], xb[3], xc[3], xm[3];
        double m0 = __ddiv_rn(__dadd_rn(__dadd_rn(P.a0, P.b0), P.c0), 3.0);
        double m1 = __ddiv_rn(__dadd_rn(__dadd_rn(P.a1, P.b1), P.c1), 3.0);
        shape_rn(a.npe, P.a0, P.a1, N); map_rn(a.npe, N, X, xa);
        shape_rn(a.npe, P.b0, P.b1, N); map_rn(a.npe, N, X, xb);
        shape_rn(a.npe, P.c0, P.c1, N); map_rn(a.npe, N, X, xc);
        shape_rn(a.npe, m0, m1, N); map_rn(a.npe, N, X, xm);
        double h = dist3_rn(xa[0], xa[1], xa[2], xb[0], xb[1], xb[2]);
        double h2 = dist3_rn(xb[0], xb[1], xb[2], xc[0], xc[1], xc[2]);
        double h3 = dist3_rn(xc[0], xc[1], xc[2], xa[0], xa[1], xa[2]);
        if (h2 > h) h = h2;
        if (h3 > h) h = h3;
        bool near = dist3_rn(xi[0], xi[1], xi[2], xm[0], xm[1], xm[2]) < __dmul_rn(a.tau, h);
        if (P.depth >= a.maxdepth || !near) {
            double det = fabs((P.b0 - P.a0) * (P.c1 - P.a1) - (P.b1 - P.a1) * (P.c0 - P.a0));
            for (int q = 0; q < NQ; q++) {
                double ps = P.a0 + c_rule.s[q] * (P.b0 - P.a0) + c_rule.t[q] * (P.c0 - P.a0);
                double pt = P.a1 + c_rule.s[q] * (P.b1 - P.a1) + c_rule.t[q] * (P.c1 - P.a1);
                acc_point(a, X, xi, ps, pt, c_rule.w[q] * det, A);
            }
            continue;
        }
        double ab0 = __dmul_rn(0.5, __dadd_rn(P.a0, P.b0)), ab1 = __dmul_rn(0.5, __dadd_rn(P.a1, P.b1));
        double bc0 = __dmul_rn(0.5, __dadd_rn(P.b0, P.c0)), bc1 = __dmul_rn(0.5, __dadd_rn(P.b1, P.c1));
        double ca0 = __dmul_rn(0.5, __dadd_rn(P.c0, P.a0)), ca1 = __dmul_rn(0.5, __dadd_rn(P.c1, P.a1));
        int d = P.depth + 1;
        // pushed in reverse so that they are processed in the listed order
        st[sp++] = {ab0, ab1, bc0, bc1, ca0, ca1, d};
        st[sp++] = {ca0, ca1, bc0, bc1, P.c0, P.c1, d};
        st[sp++] = {ab0, ab1, P.b0, P.b1, bc0, bc1, d};
        st[sp++] = {P.a0, P.a1, ab0, ab1, ca0, ca1, d};
    }
}

// One special (node, element) pair per thread: values (special - regular)
// for every local node, written in the pair's slot of the CSR arrays.
__global__ void k_special_integrate(CorrArgs a, int npairs, const int *__restrict__ pair_node,
                                    const int *__restrict__ pair_e, double *valD, double *valS, double *d0row) {
    int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= npairs) return;
    int node = pair_node[pr], e = pair_e[pr];
    double X[18], xi[3] = {a.nodes[3 * (size_t)node], a.nodes[3 * (size_t)node + 1], a.nodes[3 * (size_t)node + 2]};
    load_elem(a.nodes, a.el_phi + (size_t)e * a.npe, a.npe, X);
    int as = -1;
    int cls = classify_pair(a, node, xi, e, &as);
    Acc sp, rg;
    for (int v = 0; v < 6; v++) {
        sp.Sre[v] = sp.Sim[v] = sp.Dre[v] = sp.Dim[v] = sp.D0[v] = 0.0;
        rg.Sre[v] = rg.Sim[v] = rg.Dre[v] = rg.Dim[v] = rg.D0[v] = 0.0;
    }
    if (cls == 1) integrate_singular(a, X, xi, as, sp);
    else integrate_subdivided(a, X, xi, sp);
    for (int q = 0; q < NQ; q++) acc_point(a, X, xi, c_rule.s[q], c_rule.t[q], c_rule.w[q], rg);
    const int C = a.green == BEM_HELMHOLTZ ? 2 : 1;
    double d0 = 0.0;
    for (int v = 0; v < a.npe; v++) {
        size_t o = ((size_t)pr * a.npe + v) * C;
        valD[o] = sp.Dre[v] - rg.Dre[v];
        valS[o] = sp.Sre[v] - rg.Sre[v];
        if (C == 2) {
            valD[o + 1] = sp.Dim[v] - rg.Dim[v];
            valS[o + 1] = sp.Sim[v] - rg.Sim[v];
        }
        d0 += sp.D0[v] - rg.D0[v];
    }
    d0row[pr] = d0;
}

__global__ void k_pair_nodes(int N, const int *__restrict__ off, int *pair_node) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int p = off[i]; p < off[i + 1]; p++) pair_node[p] = i;
}

__global__ void k_corr_csr(int npairs, int npe, const int *__restrict__ pair_e, const int *__restrict__ el_phi,
                           const int *__restrict__ el_chi, int *colD, int *colS) {
    int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= npairs) return;
    int e = pair_e[pr];
    for (int v = 0; v < npe; v++) {
        colD[(size_t)pr * npe + v] = el_phi[(size_t)e * npe + v];
        colS[(size_t)pr * npe + v] = el_chi[(size_t)e * npe + v];
    }
}

__global__ void k_rows_ptr(int N, int npe, const int *__restrict__ off, int *ptr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > N) return;
    ptr[i] = off[i] * npe;
}

// per node: sum of the D0 correction over its special pairs
__global__ void k_d0_rowsum(int N, const int *__restrict__ off, const double *__restrict__ d0pair, double *d0row) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int p = off[i]; p < off[i + 1]; p++) s += d0pair[p];
    d0row[i] = s;
}

__global__ void k_to_float(int64_t n, const double *__restrict__ a, float *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

int build_correction(bem_plan *P, cudaStream_t s) {
    Tree &t = P->t;
    Arena &A = P->arena;
    const int N = (int)P->N, E = (int)P->E, npe = P->npe;
    double *ecx, *ecy, *ecz, *eh, *rho;
    BEM_TRY(A.alloc(&ecx, E)); BEM_TRY(A.alloc(&ecy, E)); BEM_TRY(A.alloc(&ecz, E)); BEM_TRY(A.alloc(&eh, E));
    BEM_TRY(A.alloc(&rho, t.nbox));
    (k_elem_centroid<<<(E + 255) / 256, 256, 0, s>>>(E, npe, t.el_phi, P->nodes, ecx, ecy, ecz, eh), ::bem::count_launch());
    CorrArgs a{N, E, npe, P->green, P->prm.n_duffy, P->prm.max_subdiv, P->k, P->prm.tau_near, P->nodes,
               t.el_phi, t.el_chi, ecx, ecy, ecz, eh, t.cx, t.cy, t.cz, rho, t.child0, t.nchild, t.eb, t.ee};
    (k_box_search_radius<<<t.nbox, 256, 0, s>>>(a, t.nbox, rho), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    int *cnt, *off, *tot;
    BEM_TRY(A.alloc(&cnt, N + 1));
    BEM_TRY(A.alloc(&off, N + 1));
    BEM_TRY(A.alloc(&tot, 1));
    BEM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (N + 1), s));
    (k_special_count<<<(N + 127) / 128, 128, 0, s>>>(a, cnt), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    BEM_TRY(scan_exclusive(cnt, off, N + 1, tot, s));
    int npairs = 0;
    BEM_CUDA(cudaMemcpyAsync(&npairs, tot, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    int *pair_e, *pair_node;
    BEM_TRY(A.alloc(&pair_e, npairs));
    BEM_TRY(A.alloc(&pair_node, npairs));
    (k_special_write<<<(N + 127) / 128, 128, 0, s>>>(a, off, pair_e), ::bem::count_launch());
    (k_pair_nodes<<<(N + 255) / 256, 256, 0, s>>>(N, off, pair_node), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    const int C = P->green == BEM_HELMHOLTZ ? 2 : 1;
    Correction &K = P->corr;
    K.nnzD = K.nnzS = (int64_t)npairs * npe;
    BEM_TRY(A.alloc(&K.ptrD, N + 1));
    BEM_TRY(A.alloc(&K.colD, K.nnzD));
    BEM_TRY(A.alloc(&K.colS, K.nnzS));
    BEM_TRY(A.alloc(&K.valD, K.nnzD * C));
    BEM_TRY(A.alloc(&K.valS, K.nnzS * C));
    K.ptrS = K.ptrD;
    double *d0pair, *d0row;
    BEM_TRY(A.alloc(&d0pair, npairs));
    BEM_TRY(A.alloc(&d0row, N));
    (k_rows_ptr<<<(N + 256) / 256, 256, 0, s>>>(N, npe, off, K.ptrD), ::bem::count_launch());
    (k_corr_csr<<<(npairs + 255) / 256, 256, 0, s>>>(npairs, npe, pair_e, t.el_phi, t.el_chi, K.colD, K.colS), ::bem::count_launch());
    (k_special_integrate<<<(npairs + 63) / 64, 64, 0, s>>>(a, npairs, pair_node, pair_e, K.valD, K.valS, d0pair), ::bem::count_launch());
    (k_d0_rowsum<<<(N + 255) / 256, 256, 0, s>>>(N, off, d0pair, d0row), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    BEM_TRY(A.alloc(&K.fvalD, K.nnzD * C));
    BEM_TRY(A.alloc(&K.fvalS, K.nnzS * C));
    int64_t nv = K.nnzD * C;
    (k_to_float<<<(int)((nv + 255) / 256), 256, 0, s>>>(nv, K.valD, K.fvalD), ::bem::count_launch());
    (k_to_float<<<(int)((nv + 255) / 256), 256, 0, s>>>(nv, K.valS, K.fvalS), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    // the diagonal starts as 1 + (correction row sum of D0); the regular part
    // is added by one Laplace double-layer product on phi = 1
    P->C = d0row;
    BEM_CUDA(cudaStreamSynchronize(s));
    A.release(cnt); A.release(tot); A.release(pair_node); A.release(d0pair);
    A.release(ecx); A.release(ecy); A.release(ecz); A.release(eh); A.release(rho); A.release(off);
    A.release(pair_e);
    return BEM_OK;
}

}  // namespace bem
