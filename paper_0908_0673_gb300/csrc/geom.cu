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

#include <mutex>

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
// Gauss-Legendre nodes and weights of every order n = 1..64, order n at
// offset n (n - 1) / 2, so that plans with different Duffy orders share them.
constexpr int GL_MAXN = 64;
__constant__ double c_glx[GL_MAXN * (GL_MAXN + 1) / 2], c_glw[GL_MAXN * (GL_MAXN + 1) / 2];

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

// The 7-point rule and the Gauss-Legendre tables are the same for every
// plan: written to constant memory once per device, under a lock, because
// plans are built from several host threads while other plans' kernels run.
static int init_rule_tables(int device) {
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0 || device >= 64) { set_error("device %d out of range", device); return BEM_EINVAL; }
    if (done[device]) return BEM_OK;
    Rule7 r = make_rule7();
    BEM_CUDA(cudaMemcpyToSymbol(c_rule, &r, sizeof(r)));
    std::vector<double> gx(GL_MAXN * (GL_MAXN + 1) / 2), gw(gx.size());
    for (int n = 1; n <= GL_MAXN; n++) gauss_legendre(n, &gx[n * (n - 1) / 2], &gw[n * (n - 1) / 2]);
    BEM_CUDA(cudaMemcpyToSymbol(c_glx, gx.data(), sizeof(double) * gx.size()));
    BEM_CUDA(cudaMemcpyToSymbol(c_glw, gw.data(), sizeof(double) * gw.size()));
    done[device] = true;
    return BEM_OK;
}

int build_geometry(bem_plan *P, cudaStream_t s) {
    Tree &t = P->t;
    Arena &A = P->arena;
    BEM_TRY(init_rule_tables(P->device));
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

// ---------------------------------------------------------------------------
// Special-pair quadrature, one warp per (node, element) pair.
//
// Point arithmetic works in the element's local frame: with d_a = X_a - x_i,
//   r = x_i - x(s,t) = -sum N_a d_a,  tangents = sum dN_a d_a,
// so distances keep full relative precision however close the point is to
// the collocation node (which lets the mixed-precision plan run it in
// float32).  Subdivision decisions use absolute float64 coordinates in the
// fixed operation order of the oracle, so each piece gets the same rule.
// Lanes share the Duffy points of a self element; near-singular pieces are
// refined level by level from a per-warp queue in shared memory.  The
// regular 7-point rule is added with negative weights, so the warp produces
// (special - regular) directly.
// ---------------------------------------------------------------------------
constexpr int SW_WARPS = 4, SW_CAP = 192;

struct PieceF {
    float a0, a1, b0, b1, c0, c1;   // parametric corners (dyadic, exact in float32)
    int depth;
};

template <class R, int NPE>
__device__ __forceinline__ void shape_all(R s, R t, R N[NPE], R Ns[NPE], R Nt[NPE]) {
    const R L0 = (R)1 - s - t;
    if (NPE == 3) {
        N[0] = L0; N[1] = s; N[2] = t;
        Ns[0] = -1; Ns[1] = 1; Ns[2] = 0;
        Nt[0] = -1; Nt[1] = 0; Nt[2] = 1;
    } else {
        N[0] = L0 * (2 * L0 - 1); N[1] = s * (2 * s - 1); N[2] = t * (2 * t - 1);
        N[3 % NPE] = 4 * L0 * s; N[4 % NPE] = 4 * s * t; N[5 % NPE] = 4 * t * L0;
        Ns[0] = 1 - 4 * L0; Ns[1] = 4 * s - 1; Ns[2] = 0;
        Ns[3 % NPE] = 4 * (L0 - s); Ns[4 % NPE] = 4 * t; Ns[5 % NPE] = -4 * t;
        Nt[0] = 1 - 4 * L0; Nt[1] = 0; Nt[2] = 4 * t - 1;
        Nt[3 % NPE] = -4 * s; Nt[4 % NPE] = 4 * s; Nt[5 % NPE] = 4 * (L0 - t);
    }
}

// acc[0..4][a]: Re S, Im S, Re D, Im D, D0 (Laplace double layer)
template <class R, bool HELM, int NPE>
__device__ __forceinline__ void acc_local(const R *d, R kk, R s, R t, R wref, R (&acc)[5][NPE]) {
    R N[NPE], Ns[NPE], Nt[NPE];
    shape_all<R, NPE>(s, t, N, Ns, Nt);
    R rx = 0, ry = 0, rz = 0, ux = 0, uy = 0, uz = 0, vx = 0, vy = 0, vz = 0;
#pragma unroll
    for (int a = 0; a < NPE; a++) {
        const R dx = d[3 * a], dy = d[3 * a + 1], dz = d[3 * a + 2];
        rx -= N[a] * dx; ry -= N[a] * dy; rz -= N[a] * dz;
        ux += Ns[a] * dx; uy += Ns[a] * dy; uz += Ns[a] * dz;
        vx += Nt[a] * dx; vy += Nt[a] * dy; vz += Nt[a] * dz;
    }
    const R nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;   // |n| = J
    const R J = sqrt(nx * nx + ny * ny + nz * nz);
    const R r2 = rx * rx + ry * ry + rz * rz;
    const R inv = (R)1 / sqrt(r2);
    const R c4 = (R)(0.25 / M_PI) * wref;
    const R wS = c4 * J * inv;                                   // w J G0
    const R wD = c4 * (rx * nx + ry * ny + rz * nz) * inv * inv * inv;   // w J dG0/dn1
    R sr = wS, si = 0, dr = wD, di = 0;
    if (HELM) {
        const R R1 = r2 * inv, kr = kk * R1;
        R sn, cs;
        sincos(kr, &sn, &cs);
        sr = cs * wS; si = sn * wS;
        dr = (cs + kr * sn) * wD;
        di = (sn - kr * cs) * wD;
    }
#pragma unroll
    for (int a = 0; a < NPE; a++) {
        acc[0][a] += N[a] * sr;
        acc[2][a] += N[a] * dr;
        acc[4][a] += N[a] * wD;
        if (HELM) {
            acc[1][a] += N[a] * si;
            acc[3][a] += N[a] * di;
        }
    }
}

// float64 subdivision decision in the oracle's operation order: true when
// the piece must be split.
template <int NPE>
__device__ __forceinline__ bool must_split(const double *X, const double xi[3], double tau, int maxdepth,
                                           const PieceF &P) {
    if (P.depth >= maxdepth) return false;
    double N[6], xa[3], xb[3], xc[3], xm[3];
    const double a0 = P.a0, a1 = P.a1, b0 = P.b0, b1 = P.b1, c0 = P.c0, c1 = P.c1;
    const double m0 = __ddiv_rn(__dadd_rn(__dadd_rn(a0, b0), c0), 3.0);
    const double m1 = __ddiv_rn(__dadd_rn(__dadd_rn(a1, b1), c1), 3.0);
    shape_rn(NPE, a0, a1, N); map_rn(NPE, N, X, xa);
    shape_rn(NPE, b0, b1, N); map_rn(NPE, N, X, xb);
    shape_rn(NPE, c0, c1, N); map_rn(NPE, N, X, xc);
    shape_rn(NPE, m0, m1, N); map_rn(NPE, N, X, xm);
    double h = dist3_rn(xa[0], xa[1], xa[2], xb[0], xb[1], xb[2]);
    const double h2 = dist3_rn(xb[0], xb[1], xb[2], xc[0], xc[1], xc[2]);
    const double h3 = dist3_rn(xc[0], xc[1], xc[2], xa[0], xa[1], xa[2]);
    if (h2 > h) h = h2;
    if (h3 > h) h = h3;
    return dist3_rn(xi[0], xi[1], xi[2], xm[0], xm[1], xm[2]) < __dmul_rn(tau, h);
}

// float32 estimate of the same decision in the element's local frame (node
// offsets from the collocation point, df[3a..3a+2]).  Its relative error is
// ~1e-6, so when |d - tau h| exceeds 1e-4 tau h the answer equals the float64
// one; otherwise the exact float64 test decides.
template <int NPE>
__device__ __forceinline__ bool must_split_fast(const float *df, const double *X, const double xi[3], double tau,
                                                int maxdepth, const PieceF &P) {
    if (P.depth >= maxdepth) return false;
    const float cs[4][2] = {{P.a0, P.a1}, {P.b0, P.b1}, {P.c0, P.c1},
                            {(P.a0 + P.b0 + P.c0) * (1.f / 3.f), (P.a1 + P.b1 + P.c1) * (1.f / 3.f)}};
    float x[4][3];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        float N[NPE], Ns[NPE], Nt[NPE];
        shape_all<float, NPE>(cs[q][0], cs[q][1], N, Ns, Nt);
        float v0 = 0.f, v1 = 0.f, v2 = 0.f;
#pragma unroll
        for (int a = 0; a < NPE; a++) {
            v0 = fmaf(N[a], df[3 * a], v0);
            v1 = fmaf(N[a], df[3 * a + 1], v1);
            v2 = fmaf(N[a], df[3 * a + 2], v2);
        }
        x[q][0] = v0; x[q][1] = v1; x[q][2] = v2;
    }
    auto dst = [&](int i, int j) {
        const float e0 = x[i][0] - x[j][0], e1 = x[i][1] - x[j][1], e2 = x[i][2] - x[j][2];
        return sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
    };
    const float h = fmaxf(dst(0, 1), fmaxf(dst(1, 2), dst(2, 0)));
    const float d = sqrtf(x[3][0] * x[3][0] + x[3][1] * x[3][1] + x[3][2] * x[3][2]);   // |x(m) - x_i|
    const float th = (float)tau * h, q = d - th;
    if (fabsf(q) > 1e-4f * th) return q < 0.f;
    return must_split<NPE>(X, xi, tau, maxdepth, P);
}

__device__ __forceinline__ void split4(const PieceF &P, PieceF out[4]) {
    const float ab0 = 0.5f * (P.a0 + P.b0), ab1 = 0.5f * (P.a1 + P.b1);
    const float bc0 = 0.5f * (P.b0 + P.c0), bc1 = 0.5f * (P.b1 + P.c1);
    const float ca0 = 0.5f * (P.c0 + P.a0), ca1 = 0.5f * (P.c1 + P.a1);
    const int d = P.depth + 1;
    out[0] = {P.a0, P.a1, ab0, ab1, ca0, ca1, d};
    out[1] = {ab0, ab1, P.b0, P.b1, bc0, bc1, d};
    out[2] = {ca0, ca1, bc0, bc1, P.c0, P.c1, d};
    out[3] = {ab0, ab1, bc0, bc1, ca0, ca1, d};
}

template <class R, bool HELM, int NPE>
__device__ __forceinline__ void leaf7(const R *d, R kk, const PieceF &P, R (&acc)[5][NPE]) {
    const double det = fabs(((double)P.b0 - P.a0) * ((double)P.c1 - P.a1) - ((double)P.b1 - P.a1) * ((double)P.c0 - P.a0));
    for (int q = 0; q < NQ; q++) {
        const double ps = P.a0 + c_rule.s[q] * ((double)P.b0 - P.a0) + c_rule.t[q] * ((double)P.c0 - P.a0);
        const double pt = P.a1 + c_rule.s[q] * ((double)P.b1 - P.a1) + c_rule.t[q] * ((double)P.c1 - P.a1);
        acc_local<R, HELM, NPE>(d, kk, (R)ps, (R)pt, (R)(c_rule.w[q] * det), acc);
    }
}

// serial depth-first refinement of one piece (queue overflow path)
template <class R, bool HELM, int NPE>
__device__ void refine_serial(const double *X, const double xi[3], const R *d, const float *df, R kk, double tau,
                              int maxdepth, PieceF root, R (&acc)[5][NPE]) {
    PieceF st[3 * 10 + 4];
    int sp = 0;
    st[sp++] = root;
    while (sp > 0) {
        const PieceF P = st[--sp];
        if (!must_split_fast<NPE>(df, X, xi, tau, maxdepth, P)) {
            leaf7<R, HELM, NPE>(d, kk, P, acc);
            continue;
        }
        PieceF ch[4];
        split4(P, ch);
        for (int c = 3; c >= 0; c--) st[sp++] = ch[c];
    }
}

template <class R, bool HELM, int NPE>
__global__ void __launch_bounds__(32 * SW_WARPS) k_special_warp(CorrArgs a, int npairs, const int *__restrict__ pair_node,
                                                                const int *__restrict__ pair_e, double *valD,
                                                                double *valS, double *d0pair) {
    __shared__ PieceF q[SW_WARPS][2][SW_CAP];
    __shared__ double sX[SW_WARPS][18];
    __shared__ R sd[SW_WARPS][18];
    __shared__ float sdf[SW_WARPS][18];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pr = blockIdx.x * SW_WARPS + warp;
    if (pr >= npairs) return;                       // uniform within the warp
    const int node = pair_node[pr], e = pair_e[pr];
    const double xi[3] = {a.nodes[3 * (size_t)node], a.nodes[3 * (size_t)node + 1], a.nodes[3 * (size_t)node + 2]};
    if (lane < 3 * NPE) {
        const int v = lane / 3, c = lane % 3;
        const double xv = a.nodes[3 * (size_t)a.el_phi[(size_t)e * NPE + v] + c];
        sX[warp][lane] = xv;
        sd[warp][lane] = (R)(xv - xi[c]);
        sdf[warp][lane] = (float)(xv - xi[c]);
    }
    __syncwarp();
    const double *X = sX[warp];
    const R *d = sd[warp];
    const float *df = sdf[warp];
    const R kk = (R)a.k;
    int as = -1;
    for (int v = 0; v < NPE; v++)
        if (a.el_phi[(size_t)e * NPE + v] == node) as = v;
    R acc[5][NPE];
#pragma unroll
    for (int j = 0; j < 5; j++)
#pragma unroll
        for (int v = 0; v < NPE; v++) acc[j][v] = 0;
    // minus the regular 7-point rule
    if (lane < NQ) acc_local<R, HELM, NPE>(d, kk, (R)c_rule.s[lane], (R)c_rule.t[lane], (R)(-c_rule.w[lane]), acc);
    if (as >= 0) {
        // self element: Duffy rule collapsed at the singular node, split at a mid-side node
        const double c0[2] = {0.0, 0.0}, c1[2] = {1.0, 0.0}, c2[2] = {0.0, 1.0};
        const double mm[3][2] = {{0.5, 0.0}, {0.5, 0.5}, {0.0, 0.5}};
        const int nsub = as < 3 ? 1 : 2, nd = a.nd, per = nd * nd;
        for (int j = lane; j < nsub * per; j += 32) {
            const int sub = j / per, rem = j - sub * per, iu = rem / nd, iv = rem - iu * nd;
            const double *P, *Q1, *Q2;
            switch (as) {
            case 0: P = c0; Q1 = c1; Q2 = c2; break;
            case 1: P = c1; Q1 = c2; Q2 = c0; break;
            case 2: P = c2; Q1 = c0; Q2 = c1; break;
            case 3: P = mm[0]; Q1 = sub ? c2 : c1; Q2 = sub ? c0 : c2; break;
            case 4: P = mm[1]; Q1 = sub ? c0 : c2; Q2 = sub ? c1 : c0; break;
            default: P = mm[2]; Q1 = sub ? c1 : c0; Q2 = sub ? c2 : c1; break;
            }
            const double det = fabs((Q1[0] - P[0]) * (Q2[1] - P[1]) - (Q1[1] - P[1]) * (Q2[0] - P[0]));
            const int go = nd * (nd - 1) / 2;
            const double u = 0.5 * (1.0 + c_glx[go + iu]), wu = 0.5 * c_glw[go + iu];
            const double v = 0.5 * (1.0 + c_glx[go + iv]), wv = 0.5 * c_glw[go + iv];
            const double s = P[0] + u * (Q1[0] - P[0]) + u * v * (Q2[0] - Q1[0]);
            const double t = P[1] + u * (Q1[1] - P[1]) + u * v * (Q2[1] - Q1[1]);
            acc_local<R, HELM, NPE>(d, kk, (R)s, (R)t, (R)(wu * wv * u * det), acc);
        }
    } else {
        // near-singular element: level-synchronous 4-way refinement
        PieceF *cur = q[warp][0], *nxt = q[warp][1];
        int ncur = 1;
        if (lane == 0) cur[0] = {0.f, 0.f, 1.f, 0.f, 0.f, 1.f, 0};
        __syncwarp();
        while (ncur > 0) {
            int nnext = 0;
            for (int base = 0; base < ncur; base += 32) {
                const int i = base + lane;
                PieceF P = {};
                bool split = false;
                if (i < ncur) {
                    P = cur[i];
                    split = must_split_fast<NPE>(df, X, xi, a.tau, a.maxdepth, P);
                }
                const unsigned m = __ballot_sync(0xffffffffu, split);
                const int pos = nnext + 4 * __popc(m & ((1u << lane) - 1u));
                if (i < ncur) {
                    if (!split) {
                        leaf7<R, HELM, NPE>(d, kk, P, acc);
                    } else if (pos + 4 <= SW_CAP) {
                        PieceF ch[4];
                        split4(P, ch);
                        for (int c = 0; c < 4; c++) nxt[pos + c] = ch[c];
                    } else {
                        refine_serial<R, HELM, NPE>(X, xi, d, df, kk, a.tau, a.maxdepth, P, acc);
                    }
                }
                nnext = min(SW_CAP, nnext + 4 * __popc(m));
                nnext -= (nnext % 4);
            }
            __syncwarp();
            PieceF *sw = cur; cur = nxt; nxt = sw;
            ncur = nnext;
        }
    }
    // warp sums
#pragma unroll
    for (int j = 0; j < 5; j++) {
        if (!HELM && (j == 1 || j == 3)) continue;
#pragma unroll
        for (int v = 0; v < NPE; v++)
            for (int off = 16; off; off >>= 1) acc[j][v] += __shfl_xor_sync(0xffffffffu, acc[j][v], off);
    }
    if (lane == 0) {
        const int C = HELM ? 2 : 1;
        double d0 = 0.0;
        for (int v = 0; v < NPE; v++) {
            const size_t o = ((size_t)pr * NPE + v) * C;
            valS[o] = (double)acc[0][v];
            valD[o] = (double)acc[2][v];
            if (HELM) {
                valS[o + 1] = (double)acc[1][v];
                valD[o + 1] = (double)acc[3][v];
            }
            d0 += (double)acc[4][v];
        }
        d0pair[pr] = d0;
    }
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
    {
        const int blocks = (npairs + SW_WARPS - 1) / SW_WARPS;
        const bool mx = P->prm.precision == BEM_MIXED, helm = P->green == BEM_HELMHOLTZ;
#define BEM_SW(R, H, NP) (k_special_warp<R, H, NP><<<blocks, 32 * SW_WARPS, 0, s>>>(a, npairs, pair_node, pair_e, K.valD, K.valS, d0pair), ::bem::count_launch())
        if (npairs > 0) {
            if (npe == 3) {
                if (mx) { if (helm) BEM_SW(float, true, 3); else BEM_SW(float, false, 3); }
                else { if (helm) BEM_SW(double, true, 3); else BEM_SW(double, false, 3); }
            } else {
                if (mx) { if (helm) BEM_SW(float, true, 6); else BEM_SW(float, false, 6); }
                else { if (helm) BEM_SW(double, true, 6); else BEM_SW(double, false, 6); }
            }
        }
#undef BEM_SW
    }
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
