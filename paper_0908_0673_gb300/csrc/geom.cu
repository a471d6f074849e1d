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

static Rule7 make_rule7() {
    Rule7 r;
    for (int q = 0; q < NQ; q++) radon7(q, r.s[q], r.t[q], r.w[q]);
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
// float32 copies for the mixed-precision special-pair quadrature: the 7-point
// rule (s, t, w) and the Gauss-Legendre nodes and weights mapped to [0, 1]
__constant__ float c_rulef[3][7];
__constant__ float2 c_gl01f[GL_MAXN * (GL_MAXN + 1) / 2];

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

// Also writes a float32 bound per element for the pair search: the centroid
// image and a radius R_e >= max(tau h_e, max_a |X_a - c_e|), so a node
// farther than R_e (plus the float32 rounding margin) is neither a node of
// the element nor near-singular to it.
__global__ void k_elem_centroid(int E, int npe, double tau, const int *__restrict__ el_phi,
                                const double *__restrict__ nodes, double *ecx, double *ecy, double *ecz, double *eh,
                                float4 *ebnd) {
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
    double rb = tau * m;
    for (int v = 0; v < npe; v++) rb = fmax(rb, dist3_rn(X[3 * v], X[3 * v + 1], X[3 * v + 2], x[0], x[1], x[2]));
    ebnd[i] = make_float4((float)x[0], (float)x[1], (float)x[2], (float)(rb * (1.0 + 1e-6)));
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
    float rf[3][7];
    for (int q = 0; q < 7; q++) { rf[0][q] = (float)r.s[q]; rf[1][q] = (float)r.t[q]; rf[2][q] = (float)r.w[q]; }
    BEM_CUDA(cudaMemcpyToSymbol(c_rulef, rf, sizeof(rf)));
    std::vector<float2> g01(gx.size());
    for (size_t i = 0; i < gx.size(); i++) g01[i] = make_float2((float)(0.5 * (1.0 + gx[i])), (float)(0.5 * gw[i]));
    BEM_CUDA(cudaMemcpyToSymbol(c_gl01f, g01.data(), sizeof(float2) * g01.size()));
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
    const float4 *ebnd;                   // per element float32 search bound (centroid, R_e)
    const float4 *fbox;                   // per box float32 centre (x, y, z)
    const float *frho;                    // per box float32 search radius, rounded up
    const double *bcx, *bcy, *bcz, *brho; // per box centre and search radius
    const int *child0, *nchild, *eb, *ee;
    const float *nh, *nl;                 // node coordinates as float32 pairs: x = nh + nl
};

// float32 offset X_v - x_n of two nodes from their float pairs: the high
// parts' difference (exact for nearby coordinates) plus the low parts'
__device__ __forceinline__ float node_diff(const CorrArgs &a, int v, int n, int c) {
    return (a.nh[3 * (size_t)v + c] - a.nh[3 * (size_t)n + c]) + (a.nl[3 * (size_t)v + c] - a.nl[3 * (size_t)n + c]);
}

__global__ void k_nodes_split(int64_t n3, const double *__restrict__ x, float *hi, float *lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) {
        const float h = (float)x[i];
        hi[i] = h;
        lo[i] = (float)(x[i] - (double)h);
    }
}

// Per box: radius of a ball around the centre that holds every point a
// special pair can involve: max over the subtree's elements of
// max(|c_e - c| + tau h_e, max_a |X_a - c|), inflated by 1e-12.  One thread
// per element walks from its owner leaf (the leaf of its node 0) to the root
// and raises each box's radius by an integer atomic max on the bits of the
// non-negative double (rho starts at zero).
__global__ void k_elem_search_radius(CorrArgs a, const int *__restrict__ leaf_of_node, const int *__restrict__ parent,
                                     unsigned long long *rho_bits) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.E) return;
    const int *el = a.el_phi + (size_t)e * a.npe;
    const double te = a.tau * a.eh[e];
    for (int b = leaf_of_node[el[0]]; b >= 0; b = b ? parent[b] : -1) {
        double d = dist3_rn(a.ecx[e], a.ecy[e], a.ecz[e], a.bcx[b], a.bcy[b], a.bcz[b]) + te;
        for (int v = 0; v < a.npe; v++) {
            const double *p = a.nodes + 3 * (size_t)el[v];
            d = fmax(d, dist3_rn(p[0], p[1], p[2], a.bcx[b], a.bcy[b], a.bcz[b]));
        }
        atomicMax(rho_bits + b, (unsigned long long)__double_as_longlong(d * (1.0 + 1e-12)));
    }
}

__global__ void k_rho_float(int nbox, const double *__restrict__ rho, float *frho) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbox) frho[b] = (float)(rho[b] * (1.0 + 1e-6));
}

// 0 regular, 1 singular (*a_sing = local node), 2 near-singular
__device__ __forceinline__ int classify_pair(const CorrArgs &a, int node, const double xi[3], int e, int *a_sing) {
    const int *el = a.el_phi + (size_t)e * a.npe;
    for (int v = 0; v < a.npe; v++)
        if (el[v] == node) { *a_sing = v; return 1; }
    double d = dist3_rn(xi[0], xi[1], xi[2], a.ecx[e], a.ecy[e], a.ecz[e]);
    return d < __dmul_rn(a.tau, a.eh[e]) ? 2 : 0;
}

// One warp per collocation node: walks the box tree (children tested by the
// lanes in parallel, passing children pushed in reverse so that they are
// visited in order) and, in every leaf reached, tests the leaf's elements 32
// at a time; special (element) pairs are counted, or written in leaf order
// and element order within a leaf when `out_e` is given.  A float32 test with
// an inflated radius filters boxes (visiting a box the exact test would skip
// only adds candidates); elements pass a float32 rejection and then the
// exact float64 classification.
constexpr int SS_WARPS = 4, SS_STACK = 8 * 24;
constexpr int SS_CAP = 192;         // special elements per node kept by the counting search

__device__ __forceinline__ bool box_may_hold(const CorrArgs &a, int b, const float xf[3], float ax) {
    const float4 c = a.fbox[b];
    const float dx = xf[0] - c.x, dy = xf[1] - c.y, dz = xf[2] - c.z, rh = a.frho[b];
    const float lim = rh + 1e-5f * (ax + fabsf(c.x) + fabsf(c.y) + fabsf(c.z) + rh);
    return dx * dx + dy * dy + dz * dz <= lim * lim;
}

__device__ int find_special_warp(const CorrArgs &a, int node, int *out_e, int *stack, int cap = 1 << 30) {
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
    const double xi[3] = {a.nodes[3 * (size_t)node], a.nodes[3 * (size_t)node + 1], a.nodes[3 * (size_t)node + 2]};
    const float xf[3] = {(float)xi[0], (float)xi[1], (float)xi[2]};
    const float ax = fabsf(xf[0]) + fabsf(xf[1]) + fabsf(xf[2]);
    int sp = 0, cnt = 0;
    if (lane == 0) stack[0] = 0;
    sp = 1;
    __syncwarp();
    while (sp > 0) {
        const int b = stack[--sp];
        __syncwarp();
        const int nc = a.nchild[b];
        if (nc != 0) {
            const int c0 = a.child0[b];
            const unsigned m = __ballot_sync(FULL, lane < nc && box_may_hold(a, c0 + lane, xf, ax));
            const int k = __popc(m);
            // passing children in reverse order: lane holding child c writes at sp + (passing children after c)
            if (lane < nc && ((m >> lane) & 1u)) stack[sp + __popc(m >> (lane + 1))] = c0 + lane;
            sp += k;
            __syncwarp();
            continue;
        }
        for (int base = a.eb[b]; base < a.ee[b]; base += 32) {
            const int e = base + lane;
            bool hit = false;
            if (e < a.ee[b]) {
                const float4 c = a.ebnd[e];
                const float dx = xf[0] - c.x, dy = xf[1] - c.y, dz = xf[2] - c.z;
                const float lim = c.w + 1e-5f * (ax + fabsf(c.x) + fabsf(c.y) + fabsf(c.z) + c.w);
                if (dx * dx + dy * dy + dz * dz <= lim * lim) {
                    int as;
                    hit = classify_pair(a, node, xi, e, &as) != 0;
                }
            }
            const unsigned m = __ballot_sync(FULL, hit);
            if (out_e && hit && cnt + __popc(m & lt) < cap) out_e[cnt + __popc(m & lt)] = e;
            cnt += __popc(m);
        }
    }
    return cnt;
}

// Counts every node's special pairs and keeps the first `cap` of their
// elements in tmp[node * cap ...]; *overflow is set when a node has more.
__global__ void __launch_bounds__(32 * SS_WARPS) k_special_count(CorrArgs a, int *cnt, int *tmp, int cap,
                                                                int *overflow) {
    __shared__ int stack[SS_WARPS][SS_STACK];
    const int w = threadIdx.x >> 5, i = blockIdx.x * SS_WARPS + w;
    if (i >= a.N) return;                              // uniform within the warp
    const int c = find_special_warp(a, i, tmp + (size_t)i * cap, stack[w], cap);
    if ((threadIdx.x & 31) == 0) {
        cnt[i] = c;
        if (c > cap) atomicOr(overflow, 1);
    }
}

// the kept elements of every node into the pair list at the node's offset
__global__ void k_special_copy(int N, const int *__restrict__ off, const int *__restrict__ tmp, int cap, int *pair_e) {
    const int i = blockIdx.x, n = off[i + 1] - off[i];
    for (int j = threadIdx.x; j < n; j += blockDim.x) pair_e[off[i] + j] = tmp[(size_t)i * cap + j];
}

__global__ void __launch_bounds__(32 * SS_WARPS) k_special_write(CorrArgs a, const int *__restrict__ off, int *pair_e) {
    __shared__ int stack[SS_WARPS][SS_STACK];
    const int w = threadIdx.x >> 5, i = blockIdx.x * SS_WARPS + w;
    if (i >= a.N) return;
    find_special_warp(a, i, pair_e + off[i], stack[w]);
}

// ---------------------------------------------------------------------------
// Special-pair quadrature, one warp per (node, element) pair.
//
// Point arithmetic works in the element's local frame: with d_a = X_a - x_i,
//   r = x_i - x(s,t) = -sum N_a d_a,  tangents = sum dN_a d_a,
// so distances keep full relative precision however close the point is to
// the collocation node (which lets the mixed-precision plan run it in
// float32).  At a Duffy point (s,t) = P + delta of a self element, P the
// parametric position of the node, the shape values are taken as
//   N_a(P + delta) = [a = a_sing] + (grad N_a(P) + grad N_a(P + delta)) . delta / 2,
// which is exact for shape functions of degree two or less and keeps the
// small N_a next to the node at full relative precision as well.
//
// Per pair the warp works in three steps.  Quadrature points are written to
// a per-warp ring in shared memory: the regular 7-point rule with negative
// weights first, then the 7 points of every leaf piece of the subdivision.
// Every 32 pending points are evaluated, one per lane.  Finally the lanes'
// partial sums are reduced by a transposing butterfly that leaves value l
// of the pair on lane l for the store.  Subdivision decisions use a float32
// estimate with a margin and fall back to the float64 test in the oracle's
// operation order, so each piece gets the same rule on both sides; pieces
// are refined level by level from a per-warp queue.  Self elements take
// their Duffy points by index, all lanes at once.  Points go to lanes in a
// fixed order, so the stored values are the same on every run.
// ---------------------------------------------------------------------------
constexpr int SP_WARPS = 4;        // warps per block
constexpr int SP_PAIRS_PER_WARP = 16;   // pairs per warp (grid-stride), launch granularity
constexpr float SP_UNIT = 1024.f;  // piece corners are multiples of 2^-10 (max_subdiv <= 10)

struct PieceF {
    float a0, a1, b0, b1, c0, c1;   // parametric corners (dyadic, exact in float32)
    int depth;
};

// values a pair stores (2 NPE C + 1), rounded up to 16 or 32 lanes
__host__ __device__ constexpr int sp_nvp(bool helm, int npe) { return 2 * npe * (helm ? 2 : 1) + 1 <= 16 ? 16 : 32; }

// a queued piece: corners in units of 2^-10, two to a word, then the depth
__device__ __forceinline__ uint4 pack_piece(const PieceF &P) {
    auto u = [](float x) { return (unsigned)(x * SP_UNIT); };
    return make_uint4(u(P.a0) | u(P.a1) << 16, u(P.b0) | u(P.b1) << 16, u(P.c0) | u(P.c1) << 16, (unsigned)P.depth);
}

__device__ __forceinline__ PieceF unpack_piece(uint4 q) {
    const float k = 1.f / SP_UNIT;
    return {(q.x & 0xffffu) * k, (q.x >> 16) * k, (q.y & 0xffffu) * k, (q.y >> 16) * k,
            (q.z & 0xffffu) * k, (q.z >> 16) * k, (int)q.w};
}

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

// rule tables in the working precision
template <class R> __device__ __forceinline__ R rule_s(int q);
template <class R> __device__ __forceinline__ R rule_t(int q);
template <class R> __device__ __forceinline__ R rule_w(int q);
template <> __device__ __forceinline__ float rule_s<float>(int q) { return c_rulef[0][q]; }
template <> __device__ __forceinline__ float rule_t<float>(int q) { return c_rulef[1][q]; }
template <> __device__ __forceinline__ float rule_w<float>(int q) { return c_rulef[2][q]; }
template <> __device__ __forceinline__ double rule_s<double>(int q) { return c_rule.s[q]; }
template <> __device__ __forceinline__ double rule_t<double>(int q) { return c_rule.t[q]; }
template <> __device__ __forceinline__ double rule_w<double>(int q) { return c_rule.w[q]; }
// Gauss-Legendre node and weight mapped to [0, 1]
template <class R> __device__ __forceinline__ void gl01(int i, R &u, R &wu);
template <> __device__ __forceinline__ void gl01<float>(int i, float &u, float &wu) { u = c_gl01f[i].x; wu = c_gl01f[i].y; }
template <> __device__ __forceinline__ void gl01<double>(int i, double &u, double &wu) {
    u = 0.5 * (1.0 + c_glx[i]);
    wu = 0.5 * c_glw[i];
}

// The values a pair stores, per lane partial sums: S at a*C + c, D at
// NPE*C + a*C + c (c = 0 real, 1 imaginary), the Laplace double layer of a
// constant density (D0 row sum) at 2*NPE*C.
template <class R, bool HELM, int NPE>
__device__ __forceinline__ void point_acc(const R *d, R kk, const R (&N)[NPE], const R (&Ns)[NPE], const R (&Nt)[NPE],
                                          R wref, R (&v)[sp_nvp(HELM, NPE)]) {
    constexpr int C = HELM ? 2 : 1;
    R rx = 0, ry = 0, rz = 0, ux = 0, uy = 0, uz = 0, vx = 0, vy = 0, vz = 0;
#pragma unroll
    for (int a = 0; a < NPE; a++) {
        const R dx = d[3 * a], dy = d[3 * a + 1], dz = d[3 * a + 2];
        rx -= N[a] * dx; ry -= N[a] * dy; rz -= N[a] * dz;
        ux += Ns[a] * dx; uy += Ns[a] * dy; uz += Ns[a] * dz;
        vx += Nt[a] * dx; vy += Nt[a] * dy; vz += Nt[a] * dz;
    }
    const R nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;   // |n| = J
    const R n2 = nx * nx + ny * ny + nz * nz, r2 = rx * rx + ry * ry + rz * rz;
    R J, inv;
    if constexpr (sizeof(R) == sizeof(float)) {
        // float32 sums: the hardware reciprocal square root (2 ulp) in place of
        // the correctly rounded square root and division
        J = n2 * rsqrtf(n2);
        inv = rsqrtf(r2);
    } else {
        J = sqrt(n2);
        inv = (R)1 / sqrt(r2);
    }
    const R c4 = (R)(0.25 / M_PI) * wref;
    const R wS = c4 * J * inv;                                           // w J G0
    const R wD = c4 * (rx * nx + ry * ny + rz * nz) * inv * inv * inv;   // w J dG0/dn1
    R sr = wS, si = 0, dr = wD, di = 0;
    if (HELM) {
        const R kr = kk * (r2 * inv);
        R sn, cs;
        sincos(kr, &sn, &cs);
        sr = cs * wS; si = sn * wS;
        dr = (cs + kr * sn) * wD;
        di = (sn - kr * cs) * wD;
    }
#pragma unroll
    for (int a = 0; a < NPE; a++) {
        v[a * C] += N[a] * sr;
        v[NPE * C + a * C] += N[a] * dr;
        if (HELM) {
            v[a * C + 1] += N[a] * si;
            v[NPE * C + a * C + 1] += N[a] * di;
        }
    }
    v[2 * NPE * C] += wD;
}

// The element's map in monomial form, X(s,t) - x_i = sum_k A_k m_k(s,t) with
// m = (1, s, t, s^2, st, t^2), from the node offsets d_a = X_a - x_i (6-node
// shapes expanded: N0 = 1 - 3s - 3t + 2s^2 + 4st + 2t^2, N1 = 2s^2 - s,
// N2 = 2t^2 - t, N3 = 4s - 4s^2 - 4st, N4 = 4st, N5 = 4t - 4st - 4t^2; 3-node:
// N0 = 1 - s - t, N1 = s, N2 = t).  A[3k + c] = coefficient k, component c.
template <class R, int NPE>
__device__ __forceinline__ R mono_coef(const R *d, int k, int c) {
    const R d0 = d[c], d1 = d[3 + c], d2 = d[6 + c];
    if constexpr (NPE == 3) return k == 0 ? d0 : k == 1 ? d1 - d0 : k == 2 ? d2 - d0 : (R)0;
    const R d3 = d[9 + c], d4 = d[12 + c], d5 = d[15 + c];
    switch (k) {
        case 0: return d0;
        case 1: return 4 * d3 - 3 * d0 - d1;
        case 2: return 4 * d5 - 3 * d0 - d2;
        case 3: return 2 * (d0 + d1) - 4 * d3;
        case 4: return 4 * ((d0 + d4) - (d3 + d5));
        default: return 2 * (d0 + d2) - 4 * d5;
    }
}

// point_acc with the geometry from the monomial coefficients: position and
// both tangents in 8 operations per component instead of 3 NPE, and only the
// shape values themselves (they weight the stored values)
template <class R, bool HELM, int NPE>
__device__ __forceinline__ void point_acc_mono(const R *A, R kk, R s, R t, R wref, R (&v)[sp_nvp(HELM, NPE)]) {
    constexpr int C = HELM ? 2 : 1;
    R N[NPE];
    const R L0 = 1 - s - t;
    if (NPE == 3) {
        N[0] = L0; N[1] = s; N[2] = t;
    } else {
        N[0] = L0 * (2 * L0 - 1); N[1] = s * (2 * s - 1); N[2] = t * (2 * t - 1);
        N[3 % NPE] = 4 * L0 * s; N[4 % NPE] = 4 * s * t; N[5 % NPE] = 4 * t * L0;
    }
    R r[3], u[3], w[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const R a0 = A[c], a1 = A[3 + c], a2 = A[6 + c], a3 = A[9 + c], a4 = A[12 + c], a5 = A[15 + c];
        const R xs = a1 + a3 * s + a4 * t;             // X_s = a1 + 2 a3 s + a4 t = xs + a3 s
        const R xt = a2 + a5 * t;                      // X_t = a2 + a4 s + 2 a5 t = xt + a5 t + a4 s
        r[c] = -(a0 + s * xs + t * xt);                // r = x_i - X(s,t)
        u[c] = xs + a3 * s;
        w[c] = xt + a5 * t + a4 * s;
    }
    const R nx = u[1] * w[2] - u[2] * w[1], ny = u[2] * w[0] - u[0] * w[2], nz = u[0] * w[1] - u[1] * w[0];
    const R n2 = nx * nx + ny * ny + nz * nz, r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    R J, inv;
    if constexpr (sizeof(R) == sizeof(float)) {
        J = n2 * rsqrtf(n2);
        inv = rsqrtf(r2);
    } else {
        J = sqrt(n2);
        inv = (R)1 / sqrt(r2);
    }
    const R c4 = (R)(0.25 / M_PI) * wref;
    const R wS = c4 * J * inv;
    const R wD = c4 * (r[0] * nx + r[1] * ny + r[2] * nz) * inv * inv * inv;
    R sr = wS, si = 0, dr = wD, di = 0;
    if (HELM) {
        const R kr = kk * (r2 * inv);
        R sn, cs;
        sincos(kr, &sn, &cs);
        sr = cs * wS; si = sn * wS;
        dr = (cs + kr * sn) * wD;
        di = (sn - kr * cs) * wD;
    }
#pragma unroll
    for (int a = 0; a < NPE; a++) {
        v[a * C] += N[a] * sr;
        v[NPE * C + a * C] += N[a] * dr;
        if (HELM) {
            v[a * C + 1] += N[a] * si;
            v[NPE * C + a * C + 1] += N[a] * di;
        }
    }
    v[2 * NPE * C] += wD;
}

template <class R, bool HELM, int NPE>
__device__ __forceinline__ void eval_st(const R *d, R kk, R s, R t, R w, R (&v)[sp_nvp(HELM, NPE)]) {
    R N[NPE], Ns[NPE], Nt[NPE];
    shape_all<R, NPE>(s, t, N, Ns, Nt);
    point_acc<R, HELM, NPE>(d, kk, N, Ns, Nt, w, v);
}

// q-th point of the 7-point rule on a piece, with its weight
template <class R>
__device__ __forceinline__ void leaf_point(const PieceF &P, int q, R &s, R &t, R &w) {
    const R e0 = (R)P.b0 - (R)P.a0, e1 = (R)P.b1 - (R)P.a1, f0 = (R)P.c0 - (R)P.a0, f1 = (R)P.c1 - (R)P.a1;
    const R det = fabs(e0 * f1 - e1 * f0);   // exact: products of dyadic numbers
    const R rs = rule_s<R>(q), rt = rule_t<R>(q);
    s = (R)P.a0 + rs * e0 + rt * f0;
    t = (R)P.a1 + rs * e1 + rt * f1;
    w = rule_w<R>(q) * det;
}

// float64 subdivision decision in the oracle's operation order: true when
// the piece must be split.
template <int NPE>
__device__ __noinline__ bool must_split(const double *X, const double xi[3], double tau, int maxdepth,
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

// A queued piece with the images of its corners in the element's local frame
// (node offsets from the collocation point), so that a decision maps only the
// centroid and a split only the three edge midpoints.
struct __align__(16) QPiece {
    uint4 piece;                    // pack_piece
    float4 A, B, Cc;                // corner images (w unused)
};

template <int NPE>
__device__ __forceinline__ float4 map_f(const float *df, float s, float t) {
    float N[NPE], Ns[NPE], Nt[NPE];
    shape_all<float, NPE>(s, t, N, Ns, Nt);
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;
#pragma unroll
    for (int a = 0; a < NPE; a++) {
        v0 = fmaf(N[a], df[3 * a], v0);
        v1 = fmaf(N[a], df[3 * a + 1], v1);
        v2 = fmaf(N[a], df[3 * a + 2], v2);
    }
    return make_float4(v0, v1, v2, 0.f);
}

__device__ __forceinline__ float dist2f(float4 p, float4 q) {
    const float e0 = p.x - q.x, e1 = p.y - q.y, e2 = p.z - q.z;
    return e0 * e0 + e1 * e1 + e2 * e2;
}

// The subdivision decision from the corner images: |x(m) - x_i|^2 against
// tau^2 h^2 in float32 (relative error ~2e-6), decided there when the two
// differ by more than 2e-4 tau^2 h^2, else by the exact float64 test.
template <int NPE>
__device__ __forceinline__ bool split_test(const float *df, const QPiece &Q, const PieceF &P, const double *X,
                                           const double xi[3], float tau2, double tau, int maxdepth) {
    if (P.depth >= maxdepth) return false;
    const float4 m = map_f<NPE>(df, (P.a0 + P.b0 + P.c0) * (1.f / 3.f), (P.a1 + P.b1 + P.c1) * (1.f / 3.f));
    const float h2 = fmaxf(dist2f(Q.A, Q.B), fmaxf(dist2f(Q.B, Q.Cc), dist2f(Q.Cc, Q.A)));
    const float th = tau2 * h2, q = m.x * m.x + m.y * m.y + m.z * m.z - th;
    if (fabsf(q) > 2e-4f * th) return q < 0.f;
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

// serial depth-first refinement of one piece on one lane (queue overflow path)
template <class R, bool HELM, int NPE>
__device__ void refine_serial(const double *X, const double xi[3], const R *d, const float *df, R kk, double tau,
                              int maxdepth, PieceF root, R (&v)[sp_nvp(HELM, NPE)]) {
    PieceF st[3 * 10 + 4];
    int sp = 0;
    st[sp++] = root;
    while (sp > 0) {
        const PieceF P = st[--sp];
        if (!must_split_fast<NPE>(df, X, xi, tau, maxdepth, P)) {
            for (int q = 0; q < NQ; q++) {
                R s, t, w;
                leaf_point<R>(P, q, s, t, w);
                eval_st<R, HELM, NPE>(d, kk, s, t, w, v);
            }
            continue;
        }
        PieceF ch[4];
        split4(P, ch);
        for (int c = 3; c >= 0; c--) st[sp++] = ch[c];
    }
}

// Loads the element of a pair into the group's tables: node coordinates
// (float64) and their offsets from the collocation point (working precision
// and float32).  W lanes of the group share the 3 NPE values.
template <class R, int NPE, int W>
__device__ __forceinline__ void load_pair(const CorrArgs &a, int node, int e, int sl, double xi[3], double *X, R *d,
                                          float *df) {
    xi[0] = a.nodes[3 * (size_t)node];
    xi[1] = a.nodes[3 * (size_t)node + 1];
    xi[2] = a.nodes[3 * (size_t)node + 2];
    for (int i = sl; i < 3 * NPE; i += W) {
        const int c = i % 3, vid = a.el_phi[(size_t)e * NPE + i / 3];
        const double xv = a.nodes[3 * (size_t)vid + c];
        X[i] = xv;
        d[i] = (R)(xv - xi[c]);
        df[i] = (float)(xv - xi[c]);
    }
}

// Sums the lanes' partial values of a pair over the W lanes of its group by a
// transposing butterfly, in blocks of W values: after the steps of widths
// W/2 .. 1 (a lane keeps the half of a block selected by bit k of its lane
// index), lane l holds value l of every block.  Value l + W b goes to S at
// l + W b < NPE C, to D below 2 NPE C, to the D0 row sum at 2 NPE C.
template <class R, bool HELM, int NPE, int W>
__device__ __forceinline__ void reduce_store(R (&v)[sp_nvp(HELM, NPE)], unsigned wmask, int sl, int pr, R *valD,
                                             R *valS, double *d0pair) {
    constexpr int C = HELM ? 2 : 1, NVP = sp_nvp(HELM, NPE);
    if constexpr (W > NVP) {
        // fewer values than lanes: plain sums across the lanes beyond NVP first
#pragma unroll
        for (int k = W / 2; k >= NVP; k >>= 1)
#pragma unroll
            for (int i = 0; i < NVP; i++) v[i] += __shfl_xor_sync(wmask, v[i], k);
    }
    constexpr int BW = W < NVP ? W : NVP;          // block width
#pragma unroll
    for (int b0 = 0; b0 < NVP; b0 += BW) {
#pragma unroll
        for (int k = BW / 2; k >= 1; k >>= 1) {
            const bool up = (sl & k) != 0;
#pragma unroll
            for (int i = 0; i < k; i++) {
                const R lo = v[b0 + i], hi = v[b0 + i + k];
                v[b0 + i] = (up ? hi : lo) + __shfl_xor_sync(wmask, up ? lo : hi, k);
            }
        }
        const int vi = b0 + (sl % BW);
        if (sl < BW) {
            if (vi < NPE * C) valS[(size_t)pr * NPE * C + vi] = (R)v[b0];
            else if (vi < 2 * NPE * C) valD[(size_t)pr * NPE * C + vi - NPE * C] = (R)v[b0];
            else if (vi == 2 * NPE * C) d0pair[pr] = (double)v[b0];
        }
    }
}

// Self pairs (the collocation node is a node of the element), one warp per
// pair: the Duffy rule collapsed at the node (split at a mid-side node), then
// the regular rule subtracted, all by point index, one point per lane.
template <class R, bool HELM, int NPE>
__global__ void __launch_bounds__(32 * SP_WARPS) k_special_self(CorrArgs a, int nlist, const int *__restrict__ list,
                                                               const int *__restrict__ pair_node,
                                                               const int *__restrict__ pair_e, R *valD,
                                                               R *valS, double *d0pair) {
    constexpr int NVP = sp_nvp(HELM, NPE);
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ double sX[SP_WARPS][18];
    __shared__ R sd[SP_WARPS][18];
    __shared__ float sdf[SP_WARPS][18];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const R kk = (R)a.k;
    for (int li = blockIdx.x * SP_WARPS + warp; li < nlist; li += gridDim.x * SP_WARPS) {
        const int pr = list[li], node = pair_node[pr], e = pair_e[pr];
        double xi[3];
        __syncwarp();                                   // the previous pair's reads of the tables are done
        load_pair<R, NPE, 32>(a, node, e, lane, xi, sX[warp], sd[warp], sdf[warp]);
        int as = 0;
        for (int v = 0; v < NPE; v++)
            if (a.el_phi[(size_t)e * NPE + v] == node) as = v;
        __syncwarp();
        const R *d = sd[warp];
        R v[NVP];
#pragma unroll
        for (int i = 0; i < NVP; i++) v[i] = 0;
        const R p0 = as == 1 || as == 3 || as == 4 ? (R)(as == 1 ? 1 : 0.5) : (R)0;
        const R p1 = as == 2 || as == 4 || as == 5 ? (R)(as == 2 ? 1 : 0.5) : (R)0;
        R NP[NPE], NsP[NPE], NtP[NPE];
        shape_all<R, NPE>(p0, p1, NP, NsP, NtP);
        const int nsub = as < 3 ? 1 : 2, nd = a.nd, per = nd * nd, go = nd * (nd - 1) / 2;
        const int nduffy = nsub * per;
        for (int j = lane; j < nduffy + NQ; j += 32) {
            if (j >= nduffy) {
                const int q = j - nduffy;
                eval_st<R, HELM, NPE>(d, kk, rule_s<R>(q), rule_t<R>(q), -rule_w<R>(q), v);
                continue;
            }
            const int sub = j / per, rem = j - sub * per, iu = rem / nd, iv = rem - iu * nd;
            // the sub-triangle (P, Q1, Q2): Q1, Q2 the corners (r+1) mod 3 and
            // (r+2) mod 3 of the reference triangle, corners 0 (0,0), 1 (1,0), 2 (0,1)
            const int r = as < 3 ? as : (as - 3 + sub) % 3, k1 = (r + 1) % 3, k2 = (r + 2) % 3;
            const R q10 = (R)(k1 == 1), q11 = (R)(k1 == 2), q20 = (R)(k2 == 1), q21 = (R)(k2 == 2);
            const R det = fabs((q10 - p0) * (q21 - p1) - (q11 - p1) * (q20 - p0));
            R u, wu, w2, wv;
            gl01<R>(go + iu, u, wu);
            gl01<R>(go + iv, w2, wv);
            const R uv = u * w2;
            const R ds = u * (q10 - p0) + uv * (q20 - q10);
            const R dt = u * (q11 - p1) + uv * (q21 - q11);
            R N[NPE], Ns[NPE], Nt[NPE];
            shape_all<R, NPE>(p0 + ds, p1 + dt, N, Ns, Nt);
#pragma unroll
            for (int b = 0; b < NPE; b++)
                N[b] = (b == as ? (R)1 : (R)0) + (R)0.5 * ((NsP[b] + Ns[b]) * ds + (NtP[b] + Nt[b]) * dt);
            point_acc<R, HELM, NPE>(d, kk, N, Ns, Nt, wu * wv * u * det, v);
        }
        reduce_store<R, HELM, NPE, 32>(v, FULL, lane, pr, valD, valS, d0pair);
    }
}

// Near-singular pairs, one group of SPN_W lanes per pair (four pairs per
// warp, so that the refinement's few pieces per level keep more lanes busy):
// the regular rule with negative weights, then the leaf pieces of a
// level-synchronous 4-way refinement.  Quadrature points go to the group's
// ring and are evaluated SPN_W at a time, one per lane, in a fixed order.
constexpr int SPN_W = 8;            // lanes per pair
constexpr int SPN_WARPS = 2;        // warps per block
constexpr int SPN_G = SPN_WARPS * 32 / SPN_W;   // groups per block
constexpr int SPN_QCAP = 32;        // pieces per level buffer and group
constexpr int SPN_RING = 64;        // pending points per group: a power of two >= SPN_W - 1 + 7 SPN_W

template <class R, bool HELM, int NPE>
__global__ void __launch_bounds__(32 * SPN_WARPS) k_special_near(CorrArgs a, const int *__restrict__ nlist_dev,
                                                                const int *__restrict__ list,
                                                                const int *__restrict__ pair_node,
                                                                const int *__restrict__ pair_e, R *valD,
                                                                R *valS, double *d0pair) {
    constexpr int NVP = sp_nvp(HELM, NPE), W = SPN_W, QCAP = SPN_QCAP, RING = SPN_RING;
    __shared__ QPiece qbuf[SPN_G][2][QCAP];
    __shared__ R ring[SPN_G][3][RING];
    __shared__ double sX[SPN_G][18];
    __shared__ R sd[SPN_G][18];
    __shared__ float sdf[SPN_G][18];
    const int lane = threadIdx.x & 31, g = threadIdx.x / W, sl = threadIdx.x % W;
    const unsigned wmask = ((1u << W) - 1u) << (lane - sl);
    const unsigned lt = (1u << sl) - 1u;
    auto ballot = [&](bool p) { return (__ballot_sync(wmask, p) >> (lane - sl)) & ((1u << W) - 1u); };
    R *rs = ring[g][0], *rt = ring[g][1], *rw = ring[g][2];
    const double *X = sX[g];
    const R *d = sd[g];
    const float *df = sdf[g];
    const R kk = (R)a.k;
    const float tau2 = (float)(a.tau * a.tau);
    const int nlist = *nlist_dev;
    for (int li = blockIdx.x * SPN_G + g; li < nlist; li += gridDim.x * SPN_G) {
        const int pr = list[li], node = pair_node[pr], e = pair_e[pr];
        double xi[3];
        __syncwarp(wmask);                              // the previous pair's reads of the tables are done
        load_pair<R, NPE, W>(a, node, e, sl, xi, sX[g], sd[g], sdf[g]);
        __syncwarp(wmask);
        R v[NVP];
#pragma unroll
        for (int i = 0; i < NVP; i++) v[i] = 0;
        for (int q = sl; q < NQ; q += W) { rs[q] = rule_s<R>(q); rt[q] = rule_t<R>(q); rw[q] = -rule_w<R>(q); }
        int head = 0, tail = NQ;
        QPiece *cur = qbuf[g][0], *nxt = qbuf[g][1];
        int ncur = 0;
        auto img = [&](int vtx) { return make_float4(df[3 * vtx], df[3 * vtx + 1], df[3 * vtx + 2], 0.f); };
        if (a.maxdepth > 0) {
            // the pair was selected by the root's own test, so the root
            // splits: its four children, corner images from the nodes
            if (sl < 4) {
                const float4 v0 = img(0), v1 = img(1), v2 = img(2);
                float4 m01, m12, m20;
                if (NPE == 6) {
                    m01 = img(3 % NPE); m12 = img(4 % NPE); m20 = img(5 % NPE);
                } else {
                    m01 = map_f<NPE>(df, 0.5f, 0.f); m12 = map_f<NPE>(df, 0.5f, 0.5f); m20 = map_f<NPE>(df, 0.f, 0.5f);
                }
                // the children of split4 on the reference triangle, by lane
                const PieceF ch = sl == 0   ? PieceF{0.f, 0.f, 0.5f, 0.f, 0.f, 0.5f, 1}
                                  : sl == 1 ? PieceF{0.5f, 0.f, 1.f, 0.f, 0.5f, 0.5f, 1}
                                  : sl == 2 ? PieceF{0.f, 0.5f, 0.5f, 0.5f, 0.f, 1.f, 1}
                                            : PieceF{0.5f, 0.f, 0.5f, 0.5f, 0.f, 0.5f, 1};
                QPiece Q;
                Q.piece = pack_piece(ch);
                Q.A = sl == 0 ? v0 : sl == 2 ? m20 : m01;
                Q.B = sl == 0 ? m01 : sl == 1 ? v1 : m12;
                Q.Cc = sl == 0 ? m20 : sl == 1 ? m12 : sl == 2 ? v2 : m20;
                cur[sl] = Q;
            }
            ncur = 4;
        } else {
            // no subdivision: the special rule is the regular rule
            for (int q = sl; q < NQ; q += W) { rs[NQ + q] = rule_s<R>(q); rt[NQ + q] = rule_t<R>(q); rw[NQ + q] = rule_w<R>(q); }
            tail = 2 * NQ;
        }
        __syncwarp(wmask);
        while (ncur > 0) {
            int nnext = 0;
            for (int base = 0; base < ncur; base += W) {
                const int i = base + sl;
                PieceF P = {};
                QPiece Q;
                bool split = false, leaf = false;
                if (i < ncur) {
                    Q = cur[i];
                    P = unpack_piece(Q.piece);
                    split = split_test<NPE>(df, Q, P, X, xi, tau2, a.tau, a.maxdepth);
                    leaf = !split;
                }
                const unsigned ms = ballot(split), ml = ballot(leaf);
                if (split) {
                    const int pos = nnext + 4 * __popc(ms & lt);
                    if (pos + 4 <= QCAP) {
                        PieceF ch[4];
                        split4(P, ch);
                        const float4 mab = map_f<NPE>(df, ch[0].b0, ch[0].b1);   // (a + b) / 2
                        const float4 mca = map_f<NPE>(df, ch[0].c0, ch[0].c1);   // (c + a) / 2
                        const float4 mbc = map_f<NPE>(df, ch[1].c0, ch[1].c1);   // (b + c) / 2
                        QPiece *o = nxt + pos;
                        o[0].piece = pack_piece(ch[0]); o[0].A = Q.A; o[0].B = mab; o[0].Cc = mca;
                        o[1].piece = pack_piece(ch[1]); o[1].A = mab; o[1].B = Q.B; o[1].Cc = mbc;
                        o[2].piece = pack_piece(ch[2]); o[2].A = mca; o[2].B = mbc; o[2].Cc = Q.Cc;
                        o[3].piece = pack_piece(ch[3]); o[3].A = mab; o[3].B = mbc; o[3].Cc = mca;
                    } else {
                        refine_serial<R, HELM, NPE>(X, xi, d, df, kk, a.tau, a.maxdepth, P, v);
                    }
                }
                if (leaf) {
                    const int p0 = tail + NQ * __popc(ml & lt);
#pragma unroll
                    for (int q = 0; q < NQ; q++) {
                        R s, t, w;
                        leaf_point<R>(P, q, s, t, w);
                        const int k = (p0 + q) & (RING - 1);
                        rs[k] = s; rt[k] = t; rw[k] = w;
                    }
                }
                tail += NQ * __popc(ml);
                nnext = min(QCAP, nnext + 4 * __popc(ms));
                nnext -= nnext % 4;
                __syncwarp(wmask);
                for (; tail - head >= W; head += W) {
                    const int k = (head + sl) & (RING - 1);
                    eval_st<R, HELM, NPE>(d, kk, rs[k], rt[k], rw[k], v);
                }
                __syncwarp(wmask);                      // ring reads done before the next writes
            }
            QPiece *sw = cur; cur = nxt; nxt = sw;
            ncur = nnext;
        }
        for (; tail - head > 0; head += W) {
            const int k = (head + sl) & (RING - 1);
            if (head + sl < tail) eval_st<R, HELM, NPE>(d, kk, rs[k], rt[k], rw[k], v);
        }
        reduce_store<R, HELM, NPE, W>(v, wmask, sl, pr, valD, valS, d0pair);
    }
}

// A piece of the 4-way subdivision as a 32-bit code: its first corner a in
// units of 2^-10 (bits 0-10 and 11-21), its depth (bits 22-25) and which of
// the six edge frames (e, f) = (b - a, c - a) / 2^-depth it has (bits 26-28).
// split4 keeps the frame in children 0-2 and turns (e, f) into (f, f - e) in
// child 3, so six frames are all there are.
// The frames' components (e0 e1 f0 f1, each -1, 0 or 1) packed two bits each
// (value + 1), one byte per frame, so that a lane reads its frame from a
// register constant whatever frame the other lanes have.
constexpr int FRAMES[6][4] = {{1, 0, 0, 1}, {0, 1, -1, 1}, {-1, 1, -1, 0},
                              {-1, 0, 0, -1}, {0, -1, 1, -1}, {1, -1, 1, 0}};
constexpr unsigned long long frame_bits() {
    unsigned long long t = 0;
    for (int f = 0; f < 6; f++)
        for (int i = 0; i < 4; i++) t |= (unsigned long long)(FRAMES[f][i] + 1) << (8 * f + 2 * i);
    return t;
}
constexpr unsigned long long FRAME_BITS = frame_bits();
__device__ __forceinline__ int frame_comp(int fr, int i) { return (int)((FRAME_BITS >> (8 * fr + 2 * i)) & 3ull) - 1; }

__device__ __forceinline__ unsigned piece_code(int a0, int a1, int depth, int frame) {
    return (unsigned)a0 | ((unsigned)a1 << 11) | ((unsigned)depth << 22) | ((unsigned)frame << 26);
}

__device__ __forceinline__ PieceF code_piece(unsigned code) {
    const int a0 = code & 2047, a1 = (code >> 11) & 2047, depth = (code >> 22) & 15, fr = code >> 26;
    const int h = 1024 >> depth;
    const float k = 1.f / SP_UNIT;
    return {a0 * k, a1 * k, (a0 + frame_comp(fr, 0) * h) * k, (a1 + frame_comp(fr, 1) * h) * k,
            (a0 + frame_comp(fr, 2) * h) * k, (a1 + frame_comp(fr, 3) * h) * k, depth};
}

// child c of a coded piece (split4's numbering)
__device__ __forceinline__ unsigned child_of(unsigned code, int c) {
    const int a0 = code & 2047, a1 = (code >> 11) & 2047, depth = (code >> 22) & 15, fr = code >> 26;
    const int h = 512 >> depth;                           // half an edge
    const int b0 = a0 + (c == 1 || c == 3 ? frame_comp(fr, 0) * h : c == 2 ? frame_comp(fr, 2) * h : 0);
    const int b1 = a1 + (c == 1 || c == 3 ? frame_comp(fr, 1) * h : c == 2 ? frame_comp(fr, 3) * h : 0);
    return piece_code(b0, b1, depth + 1, c == 3 ? (fr + 1) % 6 : fr);
}

struct PieceImg {
    float4 A, B, Cc;            // corner images (node offsets from the collocation point)
};

// children's corner images from the parent's and the three edge midpoints
__device__ __forceinline__ PieceImg child_img(const PieceImg &P, float4 mab, float4 mbc, float4 mca, int c) {
    if (c == 0) return {P.A, mab, mca};
    if (c == 1) return {mab, P.B, mbc};
    if (c == 2) return {mca, mbc, P.Cc};
    return {mab, mbc, mca};
}

template <int NPE>
__device__ __forceinline__ void mid_imgs(const float *df, const PieceF &P, float4 &mab, float4 &mbc, float4 &mca) {
    mab = map_f<NPE>(df, 0.5f * (P.a0 + P.b0), 0.5f * (P.a1 + P.b1));
    mbc = map_f<NPE>(df, 0.5f * (P.b0 + P.c0), 0.5f * (P.b1 + P.c1));
    mca = map_f<NPE>(df, 0.5f * (P.c0 + P.a0), 0.5f * (P.c1 + P.a1));
}

// the float64 test for a piece the float32 estimate leaves open, with the
// element's nodes loaded for it
template <int NPE>
__device__ __noinline__ bool split_exact(const CorrArgs &a, int e, int node, const PieceF &P) {
    double xi[3], X[3 * NPE];
    for (int c = 0; c < 3; c++) xi[c] = a.nodes[3 * (size_t)node + c];
    for (int i = 0; i < 3 * NPE; i++) X[i] = a.nodes[3 * (size_t)a.el_phi[(size_t)e * NPE + i / 3] + i % 3];
    return must_split<NPE>(X, xi, a.tau, a.maxdepth, P);
}

// split_test on a coded piece, the element's float64 nodes read only when
// the estimate is too close to call
template <int NPE>
__device__ __forceinline__ bool split_coded(const float *df, unsigned code, const PieceImg &I, const CorrArgs &a, int e,
                                            int node, float tau2, int maxdepth) {
    const PieceF P = code_piece(code);
    if (P.depth >= maxdepth) return false;
    const float4 m = map_f<NPE>(df, (P.a0 + P.b0 + P.c0) * (1.f / 3.f), (P.a1 + P.b1 + P.c1) * (1.f / 3.f));
    const float h2 = fmaxf(dist2f(I.A, I.B), fmaxf(dist2f(I.B, I.Cc), dist2f(I.Cc, I.A)));
    const float th = tau2 * h2, q = m.x * m.x + m.y * m.y + m.z * m.z - th;
    if (fabsf(q) > 2e-4f * th) return q < 0.f;
    return split_exact<NPE>(a, e, node, P);
}

// Near-singular pairs, the light ones in two steps.  Most pairs refine at
// most twice or three times (the root always splits): one thread per pair
// walks the first levels unrolled in registers and writes the pair's leaf
// pieces as 32-bit codes into slots of its own, and k_near_eval then
// evaluates their points without the refinement's control flow.  The first
// walk covers two levels (16 slots per pair); the pairs with a level-2 piece
// that splits (about a tenth) are listed in pair order and walked again over
// three levels (64 slots, for up to NW_DEEP_SHARE of the pairs); the pairs
// that refine further, or beyond that share, go to k_special_near, whose 8
// lanes per pair refine level by level.  Every path decides each piece by
// split_test (the float32 estimate from the corner images, else the float64
// test), so the pieces are the same as the oracle's, and which path a pair
// takes depends on its geometry only.
constexpr int NW_T = 128;           // threads per block of the walk
constexpr int NW_DEEP_SHARE = 8;    // the second walk takes up to 1 / 8 of the pairs
constexpr int NE_W = 8;             // lanes per pair in the evaluation
constexpr int NE_WARPS = 4;         // warps per block of the evaluation

__host__ __device__ constexpr int nw_slots(int levels) { return levels == 2 ? 16 : 64; }

// LEVELS = 2: cnt[li] = leaves, or -1 and flag[li] = 1 for a deeper pair;
// LEVELS = 3: the list is the deeper pairs' (length min(nlist, *nlist_dev)),
// cnt[li] = leaves, or -1 with the pair appended to deeper[] for the refinement
template <int NPE, int LEVELS>
__global__ void __launch_bounds__(NW_T) k_near_walk(CorrArgs a, int nlist, const int *__restrict__ nlist_dev,
                                                    const int *__restrict__ list, const int *__restrict__ pair_node,
                                                    const int *__restrict__ pair_e, int *cnt, unsigned *leaves,
                                                    int *flag, int *deeper, int *ndeeper) {
    constexpr int SLOTS = nw_slots(LEVELS);
    const int li = blockIdx.x * NW_T + threadIdx.x;
    if (nlist_dev) nlist = min(nlist, *nlist_dev);
    if (li >= nlist) return;
    const int pr = list[li], node = pair_node[pr], e = pair_e[pr];
    float df[3 * NPE];
#pragma unroll
    for (int i = 0; i < 3 * NPE; i++) df[i] = node_diff(a, a.el_phi[(size_t)e * NPE + i / 3], node, i % 3);
    const float tau2 = (float)(a.tau * a.tau);
    const int maxdepth = a.maxdepth;
    unsigned *out = leaves + (size_t)li * SLOTS;
    int n = 0;
    const unsigned root = piece_code(0, 0, 0, 0);
    bool deep = false;
    if (maxdepth <= 0) {
        out[n++] = root;                                 // no subdivision: the special rule is the regular rule
    } else {
        const float4 v0 = make_float4(df[0], df[1], df[2], 0.f), v1 = make_float4(df[3], df[4], df[5], 0.f),
                     v2 = make_float4(df[6], df[7], df[8], 0.f);
        float4 m01, m12, m20;
        if (NPE == 6) {
            m01 = make_float4(df[9 % (3 * NPE)], df[10 % (3 * NPE)], df[11 % (3 * NPE)], 0.f);
            m12 = make_float4(df[12 % (3 * NPE)], df[13 % (3 * NPE)], df[14 % (3 * NPE)], 0.f);
            m20 = make_float4(df[15 % (3 * NPE)], df[16 % (3 * NPE)], df[17 % (3 * NPE)], 0.f);
        } else {
            m01 = map_f<NPE>(df, 0.5f, 0.f); m12 = map_f<NPE>(df, 0.5f, 0.5f); m20 = map_f<NPE>(df, 0.f, 0.5f);
        }
        const PieceImg rimg{v0, v1, v2};
#pragma unroll
        for (int c1 = 0; c1 < 4; c1++) {
            if (deep) break;
            const unsigned k1 = child_of(root, c1);
            const PieceImg i1 = child_img(rimg, m01, m12, m20, c1);
            if (!split_coded<NPE>(df, k1, i1, a, e, node, tau2, maxdepth)) {
                out[n++] = k1;
                continue;
            }
            float4 mab, mbc, mca;
            mid_imgs<NPE>(df, code_piece(k1), mab, mbc, mca);
            for (int c2 = 0; c2 < 4 && !deep; c2++) {
                const unsigned k2 = child_of(k1, c2);
                const PieceImg i2 = child_img(i1, mab, mbc, mca, c2);
                if (!split_coded<NPE>(df, k2, i2, a, e, node, tau2, maxdepth)) {
                    out[n++] = k2;
                    continue;
                }
                if (LEVELS == 2) {
                    deep = true;
                    break;
                }
                float4 nab, nbc, nca;
                mid_imgs<NPE>(df, code_piece(k2), nab, nbc, nca);
                for (int c3 = 0; c3 < 4 && !deep; c3++) {
                    const unsigned k3 = child_of(k2, c3);
                    const PieceImg i3 = child_img(i2, nab, nbc, nca, c3);
                    if (split_coded<NPE>(df, k3, i3, a, e, node, tau2, maxdepth)) deep = true;
                    else out[n++] = k3;
                }
            }
        }
    }
    cnt[li] = deep ? -1 : n;
    if (LEVELS == 2) flag[li] = deep ? 1 : 0;
    else if (deep) deeper[atomicAdd(ndeeper, 1)] = pr;   // their order does not matter: pairs are independent
}

// the flagged pairs of a list, in list order
__global__ void k_compact_flagged(int n, const int *__restrict__ flag, const int *__restrict__ pos,
                                  const int *__restrict__ list, int *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = list[i];
}

// the deeper pairs beyond the second walk's share go straight to the refinement
__global__ void k_deep_overflow(int cap, const int *__restrict__ ndeep, const int *__restrict__ deep_list, int *deeper,
                                int *ndeeper) {
    const int n = *ndeep;
    for (int i = cap + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        deeper[atomicAdd(ndeeper, 1)] = deep_list[i];
}

// Evaluation of the light pairs.  A block takes chunks of NE_CHUNK
// consecutive pairs of the list, ranks them by point count (descending; ties
// in list order; deep pairs last, skipped) and gives the pairs of
// neighbouring ranks to the groups of one warp, so that the four groups of a
// warp run about the same number of rounds.
constexpr int NE_CHUNK = 64;

template <class R, bool HELM, int NPE, int W>
__global__ void __launch_bounds__(32 * NE_WARPS) k_near_eval(CorrArgs a, int nlist, const int *__restrict__ nlist_dev,
                                                             int slots, const int *__restrict__ list,
                                                             const int *__restrict__ pair_node,
                                                             const int *__restrict__ pair_e, const int *__restrict__ cnt,
                                                             const unsigned *__restrict__ leaves, R *valD,
                                                             R *valS, double *d0pair) {
    constexpr int NVP = sp_nvp(HELM, NPE), G = NE_WARPS * 32 / W;
    static_assert(NE_CHUNK % G == 0 && NE_CHUNK <= 32 * NE_WARPS, "chunk");
    __shared__ R sd[G][3 * NPE];
    __shared__ R smono[G][18];                           // float32: the map's monomial coefficients
    __shared__ int skey[NE_CHUNK], sorder[NE_CHUNK];
    __shared__ R srule[3][NQ];                           // the rule in shared memory: lanes read different points
    if (threadIdx.x < NQ) {
        srule[0][threadIdx.x] = rule_s<R>(threadIdx.x);
        srule[1][threadIdx.x] = rule_t<R>(threadIdx.x);
        srule[2][threadIdx.x] = rule_w<R>(threadIdx.x);
    }
    const int tid = threadIdx.x, lane = tid & 31, g = tid / W, sl = tid % W;
    const unsigned wmask = (W == 32 ? 0xffffffffu : ((1u << W) - 1u)) << (lane - sl);
    const R kk = (R)a.k;
    if (nlist_dev) nlist = min(nlist, *nlist_dev);
    for (int c0 = blockIdx.x * NE_CHUNK; c0 < nlist; c0 += gridDim.x * NE_CHUNK) {
        __syncthreads();                                 // the previous chunk's order and keys have been read
        if (tid < NE_CHUNK) skey[tid] = c0 + tid < nlist ? cnt[c0 + tid] : -1;
        __syncthreads();
        if (tid < NE_CHUNK) {
            const int k = skey[tid];
            int r = 0;
            for (int j = 0; j < NE_CHUNK; j++) {
                const int kj = skey[j];
                r += kj > k || (kj == k && j < tid);
            }
            sorder[r] = tid;
        }
        __syncthreads();
        for (int r0 = 0; r0 < NE_CHUNK; r0 += G) {
            const int o = sorder[r0 + g], li = c0 + o;
            if (skey[o] < 0) continue;                   // empty slots and deep pairs rank last
            const int pr = list[li], node = pair_node[pr], e = pair_e[pr];
            __syncwarp(wmask);                           // the previous pair's reads of the table are done
            for (int i = sl; i < 3 * NPE; i += W) {
                const int c = i % 3, vid = a.el_phi[(size_t)e * NPE + i / 3];
                if (sizeof(R) == sizeof(float)) sd[g][i] = (R)node_diff(a, vid, node, c);
                else sd[g][i] = (R)(a.nodes[3 * (size_t)vid + c] - a.nodes[3 * (size_t)node + c]);
            }
            __syncwarp(wmask);
            constexpr bool MONO = sizeof(R) == sizeof(float);
            if (MONO) {
                for (int i = sl; i < 18; i += W) smono[g][i] = mono_coef<R, NPE>(sd[g], i / 3, i % 3);
                __syncwarp(wmask);
            }
            R v[NVP];
#pragma unroll
            for (int i = 0; i < NVP; i++) v[i] = 0;
            const int npt = NQ * (1 + skey[o]);
            const unsigned *lv = leaves + (size_t)li * slots;
            // point j = NQ pc + q: pc = 0 the regular rule (negative weights),
            // pc >= 1 leaf pc - 1; lane sl takes j = sl, sl + W, ...
            int pc = sl / NQ, q = sl % NQ;
            for (int j = sl; j < npt; j += W) {
                R s, t, w;
                const R rs = srule[0][q], rt = srule[1][q], rw = srule[2][q];
                if (pc == 0) {
                    s = rs; t = rt; w = -rw;
                } else {
                    // the q-th point of the rule on the piece, as leaf_point
                    const PieceF P = code_piece(lv[pc - 1]);
                    const R e0 = (R)P.b0 - (R)P.a0, e1 = (R)P.b1 - (R)P.a1, f0 = (R)P.c0 - (R)P.a0, f1 = (R)P.c1 - (R)P.a1;
                    s = (R)P.a0 + rs * e0 + rt * f0;
                    t = (R)P.a1 + rs * e1 + rt * f1;
                    w = rw * fabs(e0 * f1 - e1 * f0);
                }
                if (MONO) point_acc_mono<R, HELM, NPE>(smono[g], kk, s, t, w, v);
                else eval_st<R, HELM, NPE>(sd[g], kk, s, t, w, v);
                pc += W / NQ;
                q += W % NQ;
                if (q >= NQ) { q -= NQ; pc++; }
            }
            reduce_store<R, HELM, NPE, W>(v, wmask, sl, pr, valD, valS, d0pair);
        }
    }
}

// kind of every special pair: 1 if the collocation node is a node of the element
__global__ void k_pair_kind(int npairs, int npe, const int *__restrict__ pair_node, const int *__restrict__ pair_e,
                            const int *__restrict__ el_phi, int *self) {
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= npairs) return;
    const int node = pair_node[pr], e = pair_e[pr];
    int f = 0;
    for (int v = 0; v < npe; v++) f |= el_phi[(size_t)e * npe + v] == node;
    self[pr] = f;
}

// stable partition of the pairs: self pairs to list[0 .. nself), the others after
__global__ void k_pair_split(int npairs, const int *__restrict__ self, const int *__restrict__ off, int nself,
                             int *list) {
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= npairs) return;
    list[self[pr] ? off[pr] : nself + pr - off[pr]] = pr;
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

// the correction's value array in the quadrature's working precision
template <class R> static R *corr_out(float *f, double *d);
template <> float *corr_out<float>(float *f, double *) { return f; }
template <> double *corr_out<double>(float *, double *d) { return d; }

int build_correction(bem_plan *P, cudaStream_t s) {
    Tree &t = P->t;
    Arena &A = P->arena;
    const int N = (int)P->N, E = (int)P->E, npe = P->npe;
    double *ecx, *ecy, *ecz, *eh, *rho;
    BEM_TRY(A.alloc(&ecx, E)); BEM_TRY(A.alloc(&ecy, E)); BEM_TRY(A.alloc(&ecz, E)); BEM_TRY(A.alloc(&eh, E));
    float4 *ebnd;
    float *frho;
    BEM_TRY(A.alloc(&ebnd, E));
    BEM_TRY(A.alloc(&frho, t.nbox));
    BEM_TRY(A.alloc(&rho, t.nbox));
    (k_elem_centroid<<<(E + 255) / 256, 256, 0, s>>>(E, npe, P->prm.tau_near, t.el_phi, P->nodes, ecx, ecy, ecz, eh, ebnd),
     ::bem::count_launch());
    float *nh, *nl;
    BEM_TRY(A.alloc(&nh, 3 * (size_t)N));
    BEM_TRY(A.alloc(&nl, 3 * (size_t)N));
    (k_nodes_split<<<(3 * N + 255) / 256, 256, 0, s>>>(3 * (int64_t)N, P->nodes, nh, nl), ::bem::count_launch());
    CorrArgs a{N, E, npe, P->green, P->prm.n_duffy, P->prm.max_subdiv, P->k, P->prm.tau_near, P->nodes,
               t.el_phi, t.el_chi, ecx, ecy, ecz, eh, ebnd, t.fbox, frho, t.cx, t.cy, t.cz, rho, t.child0, t.nchild,
               t.eb, t.ee, nh, nl};
    BEM_CUDA(cudaMemsetAsync(rho, 0, sizeof(double) * t.nbox, s));
    (k_elem_search_radius<<<(E + 255) / 256, 256, 0, s>>>(a, t.leaf_of_node, t.parent, (unsigned long long *)rho),
     ::bem::count_launch());
    (k_rho_float<<<(t.nbox + 255) / 256, 256, 0, s>>>(t.nbox, rho, frho), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    int *cnt, *off, *tot;
    BEM_TRY(A.alloc(&cnt, N + 1));
    BEM_TRY(A.alloc(&off, N + 1));
    BEM_TRY(A.alloc(&tot, 2));
    int *sblk = nullptr;
    BEM_TRY(A.alloc(&sblk, scan_scratch(N + 1)));
    // one search: the count pass keeps up to SS_CAP elements per node, which
    // are copied into place; a node with more makes the search run again
    int *ptmp = nullptr;
    BEM_TRY(A.alloc(&ptmp, (size_t)N * SS_CAP));
    BEM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (N + 1), s));
    BEM_CUDA(cudaMemsetAsync(tot + 1, 0, sizeof(int), s));
    (k_special_count<<<(N + SS_WARPS - 1) / SS_WARPS, 32 * SS_WARPS, 0, s>>>(a, cnt, ptmp, SS_CAP, tot + 1),
     ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    BEM_TRY(scan_exclusive(cnt, off, N + 1, tot, sblk, s));
    int hcnt[2] = {0, 0};
    BEM_CUDA(cudaMemcpyAsync(hcnt, tot, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    const int npairs = hcnt[0];
    int *pair_e, *pair_node;
    BEM_TRY(A.alloc(&pair_e, npairs));
    BEM_TRY(A.alloc(&pair_node, npairs));
    if (hcnt[1]) (k_special_write<<<(N + SS_WARPS - 1) / SS_WARPS, 32 * SS_WARPS, 0, s>>>(a, off, pair_e), ::bem::count_launch());
    else (k_special_copy<<<N, 64, 0, s>>>(N, off, ptmp, SS_CAP, pair_e), ::bem::count_launch());
    (k_pair_nodes<<<(N + 255) / 256, 256, 0, s>>>(N, off, pair_node), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    const int C = P->green == BEM_HELMHOLTZ ? 2 : 1;
    Correction &K = P->corr;
    K.nnzD = K.nnzS = (int64_t)npairs * npe;
    BEM_TRY(A.alloc(&K.ptrD, N + 1));
    BEM_TRY(A.alloc(&K.colD, K.nnzD));
    BEM_TRY(A.alloc(&K.colS, K.nnzS));
    // the values in the plan's working precision: float32 for mixed plans
    // (what their products read), float64 otherwise
    const bool fcorr = P->prm.precision == BEM_MIXED;
    if (!fcorr) {
        BEM_TRY(A.alloc(&K.valD, K.nnzD * C));
        BEM_TRY(A.alloc(&K.valS, K.nnzS * C));
    }
    K.ptrS = K.ptrD;
    double *d0pair, *d0row;
    BEM_TRY(A.alloc(&d0pair, npairs));
    BEM_TRY(A.alloc(&d0row, N));
    // every allocation comes before the long kernels, so that work other
    // streams enqueue next can overlap them
    if (fcorr) {
        BEM_TRY(A.alloc(&K.fvalD, K.nnzD * C));
        BEM_TRY(A.alloc(&K.fvalS, K.nnzS * C));
    }
    (k_rows_ptr<<<(N + 256) / 256, 256, 0, s>>>(N, npe, off, K.ptrD), ::bem::count_launch());
    (k_corr_csr<<<(npairs + 255) / 256, 256, 0, s>>>(npairs, npe, pair_e, t.el_phi, t.el_chi, K.colD, K.colS), ::bem::count_launch());
    // self pairs first, then the near-singular ones (stable), so that each kernel
    // takes one kind
    int *kind = nullptr, *koff = nullptr, *klist = nullptr, *ktot = nullptr, *kblk = nullptr;
    BEM_TRY(A.alloc(&kind, std::max(1, npairs)));
    BEM_TRY(A.alloc(&koff, std::max(1, npairs)));
    BEM_TRY(A.alloc(&klist, std::max(1, npairs)));
    BEM_TRY(A.alloc(&ktot, 1));
    BEM_TRY(A.alloc(&kblk, scan_scratch(npairs)));
    int nself = 0;
    if (npairs > 0) {
        (k_pair_kind<<<(npairs + 255) / 256, 256, 0, s>>>(npairs, npe, pair_node, pair_e, t.el_phi, kind),
         ::bem::count_launch());
        BEM_TRY(scan_exclusive(kind, koff, npairs, ktot, kblk, s));
        BEM_CUDA(cudaMemcpyAsync(&nself, ktot, sizeof(int), cudaMemcpyDeviceToHost, s));
        BEM_CUDA(cudaStreamSynchronize(s));
        (k_pair_split<<<(npairs + 255) / 256, 256, 0, s>>>(npairs, kind, koff, nself, klist), ::bem::count_launch());
    }
    const int nnear = npairs - nself;
    // near-singular pairs: the two-level walk over all of them, the
    // three-level walk over those it leaves (in pair order, up to a share),
    // the refinement over the rest
    const int dcap = std::max(1024, nnear / NW_DEEP_SHARE);
    int *lcnt = nullptr, *dflag = nullptr, *dpos = nullptr, *dblk = nullptr, *deep_list = nullptr, *ndeep = nullptr;
    int *cnt2 = nullptr, *deeper = nullptr, *ndeeper = nullptr;
    unsigned *leaves = nullptr, *leaves2 = nullptr;
    BEM_TRY(A.alloc(&lcnt, std::max(1, nnear)));
    BEM_TRY(A.alloc(&dflag, std::max(1, nnear)));
    BEM_TRY(A.alloc(&dpos, std::max(1, nnear)));
    BEM_TRY(A.alloc(&dblk, scan_scratch(std::max(1, nnear))));
    BEM_TRY(A.alloc(&deep_list, std::max(1, nnear)));
    BEM_TRY(A.alloc(&ndeep, 1));
    BEM_TRY(A.alloc(&cnt2, dcap));
    BEM_TRY(A.alloc(&deeper, std::max(1, nnear)));
    BEM_TRY(A.alloc(&ndeeper, 1));
    BEM_TRY(A.alloc(&leaves, (size_t)std::max(1, nnear) * nw_slots(2)));
    BEM_TRY(A.alloc(&leaves2, (size_t)dcap * nw_slots(3)));
    BEM_CUDA(cudaMemsetAsync(ndeep, 0, sizeof(int), s));
    BEM_CUDA(cudaMemsetAsync(ndeeper, 0, sizeof(int), s));
    if (nnear > 0) {
        const int *nl = klist + nself;
        const int gw = (nnear + NW_T - 1) / NW_T, gw2 = (dcap + NW_T - 1) / NW_T;
        if (npe == 3)
            (k_near_walk<3, 2><<<gw, NW_T, 0, s>>>(a, nnear, nullptr, nl, pair_node, pair_e, lcnt, leaves, dflag,
                                                  nullptr, nullptr), ::bem::count_launch());
        else
            (k_near_walk<6, 2><<<gw, NW_T, 0, s>>>(a, nnear, nullptr, nl, pair_node, pair_e, lcnt, leaves, dflag,
                                                  nullptr, nullptr), ::bem::count_launch());
        BEM_TRY(scan_exclusive(dflag, dpos, nnear, ndeep, dblk, s));
        (k_compact_flagged<<<(nnear + 255) / 256, 256, 0, s>>>(nnear, dflag, dpos, nl, deep_list), ::bem::count_launch());
        if (npe == 3)
            (k_near_walk<3, 3><<<gw2, NW_T, 0, s>>>(a, dcap, ndeep, deep_list, pair_node, pair_e, cnt2, leaves2,
                                                   nullptr, deeper, ndeeper), ::bem::count_launch());
        else
            (k_near_walk<6, 3><<<gw2, NW_T, 0, s>>>(a, dcap, ndeep, deep_list, pair_node, pair_e, cnt2, leaves2,
                                                   nullptr, deeper, ndeeper), ::bem::count_launch());
        (k_deep_overflow<<<64, 256, 0, s>>>(dcap, ndeep, deep_list, deeper, ndeeper), ::bem::count_launch());
        BEM_LAUNCH_CHECK();
    }
    {
        const bool mx = P->prm.precision == BEM_MIXED, helm = P->green == BEM_HELMHOLTZ;
        // grid-stride loops over the pair lists, but not persistent grids:
        // about SP_PAIRS_PER_WARP pairs per warp or group, so that blocks retire
        // throughout and the diagonal's product (a stream of higher priority)
        // gets SMs while the quadrature is still running
        const int gs = (int)std::max<int64_t>(1, ((int64_t)nself + SP_WARPS * SP_PAIRS_PER_WARP - 1) /
                                                     (SP_WARPS * SP_PAIRS_PER_WARP));
        const int ge = (int)std::max<int64_t>(1, ((int64_t)nnear + 4 * NE_CHUNK - 1) / (4 * NE_CHUNK));
        const int ge2 = (int)std::max<int64_t>(1, ((int64_t)dcap + 4 * NE_CHUNK - 1) / (4 * NE_CHUNK));
        const int gn = 5 * std::max(1, P->sm_count);       // deep pairs: a few per cent, count on the device
#define BEM_SW(R, H, NP)                                                                                          \
    do {                                                                                                          \
        if (nnear > 0) {                                                                                          \
            (k_near_eval<R, H, NP, NE_W><<<ge, 32 * NE_WARPS, 0, s>>>(a, nnear, nullptr, nw_slots(2), klist + nself,\
                                                                       pair_node, pair_e, lcnt, leaves, corr_out<R>(K.fvalD, K.valD),\
                                                                       corr_out<R>(K.fvalS, K.valS), d0pair),                           \
             ::bem::count_launch());                                                                              \
            (k_near_eval<R, H, NP, NE_W><<<ge2, 32 * NE_WARPS, 0, s>>>(a, dcap, ndeep, nw_slots(3), deep_list,     \
                                                                        pair_node, pair_e, cnt2, leaves2, corr_out<R>(K.fvalD, K.valD),\
                                                                        corr_out<R>(K.fvalS, K.valS), d0pair),                          \
             ::bem::count_launch());                                                                              \
            (k_special_near<R, H, NP><<<gn, 32 * SPN_WARPS, 0, s>>>(a, ndeeper, deeper, pair_node, pair_e,         \
                                                                    corr_out<R>(K.fvalD, K.valD), corr_out<R>(K.fvalS, K.valS), d0pair), \
             ::bem::count_launch());                                                                              \
        }                                                                                                         \
        if (nself > 0)                                                                                            \
            (k_special_self<R, H, NP><<<gs, 32 * SP_WARPS, 0, s>>>(a, nself, klist, pair_node, pair_e,           \
                                                                   corr_out<R>(K.fvalD, K.valD), corr_out<R>(K.fvalS, K.valS), d0pair),                               \
             ::bem::count_launch());                                                                              \
    } while (0)
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
    BEM_LAUNCH_CHECK();
    // the diagonal starts as 1 + (correction row sum of D0); the regular part
    // is added by one Laplace double-layer product on phi = 1
    P->C = d0row;
    // the temporaries are released once the stream has finished with them
    for (void *q : {(void *)ptmp, (void *)nh, (void *)nl, (void *)lcnt, (void *)dflag, (void *)dpos, (void *)dblk, (void *)deep_list, (void *)ndeep, (void *)cnt2, (void *)deeper, (void *)ndeeper, (void *)leaves, (void *)leaves2, (void *)kind, (void *)koff, (void *)klist, (void *)ktot, (void *)kblk, (void *)cnt, (void *)tot, (void *)sblk, (void *)pair_node, (void *)d0pair, (void *)ecx, (void *)ecy, (void *)ecz,
                    (void *)eh, (void *)ebnd, (void *)frho, (void *)rho, (void *)off, (void *)pair_e})
        P->deferred.push_back(q);
    return BEM_OK;
}

}  // namespace bem
