// Accelerated field evaluation (Section 2.2, "Accelerated field evaluation"):
// the field of known surface data at points off the surface,
//     u(x) = sum over the surface of  phi dG/dn1 - G chi      (C(x) = 1 outside),
// by descending the box tree from the root for every field point: a box whose
// centre is farther than eta r_C from the point contributes its multipole
// expansion; otherwise a parent is opened and a leaf is integrated directly
// over its elements (7-point rule, or the parametric subdivision of the
// near-singular rule when the point is within tau h_e of an element).
//
// The moments are those of the product: double-layer moments of phi minus
// single-layer moments of chi, shifted up the tree (field_moments).  One warp
// per field point; the derivatives of G at the point's offset from a box come
// from the same recursions as the translation tables, evaluated per box by the
// warp; everything after the moments is float64.
#include <algorithm>
#include <cmath>

#include "bem_internal.cuh"

namespace bem {

namespace {

constexpr int FW = 4;                   // warps (field points) per block
constexpr int FSTACK = 512;             // descent stack entries per warp
constexpr int SUBSTACK = 64;            // subdivision stack entries per lane

struct FieldArgs {
    int green;
    double k, eta, side, tau;
    int maxdepth, p, np, npe, nbox;
    const double *cx, *cy, *cz, *r;
    const int *level, *child0, *nchild, *eb, *ee;
    const int *tm, *tn, *tk, *idx3;
    const int *lev_p;                   // order of each level (nullptr: p everywhere)
    const double *fact;
    const void *M;                      // float or double moments [nbox][np][C]
    int mfloat;
    const double *nodes;
    const int *el_phi, *el_chi;
    const double *phi, *chi;            // [n][C]
    int *err;
};

__device__ __forceinline__ void shape6(int npe, double s, double t, double *N, double *Ns, double *Nt) {
    const double l0 = 1.0 - s - t;
    if (npe == 3) {
        N[0] = l0; N[1] = s; N[2] = t;
        Ns[0] = -1.0; Ns[1] = 1.0; Ns[2] = 0.0;
        Nt[0] = -1.0; Nt[1] = 0.0; Nt[2] = 1.0;
        return;
    }
    N[0] = l0 * (2.0 * l0 - 1.0); N[1] = s * (2.0 * s - 1.0); N[2] = t * (2.0 * t - 1.0);
    N[3] = 4.0 * l0 * s; N[4] = 4.0 * s * t; N[5] = 4.0 * t * l0;
    Ns[0] = 1.0 - 4.0 * l0; Ns[1] = 4.0 * s - 1.0; Ns[2] = 0.0;
    Ns[3] = 4.0 * (l0 - s); Ns[4] = 4.0 * t; Ns[5] = -4.0 * t;
    Nt[0] = 1.0 - 4.0 * l0; Nt[1] = 0.0; Nt[2] = 4.0 * t - 1.0;
    Nt[3] = -4.0 * s; Nt[4] = 4.0 * s; Nt[5] = 4.0 * (l0 - t);
}

// one quadrature point: adds wref J (phi(xi) dG/dn1 - chi(xi) G) to acc
template <int C>
__device__ __forceinline__ void field_point(const FieldArgs &a, const double *x, const double *X, const double *ph,
                                            const double *ch, double s, double t, double wref, double *acc) {
    double N[6], Ns[6], Nt[6];
    shape6(a.npe, s, t, N, Ns, Nt);
    double y[3] = {0.0, 0.0, 0.0}, ts[3] = {0.0, 0.0, 0.0}, tt[3] = {0.0, 0.0, 0.0};
    double fp[2] = {0.0, 0.0}, fc[2] = {0.0, 0.0};
    for (int q = 0; q < a.npe; q++)
        for (int c = 0; c < 3; c++) {
            y[c] += N[q] * X[3 * q + c];
            ts[c] += Ns[q] * X[3 * q + c];
            tt[c] += Nt[q] * X[3 * q + c];
        }
    for (int q = 0; q < a.npe; q++)
        for (int c = 0; c < C; c++) {
            fp[c] += N[q] * ph[q * C + c];
            fc[c] += N[q] * ch[q * C + c];
        }
    const double nx = ts[1] * tt[2] - ts[2] * tt[1], ny = ts[2] * tt[0] - ts[0] * tt[2], nz = ts[0] * tt[1] - ts[1] * tt[0];
    const double J = sqrt(nx * nx + ny * ny + nz * nz);
    const double rx = x[0] - y[0], ry = x[1] - y[1], rz = x[2] - y[2];
    const double R = sqrt(rx * rx + ry * ry + rz * rz);
    const double w = wref * J;
    const double G0 = 0.25 / M_PI / R;
    const double dG0 = (rx * nx + ry * ny + rz * nz) / J * G0 / (R * R);
    if (C == 1) {
        acc[0] += w * (fp[0] * dG0 - fc[0] * G0);
    } else {
        double sn, cs;
        sincos(a.k * R, &sn, &cs);
        const double gr = cs * G0, gi = sn * G0;                       // G = e^{jkR} G0
        const double kR = a.k * R;
        const double dr = (cs + kR * sn) * dG0, di = (sn - kR * cs) * dG0;   // e^{jkR} (1 - jkR) dG0
        acc[0] += w * (fp[0] * dr - fp[1] * di - (fc[0] * gr - fc[1] * gi));
        acc[1] += w * (fp[0] * di + fp[1] * dr - (fc[0] * gi + fc[1] * gr));
    }
}

__device__ __forceinline__ void map_param(const FieldArgs &a, const double *X, double s, double t, double *y) {
    double N[6], Ns[6], Nt[6];
    shape6(a.npe, s, t, N, Ns, Nt);
    y[0] = y[1] = y[2] = 0.0;
    for (int q = 0; q < a.npe; q++)
        for (int c = 0; c < 3; c++) y[c] += N[q] * X[3 * q + c];
}

__device__ __forceinline__ double dist(const double *u, const double *v) {
    const double d0 = u[0] - v[0], d1 = u[1] - v[1], d2 = u[2] - v[2];
    return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

// one element against the field point (the near-singular rule of the product)
template <int C>
__device__ void field_element(const FieldArgs &a, const double *x, int e, double *acc) {
    const int *ep = a.el_phi + (size_t)e * a.npe, *ec = a.el_chi + (size_t)e * a.npe;
    double X[18], ph[12], ch[12];
    for (int q = 0; q < a.npe; q++) {
        for (int c = 0; c < 3; c++) X[3 * q + c] = a.nodes[3 * (size_t)ep[q] + c];
        for (int c = 0; c < C; c++) {
            ph[q * C + c] = a.phi[(size_t)ep[q] * C + c];
            ch[q * C + c] = a.chi[(size_t)ec[q] * C + c];
        }
    }
    // stack of parametric triangles (a, b, c, depth)
    double st[SUBSTACK][6];
    int sd[SUBSTACK], sp = 0;
    st[0][0] = 0.0; st[0][1] = 0.0; st[0][2] = 1.0; st[0][3] = 0.0; st[0][4] = 0.0; st[0][5] = 1.0;
    sd[0] = 0;
    sp = 1;
    while (sp > 0) {
        sp--;
        const double *T = st[sp];
        const double pa[2] = {T[0], T[1]}, pb[2] = {T[2], T[3]}, pc[2] = {T[4], T[5]};
        const int depth = sd[sp];
        double xa[3], xb[3], xc[3], xm[3];
        map_param(a, X, pa[0], pa[1], xa);
        map_param(a, X, pb[0], pb[1], xb);
        map_param(a, X, pc[0], pc[1], xc);
        map_param(a, X, (pa[0] + pb[0] + pc[0]) / 3.0, (pa[1] + pb[1] + pc[1]) / 3.0, xm);
        double h = dist(xa, xb);
        h = fmax(h, dist(xb, xc));
        h = fmax(h, dist(xc, xa));
        if (depth >= a.maxdepth || !(dist(x, xm) < a.tau * h) || sp + 4 > SUBSTACK) {
            const double det = fabs((pb[0] - pa[0]) * (pc[1] - pa[1]) - (pb[1] - pa[1]) * (pc[0] - pa[0]));
            for (int q = 0; q < 7; q++) {
                double s, t, w;
                radon7(q, s, t, w);
                field_point<C>(a, x, X, ph, ch, pa[0] + s * (pb[0] - pa[0]) + t * (pc[0] - pa[0]),
                               pa[1] + s * (pb[1] - pa[1]) + t * (pc[1] - pa[1]), w * det, acc);
            }
            continue;
        }
        const double ab[2] = {0.5 * (pa[0] + pb[0]), 0.5 * (pa[1] + pb[1])};
        const double bc[2] = {0.5 * (pb[0] + pc[0]), 0.5 * (pb[1] + pc[1])};
        const double ca[2] = {0.5 * (pc[0] + pa[0]), 0.5 * (pc[1] + pa[1])};
        const double kids[4][6] = {{pa[0], pa[1], ab[0], ab[1], ca[0], ca[1]},
                                   {ab[0], ab[1], pb[0], pb[1], bc[0], bc[1]},
                                   {ca[0], ca[1], bc[0], bc[1], pc[0], pc[1]},
                                   {ab[0], ab[1], bc[0], bc[1], ca[0], ca[1]}};
        for (int c = 3; c >= 0; c--) {
            for (int v = 0; v < 6; v++) st[sp][v] = kids[c][v];
            sd[sp] = depth + 1;
            sp++;
        }
    }
}

// derivatives D^g G(r), |g| <= p, into up[] (pairs re, im) by the recursions
// of the translation tables; the warp shares the work of each level
__device__ void warp_derivs(const FieldArgs &a, const double *r, double *Gh, double *up, double *cur) {
    const int lane = threadIdx.x & 31, p = a.p, P1 = p + 1;
    if (lane == 0) {
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], r1 = sqrt(r2), inv4pi = 0.25 / M_PI;
        if (a.green != BEM_HELMHOLTZ) {
            double g = inv4pi / r1;
            for (int h = 0; h <= p; h++) {
                Gh[2 * h] = g;
                Gh[2 * h + 1] = 0.0;
                g = -(2.0 * h + 1.0) * g / r2;
            }
        } else {
            double sn, cs;
            sincos(a.k * r1, &sn, &cs);
            double pr = sn * inv4pi / a.k, pi = -cs * inv4pi / a.k, cr = cs * inv4pi / r1, ci = sn * inv4pi / r1;
            for (int h = 0; h <= p; h++) {
                Gh[2 * h] = cr;
                Gh[2 * h + 1] = ci;
                const double nr = -((2.0 * h + 1.0) * cr + a.k * a.k * pr) / r2;
                const double ni = -((2.0 * h + 1.0) * ci + a.k * a.k * pi) / r2;
                pr = cr; pi = ci; cr = nr; ci = ni;
            }
        }
        up[0] = Gh[2 * p];
        up[1] = Gh[2 * p + 1];
    }
    __syncwarp();
    for (int h = p - 1; h >= 0; h--) {
        const int top = p - h, n = (top + 1) * (top + 2) * (top + 3) / 6;
        for (int u = lane; u < n; u += 32) {
            const int m = a.tm[u], nn = a.tn[u], k = a.tk[u];
            double v0, v1;
            if (m + nn + k == 0) {
                v0 = Gh[2 * h];
                v1 = Gh[2 * h + 1];
            } else {
                const int ax = m > 0 ? 0 : (nn > 0 ? 1 : 2);
                const int g = ax == 0 ? m : (ax == 1 ? nn : k);
                const int m1 = m - (ax == 0), n1 = nn - (ax == 1), k1 = k - (ax == 2);
                const int i1 = a.idx3[(m1 * P1 + n1) * P1 + k1];
                v0 = r[ax] * up[2 * i1];
                v1 = r[ax] * up[2 * i1 + 1];
                if (g > 1) {
                    const int i2 = a.idx3[((m1 - (ax == 0)) * P1 + (n1 - (ax == 1))) * P1 + (k1 - (ax == 2))];
                    v0 += (g - 1) * up[2 * i2];
                    v1 += (g - 1) * up[2 * i2 + 1];
                }
            }
            cur[2 * u] = v0;
            cur[2 * u + 1] = v1;
        }
        __syncwarp();
        for (int u = lane; u < n; u += 32) {
            up[2 * u] = cur[2 * u];
            up[2 * u + 1] = cur[2 * u + 1];
        }
        __syncwarp();
    }
}

template <int C>
__global__ void __launch_bounds__(FW * 32) k_field(int64_t npts, const double *__restrict__ pts, double *__restrict__ u,
                                                   const FieldArgs a) {
    extern __shared__ double fsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = a.np;
    double *Gh = fsm + (size_t)warp * (2 * (PMAX + 2) + 4 * np);
    double *up = Gh + 2 * (PMAX + 2), *cur = up + 2 * np;
    __shared__ int stack[FW][FSTACK];
    __shared__ int sp[FW];
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;   // blockDim.x / 32 <= FW points per block
    if (i >= npts) return;                            // warp-uniform
    const double x[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
    double acc[2] = {0.0, 0.0};
    if (lane == 0) {
        stack[warp][0] = 0;                           // the root
        sp[warp] = 1;
    }
    __syncwarp();
    while (sp[warp] > 0) {
        __syncwarp();
        const int b = stack[warp][sp[warp] - 1];
        __syncwarp();
        if (lane == 0) sp[warp]--;
        __syncwarp();
        const double c[3] = {a.cx[b], a.cy[b], a.cz[b]};
        const double rr[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
        const double d = sqrt(rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2]);
        if (d > a.eta * a.r[b]) {
            // multipole expansion: u += sum_g (-1)^|g| / g! D^g G(x - c) I_g,
            // I_g = (scaled moment) h^|g|
            warp_derivs(a, rr, Gh, up, cur);
            const double h = scalbn(a.side, -a.level[b]);
            const int pb = a.lev_p ? a.lev_p[a.level[b]] : a.p, npb = (pb + 1) * (pb + 2) * (pb + 3) / 6;
            for (int g = lane; g < npb; g += 32) {
                const int m = a.tm[g], n = a.tn[g], k = a.tk[g], dg = m + n + k;
                const double cf = ((dg & 1) ? -1.0 : 1.0) * pow(h, (double)dg) / (a.fact[m] * a.fact[n] * a.fact[k]);
                double mr, mi = 0.0;
                if (a.mfloat) {
                    const float *Mf = (const float *)a.M + ((size_t)b * np + g) * C;
                    mr = Mf[0];
                    if (C == 2) mi = Mf[1];
                } else {
                    const double *Md = (const double *)a.M + ((size_t)b * np + g) * C;
                    mr = Md[0];
                    if (C == 2) mi = Md[1];
                }
                acc[0] += cf * (up[2 * g] * mr - up[2 * g + 1] * mi);
                acc[1] += cf * (up[2 * g] * mi + up[2 * g + 1] * mr);
            }
            __syncwarp();
        } else if (a.nchild[b] > 0) {
            if (lane == 0) {
                const int nch = a.nchild[b];
                if (sp[warp] + nch <= FSTACK) {
                    for (int q = nch - 1; q >= 0; q--) stack[warp][sp[warp]++] = a.child0[b] + q;
                } else {
                    atomicOr(a.err, 2);               // stack full: this branch is skipped
                }
            }
            __syncwarp();
        } else {
            for (int e = a.eb[b] + lane; e < a.ee[b]; e += 32) field_element<C>(a, x, e, acc);
            __syncwarp();
        }
    }
#pragma unroll
    for (int c = 0; c < 2; c++)
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane == 0)
        for (int c = 0; c < C; c++) u[i * C + c] = acc[c];
}

}  // namespace

template <int C>
static int launch_field(bem_plan *P, int64_t npts, const double *pts, double *u, const double *phi, const double *chi,
                        cudaStream_t s) {
    const Tree &t = P->t;
    FieldArgs a{};
    a.green = P->green;
    a.k = P->k;
    a.eta = P->prm.eta;
    a.side = t.side;
    a.tau = P->prm.tau_near;
    a.maxdepth = P->prm.max_subdiv;
    a.p = P->mi.p;
    a.np = P->mi.np;
    a.npe = P->npe;
    a.nbox = t.nbox;
    a.cx = t.cx; a.cy = t.cy; a.cz = t.cz; a.r = t.r;
    a.level = t.level; a.child0 = t.child0; a.nchild = t.nchild; a.eb = t.eb; a.ee = t.ee;
    a.tm = P->d_m; a.tn = P->d_n; a.tk = P->d_k; a.idx3 = P->d_idx3;
    a.lev_p = P->lev_var ? P->d_lev_p : nullptr;
    a.fact = P->d_fact;
    a.mfloat = P->prm.precision == BEM_MIXED;
    a.M = a.mfloat ? (const void *)P->fM : (const void *)P->M;
    a.nodes = P->nodes;
    a.el_phi = t.el_phi;
    a.el_chi = t.el_chi;
    a.phi = phi;
    a.chi = chi;
    a.err = P->dev_err;
    // derivative scratch per warp; fewer warps per block at high orders
    const size_t per_warp = sizeof(double) * (2 * (PMAX + 2) + 4 * (size_t)a.np);
    const int fw = (int)std::max<size_t>(1, std::min<size_t>(FW, (size_t)(200 * 1024) / per_warp));
    const size_t sm = per_warp * fw;
    BEM_CUDA(cudaFuncSetAttribute(k_field<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int64_t nblk = (npts + fw - 1) / fw;
    if (nblk > 0) (k_field<C><<<(unsigned)nblk, fw * 32, sm, s>>>(npts, pts, u, a), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    return BEM_OK;
}

}  // namespace bem

using namespace bem;

extern "C" int bem_field(bem_plan *P, const void *phi_dev, const void *chi_dev, int64_t npts, const double *pts_dev,
                         void *u_dev, void *cuda_stream) {
    if (!P || !phi_dev || !chi_dev || npts < 0 || (npts > 0 && (!pts_dev || !u_dev))) {
        set_error("bem_field: bad argument");
        return BEM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    BEM_CUDA(cudaSetDevice(P->device));
    BEM_CUDA(cudaMemsetAsync(P->skip, 0, sizeof(int), s));
    BEM_TRY(field_moments(P, phi_dev, chi_dev, s));
    const double *ph = (const double *)phi_dev, *ch = (const double *)chi_dev;
    if (P->green == BEM_HELMHOLTZ) return launch_field<2>(P, npts, pts_dev, (double *)u_dev, ph, ch, s);
    return launch_field<1>(P, npts, pts_dev, (double *)u_dev, ph, ch, s);
}
