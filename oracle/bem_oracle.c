/*
 * bem_oracle.c -- plain, slow, FP64 CPU oracle for the FMM-accelerated
 * collocation boundary element method of Carley, "BEM3D: a free adaptive fast
 * multipole boundary element library".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or constant generator with the CUDA
 * library: every formula below is written out again from the paper.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no FMA contraction,
 * so that the integer tree, its radii and its lists follow a fixed FP64
 * operation order).
 *
 * Contents and the passage each part follows:
 *   - boundary integral equation and the discrete system: Eq. 1, Eq. 2, Eq. 3
 *     (Section 2.1), read as the exterior problem  C phi - D phi = -S chi,
 *     C_i = 1 + sum_j D0_ij (Laplace G0 even for Helmholtz);
 *   - elements: flat 3-node and curved 6-node isoparametric triangles
 *     (Section 2.2, Figure 1);
 *   - quadrature: the 7-point degree-5 symmetric rule for regular pairs,
 *     a Duffy-collapsed Gauss-Legendre product rule for self (singular)
 *     pairs, recursive 4-way subdivision for near-singular pairs (stand-ins
 *     for the rules cited in Section 2.1);
 *   - sharp-edge multi-indexing of the Neumann data (Section 2.3);
 *   - octree over vertices, leaf when fewer than B vertices (Section 3.1);
 *   - Taylor multipole moments, local expansions, coefficient shift and
 *     expansion shift (Section 3.2, Eq. 4-10);
 *   - Tausch's recursions for Green's-function derivatives (Section 3.3,
 *     Eq. 11 and the three-step scheme);
 *   - convergence radii and parent radius (Section 3.4, Eq. 12);
 *   - near-field and interaction lists and the four-step fast matrix
 *     multiplication (Section 3.6, Eq. 13).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_LAPLACE 0
#define OR_HELMHOLTZ 1
#define OR_OP_A 0 /* y = C x - D x   (phi -> left-hand side) */
#define OR_OP_B 1 /* y = -S x        (chi -> right-hand side) */

typedef double complex cplx;

static const double OR_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Quadrature rules on the reference triangle (0,0), (1,0), (0,1), area 1/2  */
/* ------------------------------------------------------------------------ */

/* Radon's 7-point rule of degree 5 (Stroud T2:5-1): the centroid plus two
 * orbits of three points; weights sum to the reference area 1/2. */
static void rule7(double s[7], double t[7], double w[7])
{
    double r15 = sqrt(15.0);
    double a = (6.0 - r15) / 21.0, b = (9.0 + 2.0 * r15) / 21.0;
    double c = (6.0 + r15) / 21.0, d = (9.0 - 2.0 * r15) / 21.0;
    double wa = (155.0 - r15) / 2400.0, wc = (155.0 + r15) / 2400.0;
    s[0] = 1.0 / 3.0; t[0] = 1.0 / 3.0; w[0] = 9.0 / 80.0;
    s[1] = a; t[1] = a; w[1] = wa;
    s[2] = b; t[2] = a; w[2] = wa;
    s[3] = a; t[3] = b; w[3] = wa;
    s[4] = c; t[4] = c; w[4] = wc;
    s[5] = d; t[5] = c; w[5] = wc;
    s[6] = c; t[6] = d; w[6] = wc;
}

void or_rule7(double *s, double *t, double *w) { rule7(s, t, w); }

/* ------------------------------------------------------------------------ */
/* Shape functions (Section 2.2): corners 0,1,2; mid-sides 3 (0-1), 4 (1-2), */
/* 5 (2-0).  L0 = 1 - s - t, L1 = s, L2 = t are the area coordinates.        */
/* ------------------------------------------------------------------------ */
static void shape(int npe, double s, double t, double N[6], double Ns[6], double Nt[6])
{
    double L0 = (1.0 - s) - t, L1 = s, L2 = t;
    if (npe == 3) {
        N[0] = L0; N[1] = L1; N[2] = L2;
        Ns[0] = -1.0; Ns[1] = 1.0; Ns[2] = 0.0;
        Nt[0] = -1.0; Nt[1] = 0.0; Nt[2] = 1.0;
        return;
    }
    N[0] = L0 * (2.0 * L0 - 1.0);
    N[1] = L1 * (2.0 * L1 - 1.0);
    N[2] = L2 * (2.0 * L2 - 1.0);
    N[3] = 4.0 * L0 * L1;
    N[4] = 4.0 * L1 * L2;
    N[5] = 4.0 * L2 * L0;
    Ns[0] = -(4.0 * L0 - 1.0); Ns[1] = 4.0 * L1 - 1.0; Ns[2] = 0.0;
    Ns[3] = 4.0 * (L0 - L1);   Ns[4] = 4.0 * L2;       Ns[5] = -4.0 * L2;
    Nt[0] = -(4.0 * L0 - 1.0); Nt[1] = 0.0;            Nt[2] = 4.0 * L2 - 1.0;
    Nt[3] = -4.0 * L1;         Nt[4] = 4.0 * L1;       Nt[5] = 4.0 * (L0 - L2);
}

void or_shape(int npe, double s, double t, double *N, double *Ns, double *Nt)
{
    shape(npe, s, t, N, Ns, Nt);
}

/* x(s,t) = sum_a N_a X_a, summed in node order. */
static void map_point(const double *X, int npe, const double N[6], double x[3])
{
    x[0] = 0.0; x[1] = 0.0; x[2] = 0.0;
    for (int a = 0; a < npe; a++) {
        x[0] = x[0] + N[a] * X[3 * a + 0];
        x[1] = x[1] + N[a] * X[3 * a + 1];
        x[2] = x[2] + N[a] * X[3 * a + 2];
    }
}

/* |a - b| with a fixed operation order: ((dx*dx + dy*dy) + dz*dz), sqrt. */
static double dist3(const double *a, const double *b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt((dx * dx + dy * dy) + dz * dz);
}

/* Geometry of an element at a parametric point: position, unit normal
 * t1 x t2 / |t1 x t2| (outward for counter-clockwise corners), Jacobian. */
typedef struct {
    double x[3], n[3], J, N[6];
} gpoint;

static void elem_point(const double *X, int npe, double s, double t, gpoint *g)
{
    double Ns[6], Nt[6], t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
    shape(npe, s, t, g->N, Ns, Nt);
    map_point(X, npe, g->N, g->x);
    for (int a = 0; a < npe; a++)
        for (int c = 0; c < 3; c++) {
            t1[c] += Ns[a] * X[3 * a + c];
            t2[c] += Nt[a] * X[3 * a + c];
        }
    double nx = t1[1] * t2[2] - t1[2] * t2[1];
    double ny = t1[2] * t2[0] - t1[0] * t2[2];
    double nz = t1[0] * t2[1] - t1[1] * t2[0];
    g->J = sqrt(nx * nx + ny * ny + nz * nz);
    g->n[0] = nx / g->J; g->n[1] = ny / g->J; g->n[2] = nz / g->J;
}

/* centroid image X(1/3,1/3) and h = longest chord between corner images. */
static void elem_centroid_h(const double *X, int npe, double cen[3], double *h)
{
    double N[6], Ns[6], Nt[6];
    shape(npe, 1.0 / 3.0, 1.0 / 3.0, N, Ns, Nt);
    map_point(X, npe, N, cen);
    double h01 = dist3(X + 0, X + 3), h12 = dist3(X + 3, X + 6), h20 = dist3(X + 6, X + 0);
    double m = h01;
    if (h12 > m) m = h12;
    if (h20 > m) m = h20;
    *h = m;
}

/* ------------------------------------------------------------------------ */
/* Integration of one element against one collocation point                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *X;      /* element nodes, [npe][3] */
    int npe;
    const double *xi;     /* collocation point */
    int green;
    double k;
    cplx S[6], D[6];      /* int L_a G dS,  int L_a dG/dn1 dS */
    double D0[6];         /* int L_a dG0/dn1 dS (Laplace) */
} acc_t;

/* One quadrature point with reference-space weight wref.  Kernels of Eq. 1:
 * G = exp(jkR)/(4 pi R), dG/dn1 = grad_{x1} G . n1
 *   = exp(jkR) (1 - jkR) ((x - x1) . n1) / (4 pi R^3). */
static void acc_point(acc_t *A, double s, double t, double wref)
{
    gpoint g;
    elem_point(A->X, A->npe, s, t, &g);
    double r[3] = {A->xi[0] - g.x[0], A->xi[1] - g.x[1], A->xi[2] - g.x[2]};
    double R = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double rn = r[0] * g.n[0] + r[1] * g.n[1] + r[2] * g.n[2];
    double w = wref * g.J;
    double G0 = 1.0 / (4.0 * OR_PI * R);
    double dG0 = rn / (4.0 * OR_PI * R * R * R);
    cplx G = G0, dG = dG0;
    if (A->green == OR_HELMHOLTZ) {
        cplx e = cexp(I * A->k * R);
        G = e * G0;
        dG = e * (1.0 - I * A->k * R) * dG0;
    }
    for (int a = 0; a < A->npe; a++) {
        A->S[a] += w * g.N[a] * G;
        A->D[a] += w * g.N[a] * dG;
        A->D0[a] += w * g.N[a] * dG0;
    }
}

static void integrate_regular(acc_t *A)
{
    double s[7], t[7], w[7];
    rule7(s, t, w);
    for (int q = 0; q < 7; q++) acc_point(A, s[q], t[q], w[q]);
}

/* Duffy rule for the triangle (P, Q1, Q2) in reference space, collapsed at P:
 * xi(u,v) = P + u (Q1 - P) + u v (Q2 - Q1), Jacobian u |det(Q1-P, Q2-P)|. */
static void integrate_duffy(acc_t *A, const double P[2], const double Q1[2], const double Q2[2],
                            const double *glx, const double *glw, int nd)
{
    double det = (Q1[0] - P[0]) * (Q2[1] - P[1]) - (Q1[1] - P[1]) * (Q2[0] - P[0]);
    det = fabs(det);
    for (int iu = 0; iu < nd; iu++) {
        double u = 0.5 * (1.0 + glx[iu]), wu = 0.5 * glw[iu];
        for (int iv = 0; iv < nd; iv++) {
            double v = 0.5 * (1.0 + glx[iv]), wv = 0.5 * glw[iv];
            double s = P[0] + u * (Q1[0] - P[0]) + u * v * (Q2[0] - Q1[0]);
            double t = P[1] + u * (Q1[1] - P[1]) + u * v * (Q2[1] - Q1[1]);
            acc_point(A, s, t, wu * wv * u * det);
        }
    }
}

static const double REF_NODE[6][2] = {
    {0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}, {0.5, 0.0}, {0.5, 0.5}, {0.0, 0.5}};

/* Self element: split at the singular node and collapse each piece there. */
static void integrate_singular(acc_t *A, int a_sing, const double *glx, const double *glw, int nd)
{
    const double *c0 = REF_NODE[0], *c1 = REF_NODE[1], *c2 = REF_NODE[2];
    switch (a_sing) {
    case 0: integrate_duffy(A, c0, c1, c2, glx, glw, nd); break;
    case 1: integrate_duffy(A, c1, c2, c0, glx, glw, nd); break;
    case 2: integrate_duffy(A, c2, c0, c1, glx, glw, nd); break;
    case 3: /* mid-side of 0-1, opposite corner 2 */
        integrate_duffy(A, REF_NODE[3], c1, c2, glx, glw, nd);
        integrate_duffy(A, REF_NODE[3], c2, c0, glx, glw, nd);
        break;
    case 4: /* mid-side of 1-2, opposite corner 0 */
        integrate_duffy(A, REF_NODE[4], c2, c0, glx, glw, nd);
        integrate_duffy(A, REF_NODE[4], c0, c1, glx, glw, nd);
        break;
    case 5: /* mid-side of 2-0, opposite corner 1 */
        integrate_duffy(A, REF_NODE[5], c0, c1, glx, glw, nd);
        integrate_duffy(A, REF_NODE[5], c1, c2, glx, glw, nd);
        break;
    }
}

/* Near-singular rule: split the parametric triangle (a, b, c) 4-way until the
 * image of its centroid is at least tau times its longest corner chord from the
 * collocation point, or depth == maxdepth; then the 7-point rule on the piece. */
static void integrate_subdivided(acc_t *A, const double a[2], const double b[2], const double c[2],
                                 int depth, double tau, int maxdepth)
{
    double N[6], Ns[6], Nt[6], xa[3], xb[3], xc[3], xm[3];
    double m[2] = {(a[0] + b[0] + c[0]) / 3.0, (a[1] + b[1] + c[1]) / 3.0};
    shape(A->npe, a[0], a[1], N, Ns, Nt); map_point(A->X, A->npe, N, xa);
    shape(A->npe, b[0], b[1], N, Ns, Nt); map_point(A->X, A->npe, N, xb);
    shape(A->npe, c[0], c[1], N, Ns, Nt); map_point(A->X, A->npe, N, xc);
    shape(A->npe, m[0], m[1], N, Ns, Nt); map_point(A->X, A->npe, N, xm);
    double h = dist3(xa, xb), h2 = dist3(xb, xc), h3 = dist3(xc, xa);
    if (h2 > h) h = h2;
    if (h3 > h) h = h3;
    if (depth >= maxdepth || !(dist3(A->xi, xm) < tau * h)) {
        double s[7], t[7], w[7];
        rule7(s, t, w);
        double det = fabs((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]));
        for (int q = 0; q < 7; q++) {
            double ps = a[0] + s[q] * (b[0] - a[0]) + t[q] * (c[0] - a[0]);
            double pt = a[1] + s[q] * (b[1] - a[1]) + t[q] * (c[1] - a[1]);
            acc_point(A, ps, pt, w[q] * det);
        }
        return;
    }
    double ab[2] = {0.5 * (a[0] + b[0]), 0.5 * (a[1] + b[1])};
    double bc[2] = {0.5 * (b[0] + c[0]), 0.5 * (b[1] + c[1])};
    double ca[2] = {0.5 * (c[0] + a[0]), 0.5 * (c[1] + a[1])};
    integrate_subdivided(A, a, ab, ca, depth + 1, tau, maxdepth);
    integrate_subdivided(A, ab, b, bc, depth + 1, tau, maxdepth);
    integrate_subdivided(A, ca, bc, c, depth + 1, tau, maxdepth);
    integrate_subdivided(A, ab, bc, ca, depth + 1, tau, maxdepth);
}

/* Pair classification (tree independent):
 *   0 regular, 1 singular (node i belongs to e), 2 near-singular
 *   (|x_i - X_e(1/3,1/3)| < tau h_e). *a_sing receives the local node. */
static int classify(const double *xi, int64_t i, const int32_t *el, const double *X, int npe,
                    double tau, int *a_sing)
{
    for (int a = 0; a < npe; a++)
        if (el[a] == i) { *a_sing = a; return 1; }
    double cen[3], h;
    elem_centroid_h(X, npe, cen, &h);
    if (dist3(xi, cen) < tau * h) return 2;
    return 0;
}

typedef struct {
    const double *nodes; int64_t nn;
    const int32_t *elems; int64_t ne; int npe;
    int green; double k;
    const double *glx, *glw; int nd;
    double tau; int maxdepth;
} problem_t;

static void gather_elem(const problem_t *P, int64_t e, double X[18])
{
    for (int a = 0; a < P->npe; a++)
        for (int c = 0; c < 3; c++) X[3 * a + c] = P->nodes[3 * (int64_t)P->elems[e * P->npe + a] + c];
}

/* Integrals of one (collocation node i, element e) pair with the rule its
 * class asks for.  Returns the class. */
static int integrate_pair(const problem_t *P, int64_t i, int64_t e, acc_t *A, int force_regular)
{
    double X[18];
    gather_elem(P, e, X);
    memset(A, 0, sizeof(*A));
    A->X = X; A->npe = P->npe; A->xi = P->nodes + 3 * i; A->green = P->green; A->k = P->k;
    int a_sing = -1;
    int cls = classify(A->xi, i, P->elems + e * P->npe, X, P->npe, P->tau, &a_sing);
    if (force_regular || cls == 0) integrate_regular(A);
    else if (cls == 1) integrate_singular(A, a_sing, P->glx, P->glw, P->nd);
    else {
        double c0[2] = {0.0, 0.0}, c1[2] = {1.0, 0.0}, c2[2] = {0.0, 1.0};
        integrate_subdivided(A, c0, c1, c2, 0, P->tau, P->maxdepth);
    }
    A->X = NULL; A->xi = NULL;
    return cls;
}

/* Dense rows of the discrete operators (Eq. 3):
 *   D[r][j]  = sum_e sum_{a: phi-index j}  int L_a dG/dn1 dS     (n_nodes cols)
 *   S[r][j]  = sum_e sum_{a: chi-index j}  int L_a G dS          (n_chi cols)
 *   D0sum[r] = sum_j D0_ij (Laplace kernel), so C_i = 1 + D0sum.
 * rows: collocation nodes to assemble (NULL -> all).  Arrays are complex,
 * interleaved (re, im). */
int or_assemble_rows(const double *nodes, int64_t nn, const int32_t *elems, int64_t ne, int npe,
                     const int32_t *chi_idx, int64_t nchi, int green, double k,
                     const double *glx, const double *glw, int nd, double tau, int maxdepth,
                     const int64_t *rows, int64_t nrows, cplx *D, cplx *S, double *D0sum)
{
    problem_t P = {nodes, nn, elems, ne, npe, green, k, glx, glw, nd, tau, maxdepth};
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; r++) {
        int64_t i = rows ? rows[r] : r;
        cplx *Dr = D ? D + r * nn : NULL;
        cplx *Sr = S ? S + r * nchi : NULL;
        double d0 = 0.0;
        if (Dr) memset(Dr, 0, sizeof(cplx) * nn);
        if (Sr) memset(Sr, 0, sizeof(cplx) * nchi);
        for (int64_t e = 0; e < ne; e++) {
            acc_t A;
            integrate_pair(&P, i, e, &A, 0);
            for (int a = 0; a < npe; a++) {
                if (Dr) Dr[elems[e * npe + a]] += A.D[a];
                if (Sr) Sr[chi_idx[e * npe + a]] += A.S[a];
                d0 += A.D0[a];
            }
        }
        if (D0sum) D0sum[r] = d0;
    }
    return 0;
}

/* Matrix-free rows of the operators: y[r] = (A x)_i = C_i x_i - (D x)_i for
 * op A (x indexed by node), y[r] = (B x)_i = -(S x)_i for op B (x indexed by
 * chi index).  Every pair is integrated on the fly, O(rows * elements). */
int or_apply_rows(const double *nodes, int64_t nn, const int32_t *elems, int64_t ne, int npe,
                  const int32_t *chi_idx, int green, double k,
                  const double *glx, const double *glw, int nd, double tau, int maxdepth,
                  int op, const cplx *x, const int64_t *rows, int64_t nrows, cplx *y)
{
    problem_t P = {nodes, nn, elems, ne, npe, green, k, glx, glw, nd, tau, maxdepth};
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; r++) {
        int64_t i = rows ? rows[r] : r;
        cplx acc = 0.0;
        double d0 = 0.0;
        for (int64_t e = 0; e < ne; e++) {
            acc_t A;
            integrate_pair(&P, i, e, &A, 0);
            for (int a = 0; a < npe; a++) {
                if (op == OR_OP_A) {
                    acc += A.D[a] * x[elems[e * npe + a]];
                    d0 += A.D0[a];
                } else {
                    acc += A.S[a] * x[chi_idx[e * npe + a]];
                }
            }
        }
        y[r] = (op == OR_OP_A) ? (1.0 + d0) * x[i] - acc : -acc;
    }
    return 0;
}

/* Field of known surface data off the surface: the representation of Eq. 1
 * with C(x) = 1 outside the body and C(x) = 0 inside (Section 2.2, the field
 * evaluated from phi and its normal derivative chi),
 *   u(x) = sum_e sum_a [ phi_a int L_a dG/dn1 dS  -  chi_a int L_a G dS ],
 * each element integrated with the 7-point rule, or with the parametric
 * subdivision where |x - centroid| < tau h_e (as for near-singular pairs).
 * x must not lie on the surface.  phi: [n_nodes], chi: [n_chi], complex. */
int or_field(const double *nodes, int64_t nn, const int32_t *elems, int64_t ne, int npe,
             const int32_t *chi_idx, int green, double k, double tau, int maxdepth,
             const cplx *phi, const cplx *chi, int64_t npts, const double *pts, cplx *u)
{
    problem_t P = {nodes, nn, elems, ne, npe, green, k, NULL, NULL, 0, tau, maxdepth};
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < npts; i++) {
        cplx acc = 0.0;
        for (int64_t e = 0; e < ne; e++) {
            double X[18];
            gather_elem(&P, e, X);
            acc_t A;
            memset(&A, 0, sizeof(A));
            A.X = X; A.npe = npe; A.xi = pts + 3 * i; A.green = green; A.k = k;
            int a_sing = -1;
            /* index -1 matches no element node: regular or near-singular only */
            if (classify(A.xi, -1, elems + e * npe, X, npe, tau, &a_sing) == 0) {
                integrate_regular(&A);
            } else {
                double c0[2] = {0.0, 0.0}, c1[2] = {1.0, 0.0}, c2[2] = {0.0, 1.0};
                integrate_subdivided(&A, c0, c1, c2, 0, tau, maxdepth);
            }
            for (int a = 0; a < npe; a++)
                acc += A.D[a] * phi[elems[e * npe + a]] - A.S[a] * chi[chi_idx[e * npe + a]];
        }
        u[i] = acc;
    }
    return 0;
}

/* The correction the fast method adds to its regular-rule sums: for every
 * special pair (class 1 or 2) and local node a, (special - regular) integral,
 * as COO triplets.  Returns the number of triplets written (npe per pair), or
 * the count needed when out arrays are NULL. */
int64_t or_correction(const double *nodes, int64_t nn, const int32_t *elems, int64_t ne, int npe,
                      const int32_t *chi_idx, int green, double k,
                      const double *glx, const double *glw, int nd, double tau, int maxdepth,
                      int64_t *row, int32_t *col_phi, int32_t *col_chi, cplx *valD, cplx *valS,
                      double *valD0)
{
    problem_t P = {nodes, nn, elems, ne, npe, green, k, glx, glw, nd, tau, maxdepth};
    int64_t cnt = 0;
    for (int64_t i = 0; i < nn; i++)
        for (int64_t e = 0; e < ne; e++) {
            double X[18], cen[3], h;
            gather_elem(&P, e, X);
            int a_sing, cls = classify(nodes + 3 * i, i, elems + e * npe, X, npe, tau, &a_sing);
            (void)cen; (void)h;
            if (cls == 0) continue;
            if (row) {
                acc_t As, Ar;
                integrate_pair(&P, i, e, &As, 0);
                integrate_pair(&P, i, e, &Ar, 1);
                for (int a = 0; a < npe; a++) {
                    row[cnt + a] = i;
                    col_phi[cnt + a] = elems[e * npe + a];
                    col_chi[cnt + a] = chi_idx[e * npe + a];
                    valD[cnt + a] = As.D[a] - Ar.D[a];
                    valS[cnt + a] = As.S[a] - Ar.S[a];
                    valD0[cnt + a] = As.D0[a] - Ar.D0[a];
                }
            }
            cnt += npe;
        }
    return cnt;
}

/* Regular-rule quadrature points of every element, in element order:
 * position, unit normal, weight*Jacobian, shape values [E*7]. */
void or_quad_points(const double *nodes, const int32_t *elems, int64_t ne, int npe,
                    double *qx, double *qn, double *qw, double *qL)
{
    double s[7], t[7], w[7];
    rule7(s, t, w);
    for (int64_t e = 0; e < ne; e++) {
        double X[18];
        for (int a = 0; a < npe; a++)
            for (int c = 0; c < 3; c++) X[3 * a + c] = nodes[3 * (int64_t)elems[e * npe + a] + c];
        for (int q = 0; q < 7; q++) {
            gpoint g;
            elem_point(X, npe, s[q], t[q], &g);
            int64_t o = e * 7 + q;
            for (int c = 0; c < 3; c++) { qx[3 * o + c] = g.x[c]; qn[3 * o + c] = g.n[c]; }
            qw[o] = w[q] * g.J;
            for (int a = 0; a < npe; a++) qL[o * npe + a] = g.N[a];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sharp-edge multi-indexing of the Neumann data (Section 2.3)               */
/* ------------------------------------------------------------------------ */

/* Visit elements in order; at each element node compute the element normal
 * there.  A node's first normal opens a cluster; a later normal joins the first
 * cluster whose opening normal lies within the angle tolerance, otherwise it
 * opens a new cluster.  Each cluster is one chi index.  Returns n_chi. */
int64_t or_chi_index(const double *nodes, int64_t nn, const int32_t *elems, int64_t ne, int npe,
                     double angle_deg, int32_t *chi_idx)
{
    double cos_tol = cos(angle_deg * OR_PI / 180.0);
    /* per node: list of (cluster normal, chi index) */
    int64_t *head = malloc(sizeof(int64_t) * nn);
    int64_t cap = ne * npe, used = 0;
    double *cn = malloc(sizeof(double) * 3 * cap);
    int64_t *cid = malloc(sizeof(int64_t) * cap), *next = malloc(sizeof(int64_t) * cap);
    for (int64_t i = 0; i < nn; i++) head[i] = -1;
    int64_t nchi = 0;
    for (int64_t e = 0; e < ne; e++) {
        double X[18];
        for (int a = 0; a < npe; a++)
            for (int c = 0; c < 3; c++) X[3 * a + c] = nodes[3 * (int64_t)elems[e * npe + a] + c];
        for (int a = 0; a < npe; a++) {
            gpoint g;
            elem_point(X, npe, REF_NODE[a][0], REF_NODE[a][1], &g);
            int64_t node = elems[e * npe + a], found = -1, last = -1;
            for (int64_t c = head[node]; c >= 0; c = next[c]) {
                double d = g.n[0] * cn[3 * c] + g.n[1] * cn[3 * c + 1] + g.n[2] * cn[3 * c + 2];
                if (d >= cos_tol) { found = cid[c]; break; }
                last = c;
            }
            if (found < 0) {
                int64_t c = used++;
                cn[3 * c] = g.n[0]; cn[3 * c + 1] = g.n[1]; cn[3 * c + 2] = g.n[2];
                cid[c] = nchi++;
                next[c] = -1;
                if (last < 0) head[node] = c; else next[last] = c;
                found = cid[c];
            }
            chi_idx[e * npe + a] = (int32_t)found;
        }
    }
    free(head); free(cn); free(cid); free(next);
    return nchi;
}

/* ------------------------------------------------------------------------ */
/* Octree over the vertices (Section 3.1) with element-extent radii          */
/* (Section 3.4) and near-field / interaction lists (Section 3.6)            */
/* ------------------------------------------------------------------------ */

#define QBITS 21

typedef struct {
    int level;
    int64_t ix, iy, iz;
    int parent, nchild, child[8], leaf;
    int64_t *nodes; int64_t nnodes;
    int64_t *elems; int64_t nelems;     /* owned elements (leaves only) */
    double c[3], r;
    int64_t *nearl, nnear, capn;
    int64_t *inter, ninter, capi;
} obox_t;

typedef struct {
    obox_t *box; int64_t nbox, capbox;
    double lo[3], side;
    int B, max_level, leaf_descend;
    double eta;
    int64_t *leaf_of_node;              /* [n_nodes] */
    int64_t *owner;                     /* [n_elems] leaf owning each element */
    int64_t nn, ne; int npe;
} otree_t;

static int64_t new_box(otree_t *T)
{
    if (T->nbox == T->capbox) {
        T->capbox = T->capbox ? 2 * T->capbox : 64;
        T->box = realloc(T->box, sizeof(obox_t) * T->capbox);
    }
    obox_t *b = &T->box[T->nbox];
    memset(b, 0, sizeof(*b));
    b->parent = -1;
    return T->nbox++;
}

static void push(int64_t **arr, int64_t *n, int64_t *cap, int64_t v)
{
    if (*n == *cap) { *cap = *cap ? 2 * *cap : 8; *arr = realloc(*arr, sizeof(int64_t) * *cap); }
    (*arr)[(*n)++] = v;
}

/* Recursive division: a box holding B or more vertices (and below the level
 * cap) is split into its non-empty octants; otherwise it is a leaf. */
static void split_box(otree_t *T, int64_t bi, const int64_t *q)
{
    obox_t *b = &T->box[bi];
    if (b->nnodes < T->B || b->level >= T->max_level) { b->leaf = 1; return; }
    int shift = QBITS - 1 - b->level;
    int64_t cnt[8] = {0};
    for (int64_t t = 0; t < b->nnodes; t++) {
        int64_t n = b->nodes[t];
        int oct = (int)(((q[3 * n] >> shift) & 1) | (((q[3 * n + 1] >> shift) & 1) << 1) |
                        (((q[3 * n + 2] >> shift) & 1) << 2));
        cnt[oct]++;
    }
    int64_t kids[8];
    for (int o = 0; o < 8; o++) {
        kids[o] = -1;
        if (!cnt[o]) continue;
        int64_t ci = new_box(T);
        b = &T->box[bi];
        obox_t *c = &T->box[ci];
        c->level = b->level + 1;
        c->ix = 2 * b->ix + (o & 1);
        c->iy = 2 * b->iy + ((o >> 1) & 1);
        c->iz = 2 * b->iz + ((o >> 2) & 1);
        c->parent = (int)bi;
        c->nodes = malloc(sizeof(int64_t) * cnt[o]);
        b->child[b->nchild++] = (int)ci;
        kids[o] = ci;
    }
    b = &T->box[bi];
    for (int64_t t = 0; t < b->nnodes; t++) {
        int64_t n = b->nodes[t];
        int oct = (int)(((q[3 * n] >> shift) & 1) | (((q[3 * n + 1] >> shift) & 1) << 1) |
                        (((q[3 * n + 2] >> shift) & 1) << 2));
        obox_t *c = &T->box[kids[oct]];
        c->nodes[c->nnodes++] = n;
    }
    int nch = b->nchild;
    int chl[8];
    memcpy(chl, b->child, sizeof(chl));
    for (int t = 0; t < nch; t++) split_box(T, chl[t], q);
}

static int separated(const otree_t *T, const obox_t *a, const obox_t *b)
{
    double d = dist3(a->c, b->c);
    return d > T->eta * (a->r + b->r);
}

/* Lists of box B from the near list of its parent (Section 3.6): a leaf entry
 * is tested itself, a non-leaf entry through its children.  With
 * leaf_descend, a leaf B keeps opening non-leaf near entries until each is
 * separated or a leaf. */
static void classify_into(otree_t *T, int64_t bi, int64_t ni)
{
    obox_t *B = &T->box[bi], *N = &T->box[ni];
    if (separated(T, B, N)) { push(&B->inter, &B->ninter, &B->capi, ni); return; }
    if (B->leaf && T->leaf_descend && !N->leaf) {
        for (int t = 0; t < N->nchild; t++) classify_into(T, bi, N->child[t]);
        return;
    }
    push(&B->nearl, &B->nnear, &B->capn, ni);
}

static void build_lists(otree_t *T, int64_t bi)
{
    obox_t *B = &T->box[bi];
    if (B->parent < 0) {
        push(&B->nearl, &B->nnear, &B->capn, bi);
    } else {
        obox_t *P = &T->box[B->parent];
        for (int64_t t = 0; t < P->nnear; t++) {
            int64_t ni = P->nearl[t];
            obox_t *N = &T->box[ni];
            if (N->leaf) classify_into(T, bi, ni);
            else
                for (int c = 0; c < N->nchild; c++) classify_into(T, bi, N->child[c]);
        }
    }
    B = &T->box[bi];
    int nch = B->nchild, chl[8];
    memcpy(chl, B->child, sizeof(chl));
    for (int c = 0; c < nch; c++) build_lists(T, chl[c]);
}

static double radius_leaf(const otree_t *T, const obox_t *b, const double *nodes,
                          const int32_t *elems, const double *qx)
{
    double r = 0.0;
    for (int64_t t = 0; t < b->nnodes; t++) {
        double d = dist3(b->c, nodes + 3 * b->nodes[t]);
        if (d > r) r = d;
    }
    for (int64_t t = 0; t < b->nelems; t++) {
        int64_t e = b->elems[t];
        for (int a = 0; a < T->npe; a++) {
            double d = dist3(b->c, nodes + 3 * (int64_t)elems[e * T->npe + a]);
            if (d > r) r = d;
        }
        for (int q = 0; q < 7; q++) {
            double d = dist3(b->c, qx + 3 * (e * 7 + q));
            if (d > r) r = d;
        }
    }
    return r;
}

/* radius of every box: leaves from their points, parents by Eq. 12,
 * r_P = max_child r_C + d_C / 2 with d_C the child diagonal. */
static void radius_up(otree_t *T, int64_t bi, const double *nodes, const int32_t *elems, const double *qx)
{
    obox_t *b = &T->box[bi];
    if (b->leaf) { b->r = radius_leaf(T, b, nodes, elems, qx); return; }
    double rmax = 0.0;
    for (int c = 0; c < b->nchild; c++) {
        radius_up(T, b->child[c], nodes, elems, qx);
        b = &T->box[bi];
        if (T->box[b->child[c]].r > rmax) rmax = T->box[b->child[c]].r;
    }
    double hc = ldexp(T->side, -(b->level + 1));
    b->r = rmax + sqrt(3.0) * hc * 0.5;
}

void *or_tree_build(const double *nodes, int64_t nn, const int32_t *elems, int64_t ne, int npe,
                    int B, int max_level, double eta, int leaf_descend)
{
    otree_t *T = calloc(1, sizeof(otree_t));
    T->B = B; T->max_level = max_level; T->eta = eta; T->leaf_descend = leaf_descend;
    T->nn = nn; T->ne = ne; T->npe = npe;
    /* root cube: centred on the bounding box, side = largest extent (1 + 2^-20) */
    double lo[3], hi[3];
    for (int c = 0; c < 3; c++) { lo[c] = nodes[c]; hi[c] = nodes[c]; }
    for (int64_t i = 1; i < nn; i++)
        for (int c = 0; c < 3; c++) {
            if (nodes[3 * i + c] < lo[c]) lo[c] = nodes[3 * i + c];
            if (nodes[3 * i + c] > hi[c]) hi[c] = nodes[3 * i + c];
        }
    double ext = hi[0] - lo[0];
    if (hi[1] - lo[1] > ext) ext = hi[1] - lo[1];
    if (hi[2] - lo[2] > ext) ext = hi[2] - lo[2];
    T->side = ext * (1.0 + ldexp(1.0, -20));
    for (int c = 0; c < 3; c++) T->lo[c] = (lo[c] + hi[c]) * 0.5 - T->side * 0.5;
    double scale = ldexp(1.0, QBITS) / T->side;
    int64_t qmax = ((int64_t)1 << QBITS) - 1;
    int64_t *q = malloc(sizeof(int64_t) * 3 * nn);
    for (int64_t i = 0; i < nn; i++)
        for (int c = 0; c < 3; c++) {
            double v = floor((nodes[3 * i + c] - T->lo[c]) * scale);
            int64_t iv = (int64_t)v;
            q[3 * i + c] = iv < 0 ? 0 : (iv > qmax ? qmax : iv);
        }
    int64_t root = new_box(T);
    T->box[root].nodes = malloc(sizeof(int64_t) * nn);
    for (int64_t i = 0; i < nn; i++) T->box[root].nodes[i] = i;
    T->box[root].nnodes = nn;
    split_box(T, root, q);
    free(q);
    /* box centres: lo + (i + 0.5) h_level */
    for (int64_t b = 0; b < T->nbox; b++) {
        obox_t *x = &T->box[b];
        double h = ldexp(T->side, -x->level);
        x->c[0] = T->lo[0] + ((double)x->ix + 0.5) * h;
        x->c[1] = T->lo[1] + ((double)x->iy + 0.5) * h;
        x->c[2] = T->lo[2] + ((double)x->iz + 0.5) * h;
    }
    /* vertex -> leaf, element -> leaf of its first corner (unique owner) */
    T->leaf_of_node = malloc(sizeof(int64_t) * nn);
    for (int64_t b = 0; b < T->nbox; b++)
        if (T->box[b].leaf)
            for (int64_t t = 0; t < T->box[b].nnodes; t++) T->leaf_of_node[T->box[b].nodes[t]] = b;
    T->owner = malloc(sizeof(int64_t) * ne);
    for (int64_t e = 0; e < ne; e++) {
        int64_t b = T->leaf_of_node[elems[e * npe]];
        T->owner[e] = b;
        obox_t *x = &T->box[b];
        x->elems = realloc(x->elems, sizeof(int64_t) * (x->nelems + 1));
        x->elems[x->nelems++] = e;
    }
    /* convergence radii need the regular quadrature points */
    double *qx = malloc(sizeof(double) * 3 * 7 * ne), *qn = malloc(sizeof(double) * 3 * 7 * ne);
    double *qw = malloc(sizeof(double) * 7 * ne), *qL = malloc(sizeof(double) * 7 * ne * npe);
    or_quad_points(nodes, elems, ne, npe, qx, qn, qw, qL);
    radius_up(T, root, nodes, elems, qx);
    free(qx); free(qn); free(qw); free(qL);
    build_lists(T, root);
    return T;
}

void or_tree_free(void *h)
{
    otree_t *T = h;
    for (int64_t b = 0; b < T->nbox; b++) {
        free(T->box[b].nodes); free(T->box[b].elems); free(T->box[b].nearl); free(T->box[b].inter);
    }
    free(T->box); free(T->leaf_of_node); free(T->owner); free(T);
}

/* counts: [n_boxes, total near entries, total interaction entries, side] */
void or_tree_counts(void *h, int64_t *cnt, double *geom)
{
    otree_t *T = h;
    int64_t nn = 0, ni = 0;
    for (int64_t b = 0; b < T->nbox; b++) { nn += T->box[b].nnear; ni += T->box[b].ninter; }
    cnt[0] = T->nbox; cnt[1] = nn; cnt[2] = ni;
    geom[0] = T->lo[0]; geom[1] = T->lo[1]; geom[2] = T->lo[2]; geom[3] = T->side;
}

/* Flat export: per box level, ix, iy, iz, parent, leaf, centre, radius;
 * CSR near and interaction lists (box indices); vertex -> leaf;
 * element -> owning leaf. */
void or_tree_export(void *h, int32_t *level, int64_t *ijk, int32_t *parent, int32_t *leaf,
                    double *centre, double *radius, int64_t *near_ptr, int64_t *near_idx,
                    int64_t *inter_ptr, int64_t *inter_idx, int64_t *leaf_of_node, int64_t *owner)
{
    otree_t *T = h;
    near_ptr[0] = 0; inter_ptr[0] = 0;
    for (int64_t b = 0; b < T->nbox; b++) {
        obox_t *x = &T->box[b];
        level[b] = x->level;
        ijk[3 * b] = x->ix; ijk[3 * b + 1] = x->iy; ijk[3 * b + 2] = x->iz;
        parent[b] = x->parent; leaf[b] = x->leaf;
        for (int c = 0; c < 3; c++) centre[3 * b + c] = x->c[c];
        radius[b] = x->r;
        near_ptr[b + 1] = near_ptr[b] + x->nnear;
        inter_ptr[b + 1] = inter_ptr[b] + x->ninter;
        memcpy(near_idx + near_ptr[b], x->nearl, sizeof(int64_t) * x->nnear);
        memcpy(inter_idx + inter_ptr[b], x->inter, sizeof(int64_t) * x->ninter);
    }
    memcpy(leaf_of_node, T->leaf_of_node, sizeof(int64_t) * T->nn);
    memcpy(owner, T->owner, sizeof(int64_t) * T->ne);
}

/* ------------------------------------------------------------------------ */
/* Taylor expansions (Section 3.2) and Green's-function derivatives          */
/* (Section 3.3)                                                              */
/* ------------------------------------------------------------------------ */

/* Multi-index alpha = (m, n, k), |alpha| <= p, enumerated by degree h, then m
 * descending, then n descending.  idx[(m*(p+1) + n)*(p+1) + k]. */
typedef struct {
    int p, np;
    int *m, *n, *k, *idx;
    double *fact;  /* fact[i] = i! */
    double *binom; /* binom[a*(p+1)+b] */
} mindex_t;

static void mindex_init(mindex_t *M, int p)
{
    M->p = p;
    M->np = (p + 1) * (p + 2) * (p + 3) / 6;
    M->m = malloc(sizeof(int) * M->np); M->n = malloc(sizeof(int) * M->np);
    M->k = malloc(sizeof(int) * M->np);
    M->idx = malloc(sizeof(int) * (p + 1) * (p + 1) * (p + 1));
    for (int t = 0; t < (p + 1) * (p + 1) * (p + 1); t++) M->idx[t] = -1;
    int c = 0;
    for (int h = 0; h <= p; h++)
        for (int m = h; m >= 0; m--)
            for (int n = h - m; n >= 0; n--) {
                int k = h - m - n;
                M->m[c] = m; M->n[c] = n; M->k[c] = k;
                M->idx[(m * (p + 1) + n) * (p + 1) + k] = c++;
            }
    M->fact = malloc(sizeof(double) * (2 * p + 2));
    M->fact[0] = 1.0;
    for (int i = 1; i <= 2 * p + 1; i++) M->fact[i] = M->fact[i - 1] * i;
    M->binom = malloc(sizeof(double) * (p + 1) * (p + 1));
    for (int a = 0; a <= p; a++)
        for (int b = 0; b <= p; b++)
            M->binom[a * (p + 1) + b] = (b > a) ? 0.0 : M->fact[a] / (M->fact[b] * M->fact[a - b]);
}

static void mindex_free(mindex_t *M)
{
    free(M->m); free(M->n); free(M->k); free(M->idx); free(M->fact); free(M->binom);
}

static int MI(const mindex_t *M, int m, int n, int k)
{
    if (m < 0 || n < 0 || k < 0 || m + n + k > M->p) return -1;
    return M->idx[(m * (M->p + 1) + n) * (M->p + 1) + k];
}

void or_mindex(int p, int32_t *mnk)
{
    mindex_t M;
    mindex_init(&M, p);
    for (int c = 0; c < M.np; c++) { mnk[3 * c] = M.m[c]; mnk[3 * c + 1] = M.n[c]; mnk[3 * c + 2] = M.k[c]; }
    mindex_free(&M);
}

/* Tausch: G^(h) = (R^-1 d/dR)^h G.  Laplace: G^(h+1) = -(2h+1) G^(h) / R^2.
 * Helmholtz: G^(h+1) = -((2h+1) G^(h) + k^2 G^(h-1)) / R^2 with
 * G^(-1) = -j exp(jkR) / (4 pi k).  Then, for h = H-1 .. 0, the Cartesian
 * derivatives of G^(h) of total order <= H - h from those of G^(h+1):
 * d^{gamma + e_c} G^(h) = gamma_c d^{gamma - e_c} G^(h+1) + r_c d^gamma G^(h+1).
 * Output D[alpha] = d^alpha G(r), |alpha| <= H, in mindex order. */
static void green_derivs(const mindex_t *M, int green, double k, const double r[3], cplx *Dout)
{
    int H = M->p, P1 = H + 1;
    double R2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], R = sqrt(R2);
    cplx *Gh = malloc(sizeof(cplx) * (H + 2));
    Gh[0] = 1.0 / (4.0 * OR_PI * R);
    cplx Gm1 = 0.0;
    if (green == OR_HELMHOLTZ) {
        cplx e = cexp(I * k * R);
        Gh[0] = e / (4.0 * OR_PI * R);
        Gm1 = -I * e / (4.0 * OR_PI * k);
    }
    for (int h = 0; h < H; h++) {
        cplx prev = (h == 0) ? Gm1 : Gh[h - 1];
        Gh[h + 1] = -((2.0 * h + 1.0) * Gh[h] + (green == OR_HELMHOLTZ ? k * k * prev : 0.0)) / R2;
    }
    /* tables over (m, n, k) for two consecutive h */
    size_t sz = (size_t)P1 * P1 * P1;
    cplx *up = calloc(sz, sizeof(cplx)), *cur = calloc(sz, sizeof(cplx));
#define T3(A, m, n, kk) A[((m) * P1 + (n)) * P1 + (kk)]
    T3(up, 0, 0, 0) = Gh[H];
    for (int h = H - 1; h >= 0; h--) {
        int top = H - h;
        for (int deg = 0; deg <= top; deg++)
            for (int m = 0; m <= deg; m++)
                for (int n = 0; n <= deg - m; n++) {
                    int kk = deg - m - n;
                    cplx v;
                    if (deg == 0) v = Gh[h];
                    else if (m > 0) v = (m > 1 ? (m - 1) * T3(up, m - 2, n, kk) : 0.0) + r[0] * T3(up, m - 1, n, kk);
                    else if (n > 0) v = (n > 1 ? (n - 1) * T3(up, m, n - 2, kk) : 0.0) + r[1] * T3(up, m, n - 1, kk);
                    else v = (kk > 1 ? (kk - 1) * T3(up, m, n, kk - 2) : 0.0) + r[2] * T3(up, m, n, kk - 1);
                    T3(cur, m, n, kk) = v;
                }
        cplx *sw = up; up = cur; cur = sw;
    }
    for (int c = 0; c < M->np; c++) Dout[c] = T3(up, M->m[c], M->n[c], M->k[c]);
#undef T3
    free(up); free(cur); free(Gh);
}

void or_green_derivs(int p, int green, double k, const double *r, cplx *D)
{
    mindex_t M;
    mindex_init(&M, p);
    green_derivs(&M, green, k, r, D);
    mindex_free(&M);
}

static double ipow(double x, int e)
{
    double v = 1.0;
    for (int i = 0; i < e; i++) v *= x;
    return v;
}

/* Moments about c of point sources (Eq. 6): I_a += sigma (x - c)^a and of
 * dipoles: I_a += mu n . grad_x (x - c)^a. */
static void p2m_point(const mindex_t *M, const double *c, const double *x, const double *nrm,
                      cplx sigma, cplx mu, cplx *Mo)
{
    double d[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    for (int a = 0; a < M->np; a++) {
        int m = M->m[a], n = M->n[a], k = M->k[a];
        cplx v = sigma * ipow(d[0], m) * ipow(d[1], n) * ipow(d[2], k);
        if (m > 0) v += mu * nrm[0] * m * ipow(d[0], m - 1) * ipow(d[1], n) * ipow(d[2], k);
        if (n > 0) v += mu * nrm[1] * n * ipow(d[0], m) * ipow(d[1], n - 1) * ipow(d[2], k);
        if (k > 0) v += mu * nrm[2] * k * ipow(d[0], m) * ipow(d[1], n) * ipow(d[2], k - 1);
        Mo[a] += v;
    }
}

/* Coefficient shift (Eq. 8): moments about child centre c to parent c'. */
static void m2m(const mindex_t *M, const double *c, const double *cp, const cplx *Mo, cplx *Ip)
{
    double d[3] = {c[0] - cp[0], c[1] - cp[1], c[2] - cp[2]};
    int P1 = M->p + 1;
    for (int a = 0; a < M->np; a++) {
        int m = M->m[a], n = M->n[a], k = M->k[a];
        cplx s = 0.0;
        for (int q = 0; q <= m; q++)
            for (int r = 0; r <= n; r++)
                for (int t = 0; t <= k; t++)
                    s += M->binom[m * P1 + q] * M->binom[n * P1 + r] * M->binom[k * P1 + t] *
                         ipow(d[0], q) * ipow(d[1], r) * ipow(d[2], t) * Mo[MI(M, m - q, n - r, k - t)];
        Ip[a] += s;
    }
}

/* Local expansion about c_t of moments about c_s (Eq. 7):
 * F_b = sum_a (-1)^|a| d^{a+b} G(c_t - c_s) / (a! b!) I_a, |a| + |b| <= p. */
static void m2l(const mindex_t *M, int green, double k, const double *ct, const double *cs,
                const cplx *Mo, cplx *F)
{
    double r[3] = {ct[0] - cs[0], ct[1] - cs[1], ct[2] - cs[2]};
    cplx *D = malloc(sizeof(cplx) * M->np);
    green_derivs(M, green, k, r, D);
    for (int b = 0; b < M->np; b++) {
        int bm = M->m[b], bn = M->n[b], bk = M->k[b];
        double bf = M->fact[bm] * M->fact[bn] * M->fact[bk];
        cplx s = 0.0;
        for (int a = 0; a < M->np; a++) {
            int am = M->m[a], an = M->n[a], ak = M->k[a];
            int g = MI(M, am + bm, an + bn, ak + bk);
            if (g < 0) continue;
            double af = M->fact[am] * M->fact[an] * M->fact[ak];
            double sgn = ((am + an + ak) & 1) ? -1.0 : 1.0;
            s += sgn * D[g] / (af * bf) * Mo[a];
        }
        F[b] += s;
    }
    free(D);
}

/* Expansion shift (Eq. 9 with its binomial coefficients): local about parent
 * centre c to child centre c': F'_b = sum_{a>=b} C(a,b) (c' - c)^{a-b} F_a. */
static void l2l(const mindex_t *M, const double *c, const double *cp, const cplx *F, cplx *Fp)
{
    double d[3] = {cp[0] - c[0], cp[1] - c[1], cp[2] - c[2]};
    int P1 = M->p + 1;
    for (int b = 0; b < M->np; b++) {
        int bm = M->m[b], bn = M->n[b], bk = M->k[b];
        cplx s = 0.0;
        for (int a = 0; a < M->np; a++) {
            int am = M->m[a], an = M->n[a], ak = M->k[a];
            if (am < bm || an < bn || ak < bk) continue;
            s += M->binom[am * P1 + bm] * M->binom[an * P1 + bn] * M->binom[ak * P1 + bk] *
                 ipow(d[0], am - bm) * ipow(d[1], an - bn) * ipow(d[2], ak - bk) * F[a];
        }
        Fp[b] += s;
    }
}

static cplx l2p(const mindex_t *M, const double *c, const double *x, const cplx *F)
{
    double d[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    cplx s = 0.0;
    for (int b = 0; b < M->np; b++) s += F[b] * ipow(d[0], M->m[b]) * ipow(d[1], M->n[b]) * ipow(d[2], M->k[b]);
    return s;
}

/* exported single operators for the expansion pins */
void or_p2m_points(int p, const double *c, int64_t npts, const double *x, const double *nrm,
                   const cplx *sigma, const cplx *mu, cplx *Mo)
{
    mindex_t M;
    mindex_init(&M, p);
    memset(Mo, 0, sizeof(cplx) * M.np);
    for (int64_t t = 0; t < npts; t++) p2m_point(&M, c, x + 3 * t, nrm + 3 * t, sigma[t], mu[t], Mo);
    mindex_free(&M);
}
void or_m2m(int p, const double *c, const double *cp, const cplx *Mo, cplx *Ip)
{
    mindex_t M; mindex_init(&M, p); memset(Ip, 0, sizeof(cplx) * M.np); m2m(&M, c, cp, Mo, Ip); mindex_free(&M);
}
void or_m2l(int p, int green, double k, const double *ct, const double *cs, const cplx *Mo, cplx *F)
{
    mindex_t M; mindex_init(&M, p); memset(F, 0, sizeof(cplx) * M.np); m2l(&M, green, k, ct, cs, Mo, F); mindex_free(&M);
}
void or_l2l(int p, const double *c, const double *cp, const cplx *F, cplx *Fp)
{
    mindex_t M; mindex_init(&M, p); memset(Fp, 0, sizeof(cplx) * M.np); l2l(&M, c, cp, F, Fp); mindex_free(&M);
}
void or_l2p(int p, const double *c, int64_t npts, const double *x, const cplx *F, cplx *y)
{
    mindex_t M; mindex_init(&M, p);
    for (int64_t t = 0; t < npts; t++) y[t] = l2p(&M, c, x + 3 * t, F);
    mindex_free(&M);
}

/* Kernel of one regular point source at xq on target xi (Eq. 1 integrands). */
static cplx point_kernel(int green, double k, int op, const double *xi, const double *xq, const double *nq)
{
    double r[3] = {xi[0] - xq[0], xi[1] - xq[1], xi[2] - xq[2]};
    double R = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    cplx e = (green == OR_HELMHOLTZ) ? cexp(I * k * R) : 1.0;
    if (op == OR_OP_B) return e / (4.0 * OR_PI * R);
    double rn = r[0] * nq[0] + r[1] * nq[1] + r[2] * nq[2];
    return e * (1.0 - I * k * R) * rn / (4.0 * OR_PI * R * R * R);
}

static void subtree_elems(const otree_t *T, int64_t b, int64_t **out, int64_t *n, int64_t *cap)
{
    const obox_t *x = &T->box[b];
    if (x->leaf) {
        for (int64_t t = 0; t < x->nelems; t++) push(out, n, cap, x->elems[t]);
        return;
    }
    for (int c = 0; c < x->nchild; c++) subtree_elems(T, x->child[c], out, n, cap);
}

/* The fast matrix multiplication (Section 3.6, four steps) of the regular
 * part of the operator -- every element integrated with the 7-point rule --
 * followed by the exact correction of the special pairs.  Result:
 *   op A:  y = C x - D x,  op B: y = -S x.
 * The diagonal C_i = 1 + sum_j D0_ij is taken from d0sum (caller supplies).
 * moments / locals (optional, [n_boxes][n_p]) receive the expansions. */
int or_fmm_apply(void *h, const double *nodes, const int32_t *elems, const int32_t *chi_idx,
                 int green, double k, int p, int op, const cplx *x, const double *d0sum,
                 const int64_t *corr_row, const int32_t *corr_col, const cplx *corr_val, int64_t ncorr,
                 cplx *y, cplx *moments, cplx *locals)
{
    otree_t *T = h;
    int npe = T->npe;
    mindex_t M;
    mindex_init(&M, p);
    int64_t nb = T->nbox, ne = T->ne, nn = T->nn, np = M.np;
    cplx *Imom = calloc(nb * np, sizeof(cplx)), *Floc = calloc(nb * np, sizeof(cplx));
    double *qx = malloc(sizeof(double) * 3 * 7 * ne), *qn = malloc(sizeof(double) * 3 * 7 * ne);
    double *qw = malloc(sizeof(double) * 7 * ne), *qL = malloc(sizeof(double) * 7 * ne * npe);
    or_quad_points(nodes, elems, ne, npe, qx, qn, qw, qL);
    /* quadrature-point strengths from the nodal data */
    cplx *f = malloc(sizeof(cplx) * 7 * ne);
    for (int64_t e = 0; e < ne; e++)
        for (int q = 0; q < 7; q++) {
            cplx s = 0.0;
            for (int a = 0; a < npe; a++) {
                int64_t j = (op == OR_OP_A) ? elems[e * npe + a] : chi_idx[e * npe + a];
                s += qL[(e * 7 + q) * npe + a] * x[j];
            }
            f[e * 7 + q] = qw[e * 7 + q] * s;
        }
    /* levels */
    int maxl = 0;
    for (int64_t b = 0; b < nb; b++) if (T->box[b].level > maxl) maxl = T->box[b].level;
    /* step 1: leaf moments */
    for (int64_t b = 0; b < nb; b++) {
        obox_t *B = &T->box[b];
        if (!B->leaf) continue;
        for (int64_t t = 0; t < B->nelems; t++) {
            int64_t e = B->elems[t];
            for (int q = 0; q < 7; q++) {
                int64_t o = e * 7 + q;
                cplx sig = (op == OR_OP_B) ? f[o] : 0.0, mu = (op == OR_OP_A) ? f[o] : 0.0;
                p2m_point(&M, B->c, qx + 3 * o, qn + 3 * o, sig, mu, Imom + b * np);
            }
        }
    }
    /* step 2: upward coefficient shift, deepest level first */
    for (int l = maxl; l >= 1; l--)
        for (int64_t b = 0; b < nb; b++) {
            obox_t *B = &T->box[b];
            if (B->level != l) continue;
            m2m(&M, B->c, T->box[B->parent].c, Imom + b * np, Imom + (int64_t)B->parent * np);
        }
    /* step 3: downward -- parent local shifted, plus interaction list */
    for (int l = 0; l <= maxl; l++)
        for (int64_t b = 0; b < nb; b++) {
            obox_t *B = &T->box[b];
            if (B->level != l) continue;
            if (B->parent >= 0) l2l(&M, T->box[B->parent].c, B->c, Floc + (int64_t)B->parent * np, Floc + b * np);
            for (int64_t t = 0; t < B->ninter; t++) {
                int64_t s = B->inter[t];
                m2l(&M, green, k, B->c, T->box[s].c, Imom + s * np, Floc + b * np);
            }
        }
    /* step 4: local expansion at each vertex plus the near-field boxes */
    int64_t *el = NULL, nel = 0, cap = 0;
    for (int64_t b = 0; b < nb; b++) {
        obox_t *B = &T->box[b];
        if (!B->leaf) continue;
        nel = 0;
        for (int64_t t = 0; t < B->nnear; t++) subtree_elems(T, B->nearl[t], &el, &nel, &cap);
        for (int64_t t = 0; t < B->nnodes; t++) {
            int64_t i = B->nodes[t];
            cplx s = l2p(&M, B->c, nodes + 3 * i, Floc + b * np);
            for (int64_t u = 0; u < nel; u++) {
                int64_t e = el[u];
                for (int q = 0; q < 7; q++) {
                    int64_t o = e * 7 + q;
                    s += point_kernel(green, k, op, nodes + 3 * i, qx + 3 * o, qn + 3 * o) * f[o];
                }
            }
            y[i] = s;
        }
    }
    free(el);
    /* special pairs: (special - regular) correction */
    for (int64_t t = 0; t < ncorr; t++) y[corr_row[t]] += corr_val[t] * x[corr_col[t]];
    for (int64_t i = 0; i < nn; i++) y[i] = (op == OR_OP_A) ? (1.0 + d0sum[i]) * x[i] - y[i] : -y[i];
    if (moments) memcpy(moments, Imom, sizeof(cplx) * nb * np);
    if (locals) memcpy(locals, Floc, sizeof(cplx) * nb * np);
    free(Imom); free(Floc); free(qx); free(qn); free(qw); free(qL); free(f);
    mindex_free(&M);
    return 0;
}
