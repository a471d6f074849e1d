// Host-side mesh preparation: validation and the sharp-edge multi-indexing of
// the Neumann data (Section 2.3).
#include <cmath>
#include <cstring>
#include <vector>

#include "bem_internal.cuh"

namespace bem {

// Outward element normal at local node a of a 3- or 6-node triangle, not
// normalised: t1 x t2 with t1 = dx/ds, t2 = dx/dt of the isoparametric map
// (the shape-function derivatives at the node are fixed numbers, tabulated).
static void node_normal(const double *X, int npe, int a, double n[3]) {
    // d N_b / ds and d N_b / dt at node a: 6-node rows at (s, t) of node a
    static const double DS6[6][6] = {{-3, -1, 0, 4, 0, 0},  {1, 3, 0, -4, 0, 0},  {1, -1, 0, 0, 4, -4},
                                     {-1, 1, 0, 0, 0, 0},   {1, 1, 0, -2, 2, -2}, {-1, -1, 0, 2, 2, -2}};
    static const double DT6[6][6] = {{-3, 0, -1, 0, 0, 4},  {1, 0, -1, -4, 4, 0}, {1, 0, 3, 0, 0, -4},
                                     {-1, 0, -1, -2, 2, 2}, {1, 0, 1, -2, 2, -2}, {-1, 0, 1, 0, 0, 0}};
    double u[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    if (npe == 3) {
        for (int c = 0; c < 3; c++) {
            u[c] = X[3 + c] - X[c];
            v[c] = X[6 + c] - X[c];
        }
    } else {
        for (int b = 0; b < 6; b++)
            for (int c = 0; c < 3; c++) {
                u[c] += DS6[a][b] * X[3 * b + c];
                v[c] += DT6[a][b] * X[3 * b + c];
            }
    }
    n[0] = u[1] * v[2] - u[2] * v[1];
    n[1] = u[2] * v[0] - u[0] * v[2];
    n[2] = u[0] * v[1] - u[1] * v[0];
}

// Elements are visited in order; at each of their nodes the element normal
// either joins the first existing cluster of that node whose opening normal is
// within the angle tolerance, or opens a new cluster (a new chi index).  The
// clusters live in one flat array: a node's first cluster at its own index,
// further ones (edges and corners) appended and chained in creation order.
int64_t mesh_chi_index(const double *nodes, int64_t nn, const int32_t *elems, int64_t ne, int npe,
                       double angle_deg, int32_t *chi) {
    const double cos_tol = std::cos(angle_deg * M_PI / 180.0);
    struct Cluster { double n[3]; int32_t id, next; };
    std::vector<Cluster> cl((size_t)nn, Cluster{{0.0, 0.0, 0.0}, -1, -1});
    int64_t count = 0;
    double X[18];
    for (int64_t e = 0; e < ne; e++) {
        for (int a = 0; a < npe; a++)
            for (int c = 0; c < 3; c++) X[3 * a + c] = nodes[3 * (int64_t)elems[e * npe + a] + c];
        for (int a = 0; a < npe; a++) {
            double n[3];
            node_normal(X, npe, a, n);
            const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            // clusters keep unit normals: cos(angle) >= cos_tol  <=>  n . m >= cos_tol |n|
            const double thr = cos_tol * len;
            int64_t k = elems[e * npe + a], last = -1;
            int32_t id = -1;
            if (cl[k].id >= 0)
                for (; k >= 0; last = k, k = cl[k].next)
                    if (n[0] * cl[k].n[0] + n[1] * cl[k].n[1] + n[2] * cl[k].n[2] >= thr) { id = cl[k].id; break; }
            if (id < 0) {
                id = (int32_t)count++;
                const Cluster c{{n[0] / len, n[1] / len, n[2] / len}, id, -1};
                if (last < 0) {
                    cl[elems[e * npe + a]] = c;                 // the node's first cluster
                } else {
                    cl[last].next = (int32_t)cl.size();
                    cl.push_back(c);
                }
            }
            chi[e * npe + a] = id;
        }
    }
    return count;
}

}  // namespace bem

bem_mesh::~bem_mesh() {
    if (d_nodes) cudaFree(d_nodes);
    if (d_elems) cudaFree(d_elems);
    if (d_chi) cudaFree(d_chi);
}

extern "C" {

int bem_mesh_create(bem_ctx *ctx, const double *nodes, int64_t n_nodes, const int32_t *elems,
                    int64_t n_elems, int elem_type, double edge_angle_deg, bem_mesh **out) {
    if (!out) { bem::set_error("bem_mesh_create: out is NULL"); return BEM_EINVAL; }
    *out = nullptr;
    if (!nodes || !elems) { bem::set_error("bem_mesh_create: NULL argument"); return BEM_EINVAL; }
    if (elem_type != BEM_TRI3 && elem_type != BEM_TRI6) {
        bem::set_error("bem_mesh_create: elem_type %d is not BEM_TRI3 or BEM_TRI6", elem_type);
        return BEM_EINVAL;
    }
    if (n_nodes < 3 || n_elems < 1 || n_nodes > (int64_t)1 << 30 || n_elems > (int64_t)1 << 28) {
        bem::set_error("bem_mesh_create: bad sizes n_nodes=%lld n_elems=%lld", (long long)n_nodes,
                       (long long)n_elems);
        return BEM_EINVAL;
    }
    if (!(edge_angle_deg > 0.0 && edge_angle_deg < 180.0)) {
        bem::set_error("bem_mesh_create: edge_angle_deg %g outside (0, 180)", edge_angle_deg);
        return BEM_EINVAL;
    }
    int npe = elem_type == BEM_TRI3 ? 3 : 6;
    for (int64_t i = 0; i < 3 * n_nodes; i++)
        if (!std::isfinite(nodes[i])) {
            bem::set_error("bem_mesh_create: node coordinate %lld is not finite", (long long)i);
            return BEM_EINVAL;
        }
    for (int64_t e = 0; e < n_elems; e++) {
        for (int a = 0; a < npe; a++) {
            int32_t v = elems[e * npe + a];
            if (v < 0 || v >= n_nodes) {
                bem::set_error("bem_mesh_create: element %lld node %d index %d out of range", (long long)e, a, v);
                return BEM_EINVAL;
            }
            for (int b = 0; b < a; b++)
                if (elems[e * npe + b] == v) {
                    bem::set_error("bem_mesh_create: element %lld repeats node %d", (long long)e, v);
                    return BEM_EINVAL;
                }
        }
        const double *p0 = nodes + 3 * (int64_t)elems[e * npe], *p1 = nodes + 3 * (int64_t)elems[e * npe + 1],
                     *p2 = nodes + 3 * (int64_t)elems[e * npe + 2];
        double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
        double v[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
        double c0 = u[1] * v[2] - u[2] * v[1], c1 = u[2] * v[0] - u[0] * v[2], c2 = u[0] * v[1] - u[1] * v[0];
        if (c0 * c0 + c1 * c1 + c2 * c2 == 0.0) {
            bem::set_error("bem_mesh_create: element %lld has zero area", (long long)e);
            return BEM_EINVAL;
        }
    }
    bem_mesh *m = new (std::nothrow) bem_mesh;
    if (!m) { bem::set_error("bem_mesh_create: out of host memory"); return BEM_ENOMEM; }
    m->ctx = ctx;
    m->n_nodes = n_nodes;
    m->n_elems = n_elems;
    m->npe = npe;
    m->elem_type = elem_type;
    m->edge_angle = edge_angle_deg;
    m->nodes.assign(nodes, nodes + 3 * n_nodes);
    m->elems.assign(elems, elems + npe * n_elems);
    m->chi.resize(npe * n_elems);
    m->n_chi = bem::mesh_chi_index(nodes, n_nodes, elems, n_elems, npe, edge_angle_deg, m->chi.data());
    *out = m;
    return BEM_OK;
}

void bem_mesh_destroy(bem_mesh *mesh) { delete mesh; }

int bem_mesh_upload(bem_mesh *m, void *cuda_stream) {
    if (!m || !m->ctx) { bem::set_error("bem_mesh_upload: mesh without a context"); return BEM_EINVAL; }
    BEM_CUDA(cudaSetDevice(m->ctx->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!m->d_nodes) {
        BEM_CUDA(cudaMalloc(&m->d_nodes, sizeof(double) * m->nodes.size()));
        BEM_CUDA(cudaMalloc(&m->d_elems, sizeof(int32_t) * m->elems.size()));
        BEM_CUDA(cudaMalloc(&m->d_chi, sizeof(int32_t) * m->chi.size()));
    }
    BEM_CUDA(cudaMemcpyAsync(m->d_nodes, m->nodes.data(), sizeof(double) * m->nodes.size(), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyAsync(m->d_elems, m->elems.data(), sizeof(int32_t) * m->elems.size(), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaMemcpyAsync(m->d_chi, m->chi.data(), sizeof(int32_t) * m->chi.size(), cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    m->dev_device = m->ctx->device;
    return BEM_OK;
}

int bem_mesh_sizes(const bem_mesh *mesh, int64_t *n_phi, int64_t *n_chi) {
    if (!mesh) { bem::set_error("bem_mesh_sizes: NULL mesh"); return BEM_EINVAL; }
    if (n_phi) *n_phi = mesh->n_nodes;
    if (n_chi) *n_chi = mesh->n_chi;
    return BEM_OK;
}

int bem_mesh_chi_index(const bem_mesh *mesh, int32_t *elem_local_to_chi) {
    if (!mesh || !elem_local_to_chi) { bem::set_error("bem_mesh_chi_index: NULL argument"); return BEM_EINVAL; }
    std::memcpy(elem_local_to_chi, mesh->chi.data(), sizeof(int32_t) * mesh->chi.size());
    return BEM_OK;
}

}  // extern "C"
