// C ABI entry points (include/bem.h): contexts, plans, the fast matrix
// multiplication as one captured CUDA graph per operator, the GMRES solve and
// the exports used for parity checks.
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "bem_internal.cuh"

namespace bem {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};
thread_local long long *tl_capture_count = nullptr;

void count_launch(long long n) {
    if (tl_capture_count) *tl_capture_count += n;
    else g_launches += n;
}

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return e == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA;
}

__global__ void k_set_slots(const void **xs, const void *x, void **ys, void *y) {
    xs[0] = x;
    ys[0] = y;
}

// Points the plan's input/output slots at x and y, in stream order.
int set_slots(bem_plan *P, const void *x, void *y, cudaStream_t s) {
    (k_set_slots<<<1, 1, 0, s>>>(P->xptr, x, P->yptr, y), ::bem::count_launch());
    BEM_LAUNCH_CHECK();
    return BEM_OK;
}

// Enqueues the full product y = A x or B x on stream s, reading the vectors
// from the plan's device slots.  The kernel sequence is captured once per
// operator into a CUDA graph (on a private stream, since the legacy default
// stream cannot be captured) and replayed afterwards.  Another host thread
// can invalidate a capture in progress (its first launch of a kernel loads
// the kernel, which synchronises the context); the partial graph is then
// dropped, this product is enqueued kernel by kernel on s, and the capture
// is tried again on the next call.
int enqueue_matvec(bem_plan *P, int op, int green, double k, cudaStream_t s) {
    cudaGraphExec_t &ge = P->graph[op];
    if (!ge) {
        if (!P->capture_stream) BEM_CUDA(cudaStreamCreateWithFlags(&P->capture_stream, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        BEM_CUDA(cudaStreamBeginCapture(P->capture_stream, cudaStreamCaptureModeThreadLocal));
        P->graph_kernels[op] = 0;
        tl_capture_count = &P->graph_kernels[op];
        int rc = enqueue_matvec_raw(P, op, green, k, 1, P->capture_stream);
        tl_capture_count = nullptr;
        cudaError_t e = cudaStreamEndCapture(P->capture_stream, &g);
        const bool invalidated = e == cudaErrorStreamCaptureInvalidated ||
                                 (rc != BEM_OK && cudaPeekAtLastError() == cudaErrorStreamCaptureInvalidated);
        if (rc != BEM_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (!invalidated) return rc != BEM_OK ? rc : cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
            cudaGetLastError();                     // not sticky: clear it and run uncaptured
            P->capture_retries++;
            P->graph_kernels[op] = 0;
            BEM_TRY(enqueue_matvec_raw(P, op, green, k, 1, s));
            P->last_op = op;
            return BEM_OK;
        }
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
    BEM_CUDA(cudaGraphLaunch(ge, s));
    count_launch(P->graph_kernels[op]);
    P->last_op = op;
    return BEM_OK;
}

static int validate_params(const bem_fmm_params &p) {
    if (p.p < 1 || p.p > PMAX) { set_error("p = %d outside [1, %d]", p.p, PMAX); return BEM_EINVAL; }
    if (p.leaf_size < 2) { set_error("leaf_size = %d < 2", p.leaf_size); return BEM_EINVAL; }
    if (!(p.eta >= 1.0 && p.eta <= 8.0)) { set_error("eta = %g outside [1, 8]", p.eta); return BEM_EINVAL; }
    if (p.max_level < 1 || p.max_level > 20) { set_error("max_level = %d outside [1, 20]", p.max_level); return BEM_EINVAL; }
    if (p.leaf_descend != 0 && p.leaf_descend != 1) { set_error("leaf_descend must be 0 or 1"); return BEM_EINVAL; }
    if (p.precision != BEM_F64 && p.precision != BEM_MIXED) { set_error("precision must be BEM_F64 or BEM_MIXED"); return BEM_EINVAL; }
    if (p.precision == BEM_MIXED && !p.leaf_descend) { set_error("BEM_MIXED needs leaf_descend = 1"); return BEM_EINVAL; }
    if (p.n_duffy < 2 || p.n_duffy > 64) { set_error("n_duffy = %d outside [2, 64]", p.n_duffy); return BEM_EINVAL; }
    if (!(p.tau_near >= 0.0 && p.tau_near <= 16.0)) { set_error("tau_near = %g outside [0, 16]", p.tau_near); return BEM_EINVAL; }
    if (p.max_subdiv < 0 || p.max_subdiv > 10) { set_error("max_subdiv = %d outside [0, 10]", p.max_subdiv); return BEM_EINVAL; }
    if (p.p_min < 0 || p.p_min > p.p) { set_error("p_min = %d outside [0, p = %d]", p.p_min, p.p); return BEM_EINVAL; }
    return BEM_OK;
}

static int plan_setup(bem_plan *P, cudaStream_t s) {
    bem_mesh *m = P->mesh;
    Arena &A = P->arena;
    A.deferring = true;                                // released blocks stay reserved until the end
    BEM_TRY(A.alloc(&P->nodes, 3 * P->N));
    BEM_TRY(A.alloc(&P->elems, P->E * P->npe));
    BEM_TRY(A.alloc(&P->chi, P->E * P->npe));
    if (m->d_nodes && m->dev_device == P->device) {
        // device-resident mesh (bem_mesh_upload): device-to-device copies
        BEM_CUDA(cudaMemcpyAsync(P->nodes, m->d_nodes, sizeof(double) * 3 * P->N, cudaMemcpyDeviceToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(P->elems, m->d_elems, sizeof(int) * P->E * P->npe, cudaMemcpyDeviceToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(P->chi, m->d_chi, sizeof(int) * P->E * P->npe, cudaMemcpyDeviceToDevice, s));
    } else {
        BEM_CUDA(cudaMemcpyAsync(P->nodes, m->nodes.data(), sizeof(double) * 3 * P->N, cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(P->elems, m->elems.data(), sizeof(int) * P->E * P->npe, cudaMemcpyHostToDevice, s));
        BEM_CUDA(cudaMemcpyAsync(P->chi, m->chi.data(), sizeof(int) * P->E * P->npe, cudaMemcpyHostToDevice, s));
    }
    BEM_TRY(A.alloc(&P->istate, 4));
    BEM_CUDA(cudaMemsetAsync(P->istate, 0, sizeof(int) * 4, s));
    P->skip = P->istate;
    P->dev_err = P->istate + 3;
    // stage timers (wall clock, stream synchronised at every boundary)
    auto t0 = std::chrono::steady_clock::now();
    auto lap = [&](int i) -> int {
        BEM_CUDA(cudaStreamSynchronize(s));
        const auto t1 = std::chrono::steady_clock::now();
        P->setup_ms[i] = std::chrono::duration<double, std::milli>(t1 - t0).count();
        t0 = t1;
        return BEM_OK;
    };
    BEM_TRY(lap(0));
    BEM_TRY(build_tree(P, s));
    BEM_TRY(lap(1));
    BEM_TRY(build_geometry(P, s));
    BEM_TRY(build_radii_lists(P, s));
    BEM_TRY(lap(2));
    // The special-pair correction (stream s) is enqueued while a second host
    // thread builds the near-field work items and the M2L offset classes; then
    // the diagonal's tables and product at the diagonal's order (s2) are
    // enqueued, and the plan's own order (alloc_fmm, its kernels on s) is
    // built while both run.  The product
    // joins s before the diagonal adds the correction's row sums.  Stage times
    // of the correction and the diagonal are the GPU spans on their streams
    // (they overlap); the class stage is host time.
    cudaStream_t s2 = P->setup_stream[1], s3 = P->setup_stream[2];
    cudaEvent_t ev[6] = {};
    for (auto &e : ev) BEM_CUDA(cudaEventCreate(&e));
    auto fin = [&](int rc) {
        for (auto &e : ev) cudaEventDestroy(e);
        return rc;
    };
    BEM_CUDA(cudaEventRecord(ev[0], s));
    BEM_CUDA(cudaStreamWaitEvent(s2, ev[0], 0));
    BEM_CUDA(cudaStreamWaitEvent(s3, ev[0], 0));
    // host work beside the correction's enqueue (which waits once for the pair
    // count): the M2L offset classes on a second thread, the near-field work
    // items on this one once the correction is enqueued (the lists were
    // synchronised above); device copies on the null stream, which the plan's
    // non-blocking streams do not wait for
    int host_rc = BEM_OK;
    std::string host_err;
    const auto h0 = std::chrono::steady_clock::now();
    std::thread worker([&] {
        cudaError_t e = cudaSetDevice(P->device);
        host_rc = e == cudaSuccess ? build_m2l_classes(P) : cuda_fail(e, "cudaSetDevice", __FILE__, __LINE__);
        if (host_rc != BEM_OK) host_err = bem_last_error();
    });
    int rc = build_correction(P, s);
    if (rc == BEM_OK) {
        cudaError_t e = cudaEventRecord(ev[1], s);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaEventRecord", __FILE__, __LINE__);
    }
    if (rc == BEM_OK) rc = build_near_items(P);
    worker.join();
    P->setup_ms[4] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h0).count();
    if (rc == BEM_OK && host_rc != BEM_OK) {
        set_error("%s", host_err.c_str());
        rc = host_rc;
    }
    if (rc != BEM_OK) {
        cudaStreamSynchronize(s);
        return fin(rc);
    }
    if (rc == BEM_OK) BEM_CUDA(cudaEventRecord(ev[2], s2));
    if (rc == BEM_OK) rc = diagonal_prepare(P, s2);
    if (rc == BEM_OK) rc = diagonal_product(P, s2);
    if (rc == BEM_OK) BEM_CUDA(cudaEventRecord(ev[3], s2));
    if (rc == BEM_OK) rc = alloc_fmm(P, s3);
    if (rc == BEM_OK) BEM_CUDA(cudaEventRecord(ev[5], s3));
    if (rc == BEM_OK) BEM_CUDA(cudaStreamWaitEvent(s, ev[5], 0));
    if (rc == BEM_OK) BEM_CUDA(cudaStreamWaitEvent(s, ev[3], 0));
    if (rc == BEM_OK) rc = diagonal_finish(P, s);
    if (rc == BEM_OK) BEM_CUDA(cudaEventRecord(ev[4], s));
    if (rc != BEM_OK) {
        cudaStreamSynchronize(s);
        cudaStreamSynchronize(s2);
        cudaStreamSynchronize(s3);
        return fin(rc);
    }
    BEM_CUDA(cudaStreamSynchronize(s));
    for (void *q : P->deferred) A.release(q);
    P->deferred.clear();
    A.end_defer();                                     // both build streams are done
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    P->setup_ms[3] = ms;
    cudaEventElapsedTime(&ms, ev[2], ev[4]);
    P->setup_ms[5] = ms;
    t0 = std::chrono::steady_clock::now();
    BEM_TRY(lap(6));
    return fin(BEM_OK);
}

template <class T>
static int fetch(std::vector<T> &h, const T *d, size_t n) {
    h.resize(n);
    if (n) BEM_CUDA(cudaMemcpy(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost));
    return BEM_OK;
}

}  // namespace bem

bem_plan::~bem_plan() {
    for (auto &g : graph)
        if (g) cudaGraphExecDestroy(g);
    if (cycle_graph) cudaGraphExecDestroy(cycle_graph);
    if (hostbuf) cudaFreeHost(hostbuf);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    for (auto st : setup_stream)
        if (st) cudaStreamDestroy(st);
}

using namespace bem;

extern "C" {

const char *bem_last_error(void) { return g_err; }

void bem_fmm_params_default(bem_fmm_params *p) {
    if (!p) return;
    p->p = 8;
    p->leaf_size = 64;
    p->eta = 2.0;
    p->max_level = 20;
    p->leaf_descend = 1;
    p->precision = BEM_F64;
    p->n_duffy = 12;
    p->tau_near = 2.0;
    p->max_subdiv = 6;
    p->p_min = 0;
}

void bem_solve_params_default(bem_solve_params *p) {
    if (!p) return;
    p->restart = 30;
    p->tol = 1e-10;
    p->max_iter = 1000;
    p->method = BEM_GMRES;
}

int bem_ctx_create(int device, bem_ctx **out) {
    if (!out) { set_error("bem_ctx_create: out is NULL"); return BEM_EINVAL; }
    *out = nullptr;
    int n = 0;
    BEM_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) { set_error("bem_ctx_create: device %d of %d", device, n); return BEM_EINVAL; }
    BEM_CUDA(cudaSetDevice(device));
    bem_ctx *c = new (std::nothrow) bem_ctx;
    if (!c) { set_error("bem_ctx_create: out of host memory"); return BEM_ENOMEM; }
    c->device = device;
    BEM_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
    c->cache = std::make_shared<DevCache>();
    if (const char *ev = std::getenv("BEM_CACHE_BYTES")) c->cache->limit = (size_t)std::strtoull(ev, nullptr, 10);
    *out = c;
    return BEM_OK;
}

void bem_ctx_destroy(bem_ctx *ctx) { delete ctx; }

int bem_plan_create(bem_mesh *mesh, int green, double k, const bem_fmm_params *params, void *cuda_stream,
                    bem_plan **out) {
    if (!out) { set_error("bem_plan_create: out is NULL"); return BEM_EINVAL; }
    *out = nullptr;
    if (!mesh) { set_error("bem_plan_create: mesh is NULL"); return BEM_EINVAL; }
    if (!mesh->ctx) { set_error("bem_plan_create: mesh was created without a context"); return BEM_EINVAL; }
    if (green != BEM_LAPLACE && green != BEM_HELMHOLTZ) { set_error("bem_plan_create: bad green %d", green); return BEM_EINVAL; }
    if (green == BEM_HELMHOLTZ && !(k > 0.0 && k < 1e6)) { set_error("bem_plan_create: Helmholtz needs k > 0 (got %g)", k); return BEM_EINVAL; }
    bem_fmm_params prm;
    bem_fmm_params_default(&prm);
    if (params) prm = *params;
    BEM_TRY(validate_params(prm));
    BEM_CUDA(cudaSetDevice(mesh->ctx->device));
    bem_plan *P = new (std::nothrow) bem_plan;
    if (!P) { set_error("bem_plan_create: out of host memory"); return BEM_ENOMEM; }
    P->mesh = mesh;
    P->device = mesh->ctx->device;
    P->sm_count = mesh->ctx->sm_count;
    P->arena.cache = mesh->ctx->cache;
    P->green = green;
    P->k = green == BEM_HELMHOLTZ ? k : 0.0;
    P->prm = prm;
    P->N = mesh->n_nodes;
    P->E = mesh->n_elems;
    P->Q = mesh->n_elems * NQ;
    P->nchi = mesh->n_chi;
    P->npe = mesh->npe;
    // set-up runs on three streams of its own, after the caller's stream; the
    // second (the diagonal's product) has the higher priority, so its blocks
    // are scheduled first as the correction's quadrature blocks retire; the
    // third builds the plan's own order meanwhile
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    {
        int least = 0, greatest = 0;
        BEM_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        BEM_CUDA(cudaStreamCreateWithPriority(&P->setup_stream[0], cudaStreamNonBlocking, least));
        BEM_CUDA(cudaStreamCreateWithPriority(&P->setup_stream[1], cudaStreamNonBlocking, greatest));
        BEM_CUDA(cudaStreamCreateWithPriority(&P->setup_stream[2], cudaStreamNonBlocking, least));
    }
    cudaStream_t s = P->setup_stream[0];
    int rc = BEM_OK;
    {
        cudaEvent_t e0;
        BEM_CUDA(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(e0, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, e0, 0);
        cudaEventDestroy(e0);
        if (e != cudaSuccess) rc = cuda_fail(e, "plan set-up stream", __FILE__, __LINE__);
    }
    if (rc == BEM_OK) rc = plan_setup(P, s);
    if (rc == BEM_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "plan set-up", __FILE__, __LINE__);
    }
    if (rc != BEM_OK) {
        for (auto st : P->setup_stream) cudaStreamSynchronize(st);
        delete P;
        return rc;
    }
    *out = P;
    return BEM_OK;
}

void bem_plan_destroy(bem_plan *plan) {
    if (!plan) return;
    cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    delete plan;
}

int bem_matvec(bem_plan *P, int op, const void *x_dev, void *y_dev, void *cuda_stream) {
    if (!P || !x_dev || !y_dev) { set_error("bem_matvec: NULL argument"); return BEM_EINVAL; }
    if (op != BEM_OP_A && op != BEM_OP_B) { set_error("bem_matvec: bad op %d", op); return BEM_EINVAL; }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    BEM_TRY(set_slots(P, x_dev, y_dev, s));
    BEM_CUDA(cudaMemsetAsync(P->skip, 0, sizeof(int), s));
    return enqueue_matvec(P, op, P->green, P->k, s);
}

int bem_solve(bem_plan *P, const void *chi_dev, void *phi_dev, int nrhs, const bem_solve_params *params,
              bem_solve_info *info, void *cuda_stream) {
    if (!P || !chi_dev || !phi_dev || nrhs < 1) { set_error("bem_solve: bad argument"); return BEM_EINVAL; }
    bem_solve_params sp;
    bem_solve_params_default(&sp);
    if (params) sp = *params;
    if (!(sp.tol > 0.0) || sp.max_iter < 1) { set_error("bem_solve: tol must be > 0 and max_iter >= 1"); return BEM_EINVAL; }
    if (sp.method != BEM_GMRES && sp.method != BEM_BICGSTAB) { set_error("bem_solve: unknown method %d", sp.method); return BEM_EINVAL; }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    BEM_CUDA(cudaMemsetAsync(P->skip, 0, sizeof(int), s));
    return solve(P, chi_dev, phi_dev, nrhs, &sp, info, s);
}

int bem_plan_tree_sizes(const bem_plan *P, bem_tree_view *v) {
    if (!P || !v) { set_error("bem_plan_tree_sizes: NULL argument"); return BEM_EINVAL; }
    v->n_boxes = P->t.nbox;
    v->n_near = P->t.n_near;
    v->n_inter = P->t.n_inter;
    v->n_nodes = P->N;
    v->n_elems = P->E;
    for (int c = 0; c < 3; c++) v->lo[c] = P->t.lo[c];
    v->side = P->t.side;
    return BEM_OK;
}

int bem_plan_export_tree(const bem_plan *P, bem_tree_view *v) {
    if (!P || !v) { set_error("bem_plan_export_tree: NULL argument"); return BEM_EINVAL; }
    BEM_CUDA(cudaSetDevice(P->device));
    BEM_CUDA(cudaDeviceSynchronize());
    const Tree &t = P->t;
    const int nb = t.nbox;
    std::vector<int> lev, ix, iy, iz, par, nch, np_, ni, ip, ii, lon, perm, eb;
    std::vector<double> cx, cy, cz, r;
    BEM_TRY(fetch(lev, t.level, nb)); BEM_TRY(fetch(ix, t.ix, nb)); BEM_TRY(fetch(iy, t.iy, nb));
    BEM_TRY(fetch(iz, t.iz, nb)); BEM_TRY(fetch(par, t.parent, nb)); BEM_TRY(fetch(nch, t.nchild, nb));
    BEM_TRY(fetch(cx, t.cx, nb)); BEM_TRY(fetch(cy, t.cy, nb)); BEM_TRY(fetch(cz, t.cz, nb)); BEM_TRY(fetch(r, t.r, nb));
    BEM_TRY(fetch(np_, t.near_ptr, nb + 1)); BEM_TRY(fetch(ni, t.near_idx, t.n_near));
    BEM_TRY(fetch(ip, t.inter_ptr, nb + 1)); BEM_TRY(fetch(ii, t.inter_idx, t.n_inter));
    BEM_TRY(fetch(lon, t.leaf_of_node, P->N)); BEM_TRY(fetch(perm, t.elem_perm, P->E));
    std::vector<int> e_eb, e_ee;
    BEM_TRY(fetch(e_eb, t.eb, nb)); BEM_TRY(fetch(e_ee, t.ee, nb));
    for (int b = 0; b < nb; b++) {
        if (v->level) v->level[b] = lev[b];
        if (v->ijk) { v->ijk[3 * b] = ix[b]; v->ijk[3 * b + 1] = iy[b]; v->ijk[3 * b + 2] = iz[b]; }
        if (v->parent) v->parent[b] = par[b];
        if (v->leaf) v->leaf[b] = nch[b] == 0;
        if (v->centre) { v->centre[3 * b] = cx[b]; v->centre[3 * b + 1] = cy[b]; v->centre[3 * b + 2] = cz[b]; }
        if (v->radius) v->radius[b] = r[b];
    }
    for (int b = 0; b <= nb; b++) {
        if (v->near_ptr) v->near_ptr[b] = np_[b];
        if (v->inter_ptr) v->inter_ptr[b] = ip[b];
    }
    if (v->near_idx) for (int64_t u = 0; u < t.n_near; u++) v->near_idx[u] = ni[u];
    if (v->inter_idx) for (int64_t u = 0; u < t.n_inter; u++) v->inter_idx[u] = ii[u];
    if (v->leaf_of_node) for (int64_t i = 0; i < P->N; i++) v->leaf_of_node[i] = lon[i];
    if (v->owner)
        for (int b = 0; b < nb; b++)
            if (nch[b] == 0)
                for (int i = e_eb[b]; i < e_ee[b]; i++) v->owner[perm[i]] = b;
    return BEM_OK;
}

int bem_plan_export_correction(const bem_plan *P, int64_t *counts, int64_t *rowD, int64_t *colD, double *valD,
                               int64_t *rowS, int64_t *colS, double *valS) {
    if (!P || !counts) { set_error("bem_plan_export_correction: NULL argument"); return BEM_EINVAL; }
    const Correction &K = P->corr;
    counts[0] = K.nnzD;
    counts[1] = K.nnzS;
    if (!rowD && !rowS) return BEM_OK;
    BEM_CUDA(cudaSetDevice(P->device));
    BEM_CUDA(cudaDeviceSynchronize());
    const int C = P->green == BEM_HELMHOLTZ ? 2 : 1;
    std::vector<int> ptr, cD, cS;
    std::vector<double> vD, vS;
    BEM_TRY(fetch(ptr, K.ptrD, P->N + 1));
    BEM_TRY(fetch(cD, K.colD, K.nnzD)); BEM_TRY(fetch(cS, K.colS, K.nnzS));
    if (K.valD) {
        BEM_TRY(fetch(vD, K.valD, K.nnzD * C)); BEM_TRY(fetch(vS, K.valS, K.nnzS * C));
    } else {                                           // mixed plans hold float32 values
        std::vector<float> fD, fS;
        BEM_TRY(fetch(fD, K.fvalD, K.nnzD * C)); BEM_TRY(fetch(fS, K.fvalS, K.nnzS * C));
        vD.assign(fD.begin(), fD.end());
        vS.assign(fS.begin(), fS.end());
    }
    for (int64_t i = 0; i < P->N; i++)
        for (int q = ptr[i]; q < ptr[i + 1]; q++) {
            if (rowD) { rowD[q] = i; colD[q] = cD[q]; for (int c = 0; c < C; c++) valD[q * C + c] = vD[q * C + c]; }
            if (rowS) { rowS[q] = i; colS[q] = cS[q]; for (int c = 0; c < C; c++) valS[q * C + c] = vS[q * C + c]; }
        }
    return BEM_OK;
}

int bem_plan_export_expansions(const bem_plan *P, int32_t *mnk, double *moments, double *locals) {
    if (!P) { set_error("bem_plan_export_expansions: NULL plan"); return BEM_EINVAL; }
    const MIndex &mi = P->mi;
    if (mnk)
        for (int a = 0; a < mi.np; a++) { mnk[3 * a] = mi.m[a]; mnk[3 * a + 1] = mi.n[a]; mnk[3 * a + 2] = mi.k[a]; }
    if (!moments && !locals) return BEM_OK;
    BEM_CUDA(cudaSetDevice(P->device));
    BEM_CUDA(cudaDeviceSynchronize());
    const int C = P->green == BEM_HELMHOLTZ ? 2 : 1;
    const size_t n = (size_t)P->t.nbox * mi.np * C;
    std::vector<double> hm(n), hl(n);
    if (P->prm.precision == BEM_MIXED) {
        std::vector<float> fm, fl;
        BEM_TRY(fetch(fm, (const float *)P->fM, n));
        BEM_TRY(fetch(fl, (const float *)P->fL, n));
        for (size_t i = 0; i < n; i++) { hm[i] = fm[i]; hl[i] = fl[i]; }
    } else {
        BEM_TRY(fetch(hm, (const double *)P->M, n));
        BEM_TRY(fetch(hl, (const double *)P->L, n));
    }
    std::vector<int> lev;
    BEM_TRY(fetch(lev, P->t.level, P->t.nbox));
    for (int b = 0; b < P->t.nbox; b++) {
        const double h = std::ldexp(P->t.side, -lev[b]);
        for (int a = 0; a < mi.np; a++) {
            const int d = mi.m[a] + mi.n[a] + mi.k[a];
            const double up = std::pow(h, d);
            for (int c = 0; c < C; c++) {
                const size_t o = ((size_t)b * mi.np + a) * C + c;
                if (moments) moments[o] = hm[o] * up;
                if (locals) locals[o] = hl[o] / up;
            }
        }
    }
    return BEM_OK;
}

int bem_plan_diagonal(const bem_plan *P, double *c) {
    if (!P || !c) { set_error("bem_plan_diagonal: NULL argument"); return BEM_EINVAL; }
    BEM_CUDA(cudaSetDevice(P->device));
    BEM_CUDA(cudaDeviceSynchronize());
    BEM_CUDA(cudaMemcpy(c, P->C, sizeof(double) * P->N, cudaMemcpyDeviceToHost));
    return BEM_OK;
}

int bem_plan_footprint(const bem_plan *P, size_t *hbm_bytes) {
    if (!P || !hbm_bytes) { set_error("bem_plan_footprint: NULL argument"); return BEM_EINVAL; }
    *hbm_bytes = P->arena.bytes;
    return BEM_OK;
}

int bem_plan_device_status(const bem_plan *P, int *status) {
    if (!P || !status) { set_error("bem_plan_device_status: NULL argument"); return BEM_EINVAL; }
    BEM_CUDA(cudaSetDevice(P->device));
    BEM_CUDA(cudaDeviceSynchronize());
    BEM_CUDA(cudaMemcpy(status, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    return BEM_OK;
}

int bem_plan_peak_footprint(const bem_plan *P, size_t *hbm_bytes) {
    if (!P || !hbm_bytes) { set_error("bem_plan_peak_footprint: NULL argument"); return BEM_EINVAL; }
    *hbm_bytes = P->arena.peak;
    return BEM_OK;
}

int bem_plan_setup_times(const bem_plan *P, double *ms) {
    if (!P || !ms) { set_error("bem_plan_setup_times: NULL argument"); return BEM_EINVAL; }
    for (int i = 0; i < BEM_NSETUP; i++) ms[i] = P->setup_ms[i];
    return BEM_OK;
}

int bem_launch_count(long long *count) {
    if (!count) { set_error("bem_launch_count: NULL argument"); return BEM_EINVAL; }
    *count = g_launches.load();
    return BEM_OK;
}

int bem_plan_stage_times(bem_plan *P, int op, const void *x_dev, void *y_dev, int reps, double *ms,
                         void *cuda_stream) {
    if (!P || !x_dev || !y_dev || !ms || reps < 1) { set_error("bem_plan_stage_times: bad argument"); return BEM_EINVAL; }
    if (op != BEM_OP_A && op != BEM_OP_B) { set_error("bem_plan_stage_times: bad op %d", op); return BEM_EINVAL; }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t ev[BEM_NSTAGES + 1];
    for (auto &e : ev) BEM_CUDA(cudaEventCreate(&e));
    for (int i = 0; i < BEM_NSTAGES; i++) ms[i] = 0.0;
    int rc = set_slots(P, x_dev, y_dev, s);
    if (rc == BEM_OK) rc = cudaMemsetAsync(P->skip, 0, sizeof(int), s) == cudaSuccess ? BEM_OK : BEM_ECUDA;
    for (int r = 0; r < reps && rc == BEM_OK; r++) {
        rc = enqueue_matvec_raw(P, op, P->green, P->k, 1, s, ev);
        if (rc != BEM_OK) break;
        cudaError_t e = cudaEventSynchronize(ev[BEM_NSTAGES]);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaEventSynchronize", __FILE__, __LINE__); break; }
        for (int i = 0; i < BEM_NSTAGES; i++) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
            ms[i] += t / reps;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return rc;
}

int bem_plan_stats(const bem_plan *P, int64_t *st) {
    if (!P || !st) { set_error("bem_plan_stats: NULL argument"); return BEM_EINVAL; }
    st[0] = P->t.nbox;
    st[1] = P->t.nleaf;
    st[2] = P->t.nlev;
    st[3] = P->t.n_near;
    st[4] = P->t.n_inter;
    st[5] = P->near_pairs;
    st[6] = P->corr.nnzD;
    st[7] = P->corr.nnzS;
    st[8] = P->Q;
    st[9] = P->mi.np;
    st[10] = P->graph_kernels[0];
    st[11] = P->graph_kernels[1];
    st[12] = P->sy_tc;
    st[13] = P->sy_ncls;
    return BEM_OK;
}

}  // extern "C"
