"""Request serving over the C ABI: continuous batching with admission by
device-memory footprint.

A request is one boundary-value problem as the paper states it (Section 2):
a surface mesh, the Green's function (Laplace, or Helmholtz with wavenumber
k) and the Neumann data of one or more right-hand sides; the answer is the
surface potential of each.  The server

* admits a request once it has arrived, a batch slot is free for it and the
  device-memory reservation of everything admitted plus the request's
  estimated peak footprint fits the budget (requests that could never fit are
  refused at once);
* builds its plan (tree, lists, correction, translation tables, diagonal) on
  a set-up thread, so set-up overlaps the device work of solves in flight;
* runs its right-hand sides one after another in its slot of a
  ``bem_batch`` while the solves of other requests advance on their own
  streams: requests that arrive while others are on the device join as soon
  as a slot and memory free up;
* keeps the plan (and its Krylov basis) resident until the request's last
  right-hand side is done, then frees it on the set-up thread.

Latency is completion minus arrival.  The engine interface (build / submit /
progress / poll / fetch / release / destroy) separates the scheduling logic
from the device so that the scheduler can be exercised without a GPU.
"""
from __future__ import annotations

import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import bem
from . import inputs as I
from . import tune


# ----------------------------------------------------------------------------
# requests and results
# ----------------------------------------------------------------------------

@dataclass
class Request:
    rid: int
    arrival_s: float               # seconds after the stream starts
    mesh: I.Mesh
    green: int                     # bem.BEM_LAPLACE or bem.BEM_HELMHOLTZ
    k: float
    rhs: list                      # Neumann data per right-hand side, [n_elems, npe]


@dataclass
class Result:
    rid: int
    n_elems: int
    n_nodes: int
    green: int
    k: float
    n_rhs: int
    arrival_s: float
    admitted_s: float = math.nan
    ready_s: float = math.nan      # plan built
    done_s: float = math.nan
    reserved: int = 0              # bytes reserved at admission
    peak_footprint: int = 0        # measured peak of the plan
    iters: list = field(default_factory=list)
    rel_residual: list = field(default_factory=list)
    status: str = "pending"        # ok | noconv | refused | error
    error: str = ""
    phi: list | None = None

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


class EngineError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


# ----------------------------------------------------------------------------
# footprint model
# ----------------------------------------------------------------------------

# Peak device bytes per geometric node of a plan with the default parameters
# (p = 10, leaf sizes 32-128, eta = 2, Duffy order 12, tau = 2) and a GMRES(30)
# basis, by (Green's function, precision).  The correction matrix dominates
# (a few hundred entries per row for each of D and S); then the translation
# tables, the diagonal's higher-order buffers (held while the plan's own order
# is built beside them: both sets of buffers, the stored P2M weights included,
# exist at the set-up peak) and the Krylov basis.  The values bound the
# measured peaks (9-28 kB per node on spheres, ellipsoids and graded cubes of
# 1k-18k quadratic elements, before the two orders overlapped) with a margin;
# the GPU tests check the bound.  The fixed part holds the M2L row buffers of
# the two orders, each capped at 128 MiB whatever the mesh (rows are computed
# and gathered in runs of targets), and 64 MiB of small tables.
_BYTES_PER_NODE = {
    (bem.BEM_LAPLACE, bem.BEM_F64): 36_000,
    (bem.BEM_LAPLACE, bem.BEM_MIXED): 36_000,
    (bem.BEM_HELMHOLTZ, bem.BEM_F64): 44_000,
    (bem.BEM_HELMHOLTZ, bem.BEM_MIXED): 44_000,
}
_BYTES_FIXED = (64 + 2 * 128) << 20


def estimate_peak_footprint(n_nodes: int, green: int, precision: int) -> int:
    """Upper estimate of a plan's peak device memory, used for admission."""
    return _BYTES_FIXED + _BYTES_PER_NODE[(green, precision)] * int(n_nodes)


# ----------------------------------------------------------------------------
# engine over the C ABI
# ----------------------------------------------------------------------------

class _Handle:
    __slots__ = ("req", "mesh", "plan", "chi", "phi", "peak", "n_phi")


class CudaEngine:
    """Plans, device buffers and a ``bem_batch`` on one GPU.

    ``build`` and ``destroy`` run on set-up threads; everything else on the
    scheduler thread."""

    def __init__(self, device: int = 0, precision: int = bem.BEM_MIXED, max_slots: int = 8,
                 fmm: dict | None = None, solve: dict | None = None, warmup: bool = True):
        import torch
        self.torch = torch
        self.device = device
        self.precision = precision
        self.max_slots = max_slots
        self.ctx = bem.bem_ctx_create(device)
        self.batch = bem.bem_batch_create(self.ctx, max_slots)
        self.fmm = dict(fmm or {})          # fixed parameters; the rest per mesh from the autotuner's table
        self.solve = dict(restart=30, tol=1e-10, max_iter=600)
        self.solve.update(solve or {})
        self.sp = bem.bem_solve_params_default(**self.solve)
        self._tls = threading.local()
        if warmup:
            self._warmup()

    def _warmup(self):
        # One tiny solve of every element type and Green's function, on this
        # thread, before set-up threads exist: the first launch of each kernel
        # loads it, and a load in one thread invalidates a graph capture that
        # another thread has in progress.
        for et in (I.TRI3, I.TRI6):
            m = I.geodesic(2, et)
            for green, k in ((bem.BEM_LAPLACE, 0.0), (bem.BEM_HELMHOLTZ, 1.0)):
                rhs = [I.helmholtz_point_source(m, (0.1, 0.0, 0.0), k)[1] if k else I.point_source(m, (0.1, 0.0, 0.0))[1]]
                h = self.build(Request(-1, 0.0, m, green, k, rhs))
                bem.bem_solve(h.plan, h.chi[0], h.phi[0], 1, self.sp, self._stream())
                self._stream().synchronize()
                self.destroy(h)

    def estimate(self, req: Request) -> int:
        return estimate_peak_footprint(req.mesh.n_nodes, req.green, self.precision)

    def budget(self) -> int:
        free, _ = self.torch.cuda.mem_get_info(self.device)
        return int(0.85 * free)

    def _stream(self):
        s = getattr(self._tls, "stream", None)
        if s is None:
            s = self._tls.stream = self.torch.cuda.Stream(device=self.device)
        return s

    def build(self, req: Request) -> _Handle:
        t = self.torch
        m = req.mesh
        try:
            mesh = bem.bem_mesh_create(self.ctx, m.nodes, m.elems, m.elem_type)
        except bem.BemError as e:
            raise EngineError(e.code, str(e)) from None
        plan = None
        try:
            n_phi, n_chi = bem.bem_mesh_sizes(mesh)
            idx = bem.bem_mesh_chi_index(mesh, m.n_elems, m.npe)
            s = self._stream()
            prm = tune.choose(m.n_elems, req.green, self.precision)
            prm.update(self.fmm)
            prm["precision"] = self.precision
            plan = bem.bem_plan_create(mesh, req.green, req.k, bem.bem_fmm_params_default(**prm), s)
            cplx = req.green == bem.BEM_HELMHOLTZ
            dt = t.complex128 if cplx else t.float64
            chi = np.zeros((len(req.rhs), n_chi), np.complex128 if cplx else np.float64)
            for r, ce in enumerate(req.rhs):
                chi[r, idx.ravel()] = np.asarray(ce).ravel()
            with t.cuda.stream(s):
                chi_d = t.from_numpy(chi).pin_memory().to(f"cuda:{self.device}", dtype=dt, non_blocking=True)
                phi_d = t.empty((len(req.rhs), n_phi), device=f"cuda:{self.device}", dtype=dt)
            s.synchronize()                    # batch streams do not wait on this one
        except bem.BemError as e:
            if plan is not None:
                bem.bem_plan_destroy(plan)
            bem.bem_mesh_destroy(mesh)
            raise EngineError(e.code, str(e)) from None
        h = _Handle()
        h.req, h.mesh, h.plan, h.chi, h.phi, h.n_phi = req, mesh, plan, chi_d, phi_d, n_phi
        h.peak = bem.bem_plan_peak_footprint(plan)
        return h

    def submit(self, h: _Handle, r: int) -> int:
        return bem.bem_batch_submit(self.batch, h.plan, h.chi[r], h.phi[r], self.sp)

    def progress(self) -> int:
        return bem.bem_batch_progress(self.batch)

    def poll(self, slot: int):
        done, info = bem.bem_batch_poll(self.batch, slot)
        return done, (info.iters, info.rel_residual, info.status) if done else None

    def release(self, slot: int):
        bem.bem_batch_release(self.batch, slot)

    def fetch(self, h: _Handle):
        # the slot's work is complete (its last event has passed)
        return [h.phi[r].cpu().numpy() for r in range(h.phi.shape[0])]

    def peak(self, h: _Handle) -> int:
        # includes the Krylov basis allocated by the first solve
        return max(h.peak, bem.bem_plan_peak_footprint(h.plan))

    def destroy(self, h: _Handle):
        bem.bem_plan_destroy(h.plan)
        bem.bem_mesh_destroy(h.mesh)
        h.chi = h.phi = None

    def close(self):
        bem.bem_batch_destroy(self.batch)
        bem.bem_ctx_destroy(self.ctx)


# ----------------------------------------------------------------------------
# the scheduler
# ----------------------------------------------------------------------------

class Server:
    """Continuous-batching scheduler over an engine.

    ``max_inflight`` requests hold a batch slot each (at most the engine's
    slots); ``setup_threads`` plans are built at once."""

    def __init__(self, engine, hbm_budget: int | None = None, max_inflight: int | None = None,
                 setup_threads: int = 2, keep_phi: bool = False, poll_s: float = 1e-4):
        self.eng = engine
        self.budget = engine.budget() if hbm_budget is None else int(hbm_budget)
        self.max_inflight = min(max_inflight or engine.max_slots, engine.max_slots)
        self.setup_threads = max(1, setup_threads)
        self.keep_phi = keep_phi
        self.poll_s = poll_s
        self.max_reserved = 0

    def run(self, requests: list[Request]) -> list[Result]:
        reqs = sorted(requests, key=lambda r: (r.arrival_s, r.rid))
        res = {r.rid: Result(r.rid, r.mesh.n_elems, r.mesh.n_nodes, r.green, r.k, len(r.rhs), r.arrival_s)
               for r in reqs}
        jobs: queue.Queue = queue.Queue()
        ready: queue.Queue = queue.Queue()
        clock0 = time.perf_counter()

        def now():
            return time.perf_counter() - clock0

        def worker():
            while True:
                job = jobs.get()
                if job is None:
                    return
                kind, obj = job
                if kind == "build":
                    try:
                        ready.put(("ok", obj, self.eng.build(obj)))
                    except EngineError as e:
                        ready.put(("err", obj, e))
                    except Exception as e:       # a request must never take the server down
                        ready.put(("err", obj, EngineError(bem.BEM_ECUDA, repr(e))))
                else:
                    self.eng.destroy(obj)
                    ready.put(("freed", obj.req, None))

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.setup_threads)]
        for th in threads:
            th.start()

        waiting: list[Request] = []
        nxt = 0
        reserved = 0
        admitted = 0            # admitted and not yet finished (each holds a slot)
        active = {}             # slot -> (handle, rhs index)
        handles_building = 0
        pending_free = 0
        unfinished = len(reqs)
        try:
            while unfinished or pending_free:
                t = now()
                while nxt < len(reqs) and reqs[nxt].arrival_s <= t:
                    waiting.append(reqs[nxt])
                    nxt += 1
                # admission, first come first served
                while waiting and admitted < self.max_inflight:
                    r = waiting[0]
                    need = self.eng.estimate(r)
                    if need > self.budget:
                        waiting.pop(0)
                        res[r.rid].status = "refused"
                        res[r.rid].error = f"estimated peak {need} B exceeds the budget {self.budget} B"
                        res[r.rid].done_s = now()
                        unfinished -= 1
                        continue
                    if reserved + need > self.budget:
                        break
                    waiting.pop(0)
                    reserved += need
                    self.max_reserved = max(self.max_reserved, reserved)
                    admitted += 1
                    handles_building += 1
                    res[r.rid].admitted_s = now()
                    res[r.rid].reserved = need
                    jobs.put(("build", r))
                # plans built, memory freed
                while True:
                    try:
                        kind, r, h = ready.get_nowait()
                    except queue.Empty:
                        break
                    if kind == "freed":
                        reserved -= res[r.rid].reserved
                        pending_free -= 1
                        continue
                    handles_building -= 1
                    R = res[r.rid]
                    if kind == "err":
                        R.status, R.error, R.done_s = "error", str(h), now()
                        reserved -= R.reserved
                        admitted -= 1
                        unfinished -= 1
                        continue
                    R.ready_s = now()
                    active[self.eng.submit(h, 0)] = (h, 0)
                # advance everything in flight
                if active:
                    self.eng.progress()
                moved = False
                for slot in list(active):
                    h, rr = active[slot]
                    done, info = self.eng.poll(slot)
                    if not done:
                        continue
                    moved = True
                    R = res[h.req.rid]
                    R.iters.append(info[0])
                    R.rel_residual.append(info[1])
                    if info[2] != bem.BEM_OK:
                        R.status = "noconv"
                    self.eng.release(slot)
                    del active[slot]
                    if rr + 1 < len(h.req.rhs):
                        active[self.eng.submit(h, rr + 1)] = (h, rr + 1)
                        continue
                    if self.keep_phi:
                        R.phi = self.eng.fetch(h)
                    R.peak_footprint = self.eng.peak(h)
                    R.done_s = now()
                    if R.status == "pending":
                        R.status = "ok"
                    admitted -= 1
                    unfinished -= 1
                    pending_free += 1
                    jobs.put(("free", h))
                if active and not moved:
                    time.sleep(self.poll_s)      # lets the set-up threads run
                if not active:
                    # idle: sleep until the next arrival or a set-up result
                    wait = self.poll_s
                    if nxt < len(reqs) and not waiting and not handles_building and not pending_free:
                        wait = max(self.poll_s, reqs[nxt].arrival_s - now())
                    try:
                        item = ready.get(timeout=min(wait, 0.05))
                        ready.put(item)
                    except queue.Empty:
                        pass
        finally:
            for _ in threads:
                jobs.put(None)
            for th in threads:
                th.join()
        return [res[r.rid] for r in reqs]


# ----------------------------------------------------------------------------
# synthetic request stream and summary
# ----------------------------------------------------------------------------

def synthetic_stream(n_requests: int, rate_per_s: float = 200.0, elems=(1_000, 250_000),
                     k_range=(1.0, 4.0), rhs=(1, 8), helmholtz_share: float = 0.5,
                     seed: int = 0) -> list[Request]:
    """Poisson arrivals; element counts log-uniform in ``elems``; geometry a
    geodesic sphere, an ellipsoid (semi-axes uniform in [0.5, 2]) or a graded
    cube, all with 6-node triangles; Laplace or Helmholtz (k uniform in
    ``k_range``); 1..8 right-hand sides, each the field of a point source at a
    random interior point (radius up to 0.3 of the smallest semi-axis)."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        E = math.exp(rng.uniform(math.log(elems[0]), math.log(elems[1])))
        kind = int(rng.integers(0, 3))
        if kind == 2:
            n = max(2, int(round(math.sqrt(E / 12.0))))
            mesh = I.cube(n, I.TRI6, seed=int(rng.integers(1 << 30)))
            rmax = 0.3
        else:
            f = max(2, int(round(math.sqrt(E / 20.0))))
            axes = (1.0, 1.0, 1.0) if kind == 0 else tuple(rng.uniform(0.5, 2.0, 3))
            mesh = I.geodesic(f, I.TRI6, axes=axes)
            rmax = 0.3 * min(axes)
        helm = rng.uniform() < helmholtz_share
        k = float(rng.uniform(*k_range)) if helm else 0.0
        nr = int(rng.integers(rhs[0], rhs[1] + 1))
        data = []
        for _ in range(nr):
            d = rng.standard_normal(3)
            xs = d / np.linalg.norm(d) * rmax * rng.uniform() ** (1.0 / 3.0)
            data.append(I.helmholtz_point_source(mesh, xs, k)[1] if helm else I.point_source(mesh, xs)[1])
        out.append(Request(rid, t, mesh, bem.BEM_HELMHOLTZ if helm else bem.BEM_LAPLACE, k, data))
    return out


def summarize(results: list[Result]) -> dict:
    ok = [r for r in results if r.status in ("ok", "noconv")]
    lat = np.array([r.latency_s for r in ok]) * 1e3
    t0 = min((r.arrival_s for r in results), default=0.0)
    t1 = max((r.done_s for r in ok), default=t0)
    span = max(t1 - t0, 1e-9)
    solves = sum(r.n_rhs for r in ok)
    return {
        "requests": len(results), "served": len(ok),
        "refused": sum(r.status == "refused" for r in results),
        "errors": sum(r.status == "error" for r in results),
        "not_converged": sum(r.status == "noconv" for r in results),
        "solves": solves, "makespan_s": span,
        "solves_per_s": solves / span, "requests_per_s": len(ok) / span,
        "latency_ms": {"p50": float(np.percentile(lat, 50)) if len(lat) else None,
                       "p99": float(np.percentile(lat, 99)) if len(lat) else None},
        "gmres_iters_mean": float(np.mean([i for r in ok for i in r.iters])) if ok else None,
    }
