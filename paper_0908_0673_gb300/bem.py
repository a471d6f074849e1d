"""Thin ctypes binding of the C ABI in ``include/bem.h``.

Every function keeps the C name and only marshals arguments: host arrays
become pointers, torch CUDA tensors become device pointers, streams become
``cudaStream_t`` handles.  All computation happens in ``_build/libbem.so``;
if that library is missing the import fails -- there is no fallback.
A non-zero return code raises ``BemError`` with ``bem_last_error()``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

BEM_OK, BEM_EINVAL, BEM_ENOMEM, BEM_ECUDA, BEM_ENOCONV, BEM_ETIMEOUT, BEM_EBUSY = 0, -1, -2, -3, -4, -5, -6
BEM_TRI3, BEM_TRI6 = 1, 2
BEM_LAPLACE, BEM_HELMHOLTZ = 0, 1
BEM_F64, BEM_MIXED = 0, 1
BEM_OP_A, BEM_OP_B = 0, 1
BEM_GMRES, BEM_BICGSTAB = 0, 1

# every symbol include/bem.h declares
EXPORTS = [
    "bem_fmm_params_default", "bem_solve_params_default", "bem_ctx_create", "bem_ctx_destroy",
    "bem_last_error", "bem_mesh_create", "bem_mesh_destroy", "bem_mesh_sizes", "bem_mesh_chi_index",
    "bem_plan_create", "bem_plan_destroy", "bem_matvec", "bem_solve", "bem_plan_tree_sizes",
    "bem_plan_export_tree", "bem_plan_export_correction", "bem_plan_export_expansions",
    "bem_plan_diagonal", "bem_plan_footprint", "bem_plan_stats", "bem_plan_stage_times",
    "bem_launch_count", "bem_measure_peak", "bem_mesh_upload", "bem_matvec_noalloc", "bem_plan_setup_times",
    "bem_batch_create", "bem_batch_destroy", "bem_batch_submit", "bem_batch_progress", "bem_batch_poll",
    "bem_batch_wait", "bem_batch_release", "bem_batch_stream", "bem_plan_peak_footprint",
    "bem_plan_device_status", "bem_field", "bem_group_create", "bem_group_destroy", "bem_group_solve",
    "bem_solve_stop_rule",
]
BEM_NSETUP = 7
SETUP_NAMES = ["upload", "tree", "geometry_radii_lists", "correction", "m2l_classes", "diagonal_tables", "stats"]
BEM_NSTAGES = 7
STAGE_NAMES = ["p2q", "p2m", "m2m", "m2l", "l2l", "near_l2p", "combine"]


class bem_fmm_params(C.Structure):
    _fields_ = [("p", C.c_int), ("leaf_size", C.c_int), ("eta", C.c_double), ("max_level", C.c_int),
                ("leaf_descend", C.c_int), ("precision", C.c_int), ("n_duffy", C.c_int),
                ("tau_near", C.c_double), ("max_subdiv", C.c_int), ("p_min", C.c_int)]


class bem_solve_params(C.Structure):
    _fields_ = [("restart", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int), ("method", C.c_int)]


class bem_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("rel_residual", C.c_double), ("status", C.c_int)]


class bem_tree_view(C.Structure):
    _fields_ = [("n_boxes", C.c_int64), ("n_near", C.c_int64), ("n_inter", C.c_int64),
                ("n_nodes", C.c_int64), ("n_elems", C.c_int64), ("lo", C.c_double * 3), ("side", C.c_double),
                ("level", C.c_void_p), ("ijk", C.c_void_p), ("parent", C.c_void_p), ("leaf", C.c_void_p),
                ("centre", C.c_void_p), ("radius", C.c_void_p), ("near_ptr", C.c_void_p),
                ("near_idx", C.c_void_p), ("inter_ptr", C.c_void_p), ("inter_idx", C.c_void_p),
                ("leaf_of_node", C.c_void_p), ("owner", C.c_void_p)]


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"BEM error {code}: {msg}")
        self.code = code


_lib = None


def load(build_if_missing: bool = True):
    """Load libbem.so (building it with nvcc if asked); raise if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise ImportError(f"{_build.LIB} is missing: run paper_0908_0673_gb300.build")
        _build.build()
    L = C.CDLL(_build.LIB)
    P, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    L.bem_fmm_params_default.argtypes = [P]
    L.bem_fmm_params_default.restype = None
    L.bem_solve_params_default.argtypes = [P]
    L.bem_solve_params_default.restype = None
    L.bem_ctx_create.argtypes = [i32, P]
    L.bem_ctx_destroy.argtypes = [P]
    L.bem_ctx_destroy.restype = None
    L.bem_last_error.restype = C.c_char_p
    L.bem_mesh_create.argtypes = [P, P, i64, P, i64, i32, dbl, P]
    L.bem_mesh_destroy.argtypes = [P]
    L.bem_mesh_destroy.restype = None
    L.bem_mesh_sizes.argtypes = [P, P, P]
    L.bem_mesh_chi_index.argtypes = [P, P]
    L.bem_plan_create.argtypes = [P, i32, dbl, P, P, P]
    L.bem_plan_destroy.argtypes = [P]
    L.bem_plan_destroy.restype = None
    L.bem_matvec.argtypes = [P, i32, P, P, P]
    L.bem_solve.argtypes = [P, P, P, i32, P, P, P]
    L.bem_plan_tree_sizes.argtypes = [P, P]
    L.bem_plan_export_tree.argtypes = [P, P]
    L.bem_plan_export_correction.argtypes = [P, P, P, P, P, P, P, P]
    L.bem_plan_export_expansions.argtypes = [P, P, P, P]
    L.bem_plan_diagonal.argtypes = [P, P]
    L.bem_plan_footprint.argtypes = [P, P]
    L.bem_plan_stats.argtypes = [P, P]
    L.bem_plan_stage_times.argtypes = [P, i32, P, P, i32, P, P]
    L.bem_launch_count.argtypes = [P]
    L.bem_measure_peak.argtypes = [i32, P, P]
    L.bem_mesh_upload.argtypes = [P, P]
    L.bem_matvec_noalloc.argtypes = [P, i32, P, P, P]
    L.bem_plan_setup_times.argtypes = [P, P]
    L.bem_batch_create.argtypes = [P, i32, P]
    L.bem_batch_destroy.argtypes = [P]
    L.bem_batch_destroy.restype = None
    L.bem_batch_submit.argtypes = [P, P, P, P, P, P]
    L.bem_batch_progress.argtypes = [P, P]
    L.bem_batch_poll.argtypes = [P, i32, P, P]
    L.bem_batch_wait.argtypes = [P, i32, dbl]
    L.bem_batch_release.argtypes = [P, i32]
    L.bem_batch_stream.argtypes = [P, i32]
    L.bem_batch_stream.restype = P
    L.bem_solve_stop_rule.argtypes = [i32, dbl, i32, dbl, dbl, i32, i32, P]
    for name in EXPORTS:
        if name not in ("bem_fmm_params_default", "bem_solve_params_default", "bem_ctx_destroy",
                        "bem_last_error", "bem_mesh_destroy", "bem_plan_destroy", "bem_batch_destroy",
                        "bem_batch_stream", "bem_group_destroy"):
            getattr(L, name).restype = i32
    _lib = L
    return L


def _check(code, allow=()):
    if code != BEM_OK and code not in allow:
        raise BemError(code, load().bem_last_error().decode())
    return code


def _ptr(a):
    """numpy array -> host pointer; torch tensor -> device (or host) pointer."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return C.c_void_p(s)
    return C.c_void_p(s.cuda_stream)


# ----------------------------------------------------------------------------
# the C ABI, one function each
# ----------------------------------------------------------------------------

def bem_last_error() -> str:
    return load().bem_last_error().decode()


def bem_fmm_params_default(**overrides) -> bem_fmm_params:
    p = bem_fmm_params()
    load().bem_fmm_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def bem_solve_params_default(**overrides) -> bem_solve_params:
    p = bem_solve_params()
    load().bem_solve_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def bem_ctx_create(device: int = 0):
    h = C.c_void_p()
    _check(load().bem_ctx_create(device, C.byref(h)))
    return h


def bem_ctx_destroy(ctx):
    load().bem_ctx_destroy(ctx)


def bem_mesh_create(ctx, nodes, elems, elem_type, edge_angle_deg=30.0):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    h = C.c_void_p()
    _check(load().bem_mesh_create(ctx, _ptr(nodes), nodes.shape[0], _ptr(elems), elems.shape[0],
                                  int(elem_type), float(edge_angle_deg), C.byref(h)))
    return h


def bem_mesh_destroy(mesh):
    load().bem_mesh_destroy(mesh)


def bem_mesh_upload(mesh, stream=None):
    _check(load().bem_mesh_upload(mesh, _stream(stream)))


def bem_mesh_sizes(mesh):
    a, b = C.c_int64(), C.c_int64()
    _check(load().bem_mesh_sizes(mesh, C.byref(a), C.byref(b)))
    return a.value, b.value


def bem_mesh_chi_index(mesh, n_elems, npe):
    out = np.zeros((n_elems, npe), np.int32)
    _check(load().bem_mesh_chi_index(mesh, _ptr(out)))
    return out


def bem_plan_create(mesh, green=BEM_LAPLACE, k=0.0, params=None, stream=None):
    h = C.c_void_p()
    _check(load().bem_plan_create(mesh, int(green), float(k), C.byref(params) if params is not None else None,
                                  _stream(stream), C.byref(h)))
    return h


def bem_plan_destroy(plan):
    load().bem_plan_destroy(plan)


def bem_matvec(plan, op, x, y, stream=None):
    """x, y: CUDA tensors (float64, or complex128 for Helmholtz)."""
    _check(load().bem_matvec(plan, int(op), _ptr(x), _ptr(y), _stream(stream)))


def bem_matvec_noalloc(plan, op, x, y, stream=None):
    """bem_matvec without any allocation (scratch in the library's fixed
    device array); see include/bem.h."""
    _check(load().bem_matvec_noalloc(plan, int(op), _ptr(x), _ptr(y), _stream(stream)))


def bem_solve_stop_rule(precision, tol, restarts, rel, prev_rel, iters, max_iter):
    """The solvers' decision after a true residual (host only): returns
    (ended, status); status is None while the solve goes on."""
    st = C.c_int(1)
    end = load().bem_solve_stop_rule(int(precision), float(tol), int(restarts), float(rel), float(prev_rel),
                                     int(iters), int(max_iter), C.byref(st))
    return bool(end), (st.value if end else None)


def bem_solve(plan, chi, phi, nrhs=1, params=None, stream=None):
    """Returns (code, [bem_solve_info]); code is BEM_OK or BEM_ENOCONV."""
    infos = (bem_solve_info * nrhs)()
    code = load().bem_solve(plan, _ptr(chi), _ptr(phi), int(nrhs),
                            C.byref(params) if params is not None else None, infos, _stream(stream))
    _check(code, allow=(BEM_ENOCONV,))
    return code, list(infos)


def bem_field(plan, phi, chi, pts, u, stream=None):
    """Field of the surface data at points off the surface (see include/bem.h).
    phi, chi, pts ([npts, 3] float64), u: CUDA tensors."""
    _check(load().bem_field(plan, _ptr(phi), _ptr(chi), int(pts.shape[0]), _ptr(pts), _ptr(u), _stream(stream)))


def bem_group_create(ctx, plans):
    arr = (C.c_void_p * len(plans))(*[C.c_void_p(p.value if hasattr(p, "value") else p) for p in plans])
    h = C.c_void_p()
    _check(load().bem_group_create(ctx, arr, len(plans), C.byref(h)))
    return h


def bem_group_destroy(group):
    load().bem_group_destroy(group)


def bem_group_solve(group, chis, phis, params=None):
    """chis, phis: lists of CUDA tensors (or None to leave a member out).
    Returns (code, [bem_solve_info], kernels launched)."""
    n = len(chis)
    ca = (C.c_void_p * n)(*[C.c_void_p(_ptr(c).value if c is not None else None) for c in chis])
    pa = (C.c_void_p * n)(*[C.c_void_p(_ptr(p).value if p is not None else None) for p in phis])
    infos = (bem_solve_info * n)()
    nl = C.c_longlong()
    code = load().bem_group_solve(group, ca, pa, C.byref(params) if params is not None else None, infos, C.byref(nl))
    _check(code, allow=(BEM_ENOCONV,))
    return code, list(infos), nl.value


def bem_batch_create(ctx, max_slots):
    h = C.c_void_p()
    _check(load().bem_batch_create(ctx, int(max_slots), C.byref(h)))
    return h


def bem_batch_destroy(batch):
    load().bem_batch_destroy(batch)


def bem_batch_submit(batch, plan, chi, phi, params=None) -> int:
    slot = C.c_int()
    _check(load().bem_batch_submit(batch, plan, _ptr(chi), _ptr(phi),
                                   C.byref(params) if params is not None else None, C.byref(slot)))
    return slot.value


def bem_batch_progress(batch) -> int:
    n = C.c_int()
    _check(load().bem_batch_progress(batch, C.byref(n)), allow=(BEM_ENOCONV,))
    return n.value


def bem_batch_poll(batch, slot):
    done, info = C.c_int(), bem_solve_info()
    _check(load().bem_batch_poll(batch, int(slot), C.byref(done), C.byref(info)))
    return bool(done.value), info


def bem_batch_wait(batch, slot, timeout_s=600.0):
    _check(load().bem_batch_wait(batch, int(slot), float(timeout_s)))


def bem_batch_release(batch, slot):
    _check(load().bem_batch_release(batch, int(slot)))


def bem_batch_stream(batch, slot) -> int:
    return load().bem_batch_stream(batch, int(slot)) or 0


def bem_plan_tree_sizes(plan) -> bem_tree_view:
    v = bem_tree_view()
    _check(load().bem_plan_tree_sizes(plan, C.byref(v)))
    return v


def bem_plan_export_tree(plan) -> dict:
    v = bem_plan_tree_sizes(plan)
    nb, nn, ni, N, E = v.n_boxes, v.n_near, v.n_inter, v.n_nodes, v.n_elems
    out = dict(level=np.zeros(nb, np.int32), ijk=np.zeros((nb, 3), np.int64), parent=np.zeros(nb, np.int32),
               leaf=np.zeros(nb, np.int32), centre=np.zeros((nb, 3)), radius=np.zeros(nb),
               near_ptr=np.zeros(nb + 1, np.int64), near_idx=np.zeros(nn, np.int64),
               inter_ptr=np.zeros(nb + 1, np.int64), inter_idx=np.zeros(ni, np.int64),
               leaf_of_node=np.zeros(N, np.int64), owner=np.zeros(E, np.int64))
    for k_, a in out.items():
        setattr(v, k_, a.ctypes.data)
    _check(load().bem_plan_export_tree(plan, C.byref(v)))
    out["lo"] = np.array(list(v.lo))
    out["side"] = v.side
    return out


def bem_plan_export_correction(plan, complex_=False):
    counts = np.zeros(2, np.int64)
    L = load()
    _check(L.bem_plan_export_correction(plan, _ptr(counts), None, None, None, None, None, None))
    nD, nS = int(counts[0]), int(counts[1])
    c = 2 if complex_ else 1
    rD, cD, vD = np.zeros(nD, np.int64), np.zeros(nD, np.int64), np.zeros(nD * c)
    rS, cS, vS = np.zeros(nS, np.int64), np.zeros(nS, np.int64), np.zeros(nS * c)
    _check(L.bem_plan_export_correction(plan, _ptr(counts), _ptr(rD), _ptr(cD), _ptr(vD), _ptr(rS), _ptr(cS),
                                        _ptr(vS)))
    if complex_:
        vD, vS = vD.view(np.complex128), vS.view(np.complex128)
    return dict(rowD=rD, colD=cD, valD=vD, rowS=rS, colS=cS, valS=vS)


def bem_plan_export_expansions(plan, n_boxes, n_p, complex_=False):
    c = 2 if complex_ else 1
    mnk = np.zeros((n_p, 3), np.int32)
    mom = np.zeros(n_boxes * n_p * c)
    loc = np.zeros(n_boxes * n_p * c)
    _check(load().bem_plan_export_expansions(plan, _ptr(mnk), _ptr(mom), _ptr(loc)))
    if complex_:
        mom, loc = mom.view(np.complex128), loc.view(np.complex128)
    return mnk, mom.reshape(n_boxes, n_p), loc.reshape(n_boxes, n_p)


def bem_plan_diagonal(plan, n_phi):
    out = np.zeros(n_phi)
    _check(load().bem_plan_diagonal(plan, _ptr(out)))
    return out


def bem_plan_footprint(plan) -> int:
    v = C.c_size_t()
    _check(load().bem_plan_footprint(plan, C.byref(v)))
    return v.value


def bem_plan_device_status(plan) -> int:
    v = C.c_int()
    _check(load().bem_plan_device_status(plan, C.byref(v)))
    return v.value


def bem_plan_peak_footprint(plan) -> int:
    v = C.c_size_t()
    _check(load().bem_plan_peak_footprint(plan, C.byref(v)))
    return v.value


STAT_NAMES = ["n_boxes", "n_leaves", "n_levels", "n_near", "n_inter", "near_pairs", "corr_nnz_D",
              "corr_nnz_S", "n_quad", "n_p", "graph_kernels_A", "graph_kernels_B", "m2l_tensor_cores",
              "m2l_classes"]


def bem_plan_stage_times(plan, op, x, y, reps=5, stream=None) -> dict:
    ms = np.zeros(BEM_NSTAGES)
    _check(load().bem_plan_stage_times(plan, int(op), _ptr(x), _ptr(y), int(reps), _ptr(ms), _stream(stream)))
    return dict(zip(STAGE_NAMES, ms.tolist()))


def bem_plan_setup_times(plan) -> dict:
    ms = np.zeros(BEM_NSETUP)
    _check(load().bem_plan_setup_times(plan, _ptr(ms)))
    return dict(zip(SETUP_NAMES, ms.tolist()))


def bem_launch_count() -> int:
    v = C.c_longlong()
    _check(load().bem_launch_count(C.byref(v)))
    return v.value


def bem_measure_peak(kind, stream=None) -> float:
    v = C.c_double()
    _check(load().bem_measure_peak(int(kind), C.byref(v), _stream(stream)))
    return v.value


def bem_plan_stats(plan) -> dict:
    st = np.zeros(len(STAT_NAMES), np.int64)
    _check(load().bem_plan_stats(plan, _ptr(st)))
    return dict(zip(STAT_NAMES, (int(v) for v in st)))
