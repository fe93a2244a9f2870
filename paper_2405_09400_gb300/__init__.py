"""Python binding of the ddflow C ABI (include/ddflow.h).

Argument marshalling only: every step of the method runs in the CUDA library
``lib/libddflow.so`` (built in-tree by ``_build.build()``). Importing works
without a GPU; creating a context needs one. There is no fallback: if the
library is missing, every call raises.

Functions keep the C names (dd_init, dd_iterate, dd_flow_update, dd_step,
dd_get_plan, dd_get_duals, ...); ``DomDec`` bundles them around one context.
Boxes are exchanged as ``(hdr, data)``: hdr an (nbasic, 4) int32 array of
(o1, o2, h, w) and data the packed float64 box contents.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libddflow.so")

DD_OK, DD_ERR_ARG, DD_ERR_OOM, DD_ERR_CUDA, DD_ERR_MAXITER = 0, -1, -2, -3, -4
DD_ERR_STALL, DD_ERR_FLOW, DD_ERR_POOL, DD_ERR_STATE = -5, -6, -7, -8
DD_INIT_PRODUCT, DD_INIT_USER = 0, 1
DD_WARM_PREV, DD_WARM_COLD, DD_WARM_AFFINE, DD_WARM_MLP = 0, 1, 2, 3
DD_FLAG_KEEP_PREBALANCE, DD_FLAG_COLLECT, DD_FLAG_NO_GRAPH, DD_FLAG_TRACE = 1, 2, 4, 8
DD_FLAG_MLP_EVERY_SOLVE, DD_FLAG_DEVICE_PTRS, DD_FLAG_FUSED_C2B = 16, 32, 64
DD_MLP_NIN, DD_MLP_NHID, DD_MLP_NOUT, DD_MLP_NPARAMS = 336, 256, 320, 300096
DD_MLP_GEMM_UMMA, DD_MLP_GEMM_MMA = 0, 1
DD_STATIC_MAX_PIXELS, DD_STATIC_MAX_CELLS = 1024 * 1024, 65536

EXPORTS = [
    "dd_default_options", "dd_strerror", "dd_last_error", "dd_init", "dd_set_plan", "dd_set_eps", "dd_iterate", "dd_flow_update", "dd_step",
    "dd_get_plan", "dd_get_duals", "dd_get_composite", "dd_get_cell_stats", "dd_get_objective",
    "dd_get_partition", "dd_get_neighbours", "dd_get_basic_moments", "dd_get_flow", "dd_get_prebalance",
    "dd_min_cost_flow", "dd_step_stats", "dd_get_counters", "dd_debug_cell", "dd_l1_y_error_static", "dd_destroy",
    "dd_mlp_create", "dd_mlp_set_params", "dd_mlp_get_params", "dd_mlp_forward", "dd_mlp_loss_grad",
    "dd_mlp_train_step", "dd_mlp_set_gemm", "dd_mlp_destroy", "dd_set_warmstart_weights", "dd_collect_cells", "dd_get_graph_counters",
    "dd_get_tuning", "dd_set_tuning", "dd_autotune", "dd_get_trace", "dd_probe_ex2_rate",
]


class dd_grid(C.Structure):
    _fields_ = [("N1", C.c_int32), ("N2", C.c_int32), ("h", C.c_double)]


class dd_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("fixed_iters", C.c_int32), ("trunc", C.c_double),
                ("init_kind", C.c_int32), ("warm", C.c_int32), ("threads", C.c_int32), ("flags", C.c_int32),
                ("plan_tol", C.c_double), ("omega", C.c_double), ("graph_margin", C.c_double),
                ("eps_levels", C.c_int32), ("eps_factor", C.c_double), ("eps_tol", C.c_double),
                ("tol_share", C.c_double), ("tol_gamma", C.c_double), ("anderson", C.c_int32),
                ("eps_gamma", C.c_double)]


class dd_stats(C.Structure):
    _fields_ = [("part", C.c_int32), ("ncell", C.c_int32), ("iters_max", C.c_int32), ("n_maxiter", C.c_int32),
                ("n_stalled", C.c_int32), ("iters_mean", C.c_double), ("objective", C.c_double), ("l1_x", C.c_double),
                ("lse_terms", C.c_double), ("ms_total", C.c_double), ("ms_cells", C.c_double),
                ("stored_entries", C.c_int64), ("ms_c2b", C.c_double), ("bytes_c2b", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dd_flow_stats(C.Structure):
    _fields_ = [("value", C.c_double), ("nonzero", C.c_int32), ("pivots", C.c_int32), ("moved", C.c_double),
                ("ms_costs", C.c_double), ("ms_solve", C.c_double), ("ms_exchange", C.c_double),
                ("bytes_exchange", C.c_double), ("ms_host_step", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dd_tuning(C.Structure):
    _fields_ = [("threads", C.c_int32 * 3), ("small_area", C.c_int32), ("small_side", C.c_int32),
                ("ms_default", C.c_double), ("ms_best", C.c_double), ("trials", C.c_int32),
                ("cl_size", C.c_int32), ("cl_cells", C.c_int32), ("sm_reserve", C.c_int32)]

    def as_dict(self):
        return dict(threads=list(self.threads), small_area=self.small_area, small_side=self.small_side,
                    ms_default=self.ms_default, ms_best=self.ms_best, trials=self.trials, cl_size=self.cl_size,
                    cl_cells=self.cl_cells, sm_reserve=self.sm_reserve)


class DDError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = f"{where}: {strerror(code)} ({code})"
        if code == DD_ERR_CUDA:
            msg += " [" + load().dd_last_error().decode(errors="replace") + "]"
        super().__init__(msg)


_lib = None
P = C.POINTER
_i32p, _f64p, _szp = P(C.c_int32), P(C.c_double), P(C.c_size_t)


def load():
    """Load lib/libddflow.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"ddflow library not built: {LIB_PATH} missing (run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sig = {
        "dd_default_options": (None, [P(dd_options)]),
        "dd_strerror": (C.c_char_p, [C.c_int]),
        "dd_last_error": (C.c_char_p, []),
        "dd_init": (C.c_int, [_f64p, _f64p, P(dd_grid), C.c_double, C.c_int, P(dd_options), vp, P(vp)]),
        "dd_set_plan": (C.c_int, [vp, _i32p, _f64p, C.c_size_t]),
        "dd_set_eps": (C.c_int, [vp, C.c_double]),
        "dd_iterate": (C.c_int, [vp, C.c_int, P(dd_stats)]),
        "dd_flow_update": (C.c_int, [vp, P(dd_flow_stats)]),
        "dd_step": (C.c_int, [vp, C.c_int, P(dd_stats), P(dd_stats), P(dd_flow_stats)]),
        "dd_get_plan": (C.c_int, [vp, _i32p, _f64p, _szp]),
        "dd_get_duals": (C.c_int, [vp, C.c_int, _f64p, _i32p, _f64p, _szp]),
        "dd_get_composite": (C.c_int, [vp, C.c_int, _i32p, _f64p, _szp]),
        "dd_get_cell_stats": (C.c_int, [vp, C.c_int, _i32p, _f64p]),
        "dd_get_objective": (C.c_int, [vp, _f64p, _f64p, _f64p]),
        "dd_get_partition": (C.c_int, [vp, C.c_int, _i32p, _i32p]),
        "dd_get_neighbours": (C.c_int, [vp, _i32p]),
        "dd_get_basic_moments": (C.c_int, [vp, _f64p, _f64p, _f64p, _f64p]),
        "dd_get_flow": (C.c_int, [vp, _f64p, _f64p]),
        "dd_get_prebalance": (C.c_int, [vp, _i32p, _f64p, _szp]),
        "dd_min_cost_flow": (C.c_int, [C.c_int32, _i32p, _f64p, _f64p, _f64p, _f64p, _i32p]),
        "dd_step_stats": (C.c_int, [vp, P(dd_stats), P(dd_stats), P(dd_flow_stats)]),
        "dd_get_counters": (C.c_int, [vp, P(C.c_int64), P(C.c_int64), P(C.c_int64)]),
        "dd_get_graph_counters": (C.c_int, [vp, P(C.c_int64), P(C.c_int64), P(C.c_int64)]),
        "dd_get_tuning": (C.c_int, [vp, P(dd_tuning)]),
        "dd_set_tuning": (C.c_int, [vp, P(dd_tuning)]),
        "dd_autotune": (C.c_int, [vp, C.c_char_p, P(dd_tuning)]),
        "dd_get_trace": (C.c_int, [vp, C.c_int, P(C.c_int64)]),
        "dd_probe_ex2_rate": (C.c_int, [vp, _f64p, _f64p]),
        "dd_debug_cell": (C.c_int, [vp, C.c_int, C.c_int, P(C.c_float), P(C.c_float), P(C.c_float), _i32p]),
        "dd_l1_y_error_static": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, vp, vp, vp, vp, vp]),
        "dd_destroy": (None, [vp]),
        "dd_mlp_create": (C.c_int, [C.c_int32, vp, P(vp)]),
        "dd_mlp_set_params": (C.c_int, [vp, P(C.c_float), C.c_int64]),
        "dd_mlp_get_params": (C.c_int, [vp, P(C.c_float), C.c_int64]),
        "dd_mlp_forward": (C.c_int, [vp, vp, C.c_int32, vp]),
        "dd_mlp_loss_grad": (C.c_int, [vp, vp, vp, vp, C.c_int32, _f64p, P(C.c_float)]),
        "dd_mlp_train_step": (C.c_int, [vp, vp, vp, vp, C.c_int32, vp, C.c_float, _f64p]),
        "dd_mlp_set_gemm": (C.c_int, [vp, C.c_int32]),
        "dd_mlp_destroy": (None, [vp]),
        "dd_set_warmstart_weights": (C.c_int, [vp, P(C.c_float), C.c_int64]),
        "dd_collect_cells": (C.c_int, [vp, C.c_int, vp, vp, C.c_int32, _i32p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().dd_strerror(int(code)).decode()


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _check(code, where, ok=(DD_OK,)):
    if code not in ok:
        raise DDError(code, where)
    return code


def default_options(**kw) -> dd_options:
    o = dd_options()
    load().dd_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def current_stream():
    """The raw handle of torch's current CUDA stream (None without torch/CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


# ---- C-named functions ------------------------------------------------------
def dd_init(mu, nu, eps, cell_size, h=None, options=None, stream=None):
    lib = load()
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    g = dd_grid(mu.shape[0], mu.shape[1], 1.0 / mu.shape[0] if h is None else h)
    ctx = C.c_void_p()
    opt = options if options is not None else default_options()
    _check(lib.dd_init(_ptr(mu, _f64p), _ptr(nu, _f64p), C.byref(g), float(eps), int(cell_size), C.byref(opt),
                       stream, C.byref(ctx)), "dd_init")
    return ctx


def dd_init_device(mu_t, nu_t, eps, cell_size, h=None, options=None, stream=None):
    """dd_init with DD_FLAG_DEVICE_PTRS: mu_t, nu_t are (N1, N2) float64 CUDA tensors
    (their device addresses are passed; the flag is added to the options)."""
    lib = load()
    opt = options if options is not None else default_options()
    opt.flags |= DD_FLAG_DEVICE_PTRS
    N1, N2 = int(mu_t.shape[0]), int(mu_t.shape[1])
    g = dd_grid(N1, N2, 1.0 / N1 if h is None else h)
    ctx = C.c_void_p()
    _check(lib.dd_init(C.cast(C.c_void_p(mu_t.data_ptr()), _f64p), C.cast(C.c_void_p(nu_t.data_ptr()), _f64p),
                       C.byref(g), float(eps), int(cell_size), C.byref(opt),
                       stream if stream is not None else current_stream(), C.byref(ctx)), "dd_init")
    return ctx


def dd_set_plan_device(ctx, hdr_t, data_t):
    """dd_set_plan on a DD_FLAG_DEVICE_PTRS context: int32 / float64 CUDA tensors."""
    _check(load().dd_set_plan(ctx, C.cast(C.c_void_p(hdr_t.data_ptr()), _i32p),
                              C.cast(C.c_void_p(data_t.data_ptr()), _f64p), int(data_t.numel())), "dd_set_plan")


def dd_get_plan_device(ctx, nbasic):
    """dd_get_plan on a DD_FLAG_DEVICE_PTRS context: (hdr, data) as CUDA tensors."""
    import torch

    cnt = C.c_size_t(0)
    lib = load()
    hdr = torch.empty((nbasic, 4), dtype=torch.int32, device="cuda")
    _check(lib.dd_get_plan(ctx, C.cast(C.c_void_p(hdr.data_ptr()), _i32p), None, C.byref(cnt)), "dd_get_plan")
    data = torch.empty(max(1, cnt.value), dtype=torch.float64, device="cuda")
    _check(lib.dd_get_plan(ctx, C.cast(C.c_void_p(hdr.data_ptr()), _i32p), C.cast(C.c_void_p(data.data_ptr()), _f64p),
                           C.byref(cnt)), "dd_get_plan")
    return hdr, data[:cnt.value]


def dd_get_duals_device(ctx, part, shape, ncell):
    """dd_get_duals on a DD_FLAG_DEVICE_PTRS context: (alpha, hdr, beta) as CUDA tensors."""
    import torch

    cnt = C.c_size_t(0)
    lib = load()
    hdr = torch.empty((ncell, 4), dtype=torch.int32, device="cuda")
    hp = C.cast(C.c_void_p(hdr.data_ptr()), _i32p)
    _check(lib.dd_get_duals(ctx, int(part), None, hp, None, C.byref(cnt)), "dd_get_duals")
    alpha = torch.empty(shape, dtype=torch.float64, device="cuda")
    beta = torch.empty(max(1, cnt.value), dtype=torch.float64, device="cuda")
    _check(lib.dd_get_duals(ctx, int(part), C.cast(C.c_void_p(alpha.data_ptr()), _f64p), hp,
                            C.cast(C.c_void_p(beta.data_ptr()), _f64p), C.byref(cnt)), "dd_get_duals")
    return alpha, hdr, beta[:cnt.value]


def dd_set_eps(ctx, eps):
    _check(load().dd_set_eps(ctx, float(eps)), "dd_set_eps")


def dd_set_plan(ctx, hdr, data):
    hdr = np.ascontiguousarray(hdr, dtype=np.int32)
    data = np.ascontiguousarray(data, dtype=np.float64)
    _check(load().dd_set_plan(ctx, _ptr(hdr, _i32p), _ptr(data, _f64p), data.size), "dd_set_plan")


def dd_iterate(ctx, part=-1):
    st = dd_stats()
    rc = _check(load().dd_iterate(ctx, int(part), C.byref(st)), "dd_iterate", ok=(DD_OK, DD_ERR_MAXITER))
    d = st.as_dict()
    d["status"] = rc
    return d


def dd_flow_update(ctx):
    st = dd_flow_stats()
    rc = _check(load().dd_flow_update(ctx, C.byref(st)), "dd_flow_update", ok=(DD_OK, DD_ERR_FLOW))
    d = st.as_dict()
    d["status"] = rc
    return d


def dd_step(ctx, n=1, stats=True):
    sa, sb, sf = dd_stats(), dd_flow_stats(), None
    sb = dd_stats()
    sf = dd_flow_stats()
    if stats:
        rc = load().dd_step(ctx, int(n), C.byref(sa), C.byref(sb), C.byref(sf))
    else:
        rc = load().dd_step(ctx, int(n), None, None, None)
    _check(rc, "dd_step", ok=(DD_OK, DD_ERR_MAXITER, DD_ERR_FLOW))
    if not stats:
        return rc
    fd = sf.as_dict()
    fd["status"] = rc  # DD_ERR_MAXITER: some cell capped; DD_ERR_FLOW: stationary flow kept
    return sa.as_dict(), sb.as_dict(), fd


def dd_step_stats(ctx):
    """Statistics of the last dd_step iteration (read back now if the step was
    replayed without them): (A stats, B stats, flow stats) dicts."""
    sa, sb, sf = dd_stats(), dd_stats(), dd_flow_stats()
    _check(load().dd_step_stats(ctx, C.byref(sa), C.byref(sb), C.byref(sf)), "dd_step_stats")
    return sa.as_dict(), sb.as_dict(), sf.as_dict()


def _boxes_call(fn, ctx, nhdr, *lead, out=None):
    cnt = C.c_size_t(0)
    hdr = np.zeros((nhdr, 4), dtype=np.int32)
    _check(fn(ctx, *lead, _ptr(hdr, _i32p), None, C.byref(cnt)), fn.__name__)
    n = cnt.value
    if out is not None and out.dtype == np.float64 and out.flags.c_contiguous and out.size >= n:
        data = out[:n]  # caller's buffer (e.g. pinned host memory)
    else:
        data = np.zeros(n, dtype=np.float64)
    _check(fn(ctx, *lead, _ptr(hdr, _i32p), _ptr(data, _f64p), C.byref(cnt)), fn.__name__)
    return hdr, data


def dd_get_plan(ctx, nbasic, out=None):
    """Current plan as (nbasic x 4 int32 headers, packed float64 boxes); `out`: an
    optional float64 buffer (e.g. pinned) the boxes are written into when large
    enough (the returned array is then a view of it)."""
    return _boxes_call(load().dd_get_plan, ctx, nbasic, out=out)


def dd_get_composite(ctx, part, ncell):
    return _boxes_call(load().dd_get_composite, ctx, ncell, C.c_int(part))


def dd_get_prebalance(ctx, nbasic):
    return _boxes_call(load().dd_get_prebalance, ctx, nbasic)


def dd_get_duals(ctx, part, shape, ncell):
    lib = load()
    cnt = C.c_size_t(0)
    hdr = np.zeros((ncell, 4), dtype=np.int32)
    _check(lib.dd_get_duals(ctx, int(part), None, _ptr(hdr, _i32p), None, C.byref(cnt)), "dd_get_duals")
    alpha = np.zeros(shape, dtype=np.float64)
    beta = np.zeros(cnt.value, dtype=np.float64)
    _check(lib.dd_get_duals(ctx, int(part), _ptr(alpha, _f64p), _ptr(hdr, _i32p), _ptr(beta, _f64p), C.byref(cnt)),
           "dd_get_duals")
    return alpha, hdr, beta


def dd_get_cell_stats(ctx, part, ncell):
    it = np.zeros(ncell, dtype=np.int32)
    er = np.zeros(ncell, dtype=np.float64)
    _check(load().dd_get_cell_stats(ctx, int(part), _ptr(it, _i32p), _ptr(er, _f64p)), "dd_get_cell_stats")
    return it, er


def dd_get_objective(ctx):
    E, lx, ly = C.c_double(), C.c_double(), C.c_double()
    _check(load().dd_get_objective(ctx, C.byref(E), C.byref(lx), C.byref(ly)), "dd_get_objective")
    return E.value, lx.value, ly.value


def dd_get_partition(ctx, part):
    n = C.c_int32()
    _check(load().dd_get_partition(ctx, int(part), None, C.byref(n)), "dd_get_partition")
    mem = np.zeros((n.value, 4), dtype=np.int32)
    _check(load().dd_get_partition(ctx, int(part), _ptr(mem, _i32p), C.byref(n)), "dd_get_partition")
    return mem


def dd_get_neighbours(ctx, nbasic):
    nbr = np.zeros((nbasic, 5), dtype=np.int32)
    _check(load().dd_get_neighbours(ctx, _ptr(nbr, _i32p)), "dd_get_neighbours")
    return nbr


def dd_get_basic_moments(ctx, nbasic):
    D, m, v = (np.zeros(nbasic) for _ in range(3))
    yb = np.zeros((nbasic, 2))
    _check(load().dd_get_basic_moments(ctx, _ptr(D, _f64p), _ptr(m, _f64p), _ptr(yb, _f64p), _ptr(v, _f64p)),
           "dd_get_basic_moments")
    return dict(D=D, mass=m, ybar=yb, var=v)


def dd_get_flow(ctx, nbasic):
    cb = np.zeros((nbasic, 5))
    w = np.zeros((nbasic, 5))
    _check(load().dd_get_flow(ctx, _ptr(cb, _f64p), _ptr(w, _f64p)), "dd_get_flow")
    return cb, w


def dd_min_cost_flow(nbr, cbar, m):
    """Host network simplex for Eq. (MinCostFlow); returns (w, value, pivots)."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    cb = np.ascontiguousarray(np.where(nbr >= 0, np.nan_to_num(cbar), 0.0), dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    w = np.zeros((len(m), 5))
    v, piv = C.c_double(), C.c_int32()
    _check(load().dd_min_cost_flow(len(m), _ptr(nbr, _i32p), _ptr(cb, _f64p), _ptr(m, _f64p), _ptr(w, _f64p),
                                   C.byref(v), C.byref(piv)), "dd_min_cost_flow")
    return w, v.value, piv.value


def dd_get_counters(ctx):
    n, a, b = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().dd_get_counters(ctx, C.byref(n), C.byref(a), C.byref(b)), "dd_get_counters")
    return dict(launches=n.value, h2d_bytes=a.value, d2h_bytes=b.value)


def dd_get_graph_counters(ctx):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().dd_get_graph_counters(ctx, C.byref(a), C.byref(b), C.byref(c)), "dd_get_graph_counters")
    return dict(captures=a.value, replays=b.value, fallbacks=c.value)


def dd_get_trace(ctx, part, ncell):
    """Per-cell solve timeline of the last half-iteration on `part`: (ncell, 8)
    int64 (start ns, end ns, SM, CTA size, end of the gather, start and end of the
    Sinkhorn iterations, 0)."""
    t = np.zeros((ncell, 8), dtype=np.int64)
    _check(load().dd_get_trace(ctx, int(part), _ptr(t, P(C.c_int64))), "dd_get_trace")
    return t


def dd_get_tuning(ctx):
    t = dd_tuning()
    _check(load().dd_get_tuning(ctx, C.byref(t)), "dd_get_tuning")
    return t.as_dict()


def dd_set_tuning(ctx, threads, small_area, small_side, cl_size=None, cl_cells=None, sm_reserve=None):
    """Launch configuration of the cell kernels; cl_size / cl_cells / sm_reserve
    None keep the context's current setting."""
    t = dd_tuning()
    _check(load().dd_get_tuning(ctx, C.byref(t)), "dd_get_tuning")
    t.threads = (C.c_int32 * 3)(*threads)
    t.small_area, t.small_side = int(small_area), int(small_side)
    if cl_size is not None:
        t.cl_size = int(cl_size)
    if cl_cells is not None:
        t.cl_cells = int(cl_cells)
    if sm_reserve is not None:
        t.sm_reserve = int(sm_reserve)
    _check(load().dd_set_tuning(ctx, C.byref(t)), "dd_set_tuning")


def dd_autotune(ctx, cache_path=None):
    t = dd_tuning()
    _check(load().dd_autotune(ctx, cache_path.encode() if cache_path else None, C.byref(t)), "dd_autotune")
    return t.as_dict()


def dd_debug_cell(ctx, part, J, amax):
    """Raw FP32 kernel values of one composite cell (diagnostics)."""
    _f32p = P(C.c_float)
    geom = np.zeros(8, dtype=np.int32)
    _check(load().dd_debug_cell(ctx, int(part), int(J), None, None, None, _ptr(geom, _i32p)), "dd_debug_cell")
    a = np.zeros(amax, dtype=np.float32)
    b = np.zeros(int(geom[6]) * int(geom[7]), dtype=np.float32)
    g = np.zeros(8, dtype=np.float32)
    _check(load().dd_debug_cell(ctx, int(part), int(J), _ptr(a, _f32p), _ptr(b, _f32p), _ptr(g, _f32p),
                                _ptr(geom, _i32p)), "dd_debug_cell")
    hx, wx = int(geom[2]), int(geom[3])
    return dict(a=a[:hx * wx].reshape(hx, wx), b=b.reshape(int(geom[6]), int(geom[7])), gauge=g, geom=geom)


def dd_l1_y_error_static(N1, N2, nbasic, hdr_ptr, data_ptr, nu_ptr, out_ptr, stream=None):
    """Allocation-free L1 Y error; all pointers are device addresses (ints)."""
    return load().dd_l1_y_error_static(int(N1), int(N2), int(nbasic), C.c_void_p(hdr_ptr), C.c_void_p(data_ptr),
                                       C.c_void_p(nu_ptr), C.c_void_p(out_ptr),
                                       stream if stream is not None else current_stream())


def dd_probe_ex2_rate(stream=None):
    """Measured ex2.approx throughput of the current device: (ex2 per second, ms)."""
    r, ms = C.c_double(), C.c_double()
    _check(load().dd_probe_ex2_rate(stream if stream is not None else current_stream(), C.byref(r), C.byref(ms)),
           "dd_probe_ex2_rate")
    return r.value, ms.value


def dd_destroy(ctx):
    if ctx:
        load().dd_destroy(ctx)


def _dptr(t):
    """Device address of a CUDA tensor (None stays None)."""
    return None if t is None else C.c_void_p(t.data_ptr())


def _params32(params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != DD_MLP_NPARAMS:
        raise ValueError(f"expected {DD_MLP_NPARAMS} parameters, got {p.size}")
    return p


def dd_set_warmstart_weights(ctx, params):
    p = _params32(params)
    _check(load().dd_set_warmstart_weights(ctx, _ptr(p, P(C.c_float)), p.size), "dd_set_warmstart_weights")


def dd_collect_cells(ctx, part):
    """Network inputs (rows x NIN, torch.bfloat16) and targets (rows x NOUT,
    torch.float32) of the last half-iteration on `part`, on the device."""
    import torch

    rows = C.c_int32()
    lib = load()
    _check(lib.dd_collect_cells(ctx, int(part), None, None, 0, C.byref(rows)), "dd_collect_cells")
    n = rows.value
    feat = torch.empty((n, DD_MLP_NIN), dtype=torch.bfloat16, device="cuda")
    targ = torch.empty((n, DD_MLP_NOUT), dtype=torch.float32, device="cuda")
    if n:
        _check(lib.dd_collect_cells(ctx, int(part), _dptr(feat), _dptr(targ), n, C.byref(rows)), "dd_collect_cells")
    return feat, targ


class MLP:
    """The warm-start network on the GPU (dd_mlp_*): parameters, forward pass,
    loss gradient and Adam steps. Tensors are torch CUDA tensors."""

    def __init__(self, max_batch, stream=None):
        self.max_batch = int(max_batch)
        self.h = C.c_void_p()
        _check(load().dd_mlp_create(self.max_batch, stream if stream is not None else current_stream(),
                                    C.byref(self.h)), "dd_mlp_create")

    def set_params(self, params):
        p = _params32(params)
        _check(load().dd_mlp_set_params(self.h, _ptr(p, P(C.c_float)), p.size), "dd_mlp_set_params")

    def get_params(self):
        p = np.zeros(DD_MLP_NPARAMS, dtype=np.float32)
        _check(load().dd_mlp_get_params(self.h, _ptr(p, P(C.c_float)), p.size), "dd_mlp_get_params")
        return p

    def set_gemm(self, kind):
        """Kernel of the forward layer products: DD_MLP_GEMM_UMMA (tcgen05, the
        default) or DD_MLP_GEMM_MMA (warp-level mma.sync)."""
        _check(load().dd_mlp_set_gemm(self.h, int(kind)), "dd_mlp_set_gemm")

    def forward(self, x):
        import torch

        y = torch.empty((x.shape[0], DD_MLP_NOUT), dtype=torch.float32, device=x.device)
        _check(load().dd_mlp_forward(self.h, _dptr(x), int(x.shape[0]), _dptr(y)), "dd_mlp_forward")
        return y

    def loss_grad(self, x, t, w):
        loss = C.c_double()
        g = np.zeros(DD_MLP_NPARAMS, dtype=np.float32)
        _check(load().dd_mlp_loss_grad(self.h, _dptr(x), _dptr(t), _dptr(w), int(x.shape[0]), C.byref(loss),
                                       _ptr(g, P(C.c_float))), "dd_mlp_loss_grad")
        return loss.value, g

    def train_step(self, x_all, t_all, idx, w, lr, want_loss=False):
        loss = C.c_double()
        _check(load().dd_mlp_train_step(self.h, _dptr(x_all), _dptr(t_all), _dptr(idx), int(idx.shape[0]), _dptr(w),
                                        float(lr), C.byref(loss) if want_loss else None), "dd_mlp_train_step")
        return loss.value if want_loss else None

    def close(self):
        if self.h:
            load().dd_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience wrapper -----------------------------------------------------
def boxes_to_arrays(boxes):
    """[(o1, o2, array), ...] -> (hdr (n, 4) int32, packed float64 data)."""
    hdr = np.array([[b[0], b[1], b[2].shape[0], b[2].shape[1]] for b in boxes], dtype=np.int32).reshape(-1, 4)
    data = np.concatenate([np.asarray(b[2], dtype=np.float64).reshape(-1) for b in boxes]) if boxes else np.zeros(0)
    return hdr, data


def arrays_to_boxes(hdr, data):
    out, k = [], 0
    for o1, o2, h, w in hdr:
        n = int(h) * int(w)
        out.append((int(o1), int(o2), data[k:k + n].reshape(int(h), int(w))))
        k += n
    return out


class DomDec:
    """One library context: DD half-iterations and flow updates on a grid problem."""

    def __init__(self, mu, nu, eps, cell_size, boxes=None, h=None, stream=None, weights=None, **opts):
        mu = np.asarray(mu, dtype=np.float64)
        self.shape = mu.shape
        self.s = int(cell_size)
        self.nbasic = (mu.shape[0] // self.s) * (mu.shape[1] // self.s)
        if boxes is not None:
            opts.setdefault("init_kind", DD_INIT_USER)
        self.options = default_options(**opts)
        self.ctx = dd_init(mu, nu, eps, cell_size, h=h, options=self.options,
                           stream=stream if stream is not None else current_stream())
        self.ncell = [len(dd_get_partition(self.ctx, p)) for p in (0, 1)]
        if boxes is not None:
            self.set_plan(boxes)
        if weights is not None:
            self.set_warmstart_weights(weights)

    def set_eps(self, eps):
        """eps of the next half-iterations (eps schedule across hybrid iterations)."""
        dd_set_eps(self.ctx, eps)
        self.eps = float(eps)

    def set_plan(self, boxes):
        hdr, data = boxes if isinstance(boxes, tuple) else boxes_to_arrays(boxes)
        dd_set_plan(self.ctx, hdr, data)

    def iterate(self, part=-1):
        return dd_iterate(self.ctx, part)

    def flow_update(self):
        return dd_flow_update(self.ctx)

    def step(self, n=1, stats=True):
        return dd_step(self.ctx, n, stats)

    def step_stats(self):
        return dd_step_stats(self.ctx)

    def plan(self):
        return arrays_to_boxes(*dd_get_plan(self.ctx, self.nbasic))

    def composite(self, part):
        return arrays_to_boxes(*dd_get_composite(self.ctx, part, self.ncell[part]))

    def prebalance(self):
        return arrays_to_boxes(*dd_get_prebalance(self.ctx, self.nbasic))

    def duals(self, part):
        alpha, hdr, beta = dd_get_duals(self.ctx, part, self.shape, self.ncell[part])
        return alpha, arrays_to_boxes(hdr, beta)

    def cell_stats(self, part):
        return dd_get_cell_stats(self.ctx, part, self.ncell[part])

    def objective(self):
        return dd_get_objective(self.ctx)

    def partition(self, part):
        return dd_get_partition(self.ctx, part)

    def neighbours(self):
        return dd_get_neighbours(self.ctx, self.nbasic)

    def basic_moments(self):
        return dd_get_basic_moments(self.ctx, self.nbasic)

    def flow(self):
        return dd_get_flow(self.ctx, self.nbasic)

    def counters(self):
        return dd_get_counters(self.ctx)

    def graph_counters(self):
        return dd_get_graph_counters(self.ctx)

    def tuning(self):
        return dd_get_tuning(self.ctx)

    def trace(self, part):
        return dd_get_trace(self.ctx, part, self.ncell[part])

    def set_tuning(self, threads, small_area, small_side, cl_size=None, cl_cells=None, sm_reserve=None):
        dd_set_tuning(self.ctx, threads, small_area, small_side, cl_size, cl_cells, sm_reserve)

    def autotune(self, cache_path=None):
        return dd_autotune(self.ctx, cache_path)

    def set_warmstart_weights(self, params):
        dd_set_warmstart_weights(self.ctx, params)

    def collect(self, part):
        return dd_collect_cells(self.ctx, part)

    def close(self):
        if self.ctx:
            dd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
