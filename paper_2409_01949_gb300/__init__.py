"""Python binding of the GB300 multilevel ELM-FBPINN library (``libelmfb.so``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  The binding fails loudly when the compiled library is missing; there
is no CPU fallback.  Entry points carry the C names of ``include/elmfb.h``;
``Solver`` is a small object wrapper over them.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); pointers are
passed through unchanged and the library copies what it needs.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libelmfb.so")

# status codes (elmfb.h)
OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_STATE, ERR_NOT_CONVERGED, ERR_BREAKDOWN, \
    ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED = range(10)
FP64, FP32, MIXED, DF32, FP32_DF32 = 0, 1, 2, 3, 4
PLACE_CELL, PLACE_ENDPOINT = 0, 1
SOLVE_LSQR, SOLVE_PCG, SOLVE_FCG_GNN, SOLVE_QR = 0, 1, 2, 3
PREC_NONE, PREC_BLOCK_JACOBI, PREC_BJ_GNN, PREC_BJ_COARSE = 0, 1, 2, 3
MAX_LEVELS = 12
MAX_ROWSETS = 16
MAX_HOLES = 4
N_STAGES = 8
STAGE_NAMES = ["create", "cell_sort", "assemble", "gram", "precond_setup", "iterate", "eval",
               "assemble_total"]


class ElmfbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"elmfb error {code}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("dim", C.c_int), ("lo", C.c_double * 2), ("hi", C.c_double * 2),
                ("n_levels", C.c_int), ("levels", C.c_int * MAX_LEVELS), ("delta", C.c_double),
                ("placement", C.c_int), ("features", C.c_int), ("seed", C.c_uint64),
                ("weight_scale", C.c_double), ("precision", C.c_int), ("n_holes", C.c_int),
                ("holes", (C.c_double * 4) * MAX_HOLES), ("ansatz_omega", C.c_double)]


class RowSet(C.Structure):
    _fields_ = [("n", C.c_int64), ("points", C.c_void_p), ("rhs", C.c_void_p),
                ("c0", C.c_double), ("c1", C.c_double * 2), ("c2", C.c_double * 2),
                ("weight", C.c_double)]


class Sizes(C.Structure):
    _fields_ = [("n_columns", C.c_int64), ("n_rows", C.c_int64), ("n_subdomains", C.c_int64),
                ("nnz", C.c_int64), ("panel_rows", C.c_int64), ("n_cells", C.c_int64),
                ("n_gram_pairs", C.c_int64), ("gram_flops", C.c_double), ("features", C.c_int),
                ("n_levels", C.c_int),
                ("dim", C.c_int), ("precision", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("method", C.c_int), ("preconditioner", C.c_int), ("max_iter", C.c_int),
                ("atol", C.c_double), ("btol", C.c_double), ("shift", C.c_double),
                ("check_every", C.c_int), ("warm_start", C.c_int), ("refine", C.c_int),
                ("gram_shift", C.c_double), ("rcond", C.c_double), ("ntol", C.c_double),
                ("coarse_levels", C.c_int), ("autotune", C.c_int), ("graph", C.c_int),
                ("batch_shared", C.c_int), ("drop_tol", C.c_double)]


class BatchItem(C.Structure):
    _fields_ = [("cfg", Config), ("n_sets", C.c_int), ("sets", C.c_void_p), ("n_eval", C.c_int64),
                ("eval_points", C.c_void_p), ("eval_out", C.c_void_p), ("eval_ref", C.c_void_p),
                ("coeffs_out", C.c_void_p), ("opts", C.c_void_p)]


class BatchResult(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("rel_l2", C.c_double),
                ("e_l1", C.c_double), ("max_abs", C.c_double), ("total_ms", C.c_double),
                ("launches", C.c_int64), ("message", C.c_char * 160)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("residual_norm", C.c_double),
                ("normal_residual_norm", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double), ("precond_retries", C.c_int), ("rank", C.c_int),
                ("sigma_max", C.c_double), ("sigma_min", C.c_double),
                ("precond_dropped", C.c_int)]


class TuningEntry(C.Structure):
    _fields_ = [("precision", C.c_int), ("features", C.c_int), ("covering_panels", C.c_int),
                ("rows_log2", C.c_int), ("unit_rows", C.c_int), ("candidates", C.c_int * 3),
                ("ms", C.c_double * 3)]


_lib = None

# name -> (restype, argtypes)
_SIGNATURES = {
    "elmfb_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Config), C.c_void_p]),
    "elmfb_destroy": (None, [C.c_void_p]),
    "elmfb_last_error": (C.c_char_p, [C.c_void_p]),
    "elmfb_assemble": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(RowSet)]),
    "elmfb_get_sizes": (C.c_int, [C.c_void_p, C.POINTER(Sizes)]),
    "elmfb_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "elmfb_get_rows": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "elmfb_default_solve_opts": (None, [C.POINTER(SolveOpts)]),
    "elmfb_solve": (C.c_int, [C.c_void_p, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
    "elmfb_get_coeffs": (C.c_int, [C.c_void_p, C.c_void_p]),
    "elmfb_get_bidiagonal": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
    "elmfb_set_coeffs": (C.c_int, [C.c_void_p, C.c_void_p]),
    "elmfb_eval": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "elmfb_error_norms": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "elmfb_stage_times": (C.c_int, [C.c_void_p, C.c_void_p]),
    "elmfb_kernel_launches": (C.c_int64, [C.c_void_p]),
    "elmfb_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "elmfb_set_profiling_only": (C.c_int, [C.c_void_p, C.c_char_p]),
    "elmfb_set_profiling_stride": (C.c_int, [C.c_void_p, C.c_int]),
    "elmfb_trim_memory": (C.c_int, [C.c_int]),
    "elmfb_kernel_stats": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "elmfb_error_norms_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                            C.c_void_p]),
    "elmfb_compute_gram": (C.c_int, [C.c_void_p]),
    "elmfb_batch_solve": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "elmfb_gnn_num_weights": (C.c_int64, [C.c_void_p]),
    "elmfb_gnn_graph": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "elmfb_gnn_set_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "elmfb_gnn_get_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "elmfb_gnn_eval": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p]),
    "elmfb_gnn_infer": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "elmfb_gnn_train": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                  C.c_uint64, C.c_void_p]),
    "elmfb_get_gram": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "elmfb_tuning_table": (C.c_int, [C.c_int, C.c_void_p]),
}


def lib():
    """Load ``libelmfb.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        l = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


def _ptr(x):
    """(pointer, keepalive) for a numpy array or torch tensor (contiguous float64 / int64)."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr"):          # torch tensor
        if not x.is_contiguous():
            x = x.contiguous()
        return x.data_ptr(), x
    a = np.ascontiguousarray(x)
    return a.ctypes.data, a


def _check(h, rc, allow=(OK,)):
    if rc not in allow:
        msg = lib().elmfb_last_error(h).decode() if h else ""
        raise ElmfbError(rc, msg)
    return rc


def default_solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().elmfb_default_solve_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _set_holes(cfg, dim, holes):
    holes = list(holes or ())
    if len(holes) > MAX_HOLES:
        raise ValueError("too many holes")
    cfg.n_holes = len(holes)
    for k, (lo, hi) in enumerate(holes):
        for i in range(dim):
            cfg.holes[k][i] = float(lo[i])
            cfg.holes[k][2 + i] = float(hi[i])


def make_config(dim, lo, hi, levels, delta, features, seed=0, weight_scale=1.0, precision=FP64,
                placement=PLACE_CELL, holes=(), ansatz_omega=0.0) -> Config:
    cfg = Config()
    cfg.dim = dim
    for i in range(dim):
        cfg.lo[i] = float(lo[i])
        cfg.hi[i] = float(hi[i])
    if len(levels) > MAX_LEVELS:
        raise ValueError("too many levels")
    cfg.n_levels = len(levels)
    for i, n in enumerate(levels):
        cfg.levels[i] = int(n)
    cfg.delta = float(delta)
    cfg.placement = int(placement)
    cfg.features = int(features)
    cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    cfg.weight_scale = float(weight_scale)
    cfg.precision = int(precision)
    _set_holes(cfg, dim, holes)
    cfg.ansatz_omega = float(ansatz_omega)
    return cfg


def config_of(problem, precision=FP64) -> Config:
    place = PLACE_CELL if problem.placement == "cell" else PLACE_ENDPOINT
    return make_config(problem.dim, problem.lo, problem.hi, problem.levels, problem.delta,
                       problem.features, problem.seed, problem.weight_scale, precision, place,
                       getattr(problem, "holes", ()), getattr(problem, "ansatz_omega", 0.0))


def _rowsets(problem, keep):
    arr = (RowSet * (1 + len(problem.boundary)))()
    for i, rs in enumerate([problem.interior] + list(problem.boundary)):
        pts = np.ascontiguousarray(rs.points, dtype=np.float64)
        rhs = np.ascontiguousarray(rs.rhs, dtype=np.float64)
        keep += [pts, rhs]
        arr[i].n = pts.shape[0]
        arr[i].points = pts.ctypes.data
        arr[i].rhs = rhs.ctypes.data
        arr[i].c0 = float(rs.c0)
        for k in range(problem.dim):
            arr[i].c1[k] = float(rs.c1[k])
            arr[i].c2[k] = float(rs.c2[k])
        arr[i].weight = float(rs.weight or 0.0)
    keep.append(arr)
    return arr


def tuning_table():
    """The autotuner's choices so far: a list of dicts, one per shape class."""
    n = lib().elmfb_tuning_table(0, None)
    if n < 0:
        raise ElmfbError(-n, "tuning table")
    arr = (TuningEntry * max(n, 1))()
    n = lib().elmfb_tuning_table(n, arr)
    return [dict(precision=e.precision, features=e.features, covering_panels=e.covering_panels,
                 rows_log2=e.rows_log2, unit_rows=e.unit_rows, candidates=list(e.candidates),
                 ms=list(e.ms)) for e in arr[:n]]


def trim_memory(device: int = -1):
    """Release the device memory cached in the library's pool."""
    rc = lib().elmfb_trim_memory(device)
    if rc != OK:
        raise ElmfbError(rc, "trim_memory failed")


def batch_solve(problems, precision=FP32, n_workers=8, opts=None, evaluate=True, coeffs=False,
                item_opts=None):
    """Solve independent problems with elmfb_batch_solve; item_opts (a list
    with a SolveOpts or None per problem) overrides `opts` per instance.

    Returns (results, u_hat list, coefficient list)."""
    n = len(problems)
    items = (BatchItem * n)()
    keep = []
    outs, cos = [], []
    for i, P in enumerate(problems):
        items[i].cfg = config_of(P, precision)
        sets = _rowsets(P, keep)
        items[i].n_sets = len(sets)
        items[i].sets = C.cast(sets, C.c_void_p)
        if evaluate:
            X = np.ascontiguousarray(P.test_points, dtype=np.float64)
            ref = np.ascontiguousarray(P.exact(P.test_points), dtype=np.float64)
            out = np.zeros(X.shape[0])
            keep += [X, ref]
            items[i].n_eval = X.shape[0]
            items[i].eval_points = X.ctypes.data
            items[i].eval_out = out.ctypes.data
            items[i].eval_ref = ref.ctypes.data
            outs.append(out)
        if coeffs:
            a = np.zeros(P.n_columns)
            items[i].coeffs_out = a.ctypes.data
            cos.append(a)
        if item_opts is not None and item_opts[i] is not None:
            keep.append(item_opts[i])
            items[i].opts = C.cast(C.pointer(item_opts[i]), C.c_void_p)
    res = (BatchResult * n)()
    o = opts if opts is not None else default_solve_opts()
    rc = lib().elmfb_batch_solve(n, items, C.byref(o), n_workers, res)
    if rc not in (OK, ERR_NOT_CONVERGED):
        bad = [(i, r.status, r.message.decode(errors="replace")) for i, r in enumerate(res)
               if r.status not in (OK, ERR_NOT_CONVERGED)]
        raise ElmfbError(rc, f"batch solve failed: {len(bad)} instance(s), first {bad[:3]}")
    return list(res), outs, cos


class Solver:
    """One handle: create -> assemble -> solve -> eval."""

    def __init__(self, dim, lo, hi, levels: Sequence[int], delta: float, features: int,
                 seed: int = 0, weight_scale: float = 1.0, precision: int = FP64,
                 placement: int = PLACE_CELL, stream: Optional[int] = None, holes=(),
                 ansatz_omega: float = 0.0):
        cfg = make_config(dim, lo, hi, levels, delta, features, seed, weight_scale, precision,
                          placement, holes, ansatz_omega)
        self.h = C.c_void_p()
        self._keep = []
        _check(None, lib().elmfb_create(C.byref(self.h), C.byref(cfg), C.c_void_p(stream or 0)))
        self.dim = dim

    @classmethod
    def from_problem(cls, problem, precision=FP64, stream=None):
        place = PLACE_CELL if problem.placement == "cell" else PLACE_ENDPOINT
        return cls(problem.dim, problem.lo, problem.hi, problem.levels, problem.delta,
                   problem.features, problem.seed, problem.weight_scale, precision, place, stream,
                   getattr(problem, "holes", ()), getattr(problem, "ansatz_omega", 0.0))

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().elmfb_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- assemble -------------------------------------------------------------
    def assemble(self, sets):
        """sets: list of dicts(points, rhs, c0, c1, c2, weight); sets[0] = interior."""
        arr = (RowSet * len(sets))()
        keep = []
        for i, s in enumerate(sets):
            pts, kp = _ptr(s["points"])
            rhs, kr = _ptr(s["rhs"])
            keep += [kp, kr]
            arr[i].n = int(s["n"]) if "n" in s else int(len(s["rhs"]))
            arr[i].points = pts
            arr[i].rhs = rhs
            arr[i].c0 = float(s.get("c0", 0.0))
            for k in range(self.dim):
                arr[i].c1[k] = float(s.get("c1", (0.0, 0.0))[k])
                arr[i].c2[k] = float(s.get("c2", (0.0, 0.0))[k])
            arr[i].weight = float(s.get("weight") or 0.0)
        _check(self.h, lib().elmfb_assemble(self.h, len(sets), arr))

    def assemble_problem(self, problem):
        sets = []
        for rs in [problem.interior] + list(problem.boundary):
            sets.append(dict(points=np.ascontiguousarray(rs.points, dtype=np.float64),
                             rhs=np.ascontiguousarray(rs.rhs, dtype=np.float64),
                             c0=rs.c0, c1=rs.c1, c2=rs.c2, weight=rs.weight))
        self.assemble(sets)

    def sizes(self) -> Sizes:
        s = Sizes()
        _check(self.h, lib().elmfb_get_sizes(self.h, C.byref(s)))
        return s

    def params(self):
        s = self.sizes()
        W = np.zeros((s.n_columns, s.dim))
        b = np.zeros(s.n_columns)
        _check(self.h, lib().elmfb_get_params(self.h, W.ctypes.data, b.ctypes.data))
        return W, b

    def get_rows(self, rows):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        s = self.sizes()
        out = np.zeros((rows.size, s.n_columns))
        hh = np.zeros(rows.size)
        _check(self.h, lib().elmfb_get_rows(self.h, rows.ctypes.data, rows.size,
                                            out.ctypes.data, hh.ctypes.data))
        return out, hh

    # -- solve ----------------------------------------------------------------
    def solve(self, opts: Optional[SolveOpts] = None, **kw) -> SolveInfo:
        if opts is None:
            opts = default_solve_opts(**kw)
        info = SolveInfo()
        _check(self.h, lib().elmfb_solve(self.h, C.byref(opts), C.byref(info)),
               allow=(OK, ERR_NOT_CONVERGED))
        return info

    def bidiagonal(self):
        """(alpha, beta) of the last LSQR solve's Golub-Kahan bidiagonal."""
        k = C.c_int64()
        _check(self.h, lib().elmfb_get_bidiagonal(self.h, 0, None, None, C.byref(k)))
        n = k.value + 1
        al = np.zeros(n)
        be = np.zeros(n)
        _check(self.h, lib().elmfb_get_bidiagonal(self.h, n, al.ctypes.data, be.ctypes.data,
                                                  None))
        return al, be

    def coeffs(self):
        a = np.zeros(self.sizes().n_columns)
        _check(self.h, lib().elmfb_get_coeffs(self.h, a.ctypes.data))
        return a

    def set_coeffs(self, a):
        p, k = _ptr(np.ascontiguousarray(a, dtype=np.float64))
        _check(self.h, lib().elmfb_set_coeffs(self.h, p))

    # -- eval -----------------------------------------------------------------
    def eval(self, xs, out=None):
        xs_c = np.ascontiguousarray(xs, dtype=np.float64) if not hasattr(xs, "data_ptr") else xs
        n = xs_c.shape[0]
        if out is None:
            out = np.zeros(n)
        px, kx = _ptr(xs_c)
        po, ko = _ptr(out)
        _check(self.h, lib().elmfb_eval(self.h, px, n, po))
        return out

    def error_norms(self, u_hat, u_ref):
        out = np.zeros(3)
        pu, ku = _ptr(u_hat if hasattr(u_hat, "data_ptr") else np.ascontiguousarray(u_hat, dtype=np.float64))
        pr, kr = _ptr(u_ref if hasattr(u_ref, "data_ptr") else np.ascontiguousarray(u_ref, dtype=np.float64))
        n = int(u_hat.shape[0])
        _check(self.h, lib().elmfb_error_norms(self.h, pu, pr, n, out.ctypes.data))
        return {"rel_l2": out[0], "e_l1": out[1], "max_abs": out[2]}

    def stage_times(self):
        out = np.zeros(N_STAGES)
        _check(self.h, lib().elmfb_stage_times(self.h, out.ctypes.data))
        return dict(zip(STAGE_NAMES, out.tolist()))

    def compute_gram(self):
        _check(self.h, lib().elmfb_compute_gram(self.h))

    def gram_blocks(self, pairs):
        """pairs: sequence of (i, j) subdomain indices -> array (n, K, K)."""
        ij = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        K = self.sizes().features
        out = np.zeros((ij.shape[0], K, K))
        _check(self.h, lib().elmfb_get_gram(self.h, ij.shape[0], ij.ctypes.data, out.ctypes.data))
        return out

    # -- learned preconditioner ------------------------------------------------
    def gnn_graph(self):
        s = self.sizes()
        ne = C.c_int64()
        _check(self.h, lib().elmfb_gnn_graph(self.h, None, None, C.byref(ne)))
        off = np.zeros(s.n_subdomains + 1, dtype=np.int32)
        nb = np.zeros(max(ne.value, 1), dtype=np.int32)
        _check(self.h, lib().elmfb_gnn_graph(self.h, off.ctypes.data, nb.ctypes.data, None))
        return [nb[off[i]:off[i + 1]].copy() for i in range(s.n_subdomains)]

    def gnn_num_weights(self) -> int:
        return int(lib().elmfb_gnn_num_weights(self.h))

    def gnn_set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(self.h, lib().elmfb_gnn_set_weights(self.h, w.ctypes.data))

    def gnn_get_weights(self):
        w = np.zeros(self.gnn_num_weights(), dtype=np.float32)
        _check(self.h, lib().elmfb_gnn_get_weights(self.h, w.ctypes.data))
        return w

    def gnn_eval(self, x, t=None, wb=None, grad=False):
        x = np.ascontiguousarray(x, dtype=np.float32)
        B = x.shape[0]
        y = np.zeros_like(x)
        g = np.zeros(self.gnn_num_weights(), dtype=np.float32) if grad else None
        loss = C.c_double(0.0)
        tp = np.ascontiguousarray(t, dtype=np.float32) if t is not None else None
        wp = np.ascontiguousarray(wb, dtype=np.float32) if wb is not None else None
        _check(self.h, lib().elmfb_gnn_eval(self.h, B, x.ctypes.data,
                                            tp.ctypes.data if tp is not None else None,
                                            wp.ctypes.data if wp is not None else None,
                                            y.ctypes.data, g.ctypes.data if g is not None else None,
                                            C.byref(loss)))
        return y, g, loss.value

    def gnn_infer(self, x):
        """The network's forward pass as FCG applies it (bfloat16 operands on
        the tensor cores, FP32 accumulation); x [batch][n_subdomains][K]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros_like(x)
        _check(self.h, lib().elmfb_gnn_infer(self.h, x.shape[0], x.ctypes.data, y.ctypes.data))
        return y

    def gnn_train(self, rhs_list, solve_iters=30, epochs=20, lr=1e-3, seed=0):
        R = np.ascontiguousarray(np.asarray(rhs_list, dtype=np.float64))
        out = np.zeros(2)
        _check(self.h, lib().elmfb_gnn_train(self.h, R.shape[0], R.ctypes.data, solve_iters,
                                             epochs, lr, seed, out.ctypes.data))
        return out

    def kernel_launches(self) -> int:
        return int(lib().elmfb_kernel_launches(self.h))

    def set_profiling(self, on: bool = True):
        _check(self.h, lib().elmfb_set_profiling(self.h, 1 if on else 0))

    def set_profiling_only(self, kernel: str):
        """Time only the named kernel (names as kernel_stats() reports them)."""
        _check(self.h, lib().elmfb_set_profiling_only(self.h, kernel.encode()))

    def set_profiling_stride(self, stride: int):
        """Time only every stride-th launch of each profiled kernel."""
        _check(self.h, lib().elmfb_set_profiling_stride(self.h, int(stride)))

    def kernel_stats(self):
        """{name: (total_ms, launches, algorithmic bytes per launch)} of the timed kernels."""
        n = 32
        names = (C.c_char_p * n)()
        ms = np.zeros(n)
        cnt = np.zeros(n, dtype=np.int64)
        by = np.zeros(n)
        k = lib().elmfb_kernel_stats(self.h, n, names, ms.ctypes.data, cnt.ctypes.data,
                                     by.ctypes.data)
        if k < 0:
            _check(self.h, -k)
        return {names[i].decode(): (float(ms[i]), int(cnt[i]), float(by[i])) for i in range(k)}
