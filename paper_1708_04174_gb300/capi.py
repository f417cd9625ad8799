"""ctypes binding of libsos (include/sos.h): argument marshalling only.

Every step of the solver runs in the library (host setup in C++, iterations
in CUDA kernels).  This module only turns an ``instances.SOSProgram``-like
description into the C structs of the header and copies results out.  It
never falls back to anything else: if ``libsos.so`` is missing or fails to
load, every call raises.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import List, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsos.so")

SOS_OK = 0
SOS_ERR_INVALID_ARG, SOS_ERR_CUDA, SOS_ERR_FACTOR, SOS_ERR_TIMEOUT, SOS_ERR_UNSUPPORTED = -1, -2, -3, -4, -5
RUNNING, SOLVED, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, MAX_ITER, NUMERICAL = 0, 1, 2, 3, 4, 5
PREC_FP64, PREC_MIXED, PREC_FP32 = 0, 1, 2

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)


class sos_block(C.Structure):
    _fields_ = [("N", C.c_int32), ("basis_exps", _i32p), ("n_weight_terms", C.c_int32),
                ("weight_exps", _i32p), ("weight_coef", _f64p)]


class sos_constraint(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("row_exps", _i32p), ("n_terms", C.c_int64), ("term_poly", _i32p),
                ("term_exps", _i32p), ("term_coef", _f64p), ("n_blocks", C.c_int32),
                ("blocks", C.POINTER(sos_block)), ("matrix_r", C.c_int32), ("term_pair", _i32p)]


class sos_program(C.Structure):
    _fields_ = [("n_vars", C.c_int32), ("t", C.c_int32), ("w", _f64p), ("n_constraints", C.c_int32),
                ("constraints", C.POINTER(sos_constraint))]


class sos_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("k_check", C.c_int32), ("cuda_stream", C.c_void_p),
                ("solve_mode", C.c_int32), ("large_method", C.c_int32), ("warm_restart", C.c_int32),
                ("weighted_form", C.c_int32), ("infeas_tol", C.c_double), ("wait_limit_us", C.c_int32),
                ("reserved", C.c_int32)]


class sos_result(C.Structure):
    _fields_ = [("x", _f64p), ("y", _f64p), ("s", _f64p), ("res_primal", C.c_double), ("res_dual", C.c_double),
                ("gap", C.c_double), ("obj_primal", C.c_double), ("obj_dual", C.c_double), ("tau", C.c_double),
                ("kappa", C.c_double), ("iters", C.c_int32), ("status", C.c_int32)]


EXPORTS = {
    "sos_setup": (C.c_int, [C.POINTER(sos_program), C.c_int32, C.POINTER(sos_options), C.POINTER(C.c_void_p)]),
    "sos_destroy": (None, [C.c_void_p]),
    "sos_last_error": (C.c_char_p, [C.c_void_p]),
    "sos_dims": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
    "sos_solve": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.POINTER(sos_result)]),
    "sos_iterate": (C.c_int, [C.c_void_p, C.c_int32]),
    "sos_sync": (C.c_int, [C.c_void_p]),
    "sos_get_iterate": (C.c_int, [C.c_void_p, _f64p, _f64p]),
    "sos_set_iterate": (C.c_int, [C.c_void_p, _f64p, _f64p]),
    "sos_get_iterate_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sos_set_iterate_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sos_monomials": (C.c_int, [C.c_int32, C.c_int32, _i32p, C.c_int64, C.POINTER(C.c_int64)]),
    "sos_host_plan": (C.c_int, [C.POINTER(sos_program), C.c_int32, C.POINTER(C.c_int64), _i32p, _f64p, _f64p,
                                _f64p]),
    "sos_stream": (C.c_void_p, [C.c_void_p]),
    "sos_set_wait_limit": (C.c_int, [C.c_void_p, C.c_int32]),
    "sos_launches_per_iteration": (C.c_int, [C.c_void_p]),
    "sos_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "sos_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "sos_psd_project": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sos_psd_project_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sos_psd_project_mixed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sos_run_stage": (C.c_int, [C.c_void_p, C.c_int32]),
    "sos_stage_bytes": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
    "sos_mlp_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_void_p, C.POINTER(C.c_void_p)]),
    "sos_mlp_destroy": (None, [C.c_void_p]),
    "sos_mlp_param_count": (C.c_int64, [C.c_void_p]),
    "sos_mlp_set_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "sos_mlp_get_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "sos_mlp_fit_scaling": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "sos_mlp_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_float)]),
    "sos_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float,
                                     C.POINTER(C.c_double)]),
    "sos_mlp_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
}

_lib = None


def lib():
    """Loads libsos.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsos.so not found at {LIB_PATH}; build it with "
                               "`python -m paper_1708_04174_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _check(rc: int, handle=None):
    if rc != SOS_OK:
        msg = lib().sos_last_error(handle)
        raise RuntimeError(f"libsos error {rc}: {msg.decode() if msg else ''}")


def monomials(n: int, degree: int) -> np.ndarray:
    """Exponents of v_degree(x) in the graded order of eq. (4) (computed by libsos)."""
    cnt = C.c_int64(0)
    _check(lib().sos_monomials(n, degree, None, 0, C.byref(cnt)))
    out = np.zeros((cnt.value, n), dtype=np.int32)
    _check(lib().sos_monomials(n, degree, _ptr(out, C.c_int32), cnt.value, C.byref(cnt)))
    return out


class _Marshalled:
    """C structs for a list of programs; keeps every array alive."""

    def __init__(self, progs: Sequence):
        self.keep: List = []
        self.progs = (sos_program * len(progs))()
        cache = {}

        def mono(n, d, lo=0):
            # v_d without its monomials of degree < lo (same order)
            if (n, d, lo) not in cache:
                full = monomials(n, d)
                cache[(n, d, lo)] = np.ascontiguousarray(full[full.sum(axis=1) >= lo])
            return cache[(n, d, lo)]

        for pi, pg in enumerate(progs):
            n = pg.n

            def as_exps(e):
                return np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1, n))

            cons = (sos_constraint * len(pg.constraints))()
            for ci, con in enumerate(pg.constraints):
                if hasattr(con, "r"):
                    self._matrix(cons[ci], con, n, mono)
                    continue
                rows = as_exps(mono(n, con.degree, getattr(con, "min_degree", 0)))
                tp, te, tc = [], [], []
                arrays = getattr(con, "term_arrays", None)
                g0a = getattr(con, "g0_arrays", None)
                polys = ([] if g0a is not None else [con.g0]) + ([] if arrays is not None else list(con.g))
                base = 0 if g0a is None else 1  # index of the first polynomial in polys
                for k, poly in enumerate(polys):
                    for e, cval in poly.items():
                        tp.append(k + base)
                        te.append(e)
                        tc.append(cval)
                tp = np.array(tp, dtype=np.int32)
                te = np.array(te, dtype=np.int32).reshape(-1, n)
                tc = np.array(tc, dtype=np.float64)
                if g0a is not None:  # g_0 given as arrays
                    tp = np.concatenate([np.zeros(len(g0a[1]), dtype=np.int32), tp])
                    te = np.concatenate([np.asarray(g0a[0], dtype=np.int32).reshape(-1, n), te])
                    tc = np.concatenate([np.asarray(g0a[1], dtype=np.float64), tc])
                if arrays is not None:  # g_1..g_t given as flat term arrays
                    _, idx, exps, coef = arrays
                    tp = np.concatenate([tp, np.asarray(idx, dtype=np.int32) + 1])
                    te = np.concatenate([te, np.asarray(exps, dtype=np.int32).reshape(-1, n)])
                    tc = np.concatenate([tc, np.asarray(coef, dtype=np.float64)])
                tp = np.ascontiguousarray(tp)
                te = as_exps(te)
                tc = np.ascontiguousarray(tc)
                blks = (sos_block * len(con.blocks))()
                for bi, blk in enumerate(con.blocks):
                    bas = as_exps(mono(n, blk.basis_degree, getattr(blk, "min_degree", 0)))
                    blks[bi].N = bas.shape[0]
                    blks[bi].basis_exps = _ptr(bas, C.c_int32)
                    if blk.weight is not None:
                        we = as_exps(np.array(list(blk.weight.keys()), dtype=np.int32))
                        wc = np.ascontiguousarray(list(blk.weight.values()), dtype=np.float64)
                        blks[bi].n_weight_terms = len(wc)
                        blks[bi].weight_exps = _ptr(we, C.c_int32)
                        blks[bi].weight_coef = _ptr(wc, C.c_double)
                        self.keep += [we, wc]
                    else:
                        blks[bi].n_weight_terms = 0
                    self.keep.append(bas)
                cons[ci].n_rows = rows.shape[0]
                cons[ci].row_exps = _ptr(rows, C.c_int32)
                cons[ci].n_terms = len(tp)
                cons[ci].term_poly = _ptr(tp, C.c_int32)
                cons[ci].term_exps = _ptr(te, C.c_int32)
                cons[ci].term_coef = _ptr(tc, C.c_double)
                cons[ci].n_blocks = len(con.blocks)
                cons[ci].blocks = blks
                self.keep += [rows, tp, te, tc, blks]
            w = np.ascontiguousarray(pg.w, dtype=np.float64)
            self.progs[pi].n_vars = n
            self.progs[pi].t = len(w)
            self.progs[pi].w = _ptr(w, C.c_double)
            self.progs[pi].n_constraints = len(pg.constraints)
            self.progs[pi].constraints = cons
            self.keep += [w, cons]


    def _matrix(self, out, con, n, mono):
        """sos_constraint of a matrix-valued constraint (Section V): the
        monomials alpha, the terms of every entry (i, j), i <= j, of P_0, P_1,
        ... with their pair, and the basis v of the block, all in x; libsos
        forms the row triples (alpha, i, j) itself."""
        al = mono(n, con.degree, con.min_degree)
        tp, te, tc, pairs = [], [], [], []
        for h, Ph in enumerate([con.P0] + list(con.P)):
            for (i, j) in con.pairs:
                for e, cval in Ph[i][j].items():
                    tp.append(h)
                    te.append(list(e))
                    tc.append(cval)
                    pairs.append((i, j))
        tp = np.ascontiguousarray(tp, dtype=np.int32)
        te = np.ascontiguousarray(np.array(te, dtype=np.int32).reshape(-1, n))
        tc = np.ascontiguousarray(tc, dtype=np.float64)
        pr = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1, 2))
        bas = np.ascontiguousarray(mono(n, con.block.basis_degree, con.block.min_degree))
        blks = (sos_block * 1)()
        blks[0].N = bas.shape[0]
        blks[0].basis_exps = _ptr(bas, C.c_int32)
        blks[0].n_weight_terms = 0
        out.n_rows = al.shape[0]
        out.row_exps = _ptr(al, C.c_int32)
        out.n_terms = len(tp)
        out.term_poly = _ptr(tp, C.c_int32)
        out.term_exps = _ptr(te, C.c_int32)
        out.term_coef = _ptr(tc, C.c_double)
        out.n_blocks = 1
        out.blocks = blks
        out.matrix_r = con.r
        out.term_pair = _ptr(pr, C.c_int32)
        self.keep += [al, tp, te, tc, pr, bas, blks]


def psd_project(in_ptr: int, out_ptr: int, N: int, stream: int = 0):
    """PSD projection of one packed symmetric matrix; device pointers."""
    _check(lib().sos_psd_project(C.c_void_p(in_ptr), C.c_void_p(out_ptr), N, C.c_void_p(stream) if stream else None))


MIXED_MAX_N = 112


def psd_project_mixed(in_ptr: int, out_ptr: int, N: int, stream: int = 0):
    """PSD projection of the mixed form: FP32 Jacobi plus an FP64-summed
    refinement for N <= MIXED_MAX_N, the tensor-core Newton-Schulz sign
    iteration above; device pointers."""
    _check(lib().sos_psd_project_mixed(C.c_void_p(in_ptr), C.c_void_p(out_ptr), N,
                                       C.c_void_p(stream) if stream else None))


NOALLOC_MAX_N = 256


def psd_project_noalloc(in_ptr: int, out_ptr: int, N: int, stream: int = 0):
    """sos_psd_project without any device allocation (fixed library scratch)."""
    _check(lib().sos_psd_project_noalloc(C.c_void_p(in_ptr), C.c_void_p(out_ptr), N,
                                         C.c_void_p(stream) if stream else None))


def host_plan(prog, weighted_form: int = 0):
    """Index map of one program as built by libsos's host setup (no GPU)."""
    m = _Marshalled([prog])
    dims = (C.c_int64 * 6)()
    _check(lib().sos_host_plan(m.progs, weighted_form, dims, None, None, None, None))
    nx, mm = dims[0], dims[1]
    ent = np.zeros(nx, dtype=np.int32)
    pd = np.zeros(mm)
    b = np.zeros(mm)
    zh = C.c_double(0)
    _check(lib().sos_host_plan(m.progs, weighted_form, dims, _ptr(ent, C.c_int32), _ptr(pd, C.c_double),
                               _ptr(b, C.c_double), C.byref(zh)))
    return {"dims": tuple(dims), "ent_row": ent, "p_diag": pd, "b": b, "zeta_h": zh.value}


class Solver:
    """One libsos handle over a batch of SOS programs (instances)."""

    def __init__(self, progs, precision: int = PREC_FP64, k_check: int = 10, stream=None, solve_mode: int = 0,
                 large_method: int = 0, warm_restart: int = 0, infeas_tol: float = 0.0, weighted_form: int = 0,
                 wait_limit_us: int = 0):
        if not isinstance(progs, (list, tuple)):
            progs = [progs]
        self.n_inst = len(progs)
        m = _Marshalled(progs)
        opts = sos_options()
        opts.precision = precision
        opts.k_check = k_check
        opts.cuda_stream = C.c_void_p(stream) if stream else None
        opts.solve_mode = solve_mode
        opts.large_method = large_method
        opts.warm_restart = warm_restart
        opts.infeas_tol = infeas_tol
        opts.weighted_form = weighted_form
        opts.wait_limit_us = wait_limit_us
        h = C.c_void_p()
        _check(lib().sos_setup(m.progs, len(progs), C.byref(opts), C.byref(h)))
        self.h = h
        self.precision = precision
        self.dims = [self._dims(i) for i in range(self.n_inst)]
        self.total = sum(d[0] + d[1] + 1 for d in self.dims)

    def _dims(self, i):
        d = (C.c_int64 * 6)()
        _check(lib().sos_dims(self.h, i, d), self.h)
        return tuple(d)

    def close(self):
        if getattr(self, "h", None):
            lib().sos_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self, iters: int):
        _check(lib().sos_iterate(self.h, iters), self.h)

    def sync(self):
        _check(lib().sos_sync(self.h), self.h)

    @property
    def stream(self) -> int:
        return lib().sos_stream(self.h) or 0

    def stats(self) -> dict:
        out = (C.c_int64 * 4)()
        _check(lib().sos_stats(self.h, out), self.h)
        return {"iterations": out[0], "blocks": out[1], "max_sweeps": out[2], "total_sweeps": out[3]}

    def tuning(self) -> dict:
        out = (C.c_int32 * 5)()
        _check(lib().sos_tuning(self.h, out), self.h)
        return {"persistent": out[0], "grid": out[1], "dynamic": out[2], "candidates": out[3],
                "us_per_iter": out[4]}

    def launches_per_iteration(self) -> int:
        return int(lib().sos_launches_per_iteration(self.h))

    def stage_bytes(self, stage: int) -> int:
        """Algorithmic bytes of one launch of a profiling stage."""
        out = C.c_int64()
        _check(lib().sos_stage_bytes(self.h, stage, C.byref(out)), self.h)
        return int(out.value)

    def run_stage(self, stage: int):
        _check(lib().sos_run_stage(self.h, stage), self.h)

    def set_wait_limit(self, us: int):
        """Bound of the grid-wide device waits, microseconds (0: about 2 s)."""
        _check(lib().sos_set_wait_limit(self.h, us), self.h)

    def get_iterate(self, out=None):
        """sos_get_iterate into new arrays, or into ``out = (u, v)``
        (contiguous float64 host arrays of ``self.total``, e.g. views of
        pinned memory)."""
        if out is None:
            u = np.zeros(self.total)
            v = np.zeros(self.total)
        else:
            u, v = out
            assert all(a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and a.shape == (self.total,)
                       for a in (u, v))
        _check(lib().sos_get_iterate(self.h, _ptr(u, C.c_double), _ptr(v, C.c_double)), self.h)
        return u, v

    def set_iterate(self, u: np.ndarray, v: np.ndarray):
        u = np.ascontiguousarray(u, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        assert u.shape == (self.total,) and v.shape == (self.total,)
        _check(lib().sos_set_iterate(self.h, _ptr(u, C.c_double), _ptr(v, C.c_double)), self.h)

    def get_iterate_device(self, u_ptr: int, v_ptr: int):
        """sos_get_iterate_device: u_ptr, v_ptr are device addresses of
        ``self.total`` doubles each; asynchronous on ``self.stream``."""
        _check(lib().sos_get_iterate_device(self.h, C.c_void_p(u_ptr), C.c_void_p(v_ptr)), self.h)

    def set_iterate_device(self, u_ptr: int, v_ptr: int):
        """sos_set_iterate_device: device addresses as above; asynchronous on
        ``self.stream``."""
        _check(lib().sos_set_iterate_device(self.h, C.c_void_p(u_ptr), C.c_void_p(v_ptr)), self.h)

    def split(self, vec: np.ndarray):
        """Per-instance (xi, y, tau) slices of a concatenated iterate."""
        out, pos = [], 0
        for d in self.dims:
            nx, mm = d[0], d[1]
            out.append((vec[pos:pos + nx], vec[pos + nx:pos + nx + mm], vec[pos + nx + mm]))
            pos += nx + mm + 1
        return out

    def solve(self, tol: float, max_iter: int, want_solution: bool = True):
        res = (sos_result * self.n_inst)()
        bufs = []
        for i, d in enumerate(self.dims):
            if want_solution:
                x, y, s = np.zeros(d[0]), np.zeros(d[1]), np.zeros(d[0])
                res[i].x, res[i].y, res[i].s = _ptr(x, C.c_double), _ptr(y, C.c_double), _ptr(s, C.c_double)
                bufs.append((x, y, s))
            else:
                bufs.append((None, None, None))
        _check(lib().sos_solve(self.h, tol, max_iter, res), self.h)
        out = []
        for i in range(self.n_inst):
            r = res[i]
            out.append({"status": r.status, "iters": r.iters, "res_primal": r.res_primal, "res_dual": r.res_dual,
                        "gap": r.gap, "obj_primal": r.obj_primal, "obj_dual": r.obj_dual, "tau": r.tau,
                        "kappa": r.kappa, "x": bufs[i][0], "y": bufs[i][1], "s": bufs[i][2]})
        return out


class MLP:
    """Warm-start network (tensor-core kernels of libsos).  Data arguments are
    device pointers (e.g. ``tensor.data_ptr()`` of contiguous float32 CUDA
    tensors); parameters and gradients are host float32 arrays."""

    def __init__(self, n_in: int, n_hidden: int, n_out: int, seed: int = 0, stream: int = 0):
        h = C.c_void_p()
        _check(lib().sos_mlp_create(n_in, n_hidden, n_out, seed, C.c_void_p(stream) if stream else None, C.byref(h)))
        self.h = h
        self.shape = (n_in, n_hidden, n_out)
        self.n_param = int(lib().sos_mlp_param_count(h))

    def close(self):
        if getattr(self, "h", None):
            lib().sos_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.n_param
        _check(lib().sos_mlp_set_params(self.h, _ptr(flat, C.c_float)))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_param, dtype=np.float32)
        _check(lib().sos_mlp_get_params(self.h, _ptr(out, C.c_float)))
        return out

    def fit_scaling(self, Y_ptr: int, rows: int):
        _check(lib().sos_mlp_fit_scaling(self.h, C.c_void_p(Y_ptr), rows))

    def gradients(self, X_ptr: int, Y_ptr: int, batch: int):
        loss = C.c_double(0)
        g = np.zeros(self.n_param, dtype=np.float32)
        _check(lib().sos_mlp_gradients(self.h, C.c_void_p(X_ptr), C.c_void_p(Y_ptr), batch, C.byref(loss),
                                       _ptr(g, C.c_float)))
        return loss.value, g

    def train_step(self, X_ptr: int, Y_ptr: int, batch: int, lr: float, want_loss: bool = False):
        loss = C.c_double(0)
        _check(lib().sos_mlp_train_step(self.h, C.c_void_p(X_ptr), C.c_void_p(Y_ptr), batch, lr,
                                        C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def predict(self, X_ptr: int, Y_ptr: int, batch: int):
        _check(lib().sos_mlp_predict(self.h, C.c_void_p(X_ptr), C.c_void_p(Y_ptr), batch))
