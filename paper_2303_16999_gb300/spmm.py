"""ctypes binding of the C ABI in ``include/spmm.h`` (argument marshalling only).

The functions ``spmm_plan_create``, ``spmm_pack_values``, ``spmm_run``,
``spmm_run_host``, ``spmm_batch_run``, ``spmm_get_status``,
``spmm_plan_get_info``, ``spmm_plan_get_array``, ``spmm_plan_destroy``,
``spmm_equal_partition`` and ``spmm_bucket_size`` carry the C names.  The
``Plan`` class wraps a plan handle for torch tensors: torch provides device
memory and streams only; every step of the product runs in the library's CUDA
kernels.  There is no CPU fallback: if ``_build/libspmm.so`` is missing this
module raises instead of computing anything.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libspmm.so")

# status codes
OK, ERR_ARG, ERR_SHAPE, ERR_PATTERN, ERR_CAPACITY, ERR_UNSUPPORTED, ERR_CUDA, ERR_OOM, \
    ERR_TIMEOUT, ERR_BUSY, ERR_NOT_PACKED = range(11)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_SHAPE", 3: "ERR_PATTERN", 4: "ERR_CAPACITY",
                5: "ERR_UNSUPPORTED", 6: "ERR_CUDA", 7: "ERR_OOM", 8: "ERR_TIMEOUT",
                9: "ERR_BUSY", 10: "ERR_NOT_PACKED"}
STATIC, DYNAMIC = 0, 1
F32, F16, BF16, E4M3 = 0, 1, 2, 3
KERNEL_AUTO, KERNEL_PLAIN, KERNEL_GATHER, KERNEL_TC = 0, 1, 2, 3
KERNELS = {"auto": 0, "plain": 1, "gather": 2, "tc": 3, "bgather": 4}
ARRAYS = {"row_ptr": 0, "col_idx": 1, "perm": 2, "items": 3, "grp_row0": 4, "grp_rows": 5,
          "grp_ebeg": 6, "ent_col": 7, "ent_tbeg": 8, "tile_row": 9, "blk_slot": 10,
          "blk_off": 11, "ws_row0": 12, "red": 13, "ent_cover": 14, "src_index": 15}

# exported symbols of include/spmm_serve.h
SERVE_EXPORTS = ["serve_create", "serve_register_weight", "serve_submit", "serve_wait",
                 "serve_stats", "serve_reset_stats", "serve_destroy", "serve_replay"]

# exported symbols of include/spmm.h (checked by the CPU test-suite)
EXPORTS = ["spmm_plan_create", "spmm_pack_values", "spmm_run", "spmm_run_host",
           "spmm_get_status", "spmm_plan_get_info", "spmm_plan_get_array",
           "spmm_plan_destroy", "spmm_equal_partition", "spmm_bucket_size", "spmm_batch_run",
           "spmm_last_error", "spmm_version", "spmm_gather_noalloc", "spmm_quantize_e4m3",
           "spmm_sddmm", "spmm_run_ell", "spmm_plan_set_wait", "spmm_tune", "spmm_tune_clear",
           "spmm_tune_size"]


class SpmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Pattern(ctypes.Structure):
    _fields_ = [("nnzb", ctypes.c_int64), ("brow", ctypes.c_void_p), ("bcol", ctypes.c_void_p)]


class DPattern(ctypes.Structure):
    _fields_ = [("d_nnzb", ctypes.c_void_p), ("d_brow", ctypes.c_void_p),
                ("d_bcol", ctypes.c_void_p)]


class PlanOpts(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("rows_per_group", ctypes.c_int32),
                ("max_per_item", ctypes.c_int32), ("host_only", ctypes.c_int32),
                ("transposed", ctypes.c_int32), ("col_tiles", ctypes.c_int32),
                ("groups", ctypes.c_int64), ("stage_geometry", ctypes.c_int32),
                ("dyn_chain", ctypes.c_int32), ("row_begin", ctypes.c_int64),
                ("row_end", ctypes.c_int64), ("k_splits", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("m", "k", "n_max", "nnzb", "nnzb_max")] + \
        [(n, ctypes.c_int32) for n in ("b", "mode", "w_dtype", "x_dtype", "kernel",
                                      "rows_per_group", "max_per_item")] + \
        [(n, ctypes.c_int64) for n in ("n_items", "n_groups", "n_entries", "n_tiles",
                                      "ws_rows", "n_reductions", "device_bytes")] + \
        [(n, ctypes.c_int32) for n in ("stage_geometry", "sddmm_form")] + \
        [(n, ctypes.c_int64) for n in ("row_begin", "row_end")] + \
        [(n, ctypes.c_int32) for n in ("col_tiles", "index_bytes")]


class TuneChoice(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("stage_geometry", ctypes.c_int32),
                ("rows_per_group", ctypes.c_int32), ("k_splits", ctypes.c_int32),
                ("col_tiles", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("choice", TuneChoice), ("best_us", ctypes.c_float),
                ("n_candidates", ctypes.c_int32), ("cand", TuneChoice * 8),
                ("cand_us", ctypes.c_float * 8)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_batch_n", ctypes.c_int64),
                ("inject_delay_us", ctypes.c_int32), ("inject_alloc_fail", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "admitted", "completed", "rejected",
                                              "failed", "queued", "in_flight", "launches")] + \
        [(n, ctypes.c_double) for n in ("mean_requests_per_launch", "mean_cols_per_launch",
                                        "p50_us", "p99_us", "mean_us", "max_us", "span_s",
                                        "throughput_rps", "tflops_nz")]


_lib = None


def lib():
    """Loads the native library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("native library %s is not built: run "
                               "`python -c \"import __graft_entry__ as g; g.build()\"`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        L.spmm_plan_create.argtypes = [i64, i64, i64, i32, i32, i32, i32, ctypes.POINTER(Pattern),
                                       i64, ctypes.POINTER(PlanOpts), ctypes.POINTER(vp)]
        L.spmm_pack_values.argtypes = [vp, vp, vp, vp]
        L.spmm_run.argtypes = [vp, vp, vp, ctypes.POINTER(DPattern), vp, i64, i64, vp, i64, vp]
        L.spmm_run_host.argtypes = [vp, vp, i64, i64, vp, i64, vp]
        L.spmm_get_status.argtypes = [vp, ctypes.POINTER(i32)]
        L.spmm_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        L.spmm_plan_get_array.argtypes = [vp, i32, vp, i64, ctypes.POINTER(i64)]
        L.spmm_plan_destroy.argtypes = [vp]
        L.spmm_plan_destroy.restype = None
        L.spmm_equal_partition.argtypes = [i64, i64, ctypes.POINTER(i64)]
        L.spmm_bucket_size.argtypes = [i64, i64, i64, i64, i64, i64]
        L.spmm_bucket_size.restype = i64
        L.spmm_batch_run.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(vp),
                                     ctypes.POINTER(i64), vp]
        L.spmm_gather_noalloc.argtypes = [i64, i64, i32, vp, vp, vp, i64, vp, vp, i64, i64, vp,
                                          i64, vp, vp]
        L.spmm_quantize_e4m3.argtypes = [i64, i32, i32, vp, vp, vp, vp]
        L.spmm_sddmm.argtypes = [vp, ctypes.POINTER(DPattern), vp, i64, vp, i64, i64, vp, i32,
                                 vp]
        L.spmm_run_ell.argtypes = [vp, vp, i32, vp, vp, i64, i64, vp, i64, vp]
        L.spmm_plan_set_wait.argtypes = [vp, i64, i32]
        L.spmm_tune.argtypes = [i64, i64, i64, i32, i32, i32, ctypes.POINTER(Pattern), vp, vp, vp,
                                i64, i32, vp, ctypes.POINTER(TuneResult)]
        L.spmm_tune_clear.restype = None
        L.spmm_tune_size.restype = i64
        L.spmm_last_error.restype = ctypes.c_char_p
        L.spmm_version.restype = ctypes.c_char_p
        L.serve_create.argtypes = [ctypes.POINTER(ServeConfig), ctypes.POINTER(vp)]
        L.serve_register_weight.argtypes = [vp, vp, ctypes.POINTER(i32)]
        L.serve_submit.argtypes = [vp, i32, vp, i64, vp, ctypes.POINTER(ctypes.c_uint64)]
        L.serve_wait.argtypes = [vp, ctypes.c_uint64, i64]
        L.serve_stats.argtypes = [vp, ctypes.POINTER(ServeStats)]
        L.serve_reset_stats.argtypes = [vp]
        L.serve_replay.argtypes = [vp, i64, vp, vp, vp, vp, vp, ctypes.POINTER(ServeStats)]
        L.serve_destroy.argtypes = [vp]
        L.serve_destroy.restype = None
        for name in EXPORTS + SERVE_EXPORTS:
            getattr(L, name)
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise SpmmError(status, lib().spmm_last_error().decode())
    return status


# --------------------------------------------------- C names, thin wrappers
def spmm_plan_create(m, k, n_max, b, mode, w_dtype, x_dtype, pattern, nnzb_max, opts):
    h = ctypes.c_void_p()
    _check(lib().spmm_plan_create(m, k, n_max, b, mode, w_dtype, x_dtype,
                                  ctypes.byref(pattern) if pattern is not None else None,
                                  nnzb_max, ctypes.byref(opts) if opts is not None else None,
                                  ctypes.byref(h)))
    return h


def spmm_pack_values(plan, d_values, d_scales, stream):
    return _check(lib().spmm_pack_values(plan, d_values, d_scales, stream))


def spmm_run(plan, d_values, d_scales, dpat, d_X, n, ldx, d_Y, ldy, stream):
    return _check(lib().spmm_run(plan, d_values, d_scales,
                                 ctypes.byref(dpat) if dpat is not None else None,
                                 d_X, n, ldx, d_Y, ldy, stream))


def spmm_run_host(plan, h_X, n, ldx, h_Y, ldy, stream):
    return _check(lib().spmm_run_host(plan, h_X, n, ldx, h_Y, ldy, stream))


def spmm_tune(m, k, b, brow, bcol, values, X, w_dtype=F16, x_dtype=None, scales=None, reps=7,
              stream=None):
    """Times the candidate launch configurations of this static product
    (device values / scales / X as torch tensors) and records the fastest
    for its (b, density, n) bucket; returns a dict with the choice and each
    candidate's median time."""
    x_dtype = w_dtype if x_dtype is None else x_dtype
    brow = np.ascontiguousarray(brow, dtype=np.int32)
    bcol = np.ascontiguousarray(bcol, dtype=np.int32)
    pat = Pattern(len(brow), brow.ctypes.data, bcol.ctypes.data)
    r = TuneResult()
    _check(lib().spmm_tune(m, k, X.shape[1], b, w_dtype, x_dtype, ctypes.byref(pat),
                           _ptr(values), _ptr(scales), _ptr(X), X.stride(0), reps,
                           _stream_handle(stream), ctypes.byref(r)))
    names = {v: k_ for k_, v in KERNELS.items()}
    def desc(c):
        return {"kernel": names.get(c.kernel, c.kernel), "stage_geometry": c.stage_geometry,
                "rows_per_group": c.rows_per_group, "k_splits": c.k_splits,
                "col_tiles": c.col_tiles}
    cands = [dict(desc(r.cand[i]), us=round(r.cand_us[i], 2)) for i in range(r.n_candidates)]
    return dict(desc(r.choice), best_us=round(r.best_us, 2), candidates=cands)


def spmm_tune_clear():
    lib().spmm_tune_clear()


def spmm_tune_size():
    return lib().spmm_tune_size()


def spmm_plan_set_wait(plan, limit_ns, stall):
    return _check(lib().spmm_plan_set_wait(plan, limit_ns, stall))


def spmm_get_status(plan):
    s = ctypes.c_int32()
    _check(lib().spmm_get_status(plan, ctypes.byref(s)))
    return s.value


def spmm_plan_get_info(plan):
    i = PlanInfo()
    _check(lib().spmm_plan_get_info(plan, ctypes.byref(i)))
    return {f: getattr(i, f) for f, _ in PlanInfo._fields_}


def spmm_plan_get_array(plan, name):
    which = ARRAYS[name]
    cnt = ctypes.c_int64()
    _check(lib().spmm_plan_get_array(plan, which, None, 0, ctypes.byref(cnt)))
    dt = np.int64 if name == "ws_row0" else np.int32
    out = np.zeros(cnt.value, dtype=dt)
    _check(lib().spmm_plan_get_array(plan, which, out.ctypes.data_as(ctypes.c_void_p),
                                     cnt.value, ctypes.byref(cnt)))
    return out


def spmm_plan_destroy(plan):
    lib().spmm_plan_destroy(plan)


def spmm_equal_partition(extent, q):
    out = (ctypes.c_int64 * q)()
    _check(lib().spmm_equal_partition(extent, q, out))
    return list(out)


def spmm_bucket_size(m, k, d_num, d_den, q_m, q_k):
    return lib().spmm_bucket_size(m, k, d_num, d_den, q_m, q_k)


def spmm_gather_noalloc(m, k, dtype, d_nnzb, d_brow, d_bcol, nnzb_max, d_values, d_X, n, ldx,
                        d_Y, ldy, d_status, stream):
    """The allocation-free dynamic b = 1 product (see include/spmm.h)."""
    return _check(lib().spmm_gather_noalloc(m, k, dtype, d_nnzb, d_brow, d_bcol, nnzb_max,
                                            d_values, d_X, n, ldx, d_Y, ldy, d_status, stream))


def spmm_quantize_e4m3(nnzb, b, src_dtype, d_src, d_codes, d_scales, stream):
    return _check(lib().spmm_quantize_e4m3(nnzb, b, src_dtype, d_src, d_codes, d_scales, stream))


def spmm_sddmm(plan, dpat, d_dY, lddy, d_X, ldx, n, d_dW, dw_dtype, stream):
    """The sampled product dW = (dY.X^T) on the plan's block mask (see include/spmm.h)."""
    return _check(lib().spmm_sddmm(plan, dpat, d_dY, lddy, d_X, ldx, n, d_dW, dw_dtype, stream))


def spmm_run_ell(plan, d_ell_cols, ell_width, d_values, d_X, n, ldx, d_Y, ldy, stream):
    """Y = W.X with W in Blocked-ELL form, b = 16 (see include/spmm.h)."""
    return _check(lib().spmm_run_ell(plan, d_ell_cols, ell_width, d_values, d_X, n, ldx, d_Y,
                                     ldy, stream))


def quantize_e4m3(values, stream=None):
    """E4M3 codes (torch.float8_e4m3fn) and FP32 per-block scales of device
    values shaped (nnzb, b, b), by the library's quantiser kernel."""
    import torch
    nnzb, b = values.shape[0], values.shape[1]
    codes = torch.empty(values.shape, dtype=torch.uint8, device=values.device)
    scales = torch.empty(nnzb, dtype=torch.float32, device=values.device)
    spmm_quantize_e4m3(nnzb, b, dtype_code(values.dtype), _ptr(values), _ptr(codes), _ptr(scales),
                       _stream_handle(stream))
    return codes.view(torch.float8_e4m3fn), scales


def spmm_version():
    return lib().spmm_version().decode()


# ------------------------------------------------------------- torch glue
def dtype_code(t):
    import torch
    return {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16,
            torch.float8_e4m3fn: E4M3}[t]


def torch_dtype(code):
    import torch
    return {F32: torch.float32, F16: torch.float16, BF16: torch.bfloat16,
            E4M3: torch.float8_e4m3fn}[code]


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Plan:
    """One SpMM plan.  Static: ``Plan(m, k, n_max, b, brow=..., bcol=...)``;
    dynamic: ``Plan(m, k, n_max, b, mode=DYNAMIC, nnzb_max=...)``.

    ``transposed=True``: the plan applies W^T for the m x k W that the pattern
    and values describe (in W's own coordinates); ``run(Y)`` then returns
    Z = W^T.Y (k x n) for Y (m x n), and ``self.m, self.k`` are k, m.

    ``col_tiles``: 128-column tiles of n per tensor-core CTA (0 automatic,
    1, or 2 where the launch allows it), as ``spmm_plan_opts.col_tiles``;
    ``groups``: near-equal tile-row groups, as ``spmm_plan_opts.groups``;
    ``stage_geometry``: 0 automatic, 1 dense-tile, 2 sparse-tile stages;
    ``dyn_chain``: dynamic TC plans re-partition through the launch chain
    instead of the one cooperative launch (identical results);
    ``rows=(row_begin, row_end)``: a static plan of that slice of the output
    rows (the pattern and values passed stay the whole W's; ``run`` returns
    the slice's rows only), as ``spmm_plan_opts.row_begin / row_end``."""

    def __init__(self, m, k, n_max, b, w_dtype=F16, x_dtype=None, brow=None, bcol=None,
                 mode=STATIC, nnzb_max=0, kernel="auto", rows_per_group=0, max_per_item=0,
                 host_only=False, transposed=False, col_tiles=0, groups=0, rows=None,
                 stage_geometry=0, dyn_chain=False, k_splits=0):
        x_dtype = w_dtype if x_dtype is None else x_dtype
        rb, re = rows if rows is not None else (0, 0)
        opts = PlanOpts(KERNELS[kernel] if isinstance(kernel, str) else kernel,
                        rows_per_group, max_per_item, 1 if host_only else 0,
                        1 if transposed else 0, col_tiles, groups, stage_geometry, 1 if dyn_chain else 0, rb, re,
                        k_splits)
        pat = None
        self._keep = None
        if mode == STATIC:
            brow = np.ascontiguousarray(brow, dtype=np.int32)
            bcol = np.ascontiguousarray(bcol, dtype=np.int32)
            self._keep = (brow, bcol)
            pat = Pattern(len(brow), brow.ctypes.data, bcol.ctypes.data)
        self.h = spmm_plan_create(m, k, n_max, b, mode, w_dtype, x_dtype, pat, nnzb_max, opts)
        if transposed:
            m, k = k, m                       # the operator the plan applies is k x m
        if rows is not None:
            m = re - rb                       # the plan writes its slice of rows only
        self.m, self.k, self.n_max, self.b = m, k, n_max, b
        self.transposed = transposed
        self.mode, self.w_dtype, self.x_dtype = mode, w_dtype, x_dtype

    def close(self):
        if self.h:
            spmm_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return spmm_plan_get_info(self.h)

    def array(self, name):
        return spmm_plan_get_array(self.h, name)

    def pack(self, values, scales=None, stream=None):
        spmm_pack_values(self.h, _ptr(values), _ptr(scales), _stream_handle(stream))

    def run(self, X, Y=None, values=None, scales=None, pattern=None, stream=None):
        """Y = W.X for device tensors; returns Y (allocated if not given)."""
        import torch
        n = X.shape[1]
        if Y is None:
            Y = torch.empty((self.m, n), dtype=X.dtype, device=X.device)
        dp = None
        if pattern is not None:
            d_nnzb, d_brow, d_bcol = pattern
            dp = DPattern(d_nnzb.data_ptr(), d_brow.data_ptr(), d_bcol.data_ptr())
        spmm_run(self.h, _ptr(values), _ptr(scales), dp, _ptr(X), n, X.stride(0), _ptr(Y),
                 Y.stride(0), _stream_handle(stream))
        return Y

    def run_host(self, X, Y, stream=None):
        """Same product with host (CPU, ideally pinned) X and Y."""
        spmm_run_host(self.h, ctypes.c_void_p(X.data_ptr()), X.shape[1], X.stride(0),
                      ctypes.c_void_p(Y.data_ptr()), Y.stride(0), _stream_handle(stream))
        return Y

    def status(self):
        return spmm_get_status(self.h)

    def set_wait(self, limit_ns=0, stall=False):
        """Limit of each device wait of the tensor-core launches (0: 2 s);
        stall=True is the failure-detection test hook (see spmm.h)."""
        spmm_plan_set_wait(self.h, int(limit_ns), 1 if stall else 0)

    def run_ell(self, ell_cols, values, X, Y=None, stream=None):
        """Y = W.X for W in Blocked-ELL form: ell_cols (m/16, E) int32 and
        values (m/16, E, 16, 16) device tensors (dynamic b = 16 plans)."""
        import torch
        n = X.shape[1]
        if Y is None:
            Y = torch.empty((self.m, n), dtype=X.dtype, device=X.device)
        width = ell_cols.shape[1] if ell_cols.dim() == 2 else 0
        spmm_run_ell(self.h, _ptr(ell_cols), width, _ptr(values), _ptr(X), n, X.stride(0),
                     _ptr(Y), Y.stride(0), _stream_handle(stream))
        return Y

    def sddmm(self, dY, X, dW=None, dw_dtype=None, pattern=None, capacity=None, stream=None):
        """dW = (dY.X^T) on the plan's block mask for device tensors dY (m x n)
        and X (k x n); returns dW (blocks, b, b) in the pattern's order
        (allocated if not given: nnzb blocks, or ``capacity`` / nnzb_max
        for dynamic plans).  dw_dtype defaults to FP32."""
        import torch
        if dW is None:
            want = torch.float32 if dw_dtype is None else dw_dtype
            if pattern is not None:
                blocks = capacity if capacity is not None else self.info()["nnzb_max"]
            else:
                blocks = self.info()["nnzb"]
            dW = torch.empty((blocks, self.b, self.b), dtype=want, device=dY.device)
        dp = None
        if pattern is not None:
            d_nnzb, d_brow, d_bcol = pattern
            dp = DPattern(d_nnzb.data_ptr(), d_brow.data_ptr(), d_bcol.data_ptr())
        spmm_sddmm(self.h, dp, _ptr(dY), dY.stride(0), _ptr(X), X.stride(0), X.shape[1],
                   _ptr(dW), dtype_code(dW.dtype), _stream_handle(stream))
        return dW


def spmm_batch_run(plans, Xs, Ys, stream=None):
    count = len(plans)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    hp = (vp * count)(*[p.h.value if hasattr(p.h, "value") else p.h for p in plans])
    xp = (vp * count)(*[x.data_ptr() for x in Xs])
    yp = (vp * count)(*[y.data_ptr() for y in Ys])
    ns = (i64 * count)(*[x.shape[1] for x in Xs])
    lx = (i64 * count)(*[x.stride(0) for x in Xs])
    ly = (i64 * count)(*[y.stride(0) for y in Ys])
    return _check(lib().spmm_batch_run(count, hp, xp, ns, lx, yp, ly, _stream_handle(stream)))


# ------------------------------------------------------------------ serving
class Server:
    """Serving loop of include/spmm_serve.h: resident weights, HBM-budget
    admission, continuous batching on ``max_inflight`` streams.  Requests
    pass host (CPU, preferably pinned) tensors X (k x n) and Y (m x n)."""

    def __init__(self, hbm_budget_bytes, max_inflight=2, max_batch=64, max_batch_n=4096,
                 inject_delay_us=0, inject_alloc_fail=0):
        cfg = ServeConfig(hbm_budget_bytes, max_inflight, max_batch, max_batch_n,
                          inject_delay_us, inject_alloc_fail)
        h = ctypes.c_void_p()
        _check(lib().serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self._plans = []
        self._live = {}

    def register(self, plan):
        w = ctypes.c_int32()
        _check(lib().serve_register_weight(self.h, plan.h, ctypes.byref(w)))
        self._plans.append(plan)
        return w.value

    def submit(self, weight_id, X, Y):
        t = ctypes.c_uint64()
        _check(lib().serve_submit(self.h, weight_id, ctypes.c_void_p(X.data_ptr()), X.shape[1],
                                  ctypes.c_void_p(Y.data_ptr()), ctypes.byref(t)))
        self._live[t.value] = (X, Y)        # keep the buffers alive until wait
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        st = lib().serve_wait(self.h, ticket, timeout_ms)
        if st != TIMEOUT_STATUS:
            self._live.pop(ticket, None)
        return _check(st)

    def stats(self):
        s = ServeStats()
        _check(lib().serve_stats(self.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServeStats._fields_}

    def reset_stats(self):
        _check(lib().serve_reset_stats(self.h))

    def replay(self, t_arrive_s, weight, n, x_ptrs, y_ptrs):
        """Native trace replay (serve_replay): arrival offsets in seconds,
        weight ids, column counts and host buffer addresses per request."""
        cnt = len(t_arrive_s)
        t = np.ascontiguousarray(t_arrive_s, dtype=np.float64)
        w = np.ascontiguousarray(weight, dtype=np.int32)
        nn = np.ascontiguousarray(n, dtype=np.int64)
        xp = np.ascontiguousarray(x_ptrs, dtype=np.uint64)
        yp = np.ascontiguousarray(y_ptrs, dtype=np.uint64)
        s = ServeStats()
        _check(lib().serve_replay(self.h, cnt, t.ctypes.data, w.ctypes.data, nn.ctypes.data,
                                  xp.ctypes.data, yp.ctypes.data, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServeStats._fields_}

    def close(self):
        if self.h:
            lib().serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TIMEOUT_STATUS = ERR_TIMEOUT
