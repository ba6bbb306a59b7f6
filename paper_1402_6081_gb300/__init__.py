"""GB300-native LGF fast multipole solver (Liska & Colonius, "A parallel fast
multipole method for elliptic difference equations").

Thin Python binding of the C ABI in include/lgf.h: the functions below carry the
same names and only marshal arguments (NumPy arrays, torch CUDA tensors, CUDA
streams) into the library; every step of a solve runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing, importing a
function raises.  Build it with ``paper_1402_6081_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes
import pathlib

import numpy as np

LGF_OK = 0
LGF_FP64 = 0
LGF_FP32 = 1
LGF_INTERP_NATIVE = 0
LGF_INTERP_BF16 = 1
LGF_INTERP_FP16 = 2
LGF_INTERP_BF16X3 = 3
LGF_INTERP_COMPENSATED = 4
LGF_INTERP_PLAIN = 5

_STATUS = {0: "LGF_OK", 1: "LGF_ERR_INVALID_ARG", 2: "LGF_ERR_UNSUPPORTED", 3: "LGF_ERR_OOM",
           4: "LGF_ERR_CUDA", 5: "LGF_ERR_TIMEOUT", 6: "LGF_ERR_BUDGET"}

LIB_PATH = pathlib.Path(__file__).resolve().parent / "_build" / "liblgf.so"

# every entry point of include/lgf.h with its ctypes signature
_SIGS = {
    "lgf_plan_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "lgf_plan_create_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "lgf_plan_create_multi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "lgf_plan_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lgf_plan_workspace_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "lgf_plan_points": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "lgf_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lgf_solve_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p]),
    "lgf_solve_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lgf_solve_host_pipelined": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                ctypes.c_void_p]),
    "lgf_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "lgf_batch_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lgf_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "lgf_plan_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "lgf_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32]),
    "lgf_measure_fma_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]),
    "lgf_plan_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "lgf_plan_timings": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lgf_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "lgf_conv_blocks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_void_p]),
    "lgf_solve_blocks_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "lgf_noalloc_max_blocks": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "lgf_last_error": (ctypes.c_char_p, []),
    "lgf_green_values": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "lgf_interp_weights": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "lgf_lebesgue_constant": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "lgf_select_interp": (ctypes.c_int, [ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


class LgfError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


def library() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_1402_6081_gb300.build.build())")
        h = ctypes.CDLL(str(LIB_PATH))
        for name, (res, args) in _SIGS.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def _check(status: int, where: str):
    if status != LGF_OK:
        raise LgfError(status, where, library().lgf_last_error().decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


def _dev_ptr(t) -> int:
    if hasattr(t, "data_ptr"):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("expected a contiguous CUDA tensor")
        return t.data_ptr()
    return int(t)


def lgf_last_error() -> str:
    return library().lgf_last_error().decode()


MAX_LEVELS = 24


class lgf_plan_options(ctypes.Structure):
    _fields_ = [("fft_size_interval", ctypes.c_int32), ("near_kernel", ctypes.c_int32),
                ("interval_kernel", ctypes.c_int32), ("single_stream", ctypes.c_int32),
                ("separate_level1", ctypes.c_int32), ("free_sms", ctypes.c_int32),
                ("fft_kernel", ctypes.c_int32), ("level_order", ctypes.c_int32 * 8),
                ("symmetric_spectra", ctypes.c_int32), ("mac_groups_per_cta", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 7)]


class lgf_plan_stats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_blocks", ctypes.c_int64),
                ("n_levels", ctypes.c_int32), ("top_product_level", ctypes.c_int32),
                ("fft_size_level0", ctypes.c_int32), ("fft_size_interval", ctypes.c_int32),
                ("pairs", ctypes.c_int64 * (MAX_LEVELS + 1)),
                ("intervals", ctypes.c_int64 * (MAX_LEVELS + 1)),
                ("groups", ctypes.c_int64 * (MAX_LEVELS + 1)),
                ("nw", ctypes.c_int64 * (MAX_LEVELS + 1)),
                ("workspace_bytes", ctypes.c_int64), ("merged_level01", ctypes.c_int32),
                ("n_problems", ctypes.c_int32), ("persistent_ctas", ctypes.c_int32),
                ("fft_kernel", ctypes.c_int32), ("compensated_interp", ctypes.c_int32)]


def lgf_plan_create(blocks, n_b: int, n_levels: int, interp_order: int,
                    precision: int = LGF_FP32, interp_mode: int = LGF_INTERP_NATIVE) -> int:
    """Plan for the block list ``blocks`` ((n, 3) block indices); returns the handle."""
    b = np.ascontiguousarray(np.asarray(blocks, dtype=np.int32).reshape(-1, 3))
    out = ctypes.c_void_p()
    _check(library().lgf_plan_create(b.ctypes.data, len(b), n_b, n_levels, interp_order,
                                     precision, interp_mode, ctypes.byref(out)), "lgf_plan_create")
    return out.value


def lgf_plan_create_ex(blocks, n_b: int, n_levels: int, interp_order: int,
                       precision: int = LGF_FP32, interp_mode: int = LGF_INTERP_NATIVE,
                       fft_size_interval: int = 0, near_kernel: int = 0, interval_kernel: int = 0,
                       single_stream: int = 0, separate_level1: int = 0, free_sms: int = 0,
                       fft_kernel: int = 0, level_orders=None, symmetric_spectra: int = 0,
                       mac_groups_per_cta: int = 0) -> int:
    """lgf_plan_create with tuning options (0 = default); level_orders maps a
    parent level (2..9) to the interpolation order between it and the level
    below (the level_order option)."""
    b = np.ascontiguousarray(np.asarray(blocks, dtype=np.int32).reshape(-1, 3))
    opts = _options(fft_size_interval, near_kernel, interval_kernel, single_stream, separate_level1, free_sms,
                    fft_kernel, level_orders, symmetric_spectra, mac_groups_per_cta)
    out = ctypes.c_void_p()
    _check(library().lgf_plan_create_ex(b.ctypes.data, len(b), n_b, n_levels, interp_order, precision,
                                        interp_mode, ctypes.byref(opts), ctypes.byref(out)),
           "lgf_plan_create_ex")
    return out.value


def _options(fft_size_interval=0, near_kernel=0, interval_kernel=0, single_stream=0, separate_level1=0,
             free_sms=0, fft_kernel=0, level_orders=None, symmetric_spectra=0, mac_groups_per_cta=0):
    opts = lgf_plan_options()
    opts.symmetric_spectra = symmetric_spectra
    opts.mac_groups_per_cta = mac_groups_per_cta
    for lvl, order in (level_orders or {}).items():
        if not 2 <= int(lvl) <= 9:
            raise ValueError("level_orders keys are parent levels 2..9")
        opts.level_order[int(lvl) - 2] = int(order)
    opts.free_sms = free_sms
    opts.fft_kernel = fft_kernel
    opts.fft_size_interval = fft_size_interval
    opts.near_kernel = near_kernel
    opts.interval_kernel = interval_kernel
    opts.single_stream = single_stream
    opts.separate_level1 = separate_level1
    return opts


def lgf_plan_create_multi(blocks_list, n_b: int, n_levels_list, interp_order: int,
                          precision: int = LGF_FP32, interp_mode: int = LGF_INTERP_NATIVE, **options) -> int:
    """One plan over several independent problems (see include/lgf.h): f and u
    hold the problems' blocks back to back in list order."""
    parts = [np.asarray(b, dtype=np.int32).reshape(-1, 3) for b in blocks_list]
    b = np.ascontiguousarray(np.concatenate(parts, axis=0))
    offs = np.zeros(len(parts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(p) for p in parts])
    lv = np.ascontiguousarray(np.asarray(n_levels_list, dtype=np.int32))
    if len(lv) != len(parts):
        raise ValueError("one level count per problem")
    opts = _options(**options)
    out = ctypes.c_void_p()
    _check(library().lgf_plan_create_multi(b.ctypes.data, offs.ctypes.data, lv.ctypes.data, len(parts), n_b,
                                           interp_order, precision, interp_mode, ctypes.byref(opts),
                                           ctypes.byref(out)), "lgf_plan_create_multi")
    return out.value


def lgf_plan_get_stats(plan: int) -> dict:
    st = lgf_plan_stats()
    _check(library().lgf_plan_get_stats(plan, ctypes.byref(st)), "lgf_plan_get_stats")
    L = st.n_levels
    return {"n_points": st.n_points, "n_blocks": st.n_blocks, "n_levels": L,
            "top_product_level": st.top_product_level, "fft_size_level0": st.fft_size_level0,
            "fft_size_interval": st.fft_size_interval, "pairs": list(st.pairs[: L + 1]),
            "intervals": list(st.intervals[: L + 1]), "groups": list(st.groups[: L + 1]),
            "nw": list(st.nw[: L + 1]), "workspace_bytes": st.workspace_bytes,
            "merged_level01": st.merged_level01, "n_problems": st.n_problems,
            "persistent_ctas": st.persistent_ctas, "fft_kernel": st.fft_kernel,
            "compensated_interp": st.compensated_interp}


def lgf_plan_workspace_bytes(plan: int) -> int:
    v = ctypes.c_size_t()
    _check(library().lgf_plan_workspace_bytes(plan, ctypes.byref(v)), "lgf_plan_workspace_bytes")
    return v.value


def lgf_plan_points(plan: int) -> int:
    v = ctypes.c_int64()
    _check(library().lgf_plan_points(plan, ctypes.byref(v)), "lgf_plan_points")
    return v.value


def lgf_solve(plan: int, f, u, stream=None) -> None:
    """u = G * f on the plan's blocks; f, u contiguous CUDA tensors (or device
    addresses) of the plan precision; asynchronous on ``stream``."""
    _check(library().lgf_solve(plan, _dev_ptr(f), _dev_ptr(u), _stream_ptr(stream)), "lgf_solve")


def lgf_solve_batch(plans, fs, us, stream=None) -> None:
    n = len(plans)
    P = (ctypes.c_void_p * n)(*plans)
    F = (ctypes.c_void_p * n)(*[_dev_ptr(f) for f in fs])
    U = (ctypes.c_void_p * n)(*[_dev_ptr(u) for u in us])
    _check(library().lgf_solve_batch(P, F, U, n, _stream_ptr(stream)), "lgf_solve_batch")


def lgf_batch_create(plans, fs, us, use_graph: int = 1) -> int:
    """Batch of independent solves (see include/lgf.h); returns the handle."""
    n = len(plans)
    P = (ctypes.c_void_p * n)(*plans)
    F = (ctypes.c_void_p * n)(*[_dev_ptr(f) for f in fs])
    U = (ctypes.c_void_p * n)(*[_dev_ptr(u) for u in us])
    out = ctypes.c_void_p()
    _check(library().lgf_batch_create(P, F, U, n, use_graph, ctypes.byref(out)), "lgf_batch_create")
    return out.value


def lgf_batch_launch(batch: int, stream=None) -> None:
    _check(library().lgf_batch_launch(batch, _stream_ptr(stream)), "lgf_batch_launch")


def lgf_batch_destroy(batch: int) -> None:
    _check(library().lgf_batch_destroy(batch), "lgf_batch_destroy")


def lgf_solve_host(plan: int, f_host, u_host, stream=None) -> None:
    """Solve with host buffers (NumPy arrays or CPU tensors, pinned preferred)."""
    fp = f_host.data_ptr() if hasattr(f_host, "data_ptr") else f_host.ctypes.data
    up = u_host.data_ptr() if hasattr(u_host, "data_ptr") else u_host.ctypes.data
    _check(library().lgf_solve_host(plan, fp, up, _stream_ptr(stream)), "lgf_solve_host")


def lgf_solve_host_pipelined(plan: int, f_hosts, u_hosts, stream=None) -> None:
    """Solves of one plan over sequences of host buffers (equal lengths; NumPy
    arrays or CPU tensors, pinned preferred), copies overlapped with the solves
    inside the library; returns with every result in host memory."""
    if len(f_hosts) != len(u_hosts):
        raise ValueError("f_hosts and u_hosts must have the same length")
    ptr = lambda a: a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
    n = len(f_hosts)
    fa = (ctypes.c_void_p * max(n, 1))(*[ptr(a) for a in f_hosts])
    ua = (ctypes.c_void_p * max(n, 1))(*[ptr(a) for a in u_hosts])
    _check(library().lgf_solve_host_pipelined(plan, fa, ua, n, _stream_ptr(stream)), "lgf_solve_host_pipelined")


def lgf_selftest_bounded_wait(complete: int, limit_us: int) -> None:
    """Run one bounded device wait (see include/lgf.h); raises LgfError with
    LGF_ERR_TIMEOUT when it runs out."""
    _check(library().lgf_selftest_bounded_wait(complete, limit_us), "lgf_selftest_bounded_wait")


def lgf_plan_sync(plan: int) -> None:
    _check(library().lgf_plan_sync(plan), "lgf_plan_sync")


def lgf_plan_set_timing(plan: int, capacity: int) -> None:
    _check(library().lgf_plan_set_timing(plan, capacity), "lgf_plan_set_timing")


def lgf_plan_timings(plan: int):
    """{kernel name: (total_ms, launches)} since the last call, and the kernel
    launches of the last solve."""
    mx = 64
    n = ctypes.c_int32()
    names = ctypes.create_string_buffer(32 * mx)
    tot = (ctypes.c_double * mx)()
    cnt = (ctypes.c_int32 * mx)()
    per = ctypes.c_int32()
    _check(library().lgf_plan_timings(plan, mx, ctypes.byref(n), names, tot, cnt, ctypes.byref(per)),
           "lgf_plan_timings")
    out = {}
    for j in range(min(n.value, mx)):
        nm = names.raw[32 * j: 32 * (j + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (tot[j], cnt[j])
    return out, per.value


def lgf_measure_fma_peak(kind: int, reps: int = 5) -> tuple[float, float]:
    """(flop/s, ms) of the best of reps all-SM FMA launches: kind 0 FP64,
    1 FP32, 2 packed FP32 pairs (see include/lgf.h)."""
    r, ms = ctypes.c_double(), ctypes.c_double()
    _check(library().lgf_measure_fma_peak(kind, reps, ctypes.byref(r), ctypes.byref(ms)), "lgf_measure_fma_peak")
    return r.value, ms.value


def lgf_conv_blocks(f, u, n_blocks: int, n_b: int, precision: int, stream=None) -> None:
    """FFT convolution of every block as its own one-block domain, in one kernel."""
    _check(library().lgf_conv_blocks(_dev_ptr(f), _dev_ptr(u), n_blocks, n_b, precision, _stream_ptr(stream)),
           "lgf_conv_blocks")


def lgf_solve_blocks_noalloc(f, u, n_blocks: int, n_b: int, precision: int, stream=None) -> None:
    """Isolated one-block solves with no device allocation (see include/lgf.h)."""
    _check(library().lgf_solve_blocks_noalloc(_dev_ptr(f), _dev_ptr(u), n_blocks, n_b, precision,
                                              _stream_ptr(stream)), "lgf_solve_blocks_noalloc")


def lgf_noalloc_max_blocks(n_b: int, precision: int) -> int:
    v = ctypes.c_int64()
    _check(library().lgf_noalloc_max_blocks(n_b, precision, ctypes.byref(v)), "lgf_noalloc_max_blocks")
    return v.value


def lgf_destroy(plan: int) -> None:
    _check(library().lgf_destroy(plan), "lgf_destroy")


def lgf_green_values(n) -> np.ndarray:
    """The library's FP64 G(n) for integer triples n (..., 3)."""
    a = np.ascontiguousarray(np.asarray(n, dtype=np.int32).reshape(-1, 3))
    out = np.empty(len(a))
    _check(library().lgf_green_values(a.ctypes.data, len(a), out.ctypes.data), "lgf_green_values")
    return out.reshape(np.shape(n)[:-1])


def lgf_interp_weights(n_b: int, n_max: int) -> np.ndarray:
    W = np.empty((2, n_b + 1, n_b + 1))
    _check(library().lgf_interp_weights(n_b, n_max, W.ctypes.data), "lgf_interp_weights")
    return W


class Solver:
    """Owns one plan: ``Solver(blocks, n_b, n_levels, order, precision)(f) -> u``
    with f, u torch CUDA tensors of shape (n_blocks, n_b, n_b, n_b).

    The keyword options are those of ``lgf_plan_options`` in include/lgf.h
    (0 = the library's choice): the interval FFT length, the product-kernel
    forms, the stream use, the separate level-1 form, the SMs left beside the
    persistent products, and the level-0 FFT form.  ``interp_mode`` selects the
    Reg/Interp arithmetic of FP32 plans (native, BF16/FP16/BF16x3 on the
    tensor cores, or compensated FP32 sums)."""

    def __init__(self, blocks, n_b: int, n_levels: int, interp_order: int, precision: int = LGF_FP32,
                 fft_size_interval: int = 0, near_kernel: int = 0, interval_kernel: int = 0,
                 single_stream: int = 0, separate_level1: int = 0, interp_mode: int = LGF_INTERP_NATIVE,
                 free_sms: int = 0, fft_kernel: int = 0, level_orders=None, symmetric_spectra: int = 0,
                 mac_groups_per_cta: int = 0):
        self.n_b = n_b
        self.precision = precision
        self.n_blocks = int(np.asarray(blocks).reshape(-1, 3).shape[0])
        self.plan = lgf_plan_create_ex(blocks, n_b, n_levels, interp_order, precision, interp_mode,
                                       fft_size_interval=fft_size_interval, near_kernel=near_kernel,
                                       interval_kernel=interval_kernel, single_stream=single_stream,
                                       separate_level1=separate_level1, free_sms=free_sms,
                                       fft_kernel=fft_kernel, level_orders=level_orders,
                                       symmetric_spectra=symmetric_spectra, mac_groups_per_cta=mac_groups_per_cta)

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == LGF_FP64 else torch.float32

    def __call__(self, f, u=None, stream=None):
        import torch
        if u is None:
            u = torch.empty_like(f)
        if f.dtype != self.dtype or u.dtype != self.dtype:
            raise TypeError(f"expected {self.dtype} tensors")
        if f.numel() != self.n_blocks * self.n_b ** 3 or u.numel() != f.numel():
            raise ValueError("f/u size does not match the plan")
        lgf_solve(self.plan, f, u, stream)
        return u

    def stats(self) -> dict:
        return lgf_plan_get_stats(self.plan)

    def workspace_bytes(self) -> int:
        return lgf_plan_workspace_bytes(self.plan)

    def close(self):
        if self.plan:
            lgf_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent uneven solves run together.

    Problems sharing (n_b, order) go into one multi-problem plan
    (lgf_plan_create_multi), so each phase of the method is one launch for all
    of them; the plans of the different classes run concurrently on a stream
    pool and, with ``use_graph``, the whole batch is one CUDA graph
    (lgf_batch_create).  ``problems`` is a list of (blocks, n_b, n_levels,
    order); ``options`` maps n_b to plan options (e.g. from the autotuner)."""

    def __init__(self, problems, precision: int = LGF_FP32, use_graph: int = 1, options=None):
        import torch
        self.precision = precision
        dt = torch.float64 if precision == LGF_FP64 else torch.float32
        options = options or {}
        classes = {}
        for i, (blocks, n_b, n_levels, order) in enumerate(problems):
            classes.setdefault((n_b, order), []).append(i)
        self.plans, self.f, self.u = [], [], []
        self.where = [None] * len(problems)   # problem -> (class, first point, n points, shape)
        for c, ((n_b, order), idx) in enumerate(sorted(classes.items())):
            blocks = [problems[i][0] for i in idx]
            levels = [problems[i][2] for i in idx]
            plan = lgf_plan_create_multi(blocks, n_b, levels, order, precision, **options.get(n_b, {}))
            self.plans.append(plan)
            n = sum(int(np.asarray(b).reshape(-1, 3).shape[0]) for b in blocks) * n_b ** 3
            self.f.append(torch.zeros(n, dtype=dt, device="cuda"))
            self.u.append(torch.empty(n, dtype=dt, device="cuda"))
            at = 0
            for i in idx:
                nb_i = int(np.asarray(problems[i][0]).reshape(-1, 3).shape[0])
                self.where[i] = (c, at, nb_i * n_b ** 3, (nb_i, n_b, n_b, n_b))
                at += nb_i * n_b ** 3
        self.batch = lgf_batch_create(self.plans, self.f, self.u, use_graph)

    def f_view(self, i):
        c, at, n, shape = self.where[i]
        return self.f[c][at:at + n].view(shape)

    def u_view(self, i):
        c, at, n, shape = self.where[i]
        return self.u[c][at:at + n].view(shape)

    def set_sources(self, fs):
        for i, f in enumerate(fs):
            self.f_view(i).copy_(f if hasattr(f, "copy_") else __import__("torch").from_numpy(np.asarray(f)))

    def __call__(self, stream=None):
        lgf_batch_launch(self.batch, stream)

    def n_points(self) -> int:
        return sum(int(f.numel()) for f in self.f)

    def close(self):
        if self.batch:
            lgf_batch_destroy(self.batch)
            self.batch = None
        for p in self.plans:
            lgf_destroy(p)
        self.plans = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lgf_lebesgue_constant(n: int) -> float:
    """Lebesgue constant of n equally spaced nodes (host; see include/lgf.h)."""
    v = ctypes.c_double()
    _check(library().lgf_lebesgue_constant(n, ctypes.byref(v)), "lgf_lebesgue_constant")
    return v.value


def lgf_select_interp(eps: float, precision: int) -> dict:
    """Sec. 2.5's choice of n_max and n_b for a target error (host).  Returns
    {"n_max", "n_b", "lebesgue", "interp_err", "reached"}; reached is False
    when no supported block size (4..32) meets eps (the largest one tried is returned)."""
    nm, nb = ctypes.c_int32(), ctypes.c_int32()
    lam, err = ctypes.c_double(), ctypes.c_double()
    st = library().lgf_select_interp(eps, precision, ctypes.byref(nm), ctypes.byref(nb), ctypes.byref(lam),
                                     ctypes.byref(err))
    if st not in (LGF_OK, 2):
        _check(st, "lgf_select_interp")
    return {"n_max": nm.value, "n_b": nb.value, "lebesgue": lam.value, "interp_err": err.value,
            "reached": st == LGF_OK}
