"""ctypes binding of libfem.so (C ABI in include/fem.h), same names as the C calls.

Argument marshalling only: every step of counting and mining runs in the CUDA
kernels of the library.  Host data is passed as numpy arrays; device data as
PyTorch CUDA tensors (their ``data_ptr()``), with the current PyTorch stream
used unless another is given.  If the library has not been built, loading it
raises :class:`FemError` -- there is no CPU fallback.

Episode records are uint8 arrays of shape [m, 16] laid out like ``fem_episode``:
bytes 0..7 node types, 8..14 interval indices, 15 the length.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

MAX_LEN = 8
PASS_RELAXED, PASS_EXACT = 0, 1
STATUS = {0: "FEM_OK", -1: "FEM_EINVAL", -2: "FEM_EUNSORTED", -3: "FEM_ETYPE",
          -4: "FEM_ERANGE", -5: "FEM_ENOMEM", -6: "FEM_EADMIT", -7: "FEM_ETIMEOUT",
          -8: "FEM_ECUDA", -9: "FEM_EOVERFLOW", -10: "FEM_ENOSTREAM", -11: "FEM_EIO"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfem.so")


class FemError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        name = STATUS.get(status, str(status))
        super().__init__(f"{what}: {name}" if what else name)


class fem_interval(ctypes.Structure):
    _fields_ = [("lo_us", ctypes.c_uint32), ("hi_us", ctypes.c_uint32)]


class fem_config(ctypes.Structure):
    _fields_ = [("segments", ctypes.c_uint32), ("threads_per_block", ctypes.c_uint32),
                ("ring_capacity", ctypes.c_uint32), ("kernel", ctypes.c_uint32)]


KERNEL_AUTO, KERNEL_MACHINE, KERNEL_CHAIN, KERNEL_PAIRS = 0, 1, 2, 3


class fem_level_stats(ctypes.Structure):
    _fields_ = [("level", ctypes.c_uint32), ("candidates", ctypes.c_uint32),
                ("survivors", ctypes.c_uint32), ("frequent", ctypes.c_uint32),
                ("segments", ctypes.c_uint32), ("ms_generate", ctypes.c_float),
                ("ms_relaxed", ctypes.c_float), ("ms_compact", ctypes.c_float),
                ("ms_exact", ctypes.c_float), ("ms_relaxed_kernel", ctypes.c_float),
                ("ms_relaxed_stitch", ctypes.c_float), ("ms_exact_kernel", ctypes.c_float),
                ("exact_segments", ctypes.c_uint32), ("touched_relaxed", ctypes.c_uint64),
                ("touched_exact", ctypes.c_uint64), ("kernel_relaxed", ctypes.c_uint32),
                ("kernel_exact", ctypes.c_uint32)]


class fem_job(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int32), ("len", ctypes.c_uint32), ("m", ctypes.c_uint32),
                ("cands", ctypes.c_void_p), ("theta", ctypes.c_uint32),
                ("exact_out", ctypes.c_void_p), ("survived_out", ctypes.c_void_p)]


class fem_server_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_uint32),
                ("n_lanes", ctypes.c_uint32)]


REQ_ONESHOT, REQ_STANDING = 0, 1

EXPORTS = ["fem_create", "fem_destroy", "fem_mem_usage", "fem_append_stream", "fem_set_config", "fem_load_stream", "fem_free_stream",
           "fem_type_counts", "fem_capacity_table", "fem_count_candidates", "fem_count_two_pass",
           "fem_count_pairs_relaxed",
           "fem_mine_levelwise", "fem_result_level", "fem_result_max_level", "fem_result_free",
           "fem_last_mine_stats", "fem_strerror", "fem_kernel_launches", "fem_select_noalloc",
           "fem_batch_create", "fem_batch_run", "fem_batch_destroy",
           "fem_server_create", "fem_server_destroy", "fem_server_open_stream",
           "fem_server_append", "fem_server_submit", "fem_server_poll", "fem_server_result",
           "fem_server_release", "fem_server_drain", "fem_tune_enable", "fem_tune_size",
           "fem_tune_save", "fem_tune_load", "fem_count_mapconcat_literal",
           "fem_mine_levelwise_ex", "fem_count_windows"]

_lib = None


def load(path: str | None = None):
    """Load libfem.so (built by ``paper_0905_2200_gb300.build``); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise FemError(-8, f"libfem.so not built at {path}; run paper_0905_2200_gb300.build")
    lib = ctypes.CDLL(path)
    vp, u32, i32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64
    I = ctypes.c_int
    sig = {
        "fem_create": (I, [ctypes.POINTER(vp), I, ctypes.c_size_t]),
        "fem_mem_usage": (I, [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
        "fem_append_stream": (I, [vp, i32, vp, vp, u64, I, vp]),
        "fem_destroy": (I, [vp]),
        "fem_set_config": (I, [vp, ctypes.POINTER(fem_config)]),
        "fem_load_stream": (I, [vp, vp, vp, u64, u32, I, vp, ctypes.POINTER(i32)]),
        "fem_free_stream": (I, [vp, i32]),
        "fem_type_counts": (I, [vp, i32, vp]),
        "fem_capacity_table": (I, [vp, i32, vp, u32, vp]),
        "fem_count_pairs_relaxed": (I, [vp, i32, vp, u32, ctypes.POINTER(fem_interval), u32, vp]),
        "fem_count_candidates": (I, [vp, i32, vp, u32, I, ctypes.POINTER(fem_interval), u32, I,
                                     vp, I, vp]),
        "fem_count_two_pass": (I, [vp, i32, vp, u32, I, ctypes.POINTER(fem_interval), u32, u32,
                                   vp, vp, I, vp]),
        "fem_mine_levelwise": (I, [vp, i32, ctypes.POINTER(fem_interval), u32, u32, u32, vp,
                                   ctypes.POINTER(vp)]),
        "fem_mine_levelwise_ex": (I, [vp, i32, ctypes.POINTER(fem_interval), u32, u32, u32, u32,
                                      vp, ctypes.POINTER(vp)]),
        "fem_result_level": (I, [vp, u32, ctypes.POINTER(u32), ctypes.POINTER(vp),
                                 ctypes.POINTER(vp)]),
        "fem_result_max_level": (u32, [vp]),
        "fem_result_free": (None, [vp]),
        "fem_last_mine_stats": (I, [vp, ctypes.POINTER(fem_level_stats), u32]),
        "fem_strerror": (ctypes.c_char_p, [I]),
        "fem_count_mapconcat_literal": (I, [vp, i32, vp, u32, I, ctypes.POINTER(fem_interval),
                                            u32, u32, vp, I, ctypes.POINTER(u32), vp]),
        "fem_count_windows": (I, [vp, i32, vp, u32, I, ctypes.POINTER(fem_interval), u32, u32,
                                  vp, I, vp]),
        "fem_tune_enable": (I, [vp, I]),
        "fem_tune_size": (I, [vp, ctypes.POINTER(u32)]),
        "fem_tune_save": (I, [vp, ctypes.c_char_p]),
        "fem_tune_load": (I, [vp, ctypes.c_char_p]),
        "fem_kernel_launches": (u64, []),
        "fem_select_noalloc": (I, [vp, u32, u32, vp, vp, vp]),
        "fem_batch_create": (I, [vp, ctypes.POINTER(fem_job), u32, ctypes.POINTER(fem_interval),
                                 u32, vp, ctypes.POINTER(vp)]),
        "fem_batch_run": (I, [vp, vp]),
        "fem_batch_destroy": (I, [vp]),
        "fem_server_create": (I, [vp, ctypes.POINTER(fem_server_config), ctypes.POINTER(vp)]),
        "fem_server_destroy": (I, [vp]),
        "fem_server_open_stream": (I, [vp, u32, u64, ctypes.POINTER(i32)]),
        "fem_server_append": (I, [vp, i32, vp, vp, u32]),
        "fem_server_submit": (I, [vp, i32, vp, u32, ctypes.POINTER(fem_interval), u32, u32, I, u32,
                                  ctypes.POINTER(u64)]),
        "fem_server_poll": (I, [vp, ctypes.POINTER(u64), u32, ctypes.POINTER(u32)]),
        "fem_server_result": (I, [vp, u64, vp, vp, ctypes.POINTER(u64)]),
        "fem_server_release": (I, [vp, u64]),
        "fem_server_drain": (I, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc, what):
    if rc != 0:
        raise FemError(rc, what)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device) of a numpy array or torch tensor."""
    if x is None:
        return None, 0
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda)
    if not (x.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data_as(ctypes.c_void_p), 0


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _intervals(intervals):
    iv = np.ascontiguousarray(np.asarray(intervals, dtype=np.uint32).reshape(-1, 2))
    arr = (fem_interval * max(len(iv), 1))()
    if len(iv):
        ctypes.memmove(arr, iv.ctypes.data, iv.nbytes)
    return arr, len(iv)


def pack_episodes(lens, types, ivl) -> np.ndarray:
    """[m, 16] uint8 episode records from len[m], types[m, 8], ivl[m, 7]."""
    lens = np.asarray(lens, dtype=np.uint8)
    m = lens.shape[0]
    rec = np.zeros((m, 16), np.uint8)
    rec[:, :8] = np.asarray(types, dtype=np.uint8).reshape(m, 8)
    rec[:, 8:15] = np.asarray(ivl, dtype=np.uint8).reshape(m, 7)
    rec[:, 15] = lens
    return rec


def unpack_episodes(rec):
    rec = np.asarray(rec, dtype=np.uint8).reshape(-1, 16)
    return rec[:, 15].copy(), rec[:, :8].copy(), rec[:, 8:15].copy()


# --------------------------------------------------------------------------- calls
def fem_create(device: int = 0, mem_budget_bytes: int = 0):
    """A context on `device`; mem_budget_bytes bounds its device memory (0: no bound)."""
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.fem_create(ctypes.byref(h), int(device), int(mem_budget_bytes)), "fem_create")
    return h


def fem_mem_usage(ctx):
    """(device bytes the context holds, its budget or 0)."""
    used, budget = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().fem_mem_usage(ctx, ctypes.byref(used), ctypes.byref(budget)), "fem_mem_usage")
    return int(used.value), int(budget.value)


def fem_destroy(ctx):
    _check(load().fem_destroy(ctx), "fem_destroy")


def fem_set_config(ctx, segments=0, threads_per_block=0, ring_capacity=0, kernel=KERNEL_AUTO,
                   reset=False):
    lib = load()
    if reset:
        _check(lib.fem_set_config(ctx, None), "fem_set_config")
        return
    cfg = fem_config(int(segments), int(threads_per_block), int(ring_capacity), int(kernel))
    _check(lib.fem_set_config(ctx, ctypes.byref(cfg)), "fem_set_config")


def fem_count_mapconcat_literal(ctx, sid, cands, intervals, segments, out=None, stream=None):
    """MapConcatenate as Section 5.2.2 prints it (comparison with the exact counts);
    returns (counts uint32[m] or `out`, (boundaries with no match, with several))."""
    lib = load()
    m = int(cands.shape[0])
    pc, dc = _ptr(cands)
    if out is None:
        out = np.zeros(m, np.uint32)
    po, do = _ptr(out)
    iv, nI = _intervals(intervals)
    diag = (ctypes.c_uint32 * 2)()
    _check(lib.fem_count_mapconcat_literal(ctx, int(sid), pc, m, dc, iv, nI, int(segments), po, do,
                                           diag, _stream_handle(stream)),
           "fem_count_mapconcat_literal")
    return out, (int(diag[0]), int(diag[1]))


def fem_count_windows(ctx, sid, cands, intervals, window_us, out=None, stream=None):
    """Window-based frequency of each candidate: uint64[m] window starts (or `out`)."""
    lib = load()
    m = int(cands.shape[0])
    pc, dc = _ptr(cands)
    if out is None:
        out = np.zeros(m, np.uint64)
    po, do = _ptr(out)
    iv, nI = _intervals(intervals)
    _check(lib.fem_count_windows(ctx, int(sid), pc, m, dc, iv, nI, int(window_us), po, do,
                                 _stream_handle(stream)), "fem_count_windows")
    return out


def fem_tune_enable(ctx, on=True):
    """Measured mapping choice on (or off) for counts whose class is not cached."""
    _check(load().fem_tune_enable(ctx, 1 if on else 0), "fem_tune_enable")


def fem_tune_size(ctx) -> int:
    n = ctypes.c_uint32()
    _check(load().fem_tune_size(ctx, ctypes.byref(n)), "fem_tune_size")
    return int(n.value)


def fem_tune_save(ctx, path):
    _check(load().fem_tune_save(ctx, os.fsencode(path)), "fem_tune_save")


def fem_tune_load(ctx, path):
    _check(load().fem_tune_load(ctx, os.fsencode(path)), "fem_tune_load")


def fem_load_stream(ctx, types, t_us, n_types, stream=None) -> int:
    """Load an event stream (numpy host arrays or CUDA tensors); returns its id."""
    lib = load()
    pt, dt = _ptr(types)
    pu, du = _ptr(t_us)
    if dt != du:
        raise ValueError("types and t_us must both be host or both be device")
    n = int(types.shape[0]) if types is not None else 0
    if (int(t_us.shape[0]) if t_us is not None else 0) != n:
        raise ValueError("types and t_us differ in length")
    sid = ctypes.c_int32()
    _check(lib.fem_load_stream(ctx, pt, pu, n, int(n_types), dt, _stream_handle(stream),
                               ctypes.byref(sid)), "fem_load_stream")
    return sid.value


def fem_append_stream(ctx, sid, types, t_us, stream=None):
    """Append events (numpy host arrays or CUDA tensors) to a resident stream."""
    lib = load()
    if not _is_torch(types):
        types = np.ascontiguousarray(types, dtype=np.uint8)
    if not _is_torch(t_us):
        t_us = np.ascontiguousarray(t_us, dtype=np.uint32)
    pt, dt = _ptr(types)
    pu, du = _ptr(t_us)
    if dt != du:
        raise ValueError("types and t_us must both be host or both be device")
    n = int(types.shape[0])
    if int(t_us.shape[0]) != n:
        raise ValueError("types and t_us differ in length")
    _check(lib.fem_append_stream(ctx, int(sid), pt, pu, n, dt, _stream_handle(stream)),
           "fem_append_stream")


def fem_free_stream(ctx, sid):
    _check(load().fem_free_stream(ctx, int(sid)), "fem_free_stream")


def fem_type_counts(ctx, sid, n_types) -> np.ndarray:
    out = np.zeros(n_types, np.uint32)
    _check(load().fem_type_counts(ctx, int(sid), out.ctypes.data_as(ctypes.c_void_p)),
           "fem_type_counts")
    return out


def fem_capacity_table(ctx, sid, widths_us, n_types) -> np.ndarray:
    """uint32[n_types, len(widths_us)]: the most events of each type in one closed window
    of each width."""
    w = np.ascontiguousarray(widths_us, dtype=np.uint32).reshape(-1)
    out = np.zeros((n_types, len(w)), np.uint32)
    _check(load().fem_capacity_table(ctx, int(sid), w.ctypes.data_as(ctypes.c_void_p), len(w),
                                     out.ctypes.data_as(ctypes.c_void_p)), "fem_capacity_table")
    return out


def fem_count_pairs_relaxed(ctx, sid, types, intervals) -> np.ndarray:
    """Relaxed counts of every ordered pair of distinct `types` with every interval, in
    level 2's canonical order (uint32[f (f - 1) len(intervals)])."""
    ty = np.ascontiguousarray(types, dtype=np.uint8).reshape(-1)
    iv, nI = _intervals(intervals)
    out = np.zeros(len(ty) * (len(ty) - 1) * nI, np.uint32)
    _check(load().fem_count_pairs_relaxed(ctx, int(sid), ty.ctypes.data_as(ctypes.c_void_p),
                                          len(ty), iv, nI, out.ctypes.data_as(ctypes.c_void_p)),
           "fem_count_pairs_relaxed")
    return out


def fem_count_candidates(ctx, sid, cands, intervals, pass_=PASS_EXACT, out=None, stream=None):
    """Count episode records `cands` ([m,16] numpy or CUDA uint8 tensor).

    Returns `out` (a uint32 numpy array, or the given device tensor)."""
    lib = load()
    m = int(cands.shape[0])
    pc, dc = _ptr(cands)
    if out is None:
        out = np.zeros(m, np.uint32)
    po, do = _ptr(out)
    iv, nI = _intervals(intervals)
    _check(lib.fem_count_candidates(ctx, int(sid), pc, m, dc, iv, nI, int(pass_), po, do,
                                    _stream_handle(stream)), "fem_count_candidates")
    return out


def fem_count_two_pass(ctx, sid, cands, intervals, theta, exact_out=None, survived_out=None,
                       stream=None):
    """Algorithm 4; returns (exact-or-zero uint32[m], survived uint8[m])."""
    lib = load()
    m = int(cands.shape[0])
    pc, dc = _ptr(cands)
    if exact_out is None:
        exact_out = np.zeros(m, np.uint32)
    if survived_out is None:
        survived_out = np.zeros(m, np.uint8)
    pe, de = _ptr(exact_out)
    ps, ds = _ptr(survived_out)
    if de != ds:
        raise ValueError("outputs must both be host or both be device")
    iv, nI = _intervals(intervals)
    _check(lib.fem_count_two_pass(ctx, int(sid), pc, m, dc, iv, nI, int(theta), pe, ps, de,
                                  _stream_handle(stream)), "fem_count_two_pass")
    return exact_out, survived_out


MINE_REPEATED_TYPES = 1


def fem_mine_levelwise(ctx, sid, intervals, theta, max_len, stream=None, raw=False,
                       repeated_types=False):
    """Problem 1: {level: [(types tuple, interval tuple, count), ...]} in canonical order.

    raw=True returns {level: (records uint8[f,16], counts uint32[f])} instead;
    repeated_types=True mines episodes whose types may repeat (fem_mine_levelwise_ex)."""
    lib = load()
    iv, nI = _intervals(intervals)
    res = ctypes.c_void_p()
    if repeated_types:
        _check(lib.fem_mine_levelwise_ex(ctx, int(sid), iv, nI, int(theta), int(max_len),
                                         MINE_REPEATED_TYPES, _stream_handle(stream),
                                         ctypes.byref(res)), "fem_mine_levelwise_ex")
    else:
        _check(lib.fem_mine_levelwise(ctx, int(sid), iv, nI, int(theta), int(max_len),
                                      _stream_handle(stream), ctypes.byref(res)),
               "fem_mine_levelwise")
    try:
        out = {}
        for level in range(1, int(max_len) + 1):
            m = ctypes.c_uint32()
            pe, pcn = ctypes.c_void_p(), ctypes.c_void_p()
            _check(lib.fem_result_level(res, level, ctypes.byref(m), ctypes.byref(pe),
                                        ctypes.byref(pcn)), "fem_result_level")
            f = m.value
            if f == 0:  # level N + 1 is generated from level N's frequent set only
                break
            rec = np.empty((f, 16), np.uint8)
            cnt = np.empty(f, np.uint32)
            ctypes.memmove(rec.ctypes.data, pe, f * 16)
            ctypes.memmove(cnt.ctypes.data, pcn, f * 4)
            if raw:
                out[level] = (rec, cnt)
            else:
                out[level] = [(tuple(int(x) for x in rec[i, : rec[i, 15]]),
                               tuple(int(x) for x in rec[i, 8: 8 + rec[i, 15] - 1]),
                               int(cnt[i])) for i in range(f)]
        return out
    finally:
        lib.fem_result_free(res)


def fem_last_mine_stats(ctx):
    arr = (fem_level_stats * 16)()
    k = load().fem_last_mine_stats(ctx, arr, 16)
    if k < 0:
        raise FemError(k, "fem_last_mine_stats")
    return [{f: getattr(arr[i], f) for f, _ in fem_level_stats._fields_} for i in range(k)]


def fem_select_noalloc(values, theta, idx_out, count_out, stream=None):
    """Indices i with values[i] >= theta into idx_out, their number into count_out[0]
    (all CUDA tensors, no allocation by the library).  Asynchronous on the stream."""
    pv, dv = _ptr(values)
    pi, di = _ptr(idx_out)
    pc, dc = _ptr(count_out)
    if not (dv and di and dc):
        raise ValueError("values, idx_out and count_out must be device tensors")
    for name, x in (("values", values), ("idx_out", idx_out), ("count_out", count_out)):
        if x.element_size() != 4:
            raise ValueError(f"{name} must hold 4-byte elements")
    if idx_out.numel() < values.numel() or count_out.numel() < 1:
        raise ValueError("idx_out needs values.numel() elements and count_out one")
    import torch
    cur = torch.cuda.current_device()
    if any(x.device.index != cur for x in (values, idx_out, count_out)):
        raise ValueError("values, idx_out and count_out must be on the current CUDA device")
    _check(load().fem_select_noalloc(pv, int(values.shape[0]), int(theta), pi, pc,
                                     _stream_handle(stream)), "fem_select_noalloc")


def fem_batch_create(ctx, jobs, intervals, stream=None):
    """jobs: iterable of dicts with stream_id, len, cands ([m,16] uint8 CUDA tensor),
    theta, exact_out (int32/uint32 CUDA tensor [m]), survived_out (uint8 CUDA tensor [m]).
    Returns a batch handle; the tensors must outlive it."""
    lib = load()
    jobs = list(jobs)
    arr = (fem_job * max(len(jobs), 1))()
    for i, j in enumerate(jobs):
        for key in ("cands", "exact_out", "survived_out"):
            if not (_is_torch(j[key]) and j[key].is_cuda):
                raise ValueError(f"job {i}: {key} must be a CUDA tensor")
        arr[i] = fem_job(int(j["stream_id"]), int(j["len"]), int(j["cands"].shape[0]),
                         j["cands"].data_ptr(), int(j["theta"]), j["exact_out"].data_ptr(),
                         j["survived_out"].data_ptr())
    iv, nI = _intervals(intervals)
    h = ctypes.c_void_p()
    _check(lib.fem_batch_create(ctx, arr, len(jobs), iv, nI, _stream_handle(stream),
                                ctypes.byref(h)), "fem_batch_create")
    return h


def fem_batch_run(batch, stream=None):
    _check(load().fem_batch_run(batch, _stream_handle(stream)), "fem_batch_run")


def fem_batch_destroy(batch):
    _check(load().fem_batch_destroy(batch), "fem_batch_destroy")


def fem_server_create(ctx, mem_budget_bytes=0, max_active=0, n_lanes=0):
    cfg = fem_server_config(int(mem_budget_bytes), int(max_active), int(n_lanes))
    h = ctypes.c_void_p()
    _check(load().fem_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h)), "fem_server_create")
    return h


def fem_server_destroy(srv):
    _check(load().fem_server_destroy(srv), "fem_server_destroy")


def fem_server_open_stream(srv, n_types, capacity_events) -> int:
    sid = ctypes.c_int32()
    _check(load().fem_server_open_stream(srv, int(n_types), int(capacity_events),
                                         ctypes.byref(sid)), "fem_server_open_stream")
    return sid.value


def fem_server_append(srv, sid, types, t_us):
    types = np.ascontiguousarray(types, dtype=np.uint8)
    t_us = np.ascontiguousarray(t_us, dtype=np.uint32)
    if types.shape != t_us.shape:
        raise ValueError("types and t_us differ in length")
    _check(load().fem_server_append(srv, int(sid), types.ctypes.data_as(ctypes.c_void_p),
                                    t_us.ctypes.data_as(ctypes.c_void_p), int(types.shape[0])),
           "fem_server_append")


def fem_server_submit(srv, sid, cands, intervals, theta, mode=REQ_ONESHOT, window_us=0):
    """Returns the request id; raises FemError (status -6, FEM_EADMIT) if not admitted."""
    cands = np.ascontiguousarray(cands, dtype=np.uint8).reshape(-1, 16)
    iv, nI = _intervals(intervals)
    rid = ctypes.c_uint64()
    _check(load().fem_server_submit(srv, int(sid), cands.ctypes.data_as(ctypes.c_void_p),
                                    int(cands.shape[0]), iv, nI, int(theta), int(mode),
                                    int(window_us), ctypes.byref(rid)), "fem_server_submit")
    return rid.value


def fem_server_poll(srv, cap=4096):
    ids = (ctypes.c_uint64 * cap)()
    n = ctypes.c_uint32()
    _check(load().fem_server_poll(srv, ids, cap, ctypes.byref(n)), "fem_server_poll")
    return [int(ids[i]) for i in range(n.value)]


def fem_server_result(srv, rid, m):
    """(counts uint32[m], flags uint8[m], events covered, status)."""
    counts = np.zeros(m, np.uint32)
    flags = np.zeros(m, np.uint8)
    ev = ctypes.c_uint64()
    rc = load().fem_server_result(srv, int(rid), counts.ctypes.data_as(ctypes.c_void_p),
                                  flags.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ev))
    return counts, flags, int(ev.value), int(rc)


def fem_server_release(srv, rid):
    _check(load().fem_server_release(srv, int(rid)), "fem_server_release")


def fem_server_drain(srv):
    _check(load().fem_server_drain(srv), "fem_server_drain")


def fem_kernel_launches() -> int:
    return int(load().fem_kernel_launches())


def fem_strerror(status: int) -> str:
    return load().fem_strerror(int(status)).decode()


class Context:
    """Small convenience owner of a context (destroyed on close/exit)."""

    def __init__(self, device=0, mem_budget_bytes=0):
        self.h = fem_create(device, mem_budget_bytes)

    def close(self):
        if self.h:
            fem_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
