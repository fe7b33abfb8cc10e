"""ctypes binding of libskyline (include/skyline.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  There is no CPU fallback -- if the library cannot be loaded,
every call raises.  Inputs may be numpy arrays (host memory; the library
copies them to the GPU) or CUDA torch tensors (device memory, used in place
on the tensor's current stream).
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

import numpy as np

from . import build as _build

SKY_OK, SKY_EINVAL, SKY_ENOMEM, SKY_ECUDA, SKY_ETIMEOUT, SKY_EBUSY, SKY_ECANCELLED = range(7)
SCHEMES = {"random": 0, "grid": 1, "angular": 2, "sliced": 3, "none": 4}
REPS = {"none": 0, "sorted": 1, "region": 2}
MERGES = {"sequential": 0, "noseq": 1}
EXECS = {"persistent": 0, "plain": 1}
IMAGES = {"values": 0, "ranks": 1}
RANK_CODES = 0x7C00  # codes of the rank images: 0 .. RANK_CODES - 1
STAGE_SKY, STAGE_GRID, STAGE_REP, STAGE_LOCAL, STAGE_MERGE = 1, 2, 3, 4, 5


class SkyParams(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("scheme", ctypes.c_int),
        ("num_partitions", ctypes.c_uint32),
        ("slices", ctypes.c_uint32 * 8),
        ("normalize", ctypes.c_uint32),
        ("slice_dim", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
        ("grid_filter", ctypes.c_uint32),
        ("rep", ctypes.c_int),
        ("reps_per_partition", ctypes.c_uint32),
        ("merge", ctypes.c_int),
        ("exec", ctypes.c_int),
        ("chunk_min", ctypes.c_uint32),
        ("chunk_max", ctypes.c_uint32),
        ("chunk_alpha_x4", ctypes.c_uint32),
        ("dom_block", ctypes.c_uint32),
        ("engine_warps", ctypes.c_uint32),
        ("engine_cands", ctypes.c_uint32),
        ("images", ctypes.c_int),
    ]


class SkyQuery(ctypes.Structure):
    _fields_ = [
        ("points", ctypes.c_void_p),
        ("n", ctypes.c_uint64),
        ("d", ctypes.c_uint32),
        ("params", ctypes.POINTER(SkyParams)),
        ("out_idx", ctypes.c_void_p),
        ("out_count", ctypes.POINTER(ctypes.c_uint64)),
        ("status", ctypes.c_int),
    ]


class SkyServeConfig(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("workers", ctypes.c_uint32),
        ("max_batch", ctypes.c_uint32),
        ("mem_budget_bytes", ctypes.c_uint64),
    ]


class SkyTicketInfo(ctypes.Structure):
    _fields_ = [
        ("queue_us", ctypes.c_double),
        ("run_us", ctypes.c_double),
        ("latency_us", ctypes.c_double),
        ("batch_queries", ctypes.c_uint32),
    ]


class SkyStats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("d", ctypes.c_uint32),
        ("partitions", ctypes.c_uint32),
        ("nonempty_partitions", ctypes.c_uint32),
        ("rounds_local", ctypes.c_uint32),
        ("rounds_merge", ctypes.c_uint32),
        ("reps_kept", ctypes.c_uint32),
        ("grid_dropped", ctypes.c_uint64),
        ("rep_dropped", ctypes.c_uint64),
        ("local_union", ctypes.c_uint64),
        ("skyline", ctypes.c_uint64),
        ("ms_total", ctypes.c_double),
        ("ms_phase", ctypes.c_double * 6),
        ("launches", ctypes.c_uint64),
        ("ms_dom_local", ctypes.c_double),
        ("ms_dom_merge", ctypes.c_double),
        ("tests_fp16", ctypes.c_uint64),
        ("tests_fp16_local", ctypes.c_uint64),
    ]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "ms_phase"}
        d["ms_phase"] = list(self.ms_phase)
        return d


EXPORTS = ["sky_params_init", "sky_create", "sky_set_stream", "sky_set_timing", "sky_skyline",
           "sky_skyline_ex", "sky_get_stats", "sky_status_str", "sky_last_error", "sky_destroy",
           "sky_probe_compare_rate", "sky_skyline_static", "sky_skyline_batch", "sky_serve_config_init", "sky_query_bytes",
           "sky_serve_start", "sky_submit", "sky_poll", "sky_wait", "sky_serve_stop", "sky_autotune", "sky_autotune_batch",
           "sky_graph_capture", "sky_graph_launch", "sky_graph_destroy", "sky_diag_engine_wait_test",
           "sky_rank_space", "sky_probe_reject_rate"]

_lock = threading.Lock()
_lib = None


class SkylineError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Loads libskyline.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"libskyline is not built ({path}); run build() first")
        L = ctypes.CDLL(path)
        P, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        L.sky_params_init.argtypes = [ctypes.POINTER(SkyParams)]
        L.sky_params_init.restype = None
        L.sky_create.argtypes = [ctypes.POINTER(P), i32, ctypes.c_size_t]
        L.sky_create.restype = i32
        L.sky_set_stream.argtypes = [P, P]
        L.sky_set_stream.restype = i32
        L.sky_set_timing.argtypes = [P, i32]
        L.sky_set_timing.restype = i32
        L.sky_skyline.argtypes = [P, P, u64, u32, ctypes.POINTER(SkyParams), P, ctypes.POINTER(u64)]
        L.sky_skyline.restype = i32
        L.sky_skyline_ex.argtypes = [P, P, u64, u32, ctypes.POINTER(SkyParams), P, ctypes.POINTER(u64), P, P]
        L.sky_skyline_ex.restype = i32
        L.sky_get_stats.argtypes = [P, u64, ctypes.POINTER(SkyStats)]
        L.sky_get_stats.restype = i32
        L.sky_status_str.argtypes = [i32]
        L.sky_status_str.restype = ctypes.c_char_p
        L.sky_last_error.argtypes = [P]
        L.sky_last_error.restype = ctypes.c_char_p
        L.sky_destroy.argtypes = [P]
        L.sky_destroy.restype = None
        L.sky_probe_compare_rate.argtypes = [P, u32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u32)]
        L.sky_probe_compare_rate.restype = i32
        L.sky_probe_reject_rate.argtypes = [P, u32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u32)]
        L.sky_probe_reject_rate.restype = i32
        L.sky_skyline_batch.argtypes = [P, ctypes.POINTER(SkyQuery), u32]
        L.sky_skyline_batch.restype = i32
        L.sky_serve_config_init.argtypes = [ctypes.POINTER(SkyServeConfig)]
        L.sky_serve_config_init.restype = None
        L.sky_query_bytes.argtypes = [u64, u32, ctypes.POINTER(SkyParams)]
        L.sky_query_bytes.restype = u64
        L.sky_autotune.argtypes = [P, P, u64, u32, ctypes.POINTER(SkyParams), u32, ctypes.POINTER(ctypes.c_double)]
        L.sky_autotune.restype = i32
        L.sky_autotune_batch.argtypes = [P, ctypes.POINTER(SkyQuery), u32, u32, ctypes.POINTER(SkyParams),
                                         ctypes.POINTER(ctypes.c_double)]
        L.sky_autotune_batch.restype = i32
        L.sky_graph_capture.argtypes = [P, ctypes.POINTER(SkyQuery), u32, ctypes.POINTER(P)]
        L.sky_graph_capture.restype = i32
        L.sky_graph_launch.argtypes = [P, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_double)]
        L.sky_graph_launch.restype = i32
        L.sky_graph_destroy.argtypes = [P]
        L.sky_graph_destroy.restype = None
        L.sky_serve_start.argtypes = [P, ctypes.POINTER(SkyServeConfig)]
        L.sky_serve_start.restype = i32
        L.sky_submit.argtypes = [P, P, u64, u32, ctypes.POINTER(SkyParams), ctypes.POINTER(u64)]
        L.sky_submit.restype = i32
        L.sky_poll.argtypes = [P, u64]
        L.sky_poll.restype = i32
        L.sky_wait.argtypes = [P, u64, P, ctypes.POINTER(u64), ctypes.c_int64, ctypes.POINTER(SkyTicketInfo)]
        L.sky_wait.restype = i32
        L.sky_serve_stop.argtypes = [P]
        L.sky_serve_stop.restype = i32
        L.sky_skyline_static.argtypes = [P, u64, u32, P, ctypes.POINTER(u64), P]
        L.sky_skyline_static.restype = i32
        L.sky_diag_engine_wait_test.argtypes = [P, u64, u32]
        L.sky_diag_engine_wait_test.restype = i32
        L.sky_rank_space.argtypes = [P, P, u64, u32, P, P, P]
        L.sky_rank_space.restype = i32
        _lib = L
        return L


def make_params(scheme="none", p: int = 1, slices=None, normalize=False, slice_dim=0, seed=0,
                grid_filter=True, rep="none", reps_per_partition=1, merge="sequential",
                exec="persistent", chunk_min=0, chunk_max=0, chunk_alpha_x4=0, dom_block=0,
                engine_warps=0, engine_cands=0, images="values") -> SkyParams:
    L = load()
    sp = SkyParams()
    L.sky_params_init(ctypes.byref(sp))
    sp.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    sp.num_partitions = int(p)
    if slices is not None:
        for i, m in enumerate(slices):
            sp.slices[i] = int(m)
    sp.normalize = int(bool(normalize))
    sp.slice_dim = int(slice_dim)
    sp.seed = int(seed) & (2 ** 64 - 1)
    sp.grid_filter = int(bool(grid_filter))
    sp.rep = REPS[rep] if isinstance(rep, str) else int(rep)
    sp.reps_per_partition = int(reps_per_partition)
    sp.merge = MERGES[merge] if isinstance(merge, str) else int(merge)
    sp.exec = EXECS[exec] if isinstance(exec, str) else int(exec)
    sp.chunk_min, sp.chunk_max = int(chunk_min), int(chunk_max)
    sp.chunk_alpha_x4, sp.dom_block = int(chunk_alpha_x4), int(dom_block)
    sp.engine_warps, sp.engine_cands = int(engine_warps), int(engine_cands)
    sp.images = IMAGES[images] if isinstance(images, str) else int(images)
    return sp


# the engine knobs of sky_params that sky_autotune chooses
KNOBS = ("chunk_min", "chunk_max", "chunk_alpha_x4", "dom_block", "engine_warps", "engine_cands")


def tune_key(n: int, d: int, params: SkyParams) -> str:
    """Key of a tuned-knobs cache entry: the workload's shape -- d, N to the
    power of two below it, and the method parameters (the knobs excluded)."""
    rec = {"d": int(d), "log2_n": max(0, int(n).bit_length() - 1), "scheme": int(params.scheme),
           "p": int(params.num_partitions), "slices": [int(v) for v in list(params.slices)[: int(d)]],
           "normalize": int(params.normalize), "slice_dim": int(params.slice_dim),
           "grid_filter": int(params.grid_filter), "rep": int(params.rep),
           "k": int(params.reps_per_partition), "merge": int(params.merge), "exec": int(params.exec),
           "images": int(params.images)}
    return json.dumps(rec, sort_keys=True)


class TuneCache:
    """Tuned engine knobs kept in a JSON file across processes: one entry
    per tune_key, holding the six knobs and the time they gave."""

    def __init__(self, path: str):
        self.path = path
        self.entries = {}
        if os.path.exists(path):
            with open(path) as fh:
                self.entries = json.load(fh)

    def get(self, key: str):
        return self.entries.get(key)

    def put(self, key: str, params: SkyParams, ms: float):
        self.entries[key] = {**{k: int(getattr(params, k)) for k in KNOBS}, "ms": float(ms)}
        self.save()

    def save(self):
        tmp = f"{self.path}.{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(self.entries, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    @staticmethod
    def apply(entry: dict, params: SkyParams) -> SkyParams:
        for k in KNOBS:
            setattr(params, k, int(entry[k]))
        return params


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


class Context:
    """One libskyline context on a CUDA device (owns its scratch memory)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self._L = load()
        h = ctypes.c_void_p()
        st = self._L.sky_create(ctypes.byref(h), int(device), int(mem_budget_bytes))
        if st != SKY_OK:
            raise SkylineError(st, self._L.sky_status_str(st).decode())
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            self._L.sky_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        if st != SKY_OK:
            raise SkylineError(st, self._L.sky_last_error(self._h).decode())

    def set_stream(self, stream_handle: int):
        self._check(self._L.sky_set_stream(self._h, ctypes.c_void_p(int(stream_handle))))

    def set_timing(self, on: bool):
        self._check(self._L.sky_set_timing(self._h, int(bool(on))))

    def probe_compare_rate(self, iterations: int = 20000):
        """Measured FP32 compares per second of the whole GPU (diagnostic)."""
        rate = ctypes.c_double(0)
        sms = ctypes.c_uint32(0)
        self._check(self._L.sky_probe_compare_rate(self._h, int(iterations), ctypes.byref(rate), ctypes.byref(sms)))
        return rate.value, sms.value

    def probe_reject_rate(self, iterations: int = 200):
        """Measured dim-compares per second of the engine's f16x2 rejection
        loop run alone (sky_probe_reject_rate; diagnostic)."""
        rate = ctypes.c_double(0)
        sms = ctypes.c_uint32(0)
        self._check(self._L.sky_probe_reject_rate(self._h, int(iterations), ctypes.byref(rate), ctypes.byref(sms)))
        return rate.value, sms.value

    def engine_wait_test(self, wait_limit_ns: int, withhold_task: int):
        """Arms the next skyline call's test hook of the engine's bounded
        waits (sky_diag_engine_wait_test): waits give up after wait_limit_ns
        without progress, and the withhold_task-th task an engine launch
        publishes is never marked published (0 = none)."""
        self._check(self._L.sky_diag_engine_wait_test(self._h, int(wait_limit_ns), int(withhold_task)))

    def stats(self, ticket: int = 0) -> dict:
        """Statistics of the last call (ticket 0) or of a serving ticket."""
        s = SkyStats()
        self._check(self._L.sky_get_stats(self._h, int(ticket), ctypes.byref(s)))
        return s.as_dict()

    def rank_space(self, points):
        """Dense ranks of every column (sky_rank_space): returns (ranks
        uint32 [N, d], distinct uint32 [d], codes uint16 [N, d]) -- numpy
        arrays for host input, CUDA torch tensors (int32, int32, int16
        holding the same bits) for a CUDA tensor."""
        if _is_cuda_tensor(points):
            import torch
            if points.dtype != torch.float32 or points.dim() != 2:
                raise ValueError("points must be a float32 [N, d] tensor")
            points = points.contiguous()
            n, d = points.shape
            self.set_stream(torch.cuda.current_stream(points.device).cuda_stream)
            ranks = torch.empty((max(n, 1), d), dtype=torch.int32, device=points.device)
            distinct = torch.empty(d, dtype=torch.int32, device=points.device)
            codes = torch.empty((max(n, 1), d), dtype=torch.int16, device=points.device)
            self._check(self._L.sky_rank_space(self._h, ctypes.c_void_p(points.data_ptr()), n, d,
                                               ctypes.c_void_p(ranks.data_ptr()),
                                               ctypes.c_void_p(distinct.data_ptr()),
                                               ctypes.c_void_p(codes.data_ptr())))
            return ranks[:n], distinct, codes[:n]
        a = np.ascontiguousarray(points, dtype=np.float32)
        if a.ndim != 2:
            raise ValueError("points must be [N, d]")
        n, d = a.shape
        self.set_stream(0)
        ranks = np.zeros((max(n, 1), d), dtype=np.uint32)
        distinct = np.zeros(d, dtype=np.uint32)
        codes = np.zeros((max(n, 1), d), dtype=np.uint16)
        self._check(self._L.sky_rank_space(self._h, a.ctypes.data_as(ctypes.c_void_p), n, d,
                                           ranks.ctypes.data_as(ctypes.c_void_p),
                                           distinct.ctypes.data_as(ctypes.c_void_p),
                                           codes.ctypes.data_as(ctypes.c_void_p)))
        return ranks[:n], distinct, codes[:n]

    def skyline(self, points, params: SkyParams | None = None, out=None, with_diag: bool = False, **kw):
        """Sky(points): ascending indices of the non-dominated points.

        points: numpy float32 [N, d] (host) or a CUDA torch float32 tensor.
        Host input returns a numpy uint32 array; device input returns a CUDA
        torch int32 tensor (a view of `out` if given).  with_diag also returns
        the per-point partition and stage arrays (Section 3 / stage codes)."""
        if params is None:
            params = make_params(**kw)
        elif kw:
            raise TypeError("pass either params or keyword parameters")
        cnt = ctypes.c_uint64(0)
        if _is_cuda_tensor(points):
            import torch
            if points.dtype != torch.float32 or points.dim() != 2:
                raise ValueError("points must be a float32 [N, d] tensor")
            points = points.contiguous()
            n, d = points.shape
            self.set_stream(torch.cuda.current_stream(points.device).cuda_stream)
            if out is None:
                out = torch.empty(max(n, 1), dtype=torch.int32, device=points.device)
            pid = stage = None
            if with_diag:
                pid = torch.empty(max(n, 1), dtype=torch.int32, device=points.device)
                stage = torch.empty(max(n, 1), dtype=torch.uint8, device=points.device)
            st = self._L.sky_skyline_ex(self._h, ctypes.c_void_p(points.data_ptr()), n, d, ctypes.byref(params),
                                        ctypes.c_void_p(out.data_ptr()), ctypes.byref(cnt),
                                        ctypes.c_void_p(pid.data_ptr()) if with_diag else None,
                                        ctypes.c_void_p(stage.data_ptr()) if with_diag else None)
            self._check(st)
            res = out[: cnt.value]
            if with_diag:
                return res, pid[:n], stage[:n]
            return res
        a = np.ascontiguousarray(points, dtype=np.float32)
        if a.ndim != 2:
            raise ValueError("points must be [N, d]")
        n, d = a.shape
        self.set_stream(0)
        res = np.zeros(max(n, 1), dtype=np.uint32)
        pid = np.zeros(max(n, 1), dtype=np.uint32) if with_diag else None
        stage = np.zeros(max(n, 1), dtype=np.uint8) if with_diag else None
        st = self._L.sky_skyline_ex(self._h, a.ctypes.data_as(ctypes.c_void_p), n, d, ctypes.byref(params),
                                    res.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt),
                                    pid.ctypes.data_as(ctypes.c_void_p) if with_diag else None,
                                    stage.ctypes.data_as(ctypes.c_void_p) if with_diag else None)
        self._check(st)
        if with_diag:
            return res[: cnt.value], pid[:n], stage[:n]
        return res[: cnt.value]

    def autotune(self, points, params: SkyParams | None = None, max_trials: int = 0, cache=None, **kw):
        """Tunes the engine knobs for this workload (sky_autotune); returns
        (tuned SkyParams, best time in ms).  points: host numpy or CUDA
        torch float32 [N, d].  cache: a TuneCache or the path of its JSON
        file; a workload of the same shape (tune_key) found there gets the
        stored knobs without a trial, and a new one is tuned and stored."""
        if params is None:
            params = make_params(**kw)
        else:
            sp = SkyParams()
            ctypes.memmove(ctypes.byref(sp), ctypes.byref(params), ctypes.sizeof(SkyParams))
            params = sp
        if cache is not None:
            if not isinstance(cache, TuneCache):
                cache = TuneCache(str(cache))
            n0, d0 = (int(v) for v in points.shape)
            key = tune_key(n0, d0, params)
            hit = cache.get(key)
            if hit is not None:
                return TuneCache.apply(hit, params), hit["ms"]
            tuned, ms = self.autotune(points, params=params, max_trials=max_trials)
            cache.put(key, tuned, ms)
            return tuned, ms
        if _is_cuda_tensor(points):
            import torch
            points = points.contiguous()
            ptr = points.data_ptr()
            self.set_stream(torch.cuda.current_stream(points.device).cuda_stream)
        else:
            points = np.ascontiguousarray(points, dtype=np.float32)
            ptr = points.ctypes.data
            self.set_stream(0)
        n, d = points.shape
        ms = ctypes.c_double(0)
        self._check(self._L.sky_autotune(self._h, ctypes.c_void_p(ptr), n, d, ctypes.byref(params),
                                         int(max_trials), ctypes.byref(ms)))
        return params, ms.value

    def autotune_batch(self, queries, max_trials: int = 0):
        """Tunes one set of engine knobs for a batch (sky_autotune_batch).
        queries: list of (points, params).  Returns (dict of the six knobs,
        best batch time in ms)."""
        nq = len(queries)
        arr = (SkyQuery * max(nq, 1))()
        keep = []
        stream_set = False
        for i, (pts, params) in enumerate(queries):
            if params is None:
                params = make_params()
            if _is_cuda_tensor(pts):
                import torch
                pts = pts.contiguous()
                if not stream_set:
                    self.set_stream(torch.cuda.current_stream(pts.device).cuda_stream)
                    stream_set = True
                arr[i].points = pts.data_ptr()
            else:
                pts = np.ascontiguousarray(pts, dtype=np.float32)
                arr[i].points = pts.ctypes.data
            arr[i].n, arr[i].d = pts.shape
            arr[i].params = ctypes.pointer(params)
            keep.append((pts, params))
        if not stream_set:
            self.set_stream(0)
        knobs = make_params()
        ms = ctypes.c_double(0)
        self._check(self._L.sky_autotune_batch(self._h, arr, nq, int(max_trials), ctypes.byref(knobs),
                                               ctypes.byref(ms)))
        return ({k: getattr(knobs, k) for k in ("chunk_min", "chunk_max", "chunk_alpha_x4", "dom_block",
                                                 "engine_warps", "engine_cands")},
                ms.value)

    def capture(self, queries):
        """Captures a batch of device-resident queries into a CUDA graph
        (sky_graph_capture).  queries: list of (CUDA float32 [N, d] tensor,
        params).  Returns a Graph whose run() replays it."""
        import torch
        nq = len(queries)
        arr = (SkyQuery * max(nq, 1))()
        keep, outs = [], []
        for i, (pts, params) in enumerate(queries):
            if params is None:
                params = make_params()
            if not _is_cuda_tensor(pts):
                raise ValueError("a captured batch needs CUDA tensors")
            pts = pts.contiguous()
            n, d = pts.shape
            out = torch.empty(max(n, 1), dtype=torch.int32, device=pts.device)
            arr[i].points, arr[i].out_idx = pts.data_ptr(), out.data_ptr()
            arr[i].n, arr[i].d = n, d
            arr[i].params = ctypes.pointer(params)
            keep.append((pts, params))
            outs.append(out)
        if nq:
            self.set_stream(torch.cuda.current_stream(queries[0][0].device).cuda_stream)
        h = ctypes.c_void_p()
        self._check(self._L.sky_graph_capture(self._h, arr, nq, ctypes.byref(h)))
        return Graph(self._L, h, keep, outs)

    # ---- serving (continuous batching) --------------------------------
    def serve_start(self, workers: int = 2, max_batch: int = 64, mem_budget_bytes: int = 0):
        cfg = SkyServeConfig()
        self._L.sky_serve_config_init(ctypes.byref(cfg))
        cfg.workers, cfg.max_batch, cfg.mem_budget_bytes = int(workers), int(max_batch), int(mem_budget_bytes)
        st = self._L.sky_serve_start(self._h, ctypes.byref(cfg))
        if st != SKY_OK:
            raise SkylineError(st, self._L.sky_status_str(st).decode())

    def submit(self, points, params: SkyParams | None = None) -> int:
        """Queues Sky(points); returns the ticket.  points (host numpy or
        CUDA torch float32 [N, d]) is kept alive by the binding until wait()."""
        if params is None:
            params = make_params()
        if _is_cuda_tensor(points):
            points = points.contiguous()
            ptr = points.data_ptr()
        else:
            points = np.ascontiguousarray(points, dtype=np.float32)
            ptr = points.ctypes.data
        n, d = points.shape
        t = ctypes.c_uint64(0)
        st = self._L.sky_submit(self._h, ctypes.c_void_p(ptr), n, d, ctypes.byref(params), ctypes.byref(t))
        if st != SKY_OK:
            raise SkylineError(st, self._L.sky_status_str(st).decode())
        if not hasattr(self, "_inflight"):
            self._inflight = {}
        self._inflight[t.value] = (points, params, n)
        return t.value

    def poll(self, ticket: int) -> bool:
        st = self._L.sky_poll(self._h, int(ticket))
        if st == SKY_OK:
            return True
        if st == SKY_EBUSY:
            return False
        raise SkylineError(st, self._L.sky_status_str(st).decode())

    def wait(self, ticket: int, timeout_us: int = -1):
        """Result of a ticket: (numpy uint32 ascending indices, info dict with
        queue_us / run_us / latency_us / batch_queries)."""
        _, _, n = self._inflight[ticket]
        out = np.zeros(max(n, 1), dtype=np.uint32)
        cnt = ctypes.c_uint64(0)
        info = SkyTicketInfo()
        st = self._L.sky_wait(self._h, int(ticket), out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt),
                              int(timeout_us), ctypes.byref(info))
        if st == SKY_EBUSY:
            raise TimeoutError(f"ticket {ticket} still in flight")
        self._inflight.pop(ticket, None)
        if st != SKY_OK:
            raise SkylineError(st, self._L.sky_status_str(st).decode())
        return out[: cnt.value], {f: getattr(info, f) for f, _ in SkyTicketInfo._fields_}

    def serve_stop(self):
        self._check(self._L.sky_serve_stop(self._h))

    def skyline_batch(self, queries):
        """Several independent queries in one batch (sky_skyline_batch).

        queries: a list of (points, params) pairs, points a host numpy or
        CUDA torch float32 [N, d] array, params a SkyParams or None.  Returns
        the list of index arrays (numpy for host input, CUDA torch int32 for
        device input)."""
        nq = len(queries)
        arr = (SkyQuery * max(nq, 1))()
        keep, outs, counts = [], [], []
        stream_set = False
        for i, (pts, params) in enumerate(queries):
            if params is None:
                params = make_params()
            cnt = ctypes.c_uint64(0)
            if _is_cuda_tensor(pts):
                import torch
                pts = pts.contiguous()
                n, d = pts.shape
                if not stream_set:
                    self.set_stream(torch.cuda.current_stream(pts.device).cuda_stream)
                    stream_set = True
                out = torch.empty(max(n, 1), dtype=torch.int32, device=pts.device)
                arr[i].points, arr[i].out_idx = pts.data_ptr(), out.data_ptr()
            else:
                pts = np.ascontiguousarray(pts, dtype=np.float32)
                n, d = pts.shape
                out = np.zeros(max(n, 1), dtype=np.uint32)
                arr[i].points = pts.ctypes.data
                arr[i].out_idx = out.ctypes.data
            arr[i].n, arr[i].d = n, d
            arr[i].params = ctypes.pointer(params)
            arr[i].out_count = ctypes.pointer(cnt)
            keep.append((pts, params))
            outs.append(out)
            counts.append(cnt)
        if not stream_set:
            self.set_stream(0)
        self._check(self._L.sky_skyline_batch(self._h, arr, nq))
        return [o[: c.value] for o, c in zip(outs, counts)]


def query_bytes(n: int, d: int, params: SkyParams | None = None) -> int:
    """Device memory one query of this shape takes in a batch (bytes)."""
    return int(load().sky_query_bytes(int(n), int(d), ctypes.byref(params) if params is not None else None))


class Graph:
    """A captured batch (sky_graph_*); keeps its inputs and outputs alive."""

    def __init__(self, L, h, keep, outs):
        self._L, self._h, self._keep, self.outs = L, h, keep, outs

    def run(self):
        """Replays the graph; returns (list of CUDA int32 index tensors, device ms)."""
        n = len(self.outs)
        counts = (ctypes.c_uint64 * max(n, 1))()
        ms = ctypes.c_double(0)
        st = self._L.sky_graph_launch(self._h, counts, ctypes.byref(ms))
        if st != SKY_OK:
            raise SkylineError(st, self._L.sky_status_str(st).decode())
        return [o[: counts[i]] for i, o in enumerate(self.outs)], ms.value

    def close(self):
        if getattr(self, "_h", None):
            self._L.sky_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


STATIC_MAX_POINTS = 65536


def skyline_static(points, out=None):
    """Sky(points) through sky_skyline_static, the entry point that allocates
    no device memory (for callers that cannot call cudaMalloc).  points: a
    CUDA float32 [N, d] tensor with N <= STATIC_MAX_POINTS; runs on the
    tensor's current stream.  Returns a CUDA int32 tensor of ascending
    indices (a view of `out` if given, which must be device memory of
    capacity >= N).  Raises SkylineError on a non-OK status."""
    import torch
    L = load()
    if not _is_cuda_tensor(points) or points.dtype != torch.float32 or points.dim() != 2:
        raise ValueError("points must be a CUDA float32 [N, d] tensor")
    points = points.contiguous()
    n, d = points.shape
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.int32, device=points.device)
    cnt = ctypes.c_uint64(0)
    stream = torch.cuda.current_stream(points.device).cuda_stream
    with torch.cuda.device(points.device):
        st = L.sky_skyline_static(ctypes.c_void_p(points.data_ptr()), n, d, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.byref(cnt), ctypes.c_void_p(stream))
    if st != SKY_OK:
        raise SkylineError(st, L.sky_status_str(st).decode())
    return out[: cnt.value]

_default_ctx = None


def skyline(points, **kw):
    """Sky(points) on CUDA device 0 with a process-wide default context."""
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context(0)
    return _default_ctx.skyline(points, **kw)
