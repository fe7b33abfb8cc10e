"""Python access to the plain CPU oracle (``sky_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may use this module; the GPU library never does.

The oracle computes the skyline of the paper (Def. 1, §2) and the intermediate
results of its partitioned pattern (Algorithm 2, §3; Grid Filtering §3.2;
representative filtering §4.1; NoSeq §4.2) with single-threaded C loops.  The
C file is compiled with gcc on first use (or by ``build()``).

Every function takes and returns numpy arrays; inputs are C-contiguous FP32
``points[N, d]``.  Scheme codes: 0 Random, 1 Grid, 2 Angular, 3 Sliced,
4 None (one partition).  Stage codes returned per point: 1 in the skyline,
2 dropped by Grid Filtering, 3 dominated by a representative, 4 dominated
inside its partition, 5 dominated in the final merge.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sky_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libskyoracle.so")
_lock = threading.Lock()
_lib = None

RANDOM, GRID, ANGULAR, SLICED, NONE = 0, 1, 2, 3, 4
REP_NONE, REP_SORTED, REP_REGION = 0, 1, 2
MERGE_SEQUENTIAL, MERGE_NOSEQ = 0, 1
ST_SKY, ST_GRID, ST_REP, ST_LOCAL, ST_MERGE = 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
        # OpenMP only serves the multi-threaded CPU timing; without it the
        # oracle is built single-threaded
        r = subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, u64, u32, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        lib.orc_dominates.argtypes = [P, P, i32]
        lib.orc_dominates.restype = i32
        lib.orc_skyline_brute.argtypes = [P, i64, i32, P]
        lib.orc_relative_skyline.argtypes = [P, i64, P, i64, i32, P]
        lib.orc_scores.argtypes = [P, i64, i32, P]
        lib.orc_dense_ranks.argtypes = [P, i64, i32, P, P]
        lib.orc_sfs_all.argtypes = [P, i64, i32, P, P]
        lib.orc_sfs_all.restype = i64
        lib.orc_key_scale.argtypes = [P, i64, i32, P]
        lib.orc_region_volume.argtypes = [P, i32, P]
        lib.orc_region_volume.restype = ctypes.c_double
        lib.orc_assign_grid.argtypes = [P, i64, i32, P, P, P]
        lib.orc_assign_angular.argtypes = [P, i64, i32, P, P, P]
        lib.orc_splitmix64.argtypes = [u64, u64]
        lib.orc_splitmix64.restype = u64
        lib.orc_assign_random.argtypes = [i64, u32, u64, P]
        lib.orc_assign_sliced.argtypes = [P, i64, i32, i32, u32, P]
        lib.orc_grid_filter.argtypes = [P, i64, i32, P, P]
        lib.orc_partitioned.argtypes = [P, i64, i32, i32, u32, P, i32, i32, u64,
                                        i32, i32, u32, i32, P, P, P]
        lib.orc_partitioned.restype = i64
        lib.orc_set_threads.argtypes = [i32]
        lib.orc_max_threads.restype = i32
        _lib = lib
        return lib


def _pts(points) -> np.ndarray:
    a = np.ascontiguousarray(points, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("points must be [N, d]")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def dominates(t, s) -> bool:
    """Def. 1: t dominates s."""
    t = np.ascontiguousarray(t, dtype=np.float32)
    s = np.ascontiguousarray(s, dtype=np.float32)
    return bool(_load().orc_dominates(_ptr(t), _ptr(s), t.shape[0]))


def skyline_brute(points) -> np.ndarray:
    """Sky(r) from Def. 1 by testing every pair; returns a bool mask."""
    p = _pts(points)
    out = np.zeros(p.shape[0], dtype=np.uint8)
    if p.shape[0]:
        _load().orc_skyline_brute(_ptr(p), p.shape[0], p.shape[1], _ptr(out))
    return out.astype(bool)


def relative_skyline(r, c) -> np.ndarray:
    """Sky_c(r) (§4.2): mask over r of the tuples no tuple of c dominates."""
    r = _pts(r)
    c = _pts(c) if len(c) else np.zeros((0, r.shape[1]), np.float32)
    out = np.zeros(r.shape[0], dtype=np.uint8)
    if r.shape[0]:
        _load().orc_relative_skyline(_ptr(r), r.shape[0], _ptr(c), c.shape[0], r.shape[1], _ptr(out))
    return out.astype(bool)


def dense_ranks(points):
    """Rank space (Def. 1 compares attributes only by order): returns
    (ranks uint32 [N, d], distinct uint32 [d]), ranks[i, a] = the number of
    distinct values of column a below points[i, a] (-0.0 == +0.0)."""
    p = _pts(points)
    ranks = np.zeros(p.shape, dtype=np.uint32)
    distinct = np.zeros(p.shape[1], dtype=np.uint32)
    _load().orc_dense_ranks(_ptr(p), p.shape[0], p.shape[1], _ptr(ranks), _ptr(distinct))
    return ranks, distinct


def scores(points) -> np.ndarray:
    """f(t): FP32 sum of the attributes, added left to right."""
    p = _pts(points)
    out = np.zeros(p.shape[0], dtype=np.float32)
    if p.shape[0]:
        _load().orc_scores(_ptr(p), p.shape[0], p.shape[1], _ptr(out))
    return out


def sfs(points):
    """Algorithm 1 over the whole input; returns (bool mask, dominance tests)."""
    p = _pts(points)
    out = np.zeros(p.shape[0], dtype=np.uint8)
    tests = np.zeros(1, dtype=np.uint64)
    _load().orc_sfs_all(_ptr(p), p.shape[0], p.shape[1], _ptr(out), _ptr(tests))
    return out.astype(bool), int(tests[0])


def skyline_indices(points) -> np.ndarray:
    """Ascending 0-based indices of Sky(r) via SFS."""
    mask, _ = sfs(points)
    return np.nonzero(mask)[0].astype(np.uint32)


def key_scale(points) -> np.ndarray:
    p = _pts(points)
    out = np.ones(p.shape[1], dtype=np.float32)
    if p.shape[0]:
        _load().orc_key_scale(_ptr(p), p.shape[0], p.shape[1], _ptr(out))
    return out


def region_volume(point, scale=None) -> float:
    """§4.1: volume of the dominance region of one point inside [0,1]^d
    (attributes divided by `scale` first when given)."""
    t = np.ascontiguousarray(point, dtype=np.float32).reshape(-1)
    sc = None if scale is None else np.ascontiguousarray(scale, dtype=np.float32)
    return float(_load().orc_region_volume(_ptr(t), t.shape[0], _ptr(sc) if sc is not None else None))


def assign_grid(points, slices, normalize: bool = False) -> np.ndarray:
    p = _pts(points)
    m = np.ascontiguousarray(slices, dtype=np.uint32)
    sc = key_scale(p) if normalize else None
    out = np.zeros(p.shape[0], dtype=np.uint32)
    if p.shape[0]:
        _load().orc_assign_grid(_ptr(p), p.shape[0], p.shape[1], _ptr(m),
                                _ptr(sc) if sc is not None else None, _ptr(out))
    return out


def assign_angular(points, slices, normalize: bool = False) -> np.ndarray:
    p = _pts(points)
    m = np.ascontiguousarray(list(slices) + [1] * (8 - len(slices)), dtype=np.uint32)
    sc = key_scale(p) if normalize else None
    out = np.zeros(p.shape[0], dtype=np.uint32)
    if p.shape[0]:
        _load().orc_assign_angular(_ptr(p), p.shape[0], p.shape[1], _ptr(m),
                                   _ptr(sc) if sc is not None else None, _ptr(out))
    return out


def splitmix64(seed: int, i: int) -> int:
    return int(_load().orc_splitmix64(seed & (2**64 - 1), i))


def assign_random(n: int, p: int, seed: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint32)
    if n:
        _load().orc_assign_random(n, p, seed & (2**64 - 1), _ptr(out))
    return out


def assign_sliced(points, p: int, dim: int = 0) -> np.ndarray:
    a = _pts(points)
    out = np.zeros(a.shape[0], dtype=np.uint32)
    if a.shape[0]:
        _load().orc_assign_sliced(_ptr(a), a.shape[0], a.shape[1], dim, p, _ptr(out))
    return out


def grid_filter(pid, d: int, slices) -> np.ndarray:
    """Grid Filtering (§3.2): mask over cells that a non-empty cell grid-dominates."""
    pid = np.ascontiguousarray(pid, dtype=np.uint32)
    m = np.ascontiguousarray(slices, dtype=np.uint32)
    P = int(np.prod(m[:d], dtype=np.int64))
    out = np.zeros(P, dtype=np.uint8)
    _load().orc_grid_filter(_ptr(pid), pid.shape[0], d, _ptr(m), _ptr(out))
    return out.astype(bool)


def set_threads(n: int) -> None:
    """Threads for Algorithm 2's parallel loops (local skylines, NoSeq checks);
    1 (the default) runs the plain single-threaded loops."""
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    """Threads OpenMP offers (1 when the oracle was built without it)."""
    return int(_load().orc_max_threads())


def partitioned(points, scheme: int = NONE, p: int = 1, slices=None, normalize: bool = False,
                slice_dim: int = 0, seed: int = 0, grid_filter: bool = True,
                rep: int = REP_NONE, reps_per_partition: int = 1,
                merge: int = MERGE_SEQUENTIAL):
    """Algorithm 2 with its options.  Returns a dict with ``indices`` (ascending
    skyline indices), ``pid`` (partition per point), ``stage`` (stage code per
    point) and ``tests`` ([local SFS tests, merge tests])."""
    a = _pts(points)
    n, d = a.shape
    m = np.ones(8, dtype=np.uint32)
    if slices is not None:
        s = list(slices)
        m[:len(s)] = s
    pid = np.zeros(n, dtype=np.uint32)
    stage = np.zeros(n, dtype=np.uint8)
    tests = np.zeros(2, dtype=np.uint64)
    k = _load().orc_partitioned(_ptr(a), n, d, scheme, p, _ptr(m), int(normalize), slice_dim,
                                seed & (2**64 - 1), int(grid_filter), rep, reps_per_partition,
                                merge, _ptr(pid), _ptr(stage), _ptr(tests))
    idx = np.nonzero(stage == ST_SKY)[0].astype(np.uint32)
    assert idx.shape[0] == k
    return {"indices": idx, "pid": pid, "stage": stage, "tests": [int(tests[0]), int(tests[1])]}
