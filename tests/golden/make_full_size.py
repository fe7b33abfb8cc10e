"""Writes full_size_skylines.json: the oracle's skyline of each full-size
workload the GPU tests check bit-exactly, stored as |Sky| and the SHA-256 of
the ascending uint32 index array (little-endian), next to the SHA-256 of the
generated FP32 input (so that a generator difference between machines is
reported as such).  Calls only oracle/ and the seeded generators.  The
result of every partitioning, representative and merge option equals this
one set (Prop. 1, Prop. 2), so one oracle run per workload serves all of
them.  Run: python tests/golden/make_full_size.py [name ...]

The skewed 2M workload's skyline holds about half a million points, out of
reach of the single-threaded SFS, so its golden comes from the oracle's
Algorithm 2 instead: Angular partitions, Sorted representatives and the
NoSeq final phase, with the two parallel loops of Algorithm 2 (local
skylines, NoSeq's per-tuple checks) on every host core.  That route is
pinned equal to the plain SFS (tests/test_oracle.py: every scheme, rep and
merge option returns the brute-force skyline; threads change nothing), and
it also records the oracle's dominance-test counts of the local phase and
of NoSeq's merge.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2411_14968_gb300 import datagen  # noqa: E402

# name -> (generator kind, N, d, seed)
WORKLOADS = {
    "anticorrelated_1m_d6": ("anticorrelated", 1_000_000, 6, 1),
    "independent_q_4m_d8": ("independent", 4_000_000, 8, 3),
    "correlated_q_4m_d8": ("correlated", 4_000_000, 8, 3),
    "skewed_200k_d6": ("skewed", 200_000, 6, 4),
    "skewed_2m_d6": ("skewed", 2_000_000, 6, 4),
}
# workloads computed by Algorithm 2 with threads (see above)
PARTITIONED = {
    "skewed_2m_d6": dict(scheme=O.ANGULAR, slices=[4, 4, 2, 2, 2], normalize=True, rep=O.REP_SORTED,
                         merge=O.MERGE_NOSEQ),
}
OUT = os.path.join(HERE, "full_size_skylines.json")


def sha(a) -> str:
    return hashlib.sha256(a.tobytes()).hexdigest()


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names or WORKLOADS:
        kind, n, d, seed = WORKLOADS[name]
        x = datagen.make(kind, n, d, seed)
        t = time.time()
        extra = {}
        if name in PARTITIONED:
            threads = os.cpu_count() or 1
            O.set_threads(threads)
            r = O.partitioned(x, **PARTITIONED[name])
            O.set_threads(1)
            idx = r["indices"].astype("<u4")
            extra = {"oracle": "Algorithm 2, Angular (4,4,2,2,2) on x / column max, 1 Sorted rep, NoSeq",
                     "oracle_threads": threads, "tests_local": r["tests"][0], "tests_noseq": r["tests"][1],
                     "local_union": int(((r["stage"] == O.ST_SKY) | (r["stage"] == O.ST_MERGE)).sum())}
        else:
            idx = O.skyline_indices(x).astype("<u4")
        data[name] = {"kind": kind, "n": n, "d": d, "seed": seed, "input_sha256": sha(x.astype("<f4")),
                      "skyline": int(idx.shape[0]), "skyline_sha256": sha(idx),
                      "oracle_seconds": round(time.time() - t, 1), **extra}
        print(name, data[name], flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
