"""Writes full_size_skylines.json: the oracle's skyline of each full-size
workload the GPU tests check bit-exactly, stored as |Sky| and the SHA-256 of
the ascending uint32 index array (little-endian), next to the SHA-256 of the
generated FP32 input (so that a generator difference between machines is
reported as such).  Calls only oracle/ and the seeded generators.  The
result of every partitioning, representative and merge option equals this
one set (Prop. 1, Prop. 2), so one oracle run per workload serves all of
them.  Run: python tests/golden/make_full_size.py [name ...]
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
        idx = O.skyline_indices(x).astype("<u4")
        data[name] = {"kind": kind, "n": n, "d": d, "seed": seed, "input_sha256": sha(x.astype("<f4")),
                      "skyline": int(idx.shape[0]), "skyline_sha256": sha(idx),
                      "oracle_seconds": round(time.time() - t, 1)}
        print(name, data[name], flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
