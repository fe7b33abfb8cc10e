"""Writes sweep_skylines.json: the oracle's skyline of every input of the
operating-parameter sweeps (Section 5, Table 1 and the figures on varying
size, dimensions and partitions) that ``bench.py --experiment sweeps`` runs
on the GPU, as |Sky| and the SHA-256 of the ascending uint32 index array
(little-endian), next to the SHA-256 of the generated FP32 input.  The
experiment checks every strategy's result against these values.  Calls only
oracle/ and the seeded generators.  One entry per input: every strategy and
partition count returns the same set (Prop. 1, Prop. 2).
Run: python tests/golden/make_sweeps.py [key ...]
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

OUT = os.path.join(HERE, "sweep_skylines.json")
# anticorrelated inputs of the sweeps: size (d = 4, seed 7), dimensions
# (N = 1e6, seed 8); the partition sweep reuses the size sweep's N = 1e6 input
SIZES = (100_000, 500_000, 1_000_000, 5_000_000, 10_000_000, 50_000_000, 100_000_000)
DIMS = (2, 3, 5, 6, 7)


def inputs():
    for n in SIZES:
        yield f"n={n},d=4,seed=7", (n, 4, 7)
    for d in DIMS:
        yield f"n=1000000,d={d},seed=8", (1_000_000, d, 8)


def sha(a) -> str:
    return hashlib.sha256(a.tobytes()).hexdigest()


def main(keys):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for key, (n, d, seed) in inputs():
        if keys and key not in keys:
            continue
        x = datagen.anticorrelated_blocks(n, d, seed)
        t = time.time()
        idx = O.skyline_indices(x).astype("<u4")
        data[key] = {"n": n, "d": d, "seed": seed, "input_sha256": sha(x.astype("<f4")),
                     "skyline": int(idx.shape[0]), "skyline_sha256": sha(idx),
                     "oracle_seconds": round(time.time() - t, 1)}
        print(key, data[key], flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
