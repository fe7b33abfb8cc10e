"""Writes workcounts_ant_1m_d6.json: the oracle's dominance-test counts on the
1,000,000-point anticorrelated d = 6 workload (seed 1) for each variant the
benchmark times.

The count of one variant is the number of pairwise dominance tests the
plain CPU oracle makes (SFS window tests of Algorithm 1 in every partition,
plus the tests of the final phase), i.e. the algorithmic work of the
dominance kernels; one test is d attribute compares.  Calls only oracle/ and
the seeded generator.  Run: python tests/golden/make_workcounts.py
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2411_14968_gb300 import datagen  # noqa: E402

N, D, SEED = 1_000_000, 6, 1
VARIANTS = {
    "sliced": dict(scheme=O.SLICED, p=64),
    "sliced_rep": dict(scheme=O.SLICED, p=64, rep=O.REP_SORTED),
    "angular": dict(scheme=O.ANGULAR, slices=[4, 2, 2, 2, 2]),
    "angular_rep": dict(scheme=O.ANGULAR, slices=[4, 2, 2, 2, 2], rep=O.REP_SORTED),
}


def main():
    x = datagen.anticorrelated(N, D, SEED)
    out = {"workload": f"anticorrelated N={N} d={D} seed={SEED}", "machine": platform.machine(), "variants": {}}
    for name, kw in VARIANTS.items():
        t = time.time()
        r = O.partitioned(x, **kw)
        st = r["stage"]
        out["variants"][name] = {
            "local_tests": r["tests"][0],
            "merge_tests": r["tests"][1],
            "skyline": int(r["indices"].shape[0]),
            "local_union": int(((st == O.ST_SKY) | (st == O.ST_MERGE)).sum()),
            "oracle_seconds": round(time.time() - t, 1),
        }
        print(name, out["variants"][name], flush=True)
    with open(os.path.join(HERE, "workcounts_ant_1m_d6.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
