"""Writes workcounts_<workload>.json: the oracle's dominance-test counts for
each variant the benchmark times -- on the 1,000,000-point anticorrelated
d = 6 workload (seed 1: workcounts_ant_1m_d6.json) and on the 2,000,000-point
skewed d = 6 workload (seed 4, Angular (4,4,2,2,2) on x / column max with
Sorted representatives, sequential final phase:
workcounts_skewed_2m_d6.json; NoSeq final phase:
workcounts_skewed_2m_d6_noseq.json), on the 200,000-point skewed workload
(seed 4) with the NoSeq final phase (workcounts_skewed_200k_d6.json), and on
the 4,000,000-point quantised independent d = 8 workload (seed 3, Grid m = 2
and Random p = 256 with seed 11, as the benchmark's configuration run:
workcounts_indep_4m_d8.json; the correlated one likewise:
workcounts_corr_4m_d8.json).

The count of one variant is the number of pairwise dominance tests the
plain CPU oracle makes (SFS window tests of Algorithm 1 in every partition,
plus the tests of the final phase), i.e. the algorithmic work of the
dominance kernels; one test is d attribute compares.  Calls only oracle/ and
the seeded generator.  The local skylines of Algorithm 2 run over every host
core (the counts do not depend on the thread count; the sequential final
phase stays single-threaded).  Run: python tests/golden/make_workcounts.py
[workload ...]
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2411_14968_gb300 import datagen  # noqa: E402

# workload -> (generator kind, N, d, seed, variants)
WORKLOADS = {
    "ant_1m_d6": ("anticorrelated", 1_000_000, 6, 1, {
        "sliced": dict(scheme=O.SLICED, p=64),
        "sliced_rep": dict(scheme=O.SLICED, p=64, rep=O.REP_SORTED),
        "angular": dict(scheme=O.ANGULAR, slices=[4, 2, 2, 2, 2]),
        "angular_rep": dict(scheme=O.ANGULAR, slices=[4, 2, 2, 2, 2], rep=O.REP_SORTED),
    }),
    "skewed_2m_d6": ("skewed", 2_000_000, 6, 4, {
        "angular_rep": dict(scheme=O.ANGULAR, slices=[4, 4, 2, 2, 2], normalize=True, rep=O.REP_SORTED),
    }),
    # the quantised independent workload, N = 4M, d = 8: Grid m = 2 and Random p = 256
    "indep_4m_d8": ("independent", 4_000_000, 8, 3, {
        "grid": dict(scheme=O.GRID, slices=[2] * 8),
        "random": dict(scheme=O.RANDOM, p=256, seed=11),
    }),
    # the quantised correlated workload, N = 4M, d = 8: the same two variants
    "corr_4m_d8": ("correlated", 4_000_000, 8, 3, {
        "grid": dict(scheme=O.GRID, slices=[2] * 8),
        "random": dict(scheme=O.RANDOM, p=256, seed=11),
    }),
    # the skewed workload with the NoSeq final phase (merge_tests = NoSeq's tests)
    "skewed_2m_d6_noseq": ("skewed", 2_000_000, 6, 4, {
        "angular_rep_noseq": dict(scheme=O.ANGULAR, slices=[4, 4, 2, 2, 2], normalize=True, rep=O.REP_SORTED,
                                  merge=O.MERGE_NOSEQ),
    }),
    # the case the NoSeq kernel's profile runs (merge_tests = NoSeq's tests)
    "skewed_200k_d6": ("skewed", 200_000, 6, 4, {
        "angular_rep_noseq": dict(scheme=O.ANGULAR, slices=[4, 4, 2, 2, 2], normalize=True, rep=O.REP_SORTED,
                                  merge=O.MERGE_NOSEQ),
    }),
}


def noseq_score_cut_minimum(x, r):
    """The fewest tests any exact NoSeq with the score cut makes (Section
    4.2 with pd_i = u minus u_i, Random / Angular): a surviving tuple t must
    be tested against every s in pd_i with score(s) <= score(t), and a
    dropped one at least once.  From the oracle's own partitions and stage
    codes; scores are the oracle's left-to-right FP32 sums."""
    st, pid = r["stage"], r["pid"]
    inu = (st == O.ST_SKY) | (st == O.ST_MERGE)
    f = O.scores(x)
    fu, pu, sky = f[inu], pid[inu], st[inu] == O.ST_SKY
    order = np.sort(fu)
    total = 0
    for part in np.unique(pu):
        own = np.sort(fu[pu == part])
        t = fu[(pu == part) & sky]
        total += int((np.searchsorted(order, t, side="right") - np.searchsorted(own, t, side="right")).sum())
    total += int((~sky).sum())
    return {"merge_tests_score_cut_min": total}


def main(names):
    for wl in names or WORKLOADS:
        run(wl)


def run(wl):
    kind, N, D, SEED, variants = WORKLOADS[wl]
    x = datagen.make(kind, N, D, SEED)
    O.set_threads(os.cpu_count() or 1)
    out = {"workload": f"{kind} N={N} d={D} seed={SEED}", "machine": platform.machine(), "variants": {}}
    for name, kw in variants.items():
        t = time.time()
        r = O.partitioned(x, **kw)
        st = r["stage"]
        out["variants"][name] = {
            "local_tests": r["tests"][0],
            "merge_tests": r["tests"][1],
            **(noseq_score_cut_minimum(x, r) if kw.get("merge") == O.MERGE_NOSEQ else {}),
            "skyline": int(r["indices"].shape[0]),
            "local_union": int(((st == O.ST_SKY) | (st == O.ST_MERGE)).sum()),
            "oracle_seconds": round(time.time() - t, 1),
        }
        print(name, out["variants"][name], flush=True)
    O.set_threads(1)
    with open(os.path.join(HERE, f"workcounts_{wl}.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
