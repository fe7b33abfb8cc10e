"""Pins for the CPU oracle: each test checks it against something other than
itself -- the paper's worked example, closed forms, a textbook algorithm for
d = 2, published generator outputs, brute force on tiny inputs, statistical
expectations and invariants the paper proves (Prop. 1, Prop. 2).
"""
import math
import os

import numpy as np
import pytest

from paper_2411_14968_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _staircase_2d(x):
    """Textbook 2-D skyline (minimisation), independent of Def. 1 code: sort by
    (x, y); walk groups of equal x; inside a group only the points at the
    group's minimum y can survive, and they survive iff that minimum is below
    every y seen at strictly smaller x."""
    n = x.shape[0]
    order = np.lexsort((x[:, 1], x[:, 0]))
    keep = np.zeros(n, bool)
    best = math.inf
    i = 0
    while i < n:
        j = i
        while j < n and x[order[j], 0] == x[order[i], 0]:
            j += 1
        grp = order[i:j]
        ymin = x[grp, 1].min()
        if ymin < best:
            keep[grp[x[grp, 1] == ymin]] = True
        best = min(best, ymin)
        i = j
    return keep


def _expected_maxima(n, d):
    """E|Sky| of n i.i.d. continuous points in d dimensions (Bentley, Kung,
    Schkolnick & Thompson 1978): A(n,1) = 1, A(n,d) = A(n-1,d) + A(n,d-1)/n."""
    a = [1.0] * (n + 1)  # A(k, 1)
    for _ in range(2, d + 1):
        b = [0.0] * (n + 1)
        for k in range(1, n + 1):
            b[k] = b[k - 1] + a[k] / k
        a = b
    return a[n]


# ---------------------------------------------------------------- Def. 1


def test_dominance_truth_table(oracle_mod):
    dom = oracle_mod.dominates
    assert dom([1, 2], [1, 3])
    assert dom([0, 0, 0], [0, 0, 1])
    assert not dom([1, 2], [1, 2])          # duplicates never dominate
    assert not dom([1, 3], [2, 2])          # incomparable
    assert not dom([1, 3], [1, 2])          # worse on one attribute
    assert not dom([-0.0, 1.0], [0.0, 1.0])  # -0 == +0
    assert dom([1, 1], [1, np.inf])
    assert not dom([np.inf], [np.inf])
    assert dom([-1.0, 5.0], [0.0, 5.0])     # negatives compare as reals


def test_example1_cars(oracle_mod):
    names, rows = [], []
    with open(os.path.join(GOLDEN, "example1_cars.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            n, a, b = line.split()
            names.append(n)
            rows.append((float(a), float(b)))
    pts = np.array(rows, np.float32)
    sky = {names[i] for i in np.nonzero(oracle_mod.skyline_brute(pts))[0]}
    assert sky == {"C1", "C2", "C4"}
    assert set(names[i] for i in oracle_mod.skyline_indices(pts)) == sky
    c = {nm: pts[i] for i, nm in enumerate(names)}
    assert oracle_mod.dominates(c["C4"], c["C3"]) and oracle_mod.dominates(c["C4"], c["C5"])
    # top-1 of monotone functions is in the skyline (Section 2)
    assert names[int(np.argmin(pts[:, 0]))] == "C1"
    assert names[int(np.argmin(pts[:, 1]))] == "C4"
    assert names[int(np.argmin(pts.sum(1)))] == "C2"


def test_d1_closed_form(oracle_mod):
    rng = np.random.default_rng(5)
    for n in (1, 2, 17, 1000):
        x = rng.integers(0, 7, size=(n, 1)).astype(np.float32)
        want = np.nonzero(x[:, 0] == x[:, 0].min())[0]
        np.testing.assert_array_equal(oracle_mod.skyline_indices(x), want)
        np.testing.assert_array_equal(np.nonzero(oracle_mod.skyline_brute(x))[0], want)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("n,levels", [(50, 8), (3000, 64), (200000, 0)])
def test_d2_staircase(oracle_mod, seed, n, levels):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 2))
    if levels:
        x = np.floor(x * levels) / levels  # many ties and duplicates
    x = x.astype(np.float32)
    want = np.nonzero(_staircase_2d(x))[0]
    np.testing.assert_array_equal(oracle_mod.skyline_indices(x), want)
    if n <= 3000:
        np.testing.assert_array_equal(np.nonzero(oracle_mod.skyline_brute(x))[0], want)


def test_perfectly_correlated(oracle_mod):
    rng = np.random.default_rng(3)
    t = rng.permutation(500).astype(np.float32)
    x = np.repeat(t[:, None], 5, axis=1)
    np.testing.assert_array_equal(oracle_mod.skyline_indices(x), [int(np.argmin(t))])


def test_all_equal_points_all_in_skyline(oracle_mod):
    x = np.full((64, 3), 0.25, np.float32)
    np.testing.assert_array_equal(oracle_mod.skyline_indices(x), np.arange(64))


def test_empty_and_single(oracle_mod):
    assert oracle_mod.skyline_indices(np.zeros((0, 3), np.float32)).shape == (0,)
    np.testing.assert_array_equal(oracle_mod.skyline_indices(np.ones((1, 4), np.float32)), [0])


# --------------------------------------------------- Algorithm 1 (SFS)


@pytest.mark.parametrize("kind", ["anticorrelated", "independent", "correlated", "skewed"])
@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
def test_sfs_equals_brute_force(oracle_mod, kind, d):
    for seed in (1, 2):
        x = datagen.make(kind, 1500, d, seed)
        np.testing.assert_array_equal(oracle_mod.sfs(x)[0], oracle_mod.skyline_brute(x))


def test_sfs_test_count_hand_case(oracle_mod):
    # A=(1,1) f=2, B=(0,3) f=3, C=(2,2) f=4.  Window after A: {A}; B vs A: 1
    # test, kept; C vs A: 1 test, dominated.  Two tests in all.
    x = np.array([[2, 2], [0, 3], [1, 1]], np.float32)
    mask, tests = oracle_mod.sfs(x)
    assert mask.tolist() == [False, True, True]
    assert tests == 2


def test_score_is_left_to_right_fp32(oracle_mod):
    # ((2^24 + 1) + 1) rounds to 2^24 at each step; the exact sum is 2^24 + 2.
    x = np.array([[2.0 ** 24, 1.0, 1.0], [1.0, 1.0, 2.0 ** 24]], np.float32)
    f = oracle_mod.scores(x)
    assert f[0] == np.float32(2.0 ** 24)
    assert f[1] == np.float32(2.0 ** 24 + 2)


def test_expected_skyline_size_uniform(oracle_mod):
    n = 20000
    for d in (3, 4):
        sizes = [int(oracle_mod.sfs(datagen.independent(n, d, s, quantised=False))[0].sum())
                 for s in range(8)]
        want = _expected_maxima(n, d)
        assert abs(np.mean(sizes) - want) < 0.1 * want, (d, np.mean(sizes), want)


# ------------------------------------------------------------ invariants


def test_invariants_permutation_monotone_maps_duplicates(oracle_mod):
    x = datagen.anticorrelated(2000, 4, 11)
    base = set(oracle_mod.skyline_indices(x).tolist())
    perm = np.random.default_rng(0).permutation(x.shape[0])
    got = oracle_mod.skyline_indices(x[perm])
    assert set(perm[got].tolist()) == base
    # strictly increasing exact maps per column: x -> 2x and x -> dense rank
    assert set(oracle_mod.skyline_indices(2 * x).tolist()) == base
    ranks = np.empty_like(x)
    for j in range(x.shape[1]):
        _, inv = np.unique(x[:, j], return_inverse=True)
        ranks[:, j] = inv.astype(np.float32)
    assert set(oracle_mod.skyline_indices(ranks).tolist()) == base
    # appending a copy of a skyline point adds the copy to the skyline
    k = min(base)
    y = np.vstack([x, x[k:k + 1]])
    assert set(oracle_mod.skyline_indices(y).tolist()) == base | {x.shape[0]}


def test_output_is_exact_skyline(oracle_mod):
    """(I1) no output dominated by an output; (I2) every other point dominated
    by some output point -- together equivalent to correctness."""
    x = datagen.skewed(1200, 5, 4)
    idx = oracle_mod.skyline_indices(x)
    s = x[idx]
    rest = np.setdiff1d(np.arange(x.shape[0]), idx)
    assert oracle_mod.relative_skyline(s, s).all()
    assert not oracle_mod.relative_skyline(x[rest], s).any()


def test_relative_skyline(oracle_mod):
    x = datagen.independent(500, 3, 9)
    np.testing.assert_array_equal(oracle_mod.relative_skyline(x, x), oracle_mod.skyline_brute(x))
    assert oracle_mod.relative_skyline(x, np.zeros((0, 3), np.float32)).all()
    c = np.zeros((1, 3), np.float32)
    r = np.array([[0, 0, 0], [0, 0, 1], [1, 1, 1]], np.float32)
    assert oracle_mod.relative_skyline(r, c).tolist() == [True, False, False]


# ------------------------------------------------------- partitioning


def test_splitmix64_published_outputs(oracle_mod):
    # first outputs of SplitMix64 started from state 0 (Steele, Lea & Flood 2014)
    assert oracle_mod.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert oracle_mod.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert oracle_mod.splitmix64(0, 2) == 0x06C45D188009454F


def test_grid_hand_values(oracle_mod):
    x = np.array([[0.25, 0.75], [0.5, 0.0], [1.0, 1.0], [-3.0, 0.49], [0.0, np.inf]], np.float32)
    # digits (0,1) (1,0) (1,1) (0,0) (0,1) with m = 2; index = c1 + 2 c2 (Section 3.2)
    assert oracle_mod.assign_grid(x, [2, 2]).tolist() == [2, 1, 3, 0, 2]
    # m = 3 and 4 per dimension: digits (0,3) (1,0) (2,3) (0,1) (0,3)
    assert oracle_mod.assign_grid(x, [3, 4]).tolist() == [9, 1, 11, 3, 9]


def test_grid_cells_are_dominance_consistent(oracle_mod):
    x = datagen.independent(400, 3, 2)
    pid = oracle_mod.assign_grid(x, [3, 3, 3])
    c = np.stack([pid % 3, (pid // 3) % 3, pid // 9], 1)
    # if c_i grid-dominates c_h then every tuple of c_i dominates every tuple of c_h
    for i in range(0, 400, 7):
        for h in range(400):
            if np.all(c[i] < c[h]):
                assert oracle_mod.dominates(x[i], x[h])


def test_grid_filter_hand_and_soundness(oracle_mod):
    m = [2, 2]
    x = np.array([[0.1, 0.1], [0.9, 0.9], [0.8, 0.2]], np.float32)
    pid = oracle_mod.assign_grid(x, m)
    assert oracle_mod.grid_filter(pid, 2, m).tolist() == [False, False, False, True]
    x2 = np.array([[0.1, 0.9], [0.9, 0.1]], np.float32)
    assert not oracle_mod.grid_filter(oracle_mod.assign_grid(x2, m), 2, m).any()
    for kind in ("independent", "correlated"):
        x = datagen.make(kind, 3000, 3, 5)
        pid = oracle_mod.assign_grid(x, [4, 4, 4])
        dropped = oracle_mod.grid_filter(pid, 3, [4, 4, 4])
        sky = oracle_mod.skyline_brute(x)
        assert not np.any(sky & dropped[pid])
        assert dropped.any()


def test_angular_matches_atan2(oracle_mod):
    rng = np.random.default_rng(8)
    for d, m in ((2, [4]), (3, [5, 5]), (6, [4, 2, 2, 2, 2]), (4, [3, 7, 2])):
        x = rng.random((5000, d)).astype(np.float32)
        x[:50, 0] = 0.0
        pid = oracle_mod.assign_angular(x, m)
        xd = x.astype(np.float64)
        w = 1
        for i in range(d - 1):
            phi = np.arctan2(np.sqrt((xd[:, i + 1:] ** 2).sum(1)), xd[:, i])
            v = 2.0 * phi * m[i] / np.pi
            want = np.minimum(np.floor(v), m[i] - 1).astype(np.int64)
            got = (pid // w) % m[i]
            near = np.abs(v - np.round(v)) < 1e-5
            bad = (got != want) & ~near
            assert not bad.any(), (d, i, np.nonzero(bad)[0][:5])
            w *= m[i]
        assert pid.max() < w


def test_random_partitions_equinumerous(oracle_mod):
    n, p = 10007, 16
    a = oracle_mod.assign_random(n, p, 42)
    cnt = np.bincount(a, minlength=p)
    assert cnt.min() == n // p and cnt.max() == -(-n // p)
    b = oracle_mod.assign_random(n, p, 43)
    assert (a != b).mean() > 0.5
    # not index order: the first 1/p of the indices spread over all partitions
    assert len(np.unique(a[: n // p])) == p


GAMMA = 0x9E3779B97F4A7C15  # SplitMix64's state increment (Steele, Lea & Flood 2014)


def test_random_hand_instances(oracle_mod):
    # Section 3.1 as read here: pid = floor(rank * p / N), rank of the point's
    # SplitMix64 key in ascending order (ties by index).  The keys below are
    # the published outputs pinned in test_splitmix64_published_outputs:
    #   seed 0: key(0) = 0xE220..., key(1) = 0x6E78..., key(2) = 0x06C4...
    # so the ascending order is point 2, 1, 0 and the ranks are (2, 1, 0).
    #   p = 3: floor(r * 3 / 3) = r           -> (2, 1, 0)
    #   p = 2: floor(r * 2 / 3): r 0,1 -> 0, r 2 -> 1 -> (1, 0, 0)
    # (rank % p would give (0, 1, 0); a descending rank or index order (0, 0, 1).)
    assert oracle_mod.assign_random(3, 3, 0).tolist() == [2, 1, 0]
    assert oracle_mod.assign_random(3, 2, 0).tolist() == [1, 0, 0]
    assert oracle_mod.assign_random(3, 1, 0).tolist() == [0, 0, 0]
    # Starting the state one increment earlier (seed = -GAMMA mod 2^64) shifts
    # the stream by one: key(i) = published output i - 1 for i >= 1, and key(0)
    # mixes the state 0, which every xor-shift and multiply keeps at 0.  Keys
    # (0, 0xE220..., 0x6E78..., 0x06C4...): ascending order 0, 3, 2, 1, so the
    # ranks of points 0..3 are (0, 3, 2, 1).
    #   p = 2: floor(r / 2)      -> (0, 1, 1, 0)
    #   p = 3: floor(3 r / 4): r 0 -> 0, 1 -> 0, 2 -> 1, 3 -> 2 -> (0, 2, 1, 0)
    #   p = 4: r                 -> (0, 3, 2, 1)
    s = (-GAMMA) % (1 << 64)
    assert oracle_mod.splitmix64(s, 0) == 0
    assert oracle_mod.splitmix64(s, 1) == 0xE220A8397B1DCDAF
    assert oracle_mod.assign_random(4, 2, s).tolist() == [0, 1, 1, 0]
    assert oracle_mod.assign_random(4, 3, s).tolist() == [0, 2, 1, 0]
    assert oracle_mod.assign_random(4, 4, s).tolist() == [0, 3, 2, 1]


def test_sliced_hand_instance_run_across_a_boundary(oracle_mod):
    # Section 3.4 as read here: order by (x_0, f, index), nominal pid =
    # floor(rank * p / N), and a run of equal (x_0, f) takes the pid of its
    # first member (the boundary moves to the end of the run).
    x = np.array([[0.25, 0.75],   # 0: f = 1.0
                  [0.75, 0.0],    # 1: f = 0.75
                  [0.0, 1.0],     # 2: f = 1.0
                  [0.25, 0.5],    # 3: f = 0.75
                  [0.5, 0.5],     # 4: f = 1.0
                  [0.25, 0.5]],   # 5: f = 0.75 (a copy of 3)
                 np.float32)
    # Order: 2 (x0 0), then x0 = 0.25 by f: 3, 5 (f 0.75, by index), 0 (f 1.0),
    # then 4 (x0 0.5), 1 (x0 0.75): ranks of points 0..5 = (3, 5, 0, 1, 4, 2).
    # Points 3 and 5 (ranks 1, 2) are one run, which starts at rank 1, so the
    # run-start ranks are (3, 5, 0, 1, 4, 1).
    #   p = 3: floor(s / 2) -> (1, 2, 0, 0, 2, 0)   (rank 2 alone would be slice 1)
    #   p = 2: floor(s / 3) -> (1, 1, 0, 0, 1, 0)
    #   p = 6: s            -> (3, 5, 0, 1, 4, 1)   (slice 2 stays empty)
    assert oracle_mod.assign_sliced(x, 3).tolist() == [1, 2, 0, 0, 2, 0]
    assert oracle_mod.assign_sliced(x, 2).tolist() == [1, 1, 0, 0, 1, 0]
    assert oracle_mod.assign_sliced(x, 6).tolist() == [3, 5, 0, 1, 4, 1]
    # slicing on attribute 1: order 1 (x1 0), 3, 5, 4 (x1 0.5; f 0.75, 0.75,
    # 1.0), 0 (0.75), 2 (1.0); run 3, 5 starts at rank 1; ranks (4, 0, 5, 1, 3, 2)
    # -> run starts (4, 0, 5, 1, 3, 1); p = 3: floor(s / 2) -> (2, 0, 2, 0, 1, 0)
    assert oracle_mod.assign_sliced(x, 3, dim=1).tolist() == [2, 0, 2, 0, 1, 0]


def test_sliced_sizes_and_dominance_order(oracle_mod):
    x = datagen.anticorrelated(4000, 4, 3)
    pid = oracle_mod.assign_sliced(x, 8)
    cnt = np.bincount(pid, minlength=8)
    assert cnt.max() - cnt.min() <= 1
    order = np.argsort(x[:, 0], kind="stable")
    assert np.all(np.diff(pid[order].astype(np.int64)) >= 0)
    # quantised data: slice boundaries never split an equal-key run, so a
    # dominator is never in a later slice (makes pd_i = {u_j : j < i} sound)
    y = datagen.independent(600, 3, 1)
    y = np.floor(y * 4) / 4
    y = y.astype(np.float32)
    q = oracle_mod.assign_sliced(y, 6)
    for s in range(600):
        for t in range(600):
            if q[s] > q[t]:
                assert not oracle_mod.dominates(y[s], y[t])


# ------------------------------------------------ Algorithm 2 and Section 4

SCHEMES = [
    ("none", {"scheme": 4}),
    ("random", {"scheme": 0, "p": 7, "seed": 99}),
    ("grid", {"scheme": 1, "slices": None}),
    ("angular", {"scheme": 2, "slices": None}),
    ("sliced", {"scheme": 3, "p": 5}),
]


@pytest.mark.parametrize("kind", ["anticorrelated", "independent", "correlated", "skewed"])
@pytest.mark.parametrize("d", [2, 3, 5, 8])
def test_partitioned_equals_skyline(oracle_mod, kind, d):
    """Prop. 1 (any partitioning) and Prop. 2 (NoSeq) with Grid Filtering and
    Sorted representatives: every variant returns Sky(r)."""
    x = datagen.make(kind, 700, d, d * 7 + 1)
    want = np.nonzero(oracle_mod.skyline_brute(x))[0]
    norm = kind == "skewed"
    for name, kw in SCHEMES:
        kw = dict(kw)
        if name == "grid":
            kw["slices"] = [2] * d if d > 3 else [3] * d
        if name == "angular":
            kw["slices"] = ([3, 2, 2, 2, 2, 2, 2][: d - 1]) if d > 1 else []
        for rep in (0, 1, 2):
            for merge in (0, 1):
                r = oracle_mod.partitioned(x, normalize=norm, rep=rep, merge=merge, **kw)
                np.testing.assert_array_equal(r["indices"], want, err_msg=f"{name} rep={rep} merge={merge}")
                st = r["stage"]
                assert np.all((st >= 1) & (st <= 5))
                # every point removed before the merge is dominated by some point
                early = np.nonzero((st == 2) | (st == 3) | (st == 4))[0]
                assert not oracle_mod.relative_skyline(x[early], x).any()
                # points dropped inside a partition are dominated inside it
                for i in np.nonzero(st == 4)[0][:50]:
                    mates = x[r["pid"] == r["pid"][i]]
                    assert not oracle_mod.relative_skyline(x[i:i + 1], mates)[0]


def test_threaded_loops_change_nothing(oracle_mod):
    """Algorithm 2's local skylines and NoSeq's checks are independent per
    partition / per tuple: with several threads the index set, partitions,
    stage codes and dominance-test counts are those of the plain loops."""
    x = datagen.anticorrelated(6000, 5, 3)
    cases = [dict(scheme=oracle_mod.SLICED, p=37), dict(scheme=oracle_mod.RANDOM, p=16, seed=3),
             dict(scheme=oracle_mod.GRID, slices=[2] * 5), dict(scheme=oracle_mod.ANGULAR, slices=[3, 2, 2, 2])]
    try:
        for kw in cases:
            for rep in (0, 1):
                for merge in (0, 1):
                    oracle_mod.set_threads(1)
                    a = oracle_mod.partitioned(x, rep=rep, merge=merge, **kw)
                    oracle_mod.set_threads(4)
                    b = oracle_mod.partitioned(x, rep=rep, merge=merge, **kw)
                    for key in ("indices", "pid", "stage"):
                        np.testing.assert_array_equal(a[key], b[key], err_msg=f"{kw} {key}")
                    assert a["tests"] == b["tests"]
    finally:
        oracle_mod.set_threads(1)


def test_partitioned_edge_cases(oracle_mod):
    for n in (0, 1, 2, 3):
        x = datagen.independent(n, 3, 1)
        want = np.nonzero(oracle_mod.skyline_brute(x))[0] if n else np.zeros(0, np.uint32)
        for name, kw in SCHEMES:
            kw = dict(kw)
            if name == "grid":
                kw["slices"] = [2, 2, 2]
            if name == "angular":
                kw["slices"] = [2, 2]
            r = oracle_mod.partitioned(x, rep=1, merge=1, **kw)
            np.testing.assert_array_equal(r["indices"], want)
    # all points identical: every point is in the skyline
    x = np.full((100, 4), 0.5, np.float32)
    r = oracle_mod.partitioned(x, scheme=3, p=10, rep=1, merge=1)
    np.testing.assert_array_equal(r["indices"], np.arange(100))


def test_region_volume_hand_values(oracle_mod):
    # §4.1: V = prod (1 - t[i]) over [0,1]; attributes outside [0,1] are
    # clamped (the part of the dominance region inside the unit cube)
    assert oracle_mod.region_volume([0.5, 0.2]) == pytest.approx(0.4)
    assert oracle_mod.region_volume([0.0, 0.0, 0.0]) == 1.0
    assert oracle_mod.region_volume([1.2, -0.3, 0.25]) == 0.0
    assert oracle_mod.region_volume([-0.5, 0.75]) == pytest.approx(0.25)
    assert oracle_mod.region_volume([1.0, 1.0], scale=[2.0, 2.0]) == pytest.approx(0.25)


def test_region_volume_is_dominance_region_measure(oracle_mod):
    # independent pin: the volume equals the fraction of uniform points of the
    # unit cube that t dominates (Monte Carlo, 4 standard errors)
    rng = np.random.default_rng(3)
    u = rng.random((200_000, 3)).astype(np.float32)
    for t in ([0.2, 0.5, 0.1], [0.7, 0.05, 0.3], [0.33, 0.33, 0.33]):
        frac = np.mean(np.all(u >= np.float32(t), axis=1))
        v = oracle_mod.region_volume(t)
        assert abs(frac - v) < 4 * np.sqrt(v * (1 - v) / u.shape[0]) + 1e-9, (t, frac, v)


def test_region_representatives_differ_from_sorted(oracle_mod):
    # one partition: A has the lowest score (the Sorted representative), B
    # the largest dominance region (the Region representative); C is
    # dominated by B only, D by A only, E by neither
    x = np.array([[0.10, 0.70],   # A: score 0.80, V = 0.9 * 0.3 = 0.27
                  [0.40, 0.45],   # B: score 0.85, V = 0.6 * 0.55 = 0.33
                  [0.50, 0.50],   # C
                  [0.15, 0.90],   # D
                  [0.05, 0.99]], np.float32)  # E (skyline)
    srt = oracle_mod.partitioned(x, rep=oracle_mod.REP_SORTED)
    reg = oracle_mod.partitioned(x, rep=oracle_mod.REP_REGION)
    np.testing.assert_array_equal(srt["indices"], [0, 1, 4])
    np.testing.assert_array_equal(reg["indices"], [0, 1, 4])
    assert srt["stage"][3] == oracle_mod.ST_REP and srt["stage"][2] == oracle_mod.ST_LOCAL
    assert reg["stage"][2] == oracle_mod.ST_REP and reg["stage"][3] == oracle_mod.ST_LOCAL
    # k = 2 Region representatives per partition: both B and A
    reg2 = oracle_mod.partitioned(x, rep=oracle_mod.REP_REGION, reps_per_partition=2)
    assert reg2["stage"][2] == oracle_mod.ST_REP and reg2["stage"][3] == oracle_mod.ST_REP


def test_grid_filter_drops_in_pipeline(oracle_mod):
    x = datagen.correlated(3000, 4, 2)
    r = oracle_mod.partitioned(x, scheme=1, slices=[2, 2, 2, 2])
    assert (r["stage"] == 2).sum() > 0


# ------------------------------------------------------------- generators


def test_generators_shapes_and_ranges():
    a = datagen.anticorrelated(5000, 6, 1)
    assert a.shape == (5000, 6) and a.dtype == np.float32
    assert a.min() >= 0 and a.max() <= 1
    s = a.astype(np.float64).sum(1) / 6
    # rejection outside [0,1]^d favours smaller plane offsets, so the median
    # sits a little below the drawn mean of 0.5
    assert 0.44 < np.median(s) < 0.51 and 0.02 < s.std() < 0.07
    q = datagen.independent(5000, 8, 1)
    assert np.all(q * 256 == np.rint(q * 256))
    c = datagen.correlated(5000, 8, 1)
    assert np.corrcoef(c[:, 0], c[:, 1])[0, 1] > 0.9
    k = datagen.skewed(20000, 6, 1)
    assert k.min() > 0
    _, counts = np.unique(k, axis=0, return_counts=True)
    assert (counts > 1).sum() > 0.05 * 20000 / 2
    assert np.all((k == k.max(0)).mean(0) > 0.03)
    np.testing.assert_array_equal(datagen.anticorrelated(100, 3, 7), datagen.anticorrelated(100, 3, 7))


def test_key_scale_column_max(oracle_mod):
    x = np.array([[0.5, -2.0, 3.0], [4.0, -1.0, np.inf]], np.float32)
    # positive finite column maxima scale the key; otherwise the scale is 1
    assert oracle_mod.key_scale(x).tolist() == [4.0, 1.0, 1.0]
    g = oracle_mod.assign_grid(np.array([[2.0, 0.0, 0.0]], np.float32), [2, 2, 2], normalize=False)
    assert g.tolist() == [1]


def test_dense_ranks_hand_instance(oracle_mod):
    # column 0 holds {1, 0.5, 1, 0.25}: distinct ascending 0.25 < 0.5 < 1, so
    # the ranks are 2, 1, 2, 0 and there are 3 distinct values; column 1
    # holds {-0.0, +0.0, 2, 2}: -0.0 and +0.0 are one value (below 2), so the
    # ranks are 0, 0, 1, 1 and there are 2
    x = np.array([[1.0, -0.0], [0.5, 0.0], [1.0, 2.0], [0.25, 2.0]], np.float32)
    ranks, distinct = oracle_mod.dense_ranks(x)
    np.testing.assert_array_equal(ranks, [[2, 0], [1, 0], [2, 1], [0, 1]])
    np.testing.assert_array_equal(distinct, [3, 2])
    # no points: no distinct values
    r0, d0 = oracle_mod.dense_ranks(np.zeros((0, 3), np.float32))
    assert r0.shape == (0, 3)
    np.testing.assert_array_equal(d0, [0, 0, 0])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dense_ranks_brute_force(oracle_mod, seed):
    # rank = how many distinct values of the column lie below the value,
    # counted with a Python set (which, like ==, takes -0.0 and +0.0 as one)
    rng = np.random.default_rng(seed)
    x = (rng.integers(-4, 5, size=(60, 4)) / 4).astype(np.float32)  # many ties, both zeros
    x[rng.random(x.shape) < 0.1] *= np.float32(-1.0)
    ranks, distinct = oracle_mod.dense_ranks(x)
    for a in range(4):
        vals = {float(v) for v in x[:, a]}
        assert distinct[a] == len(vals)
        for i in range(60):
            assert ranks[i, a] == sum(1 for v in vals if v < float(x[i, a]))


@pytest.mark.parametrize("kind,d", [("anticorrelated", 3), ("independent", 6), ("correlated", 8)])
def test_dense_ranks_keep_the_skyline(oracle_mod, kind, d):
    # Def. 1 compares attributes only by order, and the dense rank is strictly
    # increasing in the value, so the skyline of the ranks is the skyline of
    # the values; quantised inputs put ties into every column
    x = getattr(datagen, kind)(3000, d, 40 + d)
    for pts in (x, np.round(x * 16) / 16):
        pts = pts.astype(np.float32)
        ranks, distinct = oracle_mod.dense_ranks(pts)
        assert (ranks.max(axis=0) + 1 == distinct).all()
        np.testing.assert_array_equal(oracle_mod.skyline_indices(ranks.astype(np.float32)),
                                      oracle_mod.skyline_indices(pts))


def test_dense_ranks_and_skyline_properties_hypothesis(oracle_mod):
    """Generated inputs with infinities, signed zeros, subnormals and many
    ties: the dense ranks equal a Python count of smaller distinct values,
    and the skyline of the ranks is the brute-force skyline of the values."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    values = st.sampled_from([0.0, -0.0, 1e-40, -1e-40, 0.5, 1.0, 2.0, -3.0, 3.4e38, float("inf"), float("-inf")])

    @hyp.settings(max_examples=60, deadline=None)
    @hyp.given(st.integers(1, 5).flatmap(
        lambda d: st.lists(st.lists(values, min_size=d, max_size=d), min_size=1, max_size=40)))
    def check(rows):
        x = np.array(rows, np.float32)
        ranks, distinct = oracle_mod.dense_ranks(x)
        for a in range(x.shape[1]):
            vals = {float(v) for v in x[:, a]}
            assert distinct[a] == len(vals)
            for i in range(x.shape[0]):
                assert ranks[i, a] == sum(1 for v in vals if v < float(x[i, a]))
        want = np.nonzero(oracle_mod.skyline_brute(x))[0]
        np.testing.assert_array_equal(oracle_mod.skyline_indices(ranks.astype(np.float32)), want)
        np.testing.assert_array_equal(oracle_mod.skyline_indices(x), want)

    check()


def test_score_of_a_tuple_with_both_infinities(oracle_mod):
    # (0, +inf, -inf) has no FP32 sum (inf - inf); it dominates (1, +inf, 0)
    # (0 <= 1, +inf <= +inf, -inf < 0), so SFS must place it first: its score
    # is taken as +inf, the score of (1, +inf, 0), and the tie order
    # (attributes, then index) puts it before; (2, 1, 1) is incomparable
    x = np.array([[1.0, np.inf, 0.0], [0.0, np.inf, -np.inf], [2.0, 1.0, 1.0]], np.float32)
    assert oracle_mod.scores(x)[1] == np.inf
    np.testing.assert_array_equal(np.nonzero(oracle_mod.skyline_brute(x))[0], [1, 2])
    np.testing.assert_array_equal(oracle_mod.skyline_indices(x), [1, 2])
    for kw in (dict(scheme=oracle_mod.SLICED, p=2), dict(scheme=oracle_mod.NONE, rep=oracle_mod.REP_SORTED)):
        np.testing.assert_array_equal(oracle_mod.partitioned(x, **kw)["indices"], [1, 2])


def test_every_scheme_on_generated_special_values(oracle_mod):
    """Prop. 1 and Prop. 2 on generated inputs full of infinities, signed
    zeros, subnormals and ties: every partitioning, representative filter
    and final phase returns the Def. 1 brute-force skyline."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    O = oracle_mod
    values = st.sampled_from([0.0, -0.0, 1e-40, -1e-40, 0.25, 0.5, 1.0, 2.0, -3.0, 3.4e38,
                              float("inf"), float("-inf")])

    @hyp.settings(max_examples=80, deadline=None)
    @hyp.given(st.integers(2, 5).flatmap(
        lambda d: st.lists(st.lists(values, min_size=d, max_size=d), min_size=1, max_size=30)))
    def check(rows):
        x = np.array(rows, np.float32)
        d = x.shape[1]
        want = np.nonzero(O.skyline_brute(x))[0]
        for kw in (dict(scheme=O.GRID, slices=[2] * d), dict(scheme=O.GRID, slices=[3] * d, grid_filter=False),
                   dict(scheme=O.ANGULAR, slices=[2] * (d - 1)), dict(scheme=O.RANDOM, p=3, rep=O.REP_REGION),
                   dict(scheme=O.SLICED, p=4, slice_dim=d - 1, rep=O.REP_SORTED),
                   dict(scheme=O.GRID, slices=[2] * d, merge=O.MERGE_NOSEQ, rep=O.REP_SORTED),
                   dict(scheme=O.ANGULAR, slices=[2] * (d - 1), merge=O.MERGE_NOSEQ)):
            np.testing.assert_array_equal(O.partitioned(x, **kw)["indices"], want, err_msg=str(kw))

    check()


def _numpy_skyline(x):
    """Def. 1 written with numpy broadcasting, independent of the oracle's C
    code: t is dropped iff some s has s <= t in every attribute and s < t in
    one."""
    le = (x[:, None, :] <= x[None, :, :]).all(axis=2)   # le[s, t]: s <= t everywhere
    lt = (x[:, None, :] < x[None, :, :]).any(axis=2)    # lt[s, t]: s < t somewhere
    dominated = (le & lt).any(axis=0)
    return np.nonzero(~dominated)[0].astype(np.uint32)


@pytest.mark.parametrize("kind,d", [("anticorrelated", 3), ("independent", 5), ("correlated", 7), ("skewed", 4)])
def test_oracle_against_numpy_def1(oracle_mod, kind, d):
    x = datagen.make(kind, 1200, d, 50 + d)
    rng = np.random.default_rng(d)
    special = np.array([np.inf, -np.inf, -0.0, 0.0, 1e-40], np.float32)
    y = x.copy()
    mask = rng.random(y.shape) < 0.02
    y[mask] = rng.choice(special, size=int(mask.sum()))
    for pts in (x, y):
        want = _numpy_skyline(pts)
        np.testing.assert_array_equal(np.nonzero(oracle_mod.skyline_brute(pts))[0], want)
        np.testing.assert_array_equal(oracle_mod.skyline_indices(pts), want)
        r = oracle_mod.partitioned(pts, scheme=oracle_mod.SLICED, p=6, rep=oracle_mod.REP_SORTED,
                                   merge=oracle_mod.MERGE_NOSEQ)
        np.testing.assert_array_equal(r["indices"], want)


def test_test_counters_hand_instance(oracle_mod):
    # A = (1, 0.2), B = (2, 3), C = (3, 0.5), D = (4, 0.3); Sliced p = 2 on
    # x_0 ranks them A, B, C, D, so partition 0 = {A, B}, partition 1 = {C, D}.
    # Local SFS: partition 0 in score order A (1.2), B (5): B is tested once
    # against A and dies (stage 4); partition 1: C (3.5), D (4.3): D is tested
    # once against C and survives -- 2 local tests.  u = {A, C, D}.
    # NoSeq (pd_1 = u_0 = {A}): A has no potential dominators; C and D are
    # each tested once against A and die -- 2 tests.  The sequential final
    # phase over u in score order: A, then C and D are each tested once
    # against the window {A} and die -- 2 tests.  Sky = {A}.
    x = np.array([[1.0, 0.2], [2.0, 3.0], [3.0, 0.5], [4.0, 0.3]], np.float32)
    for merge in (oracle_mod.MERGE_NOSEQ, oracle_mod.MERGE_SEQUENTIAL):
        r = oracle_mod.partitioned(x, scheme=oracle_mod.SLICED, p=2, merge=merge)
        np.testing.assert_array_equal(r["pid"], [0, 0, 1, 1])
        np.testing.assert_array_equal(r["stage"], [1, 4, 5, 5])
        assert r["tests"] == [2, 2]
        np.testing.assert_array_equal(r["indices"], [0])
