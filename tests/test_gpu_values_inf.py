"""Points holding both +inf and -inf, against the CPU oracle (bit-exact
indices, partitions and stage codes).  Their FP32 sum is undefined (inf -
inf); both sides score such a point +inf, which keeps the SFS order a
linear extension of dominance."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

VARIANTS = [
    ("none", 1, None),
    ("random", 16, None),
    ("sliced", 8, None),
    ("grid", 1, "g"),
    ("angular", 1, "a"),
]


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2411_14968_gb300 import native
    c = native.Context(0)
    yield c
    c.close()


def _check(ctx, oracle_mod, x, scheme, p, slices, rep, merge):
    from oracle import oracle as O
    want = oracle_mod.partitioned(
        x, scheme={"random": O.RANDOM, "grid": O.GRID, "angular": O.ANGULAR, "sliced": O.SLICED,
                   "none": O.NONE}[scheme], p=p, slices=slices,
        rep={"none": 0, "sorted": 1}[rep], merge={"sequential": 0, "noseq": 1}[merge])
    idx, pid, stage = ctx.skyline(x, scheme=scheme, p=p, slices=slices, rep=rep, merge=merge, with_diag=True)
    tag = f"{scheme} p={p} slices={slices} rep={rep} merge={merge}"
    np.testing.assert_array_equal(idx, want["indices"], err_msg=tag)
    np.testing.assert_array_equal(pid, want["pid"], err_msg=tag + " pid")
    np.testing.assert_array_equal(stage, want["stage"], err_msg=tag + " stage")


def test_points_with_both_infinities(ctx, oracle_mod):
    rng = np.random.default_rng(12)
    x = rng.random((3000, 4)).astype(np.float32)
    x[:200, 1] = np.inf
    x[100:300, 3] = -np.inf          # 100 points hold both
    x[300:400, 1] = np.inf
    x[300:400, 2] = -np.inf          # both, in other attributes
    x[500:700] = x[:200]             # duplicates of them
    for scheme, p, sl in VARIANTS:
        slices = [3, 3, 3, 3] if sl == "g" else ([3, 2, 2] if sl == "a" else None)
        _check(ctx, oracle_mod, x, scheme, p, slices, rep="sorted", merge="noseq")
        _check(ctx, oracle_mod, x, scheme, p, slices, rep="none", merge="sequential")
