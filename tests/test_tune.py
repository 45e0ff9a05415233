"""Launch-shape table (tn_tune_set), launch report (tn_plan_step_info) and the
autotuner: host checks on CPU, and on a GPU that tuned plans give the same
results as untuned ones."""
import numpy as np
import pytest

import graphgen as g
from paper_2501_00227_gb300 import tn


@pytest.fixture(autouse=True)
def _clean_table():
    from paper_2501_00227_gb300 import build as B
    B.build()
    yield
    tn.tn_tune_set([])


def test_step_info_reports_every_step_and_follows_the_table():
    n, e = g.random_regular3(140, 1)
    p = tn.Plan(n, e, nrepeat=10, seed=1)
    try:
        info = tn.tn_plan_step_info(p.handle, "tropical_i32")
        assert info.shape == (p.info("tropical_i32")["nsteps"], 10)
        assert sorted(info[:, 0].tolist()) == list(range(info.shape[0]))      # exec order is a permutation
        tiled = info[info[:, 2] == 1]
        assert len(tiled) > 0
        nb, nm, nn, nk = (int(v) for v in tiled[np.argmax(tiled[:, 9]), 6:10])   # deepest reduction
        assert nk >= 6
        tn.tn_tune_set([("tropical_i32", nb, nm, nn, nk, 1, 3)])
        after = tn.tn_plan_step_info(p.handle, "tropical_i32")
        row = after[(after[:, 6] == nb) & (after[:, 7] == nm) & (after[:, 8] == nn) & (after[:, 9] == nk)]
        assert (row[:, 3] == 1).all() and (row[:, 4] == 3).all()
        tn.tn_tune_set([("tropical_i32", nb, nm, nn, nk, -1, 1)])         # force the general kernel
        after = tn.tn_plan_step_info(p.handle, "tropical_i32")
        row = after[(after[:, 6] == nb) & (after[:, 7] == nm) & (after[:, 8] == nn) & (after[:, 9] == nk)]
        assert (row[:, 2] == 0).all()
        tn.tn_tune_set([])
        assert (tn.tn_plan_step_info(p.handle, "tropical_i32") == info).all()
    finally:
        p.close()


@pytest.mark.parametrize("row", [("counting", 1, 5, 5, 5, 0, 1),     # 128 x 128 tile is tropical only
                                 ("modp", 1, 5, 5, 5, 6, 1),         # no tile shape 6
                                 ("tropical_i32", 1, 5, 5, 5, 1, 17),
                                 ("tropical_i32", -1, 5, 5, 5, 1, 1)])
def test_tune_set_rejects_malformed_rows(row):
    with pytest.raises(tn.TNError) as ei:
        tn.tn_tune_set([row])
    assert ei.value.code == tn.TN_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("semiring,primes", [("tropical_i32", None), ("counting", None),
                                              ("modp", tuple(tn.PRIMES31[:3]))])
def test_autotuned_plans_give_the_same_results(semiring, primes):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_00227_gb300 import tune
    plans = [tn.Plan(*g.random_regular3(100, s), nrepeat=4, seed=1) for s in (1, 2)]
    try:
        ref = [p.contract(semiring, primes) for p in plans]
        out = tune.autotune(plans, semiring, primes, min_ops_bits=16)
        assert out["shapes"] > 0 and out["candidates"] > 0
        assert [p.contract(semiring, primes) for p in plans] == ref
    finally:
        for p in plans:
            p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5])
def test_every_tile_shape_gives_the_oracle_results(tile):
    """Every GEMM-tile step forced to one tile shape (with and without k
    split) through the launch table: results equal the oracle's."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    for spec in ("reg3:60:1", "ksg:9:0.8:2"):
        n, e = g.by_name(spec)
        o = O.greedy_order(n, e, nrepeat=4, seed=1)
        p = tn.Plan(n, e, o)
        try:
            want = {"tropical_i32": O.mis_size(n, e, o), "counting": O.mis_count(n, e, o),
                    "modp": O.count_modp(n, e, o, tn.PRIMES31[:2])}
            for sr, pr in (("tropical_i32", None), ("counting", None), ("modp", tn.PRIMES31[:2])):
                if tile == 0 and sr != "tropical_i32":
                    continue
                info = tn.tn_plan_step_info(p.handle, sr, len(pr) if pr else 1)
                shapes = {tuple(int(v) for v in r[6:10]) for r in info if int(r[2]) == 1}
                for split in (1, 2):
                    tn.tn_tune_set([(sr, *sh, tile, split) for sh in shapes])
                    r = p.contract(sr, pr)
                    got = {"tropical_i32": r.get("max"), "counting": (r.get("max"), r.get("count")),
                           "modp": r.get("residues")}[sr]
                    assert got == want[sr], (spec, sr, tile, split)
        finally:
            tn.tn_tune_set([])
            p.close()
