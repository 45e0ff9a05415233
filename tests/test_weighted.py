"""Weighted networks on the GPU (tn_contract_weighted, tn_weighted_polynomial):
vertex-weighted independent sets and the spin glass of Eq. 1, against the
CPU oracle and the values Sec. 6.4 prints for the Buckyball.  Integer
results must be equal; ln Z / N is compared within float64 rounding of the
final sum.  Host-side argument checks run without a GPU."""
import json
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O
from paper_2501_00227_gb300 import properties as P
from paper_2501_00227_gb300 import tn

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_2501_00227_gb300 import build as B
    B.build()
    O.set_threads(os.cpu_count() or 1)


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _plan(n, e, seed=1):
    o = O.greedy_order(n, e, nrepeat=4, seed=seed)
    return o, tn.Plan(n, e, o)


# ------------------------------------------------------------------ host checks (no GPU)

@pytest.mark.parametrize("semiring,problem,ew,vw", [
    ("counting", 7, None, None),                                  # unknown problem
    ("modp", "is", None, [1, -1] * 5),                            # negative exponent mod p
    ("tropical_i32", "spin", [1 << 28] * 15, None),               # |J| sum above 2^28
    ("tropical_f32", "is", None, [1 << 22] * 10),                 # not exact in float32
])
def test_weighted_rejects_bad_arguments(semiring, problem, ew, vw):
    n, e = g.petersen()
    p = tn.Plan(n, e, nrepeat=1, seed=1)
    try:
        primes, xs = ([tn.PRIMES31[0]], [3]) if semiring == "modp" else (None, None)
        with pytest.raises(tn.TNError) as ei:
            tn.tn_contract_weighted(p.handle, semiring, problem, ew, vw, primes, xs, 256, 1 << 30, 0)
        assert ei.value.code == tn.TN_EINVAL
    finally:
        p.close()


def test_weighted_workspace_covers_the_plain_one():
    n, e = g.random_regular3(60, 2)
    p = tn.Plan(n, e, nrepeat=2, seed=1)
    try:
        for sr, k in (("tropical_i32", 1), ("counting", 1), ("modp", 16)):
            assert tn.tn_weighted_workspace_bytes(p.handle, sr, k) > p.workspace_bytes(sr, k)
    finally:
        p.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_counting_min_from_the_histogram(seed):
    """CountingMin(k) read off an energy histogram: the k lowest energies
    with their multiplicities, the first the counting contraction's ground
    state (host logic, histogram by brute force)."""
    n, e = g.erdos_renyi(12, 0.3, 30 + seed)
    J = g.random_weights(len(e), seed, (-2, -1, 1, 2))
    h = g.random_weights(n, seed + 5, (-1, 0, 1))
    shift, hist = O.bruteforce_spin(n, e, J, h)
    energies = sorted(O.spin_energy(n, e, [1 if (m >> i) & 1 else -1 for i in range(n)], J, h)
                      for m in range(1 << n))
    for k in (1, 3, 1000):
        got = P.counting_min(None, k, histogram=(shift, hist))
        want = {}
        for en in energies:
            if en in want or len(want) < k:
                want[en] = want.get(en, 0) + 1
        assert got == want
    o = O.greedy_order(n, e, nrepeat=2, seed=1)
    top, cnt = O.weighted_contract("counting", "spin", n, e, o, J, h)
    assert P.counting_min(None, 1, histogram=(shift, hist)) == {-top: cnt}


# ------------------------------------------------------------------ GPU parity

@pytest.mark.gpu
def test_buckyball_printed_values_gpu():
    """Sec. 6.4: CountingMin = (-66, 16000) and ln Z / N = 1.3073684577607942
    at temperature 1 for the anti-ferromagnetic Buckyball."""
    _cuda()
    gd = json.load(open(os.path.join(GOLD, "spin_glass.json")))["buckyball"]
    n, e = g.fullerene()
    o, p = _plan(n, e)
    try:
        assert P.spin_glass_ground_state(p) == (gd["ground_energy"], gd["ground_degeneracy"])
        shift, c = P.energy_histogram(p)
        assert sum(c) == 2 ** n and c[gd["ground_energy"] + shift] == gd["ground_degeneracy"]
        assert c == O.weighted_polynomial("spin", n, e, o, tn.PRIMES31[:2], 2 * shift)
        assert P.counting_min(p, 1, histogram=(shift, c)) == {gd["ground_energy"]: gd["ground_degeneracy"]}
        lz = P.log_partition_function(p, 1.0, histogram=(shift, c)) / n
        assert lz == pytest.approx(gd["log_z_per_site_beta1"], rel=1e-13, abs=0)
    finally:
        p.close()


def _spin_case(spec, seed):
    n, e = g.by_name(spec)
    return n, e, g.random_weights(len(e), seed, (-2, -1, 1, 2)), g.random_weights(n, seed + 50, (-1, 0, 1))


@pytest.mark.gpu
@pytest.mark.parametrize("spec,seed", [("petersen", 0), ("er:14:0.3:2", 1), ("reg3:40:1", 2), ("ksg:7:0.8:3", 3),
                                       ("reg3:100:1", 4)])
def test_spin_glass_matches_oracle(spec, seed):
    _cuda()
    n, e, J, h = _spin_case(spec, seed)
    o, p = _plan(n, e)
    try:
        for sr in ("tropical_i32", "tropical_f32"):
            assert p.contract_weighted(sr, "spin", J, h)["max"] == O.weighted_contract("tropical", "spin", n, e, o, J, h)
        r = p.contract_weighted("counting", "spin", J, h)
        assert (r["max"], r["count"]) == O.weighted_contract("counting", "spin", n, e, o, J, h)
        primes = [tn.PRIMES31[0]] * 3 + [tn.PRIMES31[2]] * 4
        ys = [0, 1, 2, 3, 2 ** 30 + 1, 12345, tn.PRIMES31[2] - 1]
        assert p.contract_weighted("modp", "spin", J, h, primes, ys)["residues"] == \
            O.weighted_contract("modp", "spin", n, e, o, J, h, primes, ys)
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec,seed", [("er:12:0.3:5", 0), ("reg3:20:1", 1), ("cycle:9", 2)])
def test_spin_glass_histogram_matches_bruteforce(spec, seed):
    _cuda()
    n, e, J, h = _spin_case(spec, seed)
    o, p = _plan(n, e)
    try:
        shift, hist = O.bruteforce_spin(n, e, J, h)
        assert P.energy_histogram(p, J, h) == (shift, hist)
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec,seed", [("petersen", 0), ("er:16:0.25:4", 1), ("reg3:60:3", 2), ("ksg:8:0.8:1", 3)])
def test_weighted_is_matches_oracle(spec, seed):
    _cuda()
    n, e = g.by_name(spec)
    w = g.random_weights(n, seed, (0, 1, 2, 3, 5))
    o, p = _plan(n, e)
    try:
        for sr in ("tropical_i32", "tropical_f32"):
            assert p.contract_weighted(sr, "is", vertex_w=w)["max"] == \
                O.weighted_contract("tropical", "is", n, e, o, vertex_w=w)
        r = p.contract_weighted("counting", "is", vertex_w=w)
        assert (r["max"], r["count"]) == O.weighted_contract("counting", "is", n, e, o, vertex_w=w)
        primes, xs = [tn.PRIMES31[1]] * 4, [0, 1, 2, 99991]
        assert p.contract_weighted("modp", "is", vertex_w=w, primes=primes, xs=xs)["residues"] == \
            O.weighted_contract("modp", "is", n, e, o, vertex_w=w, primes=primes, xs=xs)
        if n <= 20:
            assert p.weighted_polynomial("is", vertex_w=w) == O.bruteforce_weighted_is(n, e, w)
    finally:
        p.close()


@pytest.mark.gpu
def test_unit_weights_reproduce_the_plain_network():
    """Stored unit-weight leaves give the results of the generated ones."""
    _cuda()
    n, e = g.random_regular3(100, 2)
    o, p = _plan(n, e)
    try:
        r = p.contract_weighted("counting", "is")
        plain = p.contract("counting")
        assert (r["max"], r["count"]) == (plain["max"], plain["count"])
        assert p.contract_weighted("modp", "is", primes=tn.PRIMES31[:3], xs=[1, 1, 1])["residues"] == \
            p.contract("modp", tn.PRIMES31[:3])["residues"]
    finally:
        p.close()


@pytest.mark.gpu
def test_full_size_spin_glass_and_weighted_is():
    """The 140-vertex 3-regular graph of the bench, +-1 couplings and random
    fields / vertex weights 0..3, every element type against the oracle."""
    _cuda()
    n, e = g.random_regular3(140, 2)
    o, p = _plan(n, e)
    try:
        J = g.random_weights(len(e), 7)
        h = g.random_weights(n, 8, (-1, 0, 1))
        r = p.contract_weighted("counting", "spin", J, h)
        assert (r["max"], r["count"]) == O.weighted_contract("counting", "spin", n, e, o, J, h)
        pr, ys = [tn.PRIMES31[0]] * 2 + [tn.PRIMES31[1]] * 2, [3, 2 ** 30 + 3, 5, 77]
        assert p.contract_weighted("modp", "spin", J, h, pr, ys)["residues"] == \
            O.weighted_contract("modp", "spin", n, e, o, J, h, pr, ys)
        w = g.random_weights(n, 9, (0, 1, 2, 3))
        r = p.contract_weighted("counting", "is", vertex_w=w)
        assert (r["max"], r["count"]) == O.weighted_contract("counting", "is", n, e, o, vertex_w=w)
        val, cfg = p.single_config_max("is", vertex_w=w)
        assert val == r["max"]
        cfgb = cfg.astype(bool)
        assert not np.any(cfgb[e[:, 0]] & cfgb[e[:, 1]]) and int(w[cfgb].sum()) == val
    finally:
        p.close()
