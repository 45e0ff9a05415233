"""SingleConfigMax(k) (Sec. 5.3): k distinct independent sets with the k
largest total weights, by Lawler's partition over optimal-configuration
passes.  The partition logic is checked on the CPU with a brute-force
solver in its place; the GPU tests run it on the single-configuration pass
and compare the weights with the oracle's polynomial / weight histogram."""
import json
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O
from paper_2501_00227_gb300 import properties as P
from paper_2501_00227_gb300 import tn


class _Graph:
    """What single_config_max_k reads of a plan, without a plan handle."""

    def __init__(self, n, e):
        self.n, self.edges = n, np.asarray(e, dtype=np.int32).reshape(-1, 2)


def _brute_solver(n, e):
    """Best total weight over all 2^n subsets and the lowest-index subset
    reaching it (test stand-in for the GPU pass; n <= 16)."""
    masks = np.arange(1 << n, dtype=np.int64)
    bits = ((masks[:, None] >> np.arange(n)) & 1).astype(np.int64)
    ok = np.ones(1 << n, dtype=bool)
    for a, b in np.asarray(e).reshape(-1, 2).tolist():
        ok &= ~((bits[:, a] == 1) & (bits[:, b] == 1))

    def solve(wf):
        vals = np.where(ok, bits @ np.asarray(wf, dtype=np.int64), np.iinfo(np.int64).min)
        i = int(np.argmax(vals))
        return int(vals[i]), bits[i].astype(np.uint8)
    return solve


def _weights_of_all_sets(n, e, w):
    """Total weights of all independent sets, largest first (brute force)."""
    hist = O.bruteforce_weighted_is(n, e, w) if w is not None else O.bruteforce_poly(n, e)
    return [s for s in range(len(hist) - 1, -1, -1) for _ in range(hist[s])]


def _check(n, e, res, k, w):
    want = _weights_of_all_sets(n, e, w)[:k]
    assert [v for v, _ in res] == want
    seen = set()
    ww = np.ones(n, dtype=np.int64) if w is None else np.asarray(w, dtype=np.int64)
    for v, cfg in res:
        assert all(not (cfg[a] and cfg[b]) for a, b in np.asarray(e).reshape(-1, 2).tolist())
        assert int(ww @ cfg.astype(np.int64)) == v
        seen.add(cfg.tobytes())
    assert len(seen) == len(res)


def test_petersen_two_best_printed():
    """Sec. 5.3 prints SingleConfigMax(2) of the Petersen graph: two
    different sets of size 4 (which two depends on the solver)."""
    n, e = g.petersen()
    res = P.single_config_max_k(_Graph(n, e), 2, solve=_brute_solver(n, e))
    assert [v for v, _ in res] == [4, 4]
    _check(n, e, res, 2, None)


def _printed_configs():
    with open(os.path.join(os.path.dirname(__file__), "golden", "petersen.json")) as f:
        gd = json.load(f)
    return [np.array([int(c) for c in s], dtype=np.uint8) for s in [gd["single_config_max"]] + gd["single_config_max_2"]]


def test_printed_petersen_configurations_are_among_the_five_maximum_sets():
    """The configurations Sec. 5.3 prints for SingleConfigMax() and
    SingleConfigMax(2) are maximum independent sets of the Petersen graph
    (with its vertices numbered as the paper's); the partition enumerates
    all five maximum sets, those three among them."""
    n, e = g.petersen()
    res = P.single_config_max_k(_Graph(n, e), 5, solve=_brute_solver(n, e))
    assert [v for v, _ in res] == [4] * 5
    got = {cfg.tobytes() for _, cfg in res}
    for cfg in _printed_configs():
        assert all(not (cfg[a] and cfg[b]) for a, b in e.tolist()) and cfg.sum() == 4
        assert cfg.tobytes() in got


@pytest.mark.parametrize("spec,k", [("petersen", 12), ("er:12:0.3:2", 40), ("cycle:9", 7), ("path:3", 10),
                                    ("complete:5", 8), ("empty:4", 16)])
def test_partition_enumerates_in_weight_order(spec, k):
    n, e = g.by_name(spec)
    res = P.single_config_max_k(_Graph(n, e), k, solve=_brute_solver(n, e))
    _check(n, e, res, k, None)
    assert len(res) == min(k, sum(O.bruteforce_poly(n, e)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_partition_with_weights(seed):
    n, e = g.erdos_renyi(12, 0.3, 70 + seed)
    w = g.random_weights(n, seed, (0, 1, 2, 5))
    res = P.single_config_max_k(_Graph(n, e), 25, vertex_w=w, solve=_brute_solver(n, e))
    _check(n, e, res, 25, w)


def test_partition_with_negative_weights():
    """Negative weights: the forcing still holds (B > 2 sum|w|), and the k
    best weights match a direct enumeration of every independent set."""
    n, e = g.erdos_renyi(11, 0.3, 91)
    w = g.random_weights(n, 4, (-3, -1, 0, 2, 4))
    res = P.single_config_max_k(_Graph(n, e), 40, vertex_w=w, solve=_brute_solver(n, e))
    ee = np.asarray(e).reshape(-1, 2)
    weights = sorted((sum(int(w[v]) for v in range(n) if (m >> v) & 1) for m in range(1 << n)
                      if all(not ((m >> a) & 1 and (m >> b) & 1) for a, b in ee.tolist())), reverse=True)
    assert [v for v, _ in res] == weights[:40]
    assert len({cfg.tobytes() for _, cfg in res}) == 40
    for v, cfg in res:
        assert int(np.asarray(w, dtype=np.int64) @ cfg.astype(np.int64)) == v
        assert all(not (cfg[a] and cfg[b]) for a, b in ee.tolist())


def test_all_sets_of_a_small_graph():
    """k beyond the number of sets enumerates every independent set once."""
    n, e = g.cycle(6)
    res = P.single_config_max_k(_Graph(n, e), 100, solve=_brute_solver(n, e))
    assert len(res) == 18                                   # the Lucas number L_6
    _check(n, e, res, 100, None)


def test_default_pass_reuses_one_workspace(monkeypatch):
    """Without `solve`, every subspace goes through Plan.single_config_max
    with one workspace sized by tn_single_config_workspace_bytes (the GPU
    call replaced here by brute force)."""
    torch = pytest.importorskip("torch")
    n, e = g.petersen()
    brute = _brute_solver(n, e)
    sizes, seen = [], []
    monkeypatch.setattr(tn, "tn_single_config_workspace_bytes", lambda h: sizes.append(h) or 4096)
    monkeypatch.setattr(torch, "empty", lambda *a, **kw: ("ws", a, kw.get("device")))

    class FakePlan(_Graph):
        handle = "plan-handle"

        def single_config_max(self, problem, edge_w=None, vertex_w=None, workspace=None):
            assert problem == "is" and edge_w is None
            seen.append(workspace)
            return brute(vertex_w)

    res = P.single_config_max_k(FakePlan(n, e), 3)
    assert sizes == ["plan-handle"] and all(s == ("ws", (4096,), "cuda") for s in seen)
    _check(n, e, res, 3, None)


def test_lazy_subspaces_take_few_passes():
    """Subspaces are solved only when their bound reaches the top: the 5
    maximum sets of the Petersen graph take far fewer than 5 n passes."""
    n, e = g.petersen()
    brute, calls = _brute_solver(n, e), []

    def counted(wf):
        calls.append(1)
        return brute(wf)
    res = P.single_config_max_k(_Graph(n, e), 5, solve=counted)
    assert [v for v, _ in res] == [4] * 5
    assert len(calls) < 5 * n


def test_rejects_weights_too_large_to_force():
    n, e = g.path(4)
    with pytest.raises(ValueError):
        P.single_config_max_k(_Graph(n, e), 2, vertex_w=[1 << 25] * 4, solve=_brute_solver(n, e))


def _brute_spin_solver(n, e):
    """max over all 2^n spin configurations of -H and the lowest-index
    configuration reaching it (bit 1 = spin +1); test stand-in, n <= 16."""
    masks = np.arange(1 << n, dtype=np.int64)
    sp = 2 * ((masks[:, None] >> np.arange(n)) & 1) - 1
    e = np.asarray(e).reshape(-1, 2)

    def solve(J, h):
        neg_h = -((sp[:, e[:, 0]] * sp[:, e[:, 1]]) @ np.asarray(J, dtype=np.int64) if len(e) else 0) \
            - sp @ np.asarray(h, dtype=np.int64)
        i = int(np.argmax(neg_h))
        return int(neg_h[i]), ((sp[i] + 1) // 2).astype(np.uint8)
    return solve


def _spin_energies(n, e, J, h):
    """All 2^n energies, ascending (brute force via the oracle's histogram)."""
    shift, hist = O.bruteforce_spin(n, e, J, h)
    return [k - shift for k, c in enumerate(hist) for _ in range(c)]


def _check_spins(n, e, res, k, J, h):
    assert [en for en, _ in res] == _spin_energies(n, e, J, h)[:k]
    seen = set()
    for en, s in res:
        assert set(np.unique(s).tolist()) <= {-1, 1}
        assert O.spin_energy(n, e, s, J, h) == en
        seen.add(s.tobytes())
    assert len(seen) == len(res)


@pytest.mark.parametrize("spec,seed,k", [("petersen", 0, 30), ("er:11:0.35:2", 1, 50), ("cycle:8", 2, 256),
                                         ("path:5", 3, 40)])
def test_spin_glass_lowest_energies(spec, seed, k):
    """The k lowest energies of random +-J couplings and fields in -2..2
    equal the bottom of the brute-force energy spectrum, each configuration
    distinct and of the stated energy (all 2^n when k exceeds it)."""
    n, e = g.by_name(spec)
    J = g.random_weights(len(e), seed)
    h = g.random_weights(n, seed + 10, (-2, -1, 0, 1, 2))
    res = P.spin_glass_lowest_k(_Graph(n, e), k, J, h, solve=_brute_spin_solver(n, e))
    assert len(res) == min(k, 1 << n)
    _check_spins(n, e, res, k, J, h)


def test_spin_glass_default_couplings():
    """J = 1, h = 0 (an antiferromagnet): on an even cycle the two Neel
    states are the ground states, energy -n."""
    n, e = g.cycle(10)
    res = P.spin_glass_lowest_k(_Graph(n, e), 3, solve=_brute_spin_solver(n, e))
    assert [en for en, _ in res[:2]] == [-10, -10] and res[2][0] > -10
    assert {tuple(s.tolist()) for _, s in res[:2]} == {tuple([1, -1] * 5), tuple([-1, 1] * 5)}


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.gpu
@pytest.mark.parametrize("spec,k", [("petersen", 2), ("petersen", 20), ("er:14:0.25:3", 30), ("ksg:4:0.8:1", 12)])
def test_k_best_configurations_on_gpu(spec, k):
    _cuda()
    n, e = g.by_name(spec)
    p = tn.Plan(n, e, nrepeat=2, seed=1)
    try:
        res = P.single_config_max_k(p, k)
    finally:
        p.close()
    _check(n, e, res, k, None)


@pytest.mark.gpu
def test_printed_petersen_configurations_on_gpu():
    _cuda()
    n, e = g.petersen()
    p = tn.Plan(n, e, nrepeat=2, seed=1)
    try:
        res = P.single_config_max_k(p, 5)
    finally:
        p.close()
    assert [v for v, _ in res] == [4] * 5
    got = {cfg.tobytes() for _, cfg in res}
    assert all(cfg.tobytes() in got for cfg in _printed_configs())


@pytest.mark.gpu
def test_k_best_weighted_configurations_on_gpu():
    _cuda()
    n, e = g.erdos_renyi(13, 0.3, 5)
    w = g.random_weights(n, 3, (0, 1, 2, 3))
    p = tn.Plan(n, e, nrepeat=2, seed=1)
    try:
        res = P.single_config_max_k(p, 15, vertex_w=w)
    finally:
        p.close()
    _check(n, e, res, 15, w)


@pytest.mark.gpu
@pytest.mark.parametrize("spec,seed,k", [("petersen", 0, 12), ("er:13:0.3:4", 1, 20)])
def test_spin_glass_lowest_energies_on_gpu(spec, seed, k):
    _cuda()
    n, e = g.by_name(spec)
    J = g.random_weights(len(e), seed)
    h = g.random_weights(n, seed + 10, (-2, -1, 0, 1, 2))
    p = tn.Plan(n, e, nrepeat=2, seed=1)
    try:
        res = P.spin_glass_lowest_k(p, k, J, h)
    finally:
        p.close()
    _check_spins(n, e, res, k, J, h)


@pytest.mark.gpu
def test_buckyball_lowest_energies_on_gpu():
    """Sec. 6.4 prints the Buckyball's ground-state energy -66 with
    degeneracy 16000: its four lowest-energy configurations are distinct
    ground states."""
    _cuda()
    with open(os.path.join(os.path.dirname(__file__), "golden", "spin_glass.json")) as f:
        gd = json.load(f)["buckyball"]
    n, e = g.fullerene()
    p = tn.Plan(n, e, nrepeat=4, seed=1)
    try:
        res = P.spin_glass_lowest_k(p, 4)
    finally:
        p.close()
    assert [en for en, _ in res] == [gd["ground_energy"]] * 4
    assert len({s.tobytes() for _, s in res}) == 4
    assert all(O.spin_energy(n, e, s) == gd["ground_energy"] for _, s in res)
