"""Pins for the oracle's weighted networks: vertex-weighted independent sets
and the spin glass of Eq. 1 (Sec. 2.1.1, Sec. 6.4).  Checked against values
the paper prints (Petersen energy example, Buckyball ground state and
ln Z / N), the Ising-ring transfer-matrix closed form, and brute force over
all configurations.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
P0, P1 = O.PRIMES31[0], O.PRIMES31[1]


def _gold():
    with open(os.path.join(GOLD, "spin_glass.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------- paper values

def test_petersen_spin_energy_printed():
    gd = _gold()["petersen_energy"]
    n, e = g.petersen()
    assert O.spin_energy(n, e, gd["spins"]) == gd["energy"]


def test_fullerene_structure():
    """60 vertices, 90 edges, cubic, 12 pentagons that share no edge with
    each other, 20 hexagons: the Buckyball."""
    nx = pytest.importorskip("networkx")
    n, e = g.fullerene()
    gd = _gold()["buckyball"]
    assert (n, len(e)) == (gd["n"], gd["m"])
    assert set(np.bincount(e.reshape(-1)).tolist()) == {3}
    G = nx.Graph(e.tolist())
    cycles = list(nx.simple_cycles(G, length_bound=6))
    pent = [c for c in cycles if len(c) == 5]
    assert len(pent) == 12 and sum(len(c) == 6 for c in cycles) == 20
    pe = [{frozenset((c[i], c[(i + 1) % 5])) for i in range(5)} for c in pent]
    assert all(not (a & b) for i, a in enumerate(pe) for b in pe[i + 1:])


def test_buckyball_ground_state_printed():
    """CountingMin = (-66, 16000): the counting element type maximises -H."""
    gd = _gold()["buckyball"]
    n, e = g.fullerene()
    o = O.greedy_order(n, e, nrepeat=4, seed=1)
    assert O.weighted_contract("tropical", "spin", n, e, o) == -gd["ground_energy"]
    assert O.weighted_contract("counting", "spin", n, e, o) == (-gd["ground_energy"], gd["ground_degeneracy"])


def test_buckyball_log_partition_function_printed():
    """ln Z / N at beta = 1 from the exact energy histogram (2 primes > 2^60)."""
    gd = _gold()["buckyball"]
    n, e = g.fullerene()
    o = O.greedy_order(n, e, nrepeat=4, seed=1)
    shift = O.spin_shift(n, e)
    coeffs = O.weighted_polynomial("spin", n, e, o, O.PRIMES31[:2], 2 * shift)
    assert sum(coeffs) == 2 ** n
    assert coeffs[gd["ground_energy"] + shift] == gd["ground_degeneracy"]
    assert all(c == 0 for c in coeffs[: gd["ground_energy"] + shift])
    lz = O.log_partition_function(coeffs, shift, 1.0) / n
    assert lz == pytest.approx(gd["log_z_per_site_beta1"], rel=1e-13, abs=0)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [4, 7, 10, 16])
def test_ising_ring_transfer_matrix(n):
    """Anti-ferromagnetic ring, J = 1, h = 0: Z = (2 cosh b)^n + (-2 sinh b)^n;
    ground state -n (degeneracy 2) for even n, -(n - 2) (degeneracy 2n) for odd n."""
    nn, e = g.cycle(n)
    o = O.greedy_order(nn, e, nrepeat=2, seed=n)
    want_e, want_d = (-n, 2) if n % 2 == 0 else (-(n - 2), 2 * n)
    assert O.weighted_contract("counting", "spin", nn, e, o) == (-want_e, want_d)
    shift = O.spin_shift(nn, e)
    coeffs = O.weighted_polynomial("spin", nn, e, o, [P0], 2 * shift)
    for beta in (0.1, 0.7, 1.0, 2.5):
        z = (2 * math.cosh(beta)) ** n + (-2 * math.sinh(beta)) ** n
        assert O.log_partition_function(coeffs, shift, beta) == pytest.approx(math.log(z), rel=1e-12)


# ---------------------------------------------------------------- brute force

def _spin_cases():
    out = []
    for seed in range(3):
        n, e = g.erdos_renyi(12, 0.35, 70 + seed)
        out.append((n, e, g.random_weights(len(e), seed, (-2, -1, 1, 2)), g.random_weights(n, 10 + seed, (-1, 0, 1))))
    n, e = g.petersen()
    out.append((n, e, None, None))
    n, e = g.random_regular3(14, 3)
    out.append((n, e, g.random_weights(len(e), 5), None))
    return out


@pytest.mark.parametrize("case", range(5))
def test_spin_glass_equals_bruteforce(case):
    n, e, J, h = _spin_cases()[case]
    shift, hist = O.bruteforce_spin(n, e, J, h)
    kmin = min(k for k, c in enumerate(hist) if c)
    o = O.greedy_order(n, e, nrepeat=2, seed=case)
    assert O.weighted_contract("tropical", "spin", n, e, o, J, h) == shift - kmin
    assert O.weighted_contract("counting", "spin", n, e, o, J, h) == (shift - kmin, hist[kmin])
    primes, ys = [P0, P0, P1, P1], [0, 1, 3, 2 ** 30 + 7]
    got = O.weighted_contract("modp", "spin", n, e, o, J, h, primes, ys)
    assert got == [sum(c * pow(y, k, p) for k, c in enumerate(hist)) % p for p, y in zip(primes, ys)]
    assert O.weighted_polynomial("spin", n, e, o, [P0], 2 * shift, J, h) == hist


def test_spin_energy_matches_histogram_and_flip_symmetry():
    """With h = 0, flipping every spin keeps H (the histogram of a direct
    energy loop over all configurations equals the oracle's brute force)."""
    n, e = g.erdos_renyi(10, 0.4, 3)
    J = g.random_weights(len(e), 1, (-3, 1, 2))
    shift, hist = O.bruteforce_spin(n, e, J)
    mine = [0] * len(hist)
    for c in range(1 << n):
        s = [1 if (c >> v) & 1 else -1 for v in range(n)]
        E = O.spin_energy(n, e, s, J)
        assert O.spin_energy(n, e, [-x for x in s], J) == E
        mine[E + shift] += 1
    assert mine == hist


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_weighted_is_equals_bruteforce(seed):
    n, e = g.erdos_renyi(13, 0.3, 90 + seed)
    w = g.random_weights(n, seed, (0, 1, 2, 3))
    hist = O.bruteforce_weighted_is(n, e, w)
    top = max(k for k, c in enumerate(hist) if c)
    o = O.greedy_order(n, e, nrepeat=2, seed=seed)
    assert O.weighted_contract("tropical", "is", n, e, o, vertex_w=w) == top
    assert O.weighted_contract("counting", "is", n, e, o, vertex_w=w) == (top, hist[top])
    assert O.weighted_polynomial("is", n, e, o, [P0], int(w.sum()), vertex_w=w) == hist
    # unit weights are the plain IS network
    assert O.weighted_contract("counting", "is", n, e, o) == O.mis_count(n, e, o)


def test_negative_is_weights_allowed_in_max_plus():
    n, e = g.path(5)
    w = np.array([-1, 4, -2, 3, 0], dtype=np.int32)
    o = O.sweep_order(n, e)
    assert O.weighted_contract("tropical", "is", n, e, o, vertex_w=w) == 7        # {1, 3}
    assert O.weighted_contract("counting", "is", n, e, o, vertex_w=w) == (7, 1)
    with pytest.raises(O.OracleError):
        O.weighted_contract("modp", "is", n, e, o, vertex_w=w, primes=[P0], xs=[2])
