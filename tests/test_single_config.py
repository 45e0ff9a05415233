"""One optimal configuration (SingleConfigMax, Sec. 5.3) from the GPU's
backward pass: the maximum must equal the oracle's, and the configuration
must be valid and reach it (several optima may exist, so the configuration
itself is checked, not compared)."""
import json
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O
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


def _is_weight(e, cfg, w=None):
    """Total weight of the chosen vertices, or None if two of them are adjacent."""
    cfg = np.asarray(cfg).astype(bool)
    if np.any(cfg[e[:, 0]] & cfg[e[:, 1]]):
        return None
    return int(cfg.sum()) if w is None else int(np.asarray(w)[cfg].sum())


def test_single_config_workspace_and_argument_checks():
    n, e = g.petersen()
    p = tn.Plan(n, e, nrepeat=1, seed=1)
    try:
        assert tn.tn_single_config_workspace_bytes(p.handle) > p.workspace_bytes("tropical_i32")
        with pytest.raises(tn.TNError) as ei:
            tn.tn_single_config_max(p.handle, 5, None, None, n, 256, 1 << 30, 0)
        assert ei.value.code == tn.TN_EINVAL
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec", ["petersen", "path:1", "path:2", "empty:6", "complete:7", "cycle:11", "reg3:20:1",
                                  "er:18:0.15:2", "ksg:8:0.8:3", "reg3:100:2", "reg3:140:1"])
def test_mis_configuration(spec):
    _cuda()
    n, e = g.by_name(spec)
    o = O.greedy_order(n, e, nrepeat=4, seed=1)
    p = tn.Plan(n, e, o)
    try:
        val, cfg = p.single_config_max()
        assert val == O.mis_size(n, e, o)
        assert _is_weight(e, cfg) == val
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec,seed", [("er:14:0.3:1", 0), ("reg3:60:2", 1), ("ksg:7:0.8:2", 2)])
def test_weighted_is_configuration(spec, seed):
    _cuda()
    n, e = g.by_name(spec)
    w = g.random_weights(n, seed, (-2, 0, 1, 3, 7))
    o = O.greedy_order(n, e, nrepeat=4, seed=1)
    p = tn.Plan(n, e, o)
    try:
        val, cfg = p.single_config_max("is", vertex_w=w)
        assert val == O.weighted_contract("tropical", "is", n, e, o, vertex_w=w)
        assert _is_weight(e, cfg, w) == val
    finally:
        p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("spec,seed", [("petersen", 0), ("er:16:0.3:4", 1), ("reg3:100:3", 2)])
def test_spin_glass_ground_state_configuration(spec, seed):
    _cuda()
    n, e = g.by_name(spec)
    J = g.random_weights(len(e), seed, (-2, -1, 1, 3))
    h = g.random_weights(n, seed + 7, (-1, 0, 1))
    o = O.greedy_order(n, e, nrepeat=4, seed=1)
    p = tn.Plan(n, e, o)
    try:
        val, cfg = p.single_config_max("spin", J, h)
        assert val == O.weighted_contract("tropical", "spin", n, e, o, J, h)
        assert O.spin_energy(n, e, 2 * cfg.astype(np.int8) - 1, J, h) == -val
    finally:
        p.close()


@pytest.mark.gpu
def test_buckyball_ground_state_configuration():
    """A ground state of the Buckyball has the energy Sec. 6.4 prints (-66)."""
    _cuda()
    gd = json.load(open(os.path.join(GOLD, "spin_glass.json")))["buckyball"]
    n, e = g.fullerene()
    p = tn.Plan(n, e, nrepeat=4, seed=1)
    try:
        val, cfg = p.single_config_max("spin")
        assert -val == gd["ground_energy"]
        assert O.spin_energy(n, e, 2 * cfg.astype(np.int8) - 1) == gd["ground_energy"]
    finally:
        p.close()
