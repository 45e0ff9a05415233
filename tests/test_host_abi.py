"""Host-side checks of libtn through its C ABI (no GPU needed): the library
loads and exports every symbol include/tn.h declares; orders, plans, the
complexity report and the CRT decode agree with the oracle and the paper."""
import ctypes
import json
import math
import os

import numpy as np
import pytest

import graphgen as g
import oracle as O
from paper_2501_00227_gb300 import build as B
from paper_2501_00227_gb300 import tn

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def test_library_exports_every_declared_symbol():
    L = tn.lib()
    names = tn.declared_symbols()
    for must in ["tn_plan", "tn_order_greedy", "tn_plan_info", "tn_contract", "tn_server_create",
                 "tn_submit", "tn_poll", "tn_plan_destroy", "tn_server_destroy", "tn_strerror"]:
        assert must in names
    missing = [s for s in names if not hasattr(L, s)]
    assert not missing, missing
    assert tn.tn_strerror(tn.TN_EINVAL)


def _replay_min_cost(n, edges, order):
    """Replays an order; True iff every step picks a label-sharing pair of
    minimum output rank (Sec. 4.2.1, alpha = 0), or, when no pair shares a
    label, any pair."""
    m = len(edges)
    labels = {i: frozenset(map(int, edges[i])) for i in range(m)}
    labels.update({m + v: frozenset([v]) for v in range(n)})
    nxt = m + n
    for a, b in order:
        a, b = int(a), int(b)

        def out(i, j):
            used = set()
            for t, L in labels.items():
                if t not in (i, j):
                    used |= L
            return (labels[i] | labels[j]) & used

        live = sorted(labels)
        cands = [len(out(i, j)) for x, i in enumerate(live) for j in live[x + 1:] if labels[i] & labels[j]]
        o = out(a, b)
        if cands and (not (labels[a] & labels[b]) or len(o) != min(cands)):
            return False
        del labels[a], labels[b]
        labels[nxt] = frozenset(o)
        nxt += 1
    return True


@pytest.mark.parametrize("spec", ["petersen", "reg3:20:1", "ksg:6:0.8:3", "er:14:0.2:5", "empty:5", "cycle:9"])
def test_greedy_order_valid_and_greedy(spec):
    n, e = g.by_name(spec)
    o = tn.tn_order_greedy(n, e, 0.0, 3, 11)
    assert O.check_order(n, e, o)
    assert _replay_min_cost(n, e, o)


def test_greedy_deterministic_and_seeded():
    n, e = g.random_regular3(40, 2)
    a = tn.tn_order_greedy(n, e, 0.0, 2, 5)
    b = tn.tn_order_greedy(n, e, 0.0, 2, 5)
    assert np.array_equal(a, b)


def test_petersen_greedy_matches_printed_complexity():
    gd = json.load(open(os.path.join(GOLD, "petersen.json")))
    n, e = g.petersen()
    p = tn.tn_plan(n, e, tn.tn_order_greedy(n, e, 0.0, 10, 1))
    try:
        info = tn.tn_plan_info(p, tn.TN_TROPICAL_I32, 1)
    finally:
        tn.tn_plan_destroy(p)
    assert [info["log2_tc"], info["log2_sc"], info["log2_rwc"]] == pytest.approx(gd["greedy_complexity_log2"], abs=5e-4)


def test_c4_tree_plan_info():
    gd = json.load(open(os.path.join(GOLD, "c4_tree.json")))
    edges = [(u - 1, v - 1) for u, v in gd["edges_1based"]]
    p = tn.tn_plan(4, edges, gd["tree_steps"])
    try:
        info = tn.tn_plan_info(p, tn.TN_TROPICAL_I32, 1)
    finally:
        tn.tn_plan_destroy(p)
    assert (info["tc"], info["sc"], info["rwc"]) == (34, 4, 69)
    assert info["nsteps"] == 7


@pytest.mark.parametrize("spec", ["reg3:100:1", "reg3:140:1", "ksg:12:0.8:1", "er:30:0.1:3"])
def test_plan_complexity_equals_oracle(spec):
    n, e = g.by_name(spec)
    o = tn.tn_order_greedy(n, e, 0.0, 2, 1)
    p = tn.tn_plan(n, e, o)
    try:
        info = tn.tn_plan_info(p, tn.TN_COUNT_MODP, 3)
    finally:
        tn.tn_plan_destroy(p)
    assert (info["tc"], info["sc"], info["rwc"]) == O.complexity(n, e, o)
    # workspace at least holds the largest intermediate in every semiring
    assert info["peak_bytes"][1] >= 4 * info["sc"]
    assert info["peak_bytes"][2] >= 12 * info["sc"]
    assert info["peak_bytes"][3] >= 12 * info["sc"]


def test_plan_rejects_bad_input():
    n, e = g.cycle(5)
    o = tn.tn_order_greedy(n, e)
    for bad_edges in ([(0, 0)], [(0, 1), (1, 0)], [(0, 9)]):
        with pytest.raises(tn.TNError) as ei:
            tn.tn_plan(5, bad_edges, [(0, 1)] * (len(bad_edges) + 4))
        assert ei.value.code == tn.TN_EINVAL
    bad = o.copy(); bad[2] = bad[0]
    with pytest.raises(tn.TNError):
        tn.tn_plan(n, e, bad)                  # consumes a tensor twice
    with pytest.raises(tn.TNError):
        tn.tn_plan(n, e, o[:-1])               # incomplete order
    with pytest.raises(tn.TNError):
        tn.tn_order_greedy(n, e, -1.0)         # alpha must be >= 0


def test_single_vertex_plan():
    p = tn.tn_plan(1, np.zeros((0, 2), np.int32), np.zeros((0, 2), np.int32))
    try:
        info = tn.tn_plan_info(p, tn.TN_TROPICAL_I32, 1)
        assert info["nsteps"] == 1 and info["sc"] == 1
    finally:
        tn.tn_plan_destroy(p)


def test_result_decode_crt_matches_oracle():
    rng = np.random.default_rng(0)
    for k in (1, 3, 4, 8):
        pr = tn.PRIMES31[:k]
        x = int(rng.integers(0, 2 ** 62)) ** 3 % math.prod(pr)
        raw = bytearray(tn.TN_RAW_BYTES)
        for q, p in enumerate(pr):
            raw[16 + 4 * q: 20 + 4 * q] = (x % p).to_bytes(4, "little")
        r = tn.tn_result_decode(tn.TN_COUNT_MODP, pr, bytes(raw))
        assert (r["crt"], r["modulus"]) == O.crt([x % p for p in pr], pr)
    raw = bytearray(tn.TN_RAW_BYTES)
    raw[0:4] = (7).to_bytes(4, "little", signed=True)
    raw[8:16] = (2 ** 64 - 1).to_bytes(8, "little")
    r = tn.tn_result_decode(tn.TN_COUNTING_TROPICAL, None, bytes(raw))
    assert r["max"] == 7 and r["status"] == tn.TN_EOVERFLOW
    with pytest.raises(tn.TNError):
        tn.tn_result_decode(tn.TN_COUNT_MODP, [6, 9], bytes(raw))   # moduli not coprime


@pytest.mark.parametrize("height", ["1", "4", "64"])
@pytest.mark.parametrize("spec", ["reg3:140:1", "ksg:12:0.8:2", "er:40:0.08:1", "empty:7", "square:8"])
def test_executor_schedule_self_check(spec, height, monkeypatch):
    """The executor's task order and workspace reuse pass the library's own
    schedule check (dependencies point backwards; a step never overwrites a
    tensor some non-ancestor step still reads), with and without groups of
    tiny steps run by one CTA."""
    monkeypatch.setenv("TN_EXEC_CHECK", "1")
    monkeypatch.setenv("TN_GROUP_HEIGHT", height)
    n, e = g.by_name(spec)
    p = tn.tn_plan(n, e, tn.tn_order_greedy(n, e, 0.0, 2, 3))
    try:
        for sr in (tn.TN_TROPICAL_I32, tn.TN_COUNTING_TROPICAL, tn.TN_COUNT_MODP):
            info = tn.tn_plan_info(p, sr, 3)
            assert info["exec_tasks"] >= 2
            if height == "1":
                assert info["exec_tasks"] >= info["nsteps"]  # a task per step at least; the last one writes the result
            assert info["exec_levels"] >= 1
    finally:
        tn.tn_plan_destroy(p)


@pytest.mark.parametrize("spec", ["reg3:60:2", "ksg:8:0.8:1", "petersen"])
def test_exec_self_check_on_plan_variants(monkeypatch, spec):
    """The executor plans behind weighted networks (stored leaves), the
    backward pass (every intermediate kept) and sliced networks pass the
    schedule self-check (leaves after every intermediate; no reuse when
    kept)."""
    monkeypatch.setenv("TN_EXEC_CHECK", "1")
    n, e = g.by_name(spec)
    o = tn.tn_order_greedy(n, e, 0.0, 2, 3)
    p = tn.tn_plan(n, e, o)
    ps = tn.tn_plan_sliced(n, e, o, [0, n - 1])
    try:
        for sr in ("tropical_i32", "counting", "modp"):
            assert tn.tn_weighted_workspace_bytes(p, sr, 3) > 0
            assert tn.tn_weighted_workspace_bytes(ps, sr, 3) > 0
            assert tn.tn_sliced_workspace_bytes(ps, sr, 3, 4) > 0
        assert tn.tn_single_config_workspace_bytes(p) > 0
        info = tn.tn_plan_info(ps, tn.TN_COUNTING_TROPICAL, 1)
        assert info["exec_tasks"] >= info["nsteps"]  # a task per step at least; the last one writes the result
    finally:
        tn.tn_plan_destroy(p)
        tn.tn_plan_destroy(ps)


@pytest.mark.parametrize("kind,iters", [(3, 1024), (-1, 1024), (0, 3), (1, (1 << 24) + 1)])
def test_alu_peak_rejects_bad_arguments(kind, iters):
    out = ctypes.c_double()
    assert tn.lib().tn_alu_peak(kind, iters, None, ctypes.byref(out)) == tn.TN_EINVAL


@pytest.mark.gpu
def test_alu_peaks_are_plausible():
    """The register-only rates behind the ALU rooflines: (max,+) near one
    term per lane per clock (64 per SM), the packed 16-bit form near two, the
    folded mod-p step slower."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mp = tn.tn_alu_peak("maxplus")
    md = tn.tn_alu_peak("modp")
    assert 0.3 * sms * 64 * 1.0e9 / 1e12 < mp < 1.2 * sms * 64 * 2.2e9 / 1e12
    assert 0 < md < mp
    mp2 = tn.tn_alu_peak("maxplus16x2")
    assert 1.5 * mp < mp2 < 1.2 * sms * 128 * 2.2e9 / 1e12


@pytest.mark.parametrize("ns,ok", [(0, True), (1, True), (2_000_000_000, True), (60_000_000_000, True),
                                   (60_000_000_001, False), (2 ** 64 - 1, False)])
def test_wait_timeout_setting_bounds(ns, ok):
    """The executor's wait limit takes 0 (the default) .. 60 s; the setting is
    restored to the default afterwards."""
    try:
        if ok:
            tn.tn_set_wait_timeout_ns(ns)
        else:
            with pytest.raises(tn.TNError) as ei:
                tn.tn_set_wait_timeout_ns(ns)
            assert ei.value.code == tn.TN_EINVAL
    finally:
        tn.tn_set_wait_timeout_ns(0)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every entry point raises; nothing falls
    back to another implementation."""
    monkeypatch.setattr(tn, "_lib", None)
    monkeypatch.setattr(tn, "library_path", lambda: str(tmp_path / "libtn.so"))
    n, e = g.petersen()
    with pytest.raises(tn.TNError, match="not built"):
        tn.lib()
    with pytest.raises(tn.TNError, match="not built"):
        tn.Plan(n, e)
    with pytest.raises(tn.TNError, match="not built"):
        tn.tn_order_treesa(n, e)
