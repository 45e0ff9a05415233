"""Solution-space properties of Sec. 5.3 computed from the GPU contractions.

From the independence polynomial I(G, x) = sum_k c_k x^k (Eq. 13), computed
on the GPU by ``Plan.independence_polynomial`` (weighted mod-p contractions,
interpolation, CRT):

  counting_max(plan, k)  the k highest nonzero orders of I with their
                         coefficients (CountingMax(k), a TruncatedPoly{k}
                         in the paper): {size: number of sets};
  size_max(plan, k)      the k largest set sizes over all independent sets,
                         repeated by multiplicity, ascending (SizeMax(k), an
                         ExtendedTropical{k} in the paper).

Both also have dedicated element types (the paper's route, one
contraction): ``Plan.kbest("size_max" | "counting_max", k)`` for k up to
TN_KBEST_MAX on unit-weight networks (tn_contract_kbest), whose counts are
uint64 (saturating) and whose CountingMax(k) lists the k highest orders
including zero coefficients.  The functions here read the same numbers off
the exact polynomial instead, which costs alpha + 1 evaluations per prime,
takes any k and vertex weights, keeps exact counts, and lists the k highest
orders with nonzero coefficients.

SingleConfigMax(k) (single_config_max_k): k distinct sets with the k
largest sizes or total weights, by Lawler's partition of the solution space
over the GPU's optimal-configuration pass (tn_single_config_max), vertices
forced in or out through their weights.

For the spin glass of Eq. 1: the ground state (CountingMin) from the
counting contraction of -H, the exact energy histogram from
``Plan.weighted_polynomial``, the k lowest energies with their counts
(CountingMin(k)) and ln Z(beta) (PartitionFunction) read off that
histogram, and the k lowest-energy configurations (spin_glass_lowest_k).
"""
from __future__ import annotations


def _poly(plan, polynomial, vertex_w):
    if polynomial is not None:
        return polynomial
    if vertex_w is not None:  # sizes are total weights (weights >= 0)
        return plan.weighted_polynomial("is", vertex_w=vertex_w)
    return plan.independence_polynomial()


def counting_max(plan, k: int = 1, polynomial=None, vertex_w=None) -> dict:
    """{size: count} for the k largest sizes that occur (fewer if the graph
    has fewer distinct sizes).  k = 1 is CountingMax().  vertex_w: integer
    weights >= 0, sizes then being total weights."""
    c = _poly(plan, polynomial, vertex_w)
    sizes = [s for s in range(len(c) - 1, -1, -1) if c[s]][:k]
    return {s: c[s] for s in sorted(sizes)}


def size_max(plan, k: int = 1, polynomial=None, vertex_w=None) -> list:
    """The k largest independent-set sizes (total weights with vertex_w),
    each repeated by the number of sets of that size, in ascending order.
    k = 1 is SizeMax()."""
    c = _poly(plan, polynomial, vertex_w)
    out = []
    for s in range(len(c) - 1, -1, -1):
        take = min(c[s], k - len(out))
        out += [s] * take
        if len(out) == k:
            break
    return sorted(out)


# --------------------------------------------------------------------------- spin glass (Eq. 1)

def spin_glass_ground_state(plan, edge_w=None, vertex_w=None) -> tuple:
    """(E_min, degeneracy) of H = sum J s_i s_j + sum h s_i (the paper's
    CountingMin), from the counting contraction of -H on the GPU."""
    r = plan.contract_weighted("counting", "spin", edge_w, vertex_w)
    return -r["max"], r["count"]


def energy_histogram(plan, edge_w=None, vertex_w=None) -> tuple:
    """(shift, c) with c[k] = the exact number of spin configurations of
    energy k - shift, shift = sum|J| + sum|h| (tn_weighted_polynomial)."""
    import numpy as np
    m = len(plan.edges)
    sj = m if edge_w is None else int(np.abs(np.asarray(edge_w, dtype=np.int64)).sum())
    sh = 0 if vertex_w is None else int(np.abs(np.asarray(vertex_w, dtype=np.int64)).sum())
    return sj + sh, plan.weighted_polynomial("spin", edge_w, vertex_w)


def counting_min(plan, k: int = 1, edge_w=None, vertex_w=None, histogram=None) -> dict:
    """{energy: number of configurations} for the k lowest energies that
    occur (CountingMin(k) of Sec. 5.3 for the spin glass of Eq. 1), read off
    the exact energy histogram (energy_histogram, or `histogram` = (shift,
    c) as it returns).  k = 1 is the ground state and its degeneracy."""
    shift, c = histogram if histogram is not None else energy_histogram(plan, edge_w, vertex_w)
    levels = [i for i, v in enumerate(c) if v][:k]
    return {i - shift: c[i] for i in levels}


def log_partition_function(plan, beta: float, edge_w=None, vertex_w=None, histogram=None) -> float:
    """ln Z(beta), Z = sum_sigma e^{-beta H(sigma)} (PartitionFunction of
    Sec. 5.3), from the exact energy histogram: the largest term is factored
    out and the rest summed in float64."""
    import math
    shift, c = histogram if histogram is not None else energy_histogram(plan, edge_w, vertex_w)
    terms = [math.log(v) - beta * (k - shift) for k, v in enumerate(c) if v]
    top = max(terms)
    return top + math.log(sum(math.exp(t - top) for t in terms))


# --------------------------------------------------------------------------- k best configurations

def _k_best(n: int, k: int, sub) -> list:
    """Lawler's partition of the configurations of n binary variables: the
    best configuration x of a subspace (variables forced to 1 in F1, to 0
    in F0) splits the rest of that subspace into disjoint subspaces, one per
    free variable v_i in index order, each agreeing with x on v_1 .. v_{i-1}
    and differing on v_i.  sub(F1, F0) -> (score, config) or None (empty
    subspace) gives a subspace's best.  A subspace waits in the heap with its
    parent's score as a bound (none of its configurations beats the best of
    the subspace containing it) and is solved only when it reaches the top,
    so k configurations take about k passes when many share the top scores,
    at most k n.  Returns the k best [(score, config)], score non-increasing."""
    import heapq
    # entries (-bound, tick, cfg, f1, f0); cfg None: not solved yet
    out, heap, tick = [], [(0, 0, None, frozenset(), frozenset())], 0
    while heap and len(out) < k:
        negv, _, cfg, f1, f0 = heapq.heappop(heap)
        if cfg is None:
            r = sub(f1, f0)
            if r is not None:
                tick += 1
                heapq.heappush(heap, (-r[0], tick, r[1], f1, f0))
            continue
        out.append((-negv, cfg))
        in_, out_ = set(f1), set(f0)
        for v in range(n):
            if v in f1 or v in f0:
                continue
            f1n, f0n = (frozenset(in_), frozenset(out_ | {v})) if cfg[v] else (frozenset(in_ | {v}), frozenset(out_))
            tick += 1
            heapq.heappush(heap, (negv, tick, None, f1n, f0n))
            (in_ if cfg[v] else out_).add(v)
    return out


def _workspace_solver(plan, problem):
    """solve(edge_w, vertex_w) -> (max, config) through Plan.single_config_max
    with one workspace for every pass."""
    import torch

    from . import tn
    ws = torch.empty(tn.tn_single_config_workspace_bytes(plan.handle), dtype=torch.uint8, device="cuda")

    def solve(edge_w, vertex_w):
        return plan.single_config_max(problem, edge_w=edge_w, vertex_w=vertex_w, workspace=ws)
    return solve


def single_config_max_k(plan, k: int = 1, vertex_w=None, solve=None) -> list:
    """SingleConfigMax(k) of Sec. 5.3: k distinct independent sets whose
    total weights (sizes with vertex_w None) are the k largest over all
    independent sets, ties in any order, as [(weight, config)] by
    non-increasing weight (fewer if the graph has fewer sets).  plan: an
    unsliced Plan (the optimal-configuration pass needs every intermediate).

    Lawler's partition (_k_best) over the vertices' 0/1 values.  A
    subspace's best set comes from one optimal-configuration pass on the
    GPU (Plan.single_config_max, or `solve(weights) -> (max, config)`): with
    B = 2 sum|w| + 1, vertices of F1 weigh w + B and those of F0 w - B, so
    every optimum avoids F0 and holds all of F1 when F1 is independent (the
    subspace is empty otherwise); its weight is max - B |F1|."""
    import numpy as np
    n = plan.n
    e = np.asarray(plan.edges).reshape(-1, 2)
    w = np.ones(n, dtype=np.int64) if vertex_w is None else np.asarray(vertex_w, dtype=np.int64).reshape(-1)
    if w.size != n:
        raise ValueError("vertex_w needs one weight per vertex")
    big = 2 * int(np.abs(w).sum()) + 1
    if int(np.abs(w).sum()) + big * n > 2 ** 28:       # the int32 max-plus path's bound on sum |w|
        raise ValueError("weights too large to force vertices in or out")
    if solve is None:
        gpu = _workspace_solver(plan, "is")

        def solve(wf):
            return gpu(None, wf)
    nbr = [set() for _ in range(n)]
    for a, b in e.tolist():
        nbr[a].add(b)
        nbr[b].add(a)

    def sub(f1, f0):
        if any(nbr[v] & f1 for v in f1):
            return None
        wf = w.copy()
        wf[list(f1)] += big
        wf[list(f0)] -= big
        val, cfg = solve(wf.astype(np.int32))
        cfg = np.asarray(cfg, dtype=np.uint8)
        if any(cfg[v] == 0 for v in f1) or any(cfg[v] == 1 for v in f0):
            return None
        return int(val) - big * len(f1), cfg

    return _k_best(n, k, sub)


def spin_glass_lowest_k(plan, k: int = 1, edge_w=None, vertex_w=None, solve=None) -> list:
    """The k lowest-energy configurations of the spin glass of Eq. 1,
    H = sum J s_i s_j + sum h s_i (couplings edge_w, None: 1; fields
    vertex_w, None: 0), ties in any order, as [(energy, spins)] by
    non-decreasing energy, spins in {-1, +1}.  plan: an unsliced Plan.

    Lawler's partition (_k_best) over the spins; a subspace's best comes
    from one ground-state pass on the GPU (Plan.single_config_max of -H, or
    `solve(edge_w, vertex_w) -> (max of -H, config)`, config bit 1 = spin
    +1), spins forced through their fields: with B = sum|J| + sum|h| + 1,
    h - B forces s = +1 and h + B forces s = -1 (a wrong forced spin costs
    2B, more than any other change can gain).  Energies are those of the
    original couplings and fields."""
    import numpy as np
    n = plan.n
    e = np.asarray(plan.edges).reshape(-1, 2)
    J = np.ones(len(e), dtype=np.int64) if edge_w is None else np.asarray(edge_w, dtype=np.int64).reshape(-1)
    h = np.zeros(n, dtype=np.int64) if vertex_w is None else np.asarray(vertex_w, dtype=np.int64).reshape(-1)
    if J.size != len(e) or h.size != n:
        raise ValueError("edge_w needs one coupling per edge, vertex_w one field per vertex")
    total = int(np.abs(J).sum()) + int(np.abs(h).sum())
    big = total + 1
    if total + big * n > 2 ** 28:                     # the int32 max-plus path's bound on sum |J| + sum |h|
        raise ValueError("couplings and fields too large to force spins")
    if solve is None:
        solve = _workspace_solver(plan, "spin")
    J32 = J.astype(np.int32)

    def sub(f1, f0):
        hf = h.copy()
        hf[list(f1)] -= big
        hf[list(f0)] += big
        _, cfg = solve(J32, hf.astype(np.int32))
        cfg = np.asarray(cfg, dtype=np.uint8)
        if any(cfg[v] == 0 for v in f1) or any(cfg[v] == 1 for v in f0):
            return None                                 # cannot happen with this B; kept as a check
        sp = 2 * cfg.astype(np.int64) - 1
        energy = int((J * sp[e[:, 0]] * sp[e[:, 1]]).sum() + (h * sp).sum()) if len(e) else int((h * sp).sum())
        return -energy, cfg

    return [(-score, 2 * cfg.astype(np.int8) - 1) for score, cfg in _k_best(n, k, sub)]
