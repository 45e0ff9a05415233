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

The paper computes both with dedicated element types in one contraction;
here they are read off the exact polynomial, which costs alpha + 1
evaluations per prime instead of one wider contraction but gives the same
numbers (counts are exact integers, not saturated).

SingleConfigMax(k) (single_config_max_k): k distinct sets with the k
largest sizes or total weights, by Lawler's partition of the solution space
over the GPU's optimal-configuration pass (tn_single_config_max), vertices
forced in or out through their weights.

For the spin glass of Eq. 1: the ground state (CountingMin) from the
counting contraction of -H, the exact energy histogram from
``Plan.weighted_polynomial``, and ln Z(beta) (PartitionFunction) summed from
that histogram.
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

def single_config_max_k(plan, k: int = 1, vertex_w=None, solve=None) -> list:
    """SingleConfigMax(k) of Sec. 5.3: k distinct independent sets whose
    total weights (sizes with vertex_w None) are the k largest over all
    independent sets, ties in any order, as [(weight, config)] by
    non-increasing weight (fewer if the graph has fewer sets).

    Lawler's partition of the solution space: the best set x of a subspace
    (vertices forced in F1, forced out F0) splits the rest of that subspace
    into disjoint subspaces, one per free vertex v_i in index order, each
    agreeing with x on v_1 .. v_{i-1} and differing on v_i; the best of
    every open subspace waits in a heap.  A subspace's best set comes from
    one optimal-configuration pass on the GPU (Plan.single_config_max, or
    `solve(weights) -> (max, config)`): with B = 2 sum|w| + 1, vertices of
    F1 weigh w + B and those of F0 w - B, so every optimum avoids F0 and
    holds all of F1 when F1 is independent; its weight is max - B |F1|.
    Subspaces are solved only when their bound (the parent's weight)
    reaches the top of the heap, so k sets take far fewer than k n passes
    when many sets share the top weights."""
    import heapq

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
        import torch

        from . import tn
        ws = torch.empty(tn.tn_single_config_workspace_bytes(plan.handle), dtype=torch.uint8, device="cuda")

        def solve(wf):
            return plan.single_config_max("is", vertex_w=wf, workspace=ws)
    nbr = [set() for _ in range(n)]
    for a, b in e.tolist():
        nbr[a].add(b)
        nbr[b].add(a)

    def best(f1, f0):
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

    # heap entries (-bound, tick, cfg, f1, f0): cfg None marks a subspace not
    # solved yet, whose bound is its parent's weight (no set of a subspace
    # outweighs the best of the subspace containing it); it is solved when
    # it reaches the top and goes back in with its own weight
    out, heap, tick = [], [(0, 0, None, frozenset(), frozenset())], 0
    while heap and len(out) < k:
        negv, _, cfg, f1, f0 = heapq.heappop(heap)
        if cfg is None:
            r = best(f1, f0)
            if r is not None:
                tick += 1
                heapq.heappush(heap, (-r[0], tick, r[1], f1, f0))
            continue
        out.append((-negv, cfg))
        in_, out_ = set(f1), set(f0)
        for v in range(n):
            if v in f1 or v in f0:
                continue
            # the subspace agreeing with cfg before v and differing at v
            if not cfg[v] and nbr[v] & in_:
                pass                                    # v cannot join: the subspace is empty
            else:
                f1n, f0n = (frozenset(in_), frozenset(out_ | {v})) if cfg[v] else (frozenset(in_ | {v}), frozenset(out_))
                tick += 1
                heapq.heappush(heap, (negv, tick, None, f1n, f0n))
            (in_ if cfg[v] else out_).add(v)
    return out
