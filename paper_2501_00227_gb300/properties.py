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
