"""Solution-space properties of Sec. 5.3 that follow from the independence
polynomial I(G, x) = sum_k c_k x^k (Eq. 13), computed on the GPU by
``Plan.independence_polynomial`` (weighted mod-p contractions, interpolation,
CRT):

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
"""
from __future__ import annotations


def counting_max(plan, k: int = 1, polynomial=None) -> dict:
    """{size: count} for the k largest sizes that occur (fewer if the graph
    has fewer distinct sizes).  k = 1 is CountingMax()."""
    c = polynomial if polynomial is not None else plan.independence_polynomial()
    sizes = [s for s in range(len(c) - 1, -1, -1) if c[s]][:k]
    return {s: c[s] for s in sorted(sizes)}


def size_max(plan, k: int = 1, polynomial=None) -> list:
    """The k largest independent-set sizes, each repeated by the number of
    sets of that size, in ascending order.  k = 1 is SizeMax()."""
    c = polynomial if polynomial is not None else plan.independence_polynomial()
    out = []
    for s in range(len(c) - 1, -1, -1):
        take = min(c[s], k - len(out))
        out += [s] * take
        if len(out) == k:
            break
    return sorted(out)
