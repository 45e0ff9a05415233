"""Seeded synthetic graph generators.

This module is the single source of inputs shared by the CPU oracle and the
GPU path.  It holds no tensor-network arithmetic: it only produces simple
undirected graphs as ``(n, edges)`` with ``edges`` an ``int32`` array of shape
``(m, 2)``, 0-based, ``u != v``, no duplicate edges, each edge stored with
``u < v`` and the edge list sorted.

The families stand in for the graphs the paper studies (Sec. 2.1.1, the
``petersen``, ``square``, ``ksg`` and ``regular3`` constructors): the Petersen
graph, the L x L square lattice, King's subgraphs (an L x L grid whose sites are
kept independently with probability ``p``, joined at Chebyshev distance 1) and
random 3-regular graphs.  The paper's own graphs come from Julia generators whose
random streams are not reproducible here, so these are fresh seeded stand-ins
with the same structure.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "canonical",
    "petersen",
    "path",
    "cycle",
    "complete",
    "empty",
    "square_lattice",
    "kings_subgraph",
    "random_regular3",
    "erdos_renyi",
    "fullerene",
    "random_weights",
    "by_name",
]


def canonical(n: int, pairs) -> tuple[int, np.ndarray]:
    """Return ``(n, edges)`` with each edge as (min, max), duplicates removed, sorted."""
    e = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    if e.size:
        if (e < 0).any() or (e >= n).any():
            raise ValueError("vertex id out of range")
        if (e[:, 0] == e[:, 1]).any():
            raise ValueError("self-loop")
        e = np.sort(e, axis=1)
        e = np.unique(e, axis=0)
    return int(n), e.astype(np.int32).reshape(-1, 2)


def petersen() -> tuple[int, np.ndarray]:
    """The Petersen graph: outer 5-cycle, five spokes, inner pentagram (10 vertices, 15 edges)."""
    pairs = []
    for i in range(5):
        pairs.append((i, (i + 1) % 5))          # outer cycle
        pairs.append((i, i + 5))                # spoke
        pairs.append((5 + i, 5 + (i + 2) % 5))  # pentagram
    return canonical(10, pairs)


def path(n: int) -> tuple[int, np.ndarray]:
    return canonical(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n: int) -> tuple[int, np.ndarray]:
    if n < 3:
        raise ValueError("a simple cycle needs n >= 3")
    return canonical(n, [(i, (i + 1) % n) for i in range(n)])


def complete(n: int) -> tuple[int, np.ndarray]:
    return canonical(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def empty(n: int) -> tuple[int, np.ndarray]:
    return canonical(n, [])


def square_lattice(L: int, W: int | None = None) -> tuple[int, np.ndarray]:
    """L x W grid (row-major vertex ids), nearest-neighbour edges."""
    W = L if W is None else W
    pairs = []
    for r in range(L):
        for c in range(W):
            v = r * W + c
            if c + 1 < W:
                pairs.append((v, v + 1))
            if r + 1 < L:
                pairs.append((v, v + W))
    return canonical(L * W, pairs)


def kings_subgraph(L: int, p: float, seed: int) -> tuple[int, np.ndarray]:
    """King's subgraph: each site of an L x L grid kept with probability ``p``.

    Kept sites are numbered row-major; two kept sites are adjacent iff their
    Chebyshev distance is 1 (horizontal, vertical and both diagonals).
    """
    rng = np.random.default_rng(seed)
    keep = rng.random((L, L)) < p
    ids = -np.ones((L, L), dtype=np.int64)
    ids[keep] = np.arange(int(keep.sum()))
    pairs = []
    for r in range(L):
        for c in range(L):
            if not keep[r, c]:
                continue
            for dr, dc in ((0, 1), (1, -1), (1, 0), (1, 1)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < L and 0 <= cc < L and keep[rr, cc]:
                    pairs.append((ids[r, c], ids[rr, cc]))
    return canonical(int(keep.sum()), pairs)


def random_regular3(n: int, seed: int, max_tries: int = 10000) -> tuple[int, np.ndarray]:
    """Random 3-regular simple graph by the configuration model with rejection.

    Each vertex gets three half-edges; a uniformly random perfect matching of
    the 3n half-edges is drawn and rejected if it has a loop or a repeated edge.
    ``n`` must be even (3n half-edges must pair up).
    """
    if n % 2 or n < 4:
        raise ValueError("3-regular graphs need even n >= 4")
    rng = np.random.default_rng(seed)
    stubs = np.repeat(np.arange(n), 3)
    for _ in range(max_tries):
        perm = rng.permutation(stubs)
        e = perm.reshape(-1, 2)
        if (e[:, 0] == e[:, 1]).any():
            continue
        s = np.sort(e, axis=1)
        if len(np.unique(s, axis=0)) != len(s):
            continue
        return canonical(n, s)
    raise RuntimeError("configuration model did not produce a simple graph")


def erdos_renyi(n: int, p: float, seed: int) -> tuple[int, np.ndarray]:
    """G(n, p): each of the n(n-1)/2 pairs is an edge independently with probability p."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, k=1)
    mask = rng.random(iu.shape[0]) < p
    return canonical(n, np.stack([iu[mask], ju[mask]], axis=1))


def fullerene() -> tuple[int, np.ndarray]:
    """The Buckyball C60 (truncated icosahedron, Sec. 6.4): 60 vertices, 90
    edges.  Built combinatorially: the icosahedron's 12 vertices are the
    cyclic permutations of (0, +-1, +-phi), joined when at distance 2; each
    directed edge (u -> v) becomes a vertex near u; (u -> v) is joined to
    (v -> u) (the hexagon-hexagon edges) and to (u -> w) for the two
    neighbours w of u adjacent to v (the pentagon around u)."""
    phi = (1 + 5 ** 0.5) / 2
    pts = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            pts += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    pts = np.array(pts)
    d = np.linalg.norm(pts[:, None, :] - pts[None, :, :], axis=2)
    adj = [[j for j in range(12) if j != i and abs(d[i, j] - 2.0) < 1e-9] for i in range(12)]
    ids = {}
    for u in range(12):
        for v in adj[u]:
            ids[(u, v)] = len(ids)
    pairs = []
    for (u, v), i in ids.items():
        pairs.append((i, ids[(v, u)]))
        for w in adj[u]:
            if w in adj[v]:
                pairs.append((i, ids[(u, w)]))
    return canonical(len(ids), pairs)


def random_weights(count: int, seed: int, values=(-1, 1)) -> np.ndarray:
    """``count`` integers drawn uniformly from ``values`` (seeded): spin-glass
    couplings J_ij / fields h_i, or vertex weights."""
    rng = np.random.default_rng(seed)
    return np.asarray(values, dtype=np.int32)[rng.integers(0, len(values), size=count)]


def by_name(spec: str) -> tuple[int, np.ndarray]:
    """Parse a short graph spec, e.g. ``reg3:140:1``, ``ksg:20:0.8:1``, ``square:20``,
    ``petersen``, ``path:10``, ``cycle:9``, ``complete:5``, ``empty:6``, ``er:12:0.3:7``,
    ``fullerene``."""
    parts = spec.split(":")
    kind = parts[0]
    if kind == "petersen":
        return petersen()
    if kind == "path":
        return path(int(parts[1]))
    if kind == "cycle":
        return cycle(int(parts[1]))
    if kind == "complete":
        return complete(int(parts[1]))
    if kind == "empty":
        return empty(int(parts[1]))
    if kind == "square":
        return square_lattice(int(parts[1]))
    if kind == "ksg":
        return kings_subgraph(int(parts[1]), float(parts[2]), int(parts[3]))
    if kind == "reg3":
        return random_regular3(int(parts[1]), int(parts[2]))
    if kind == "er":
        return erdos_renyi(int(parts[1]), float(parts[2]), int(parts[3]))
    if kind == "fullerene":
        return fullerene()
    raise ValueError(f"unknown graph spec {spec!r}")
