"""Random d-regular Max-Cut graphs (Section 4.1 of the paper).

The paper places edges at random until every vertex reaches degree d and
rejects disconnected graphs; it names neither the pairing rule nor the RNG.
Reading used here: the configuration model with incremental stub pairing
(Steger and Wormald, 1999) — repeatedly pick two random unpaired stubs, keep
the pair only if it is neither a self-loop nor a repeated edge, restart from
scratch when no valid pair can be found, and reject the finished graph if it
is disconnected.  Every draw comes from one SplitMix64 stream seeded by
``seed``.
"""

from __future__ import annotations

from .rng import SplitMix64


def is_connected(n: int, edges) -> bool:
    """Breadth-first search from vertex 0 reaches all n vertices."""
    if n == 0:
        return True
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    seen = [False] * n
    seen[0] = True
    stack = [0]
    while stack:
        a = stack.pop()
        for b in adj[a]:
            if not seen[b]:
                seen[b] = True
                stack.append(b)
    return all(seen)


def _pair_stubs(n: int, d: int, rng: SplitMix64):
    stubs = [v for v in range(n) for _ in range(d)]
    present = set()
    edges = []
    misses = 0
    while stubs:
        i = rng.randbelow(len(stubs))
        j = rng.randbelow(len(stubs) - 1)
        if j >= i:
            j += 1
        a, b = stubs[i], stubs[j]
        key = (a, b) if a < b else (b, a)
        if a == b or key in present:
            misses += 1
            if misses > 64 + 8 * len(stubs):
                return None  # stuck: restart the whole pairing
            continue
        misses = 0
        present.add(key)
        edges.append(key)
        # swap-remove the two stubs (higher index first)
        for k in sorted((i, j), reverse=True):
            stubs[k] = stubs[-1]
            stubs.pop()
    return edges


def random_regular_graph(n: int, d: int, seed: int):
    """Seeded connected simple d-regular graph on n vertices.

    Returns a sorted list of ``(a, b)`` tuples with ``a < b``.
    """
    if n <= d or (n * d) % 2:
        raise ValueError(f"no simple {d}-regular graph on {n} vertices")
    rng = SplitMix64(seed)
    while True:
        edges = _pair_stubs(n, d, rng)
        if edges is None:
            continue
        if is_connected(n, edges):
            return sorted(edges)


def ring_plus_pairs_graph(n: int, seed: int):
    """3-regular graph built from a ring plus random chords (Section 5).

    The paper's 100-qubit example starts from the n-cycle and joins random
    pairs of vertices until every vertex has degree 3.  Pairs that would form
    a repeated edge are redrawn; a stuck matching restarts.
    """
    if n % 2 or n < 4:
        raise ValueError("ring plus pairs needs an even n >= 4")
    rng = SplitMix64(seed)
    ring = [(i, (i + 1) % n) for i in range(n)]
    ring = [(min(a, b), max(a, b)) for a, b in ring]
    while True:
        present = set(ring)
        free = list(range(n))
        chords = []
        misses = 0
        ok = True
        while free:
            i = rng.randbelow(len(free))
            j = rng.randbelow(len(free) - 1)
            if j >= i:
                j += 1
            a, b = free[i], free[j]
            key = (min(a, b), max(a, b))
            if key in present:
                misses += 1
                if misses > 64 + 8 * len(free):
                    ok = False
                    break
                continue
            misses = 0
            present.add(key)
            chords.append(key)
            for k in sorted((i, j), reverse=True):
                free[k] = free[-1]
                free.pop()
        if ok:
            return sorted(ring + chords)
