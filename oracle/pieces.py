"""Piece decomposition of the DoFs (Sec. 5, Fig. decomp) -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Pieces are the patch interiors and the interface pieces: edges and vertices
(d = 2) or faces, edges and vertices (d = 3) of the patches.  A boundary DoF
of a patch lies on the entity formed by the sides it touches (index 0 or
N-1 in some directions).  Entities of different patches are the same piece
when the interfaces identify them; in the SIPG case an interface piece
therefore takes the DoFs of all patches sharing that entity (Sec. 5, the
discussion before Theorem 2 and Fig. decomp right).

Order (integer work, compared bit-exactly with the library): all interior
pieces by patch id, then interface pieces by their smallest global DoF; the
DoFs of a piece in increasing global order.
"""
import numpy as np

from . import discretize


def _entity_key(multi, shape):
    """Sides touched by a local DoF: tuple of (direction, end) pairs."""
    key = []
    for a, n in enumerate(shape):
        if multi[a] == 0:
            key.append((a, 0))
        elif multi[a] == n - 1:
            key.append((a, 1))
    return tuple(key)


def _map_key(key, iface, d):
    """Entity key on patch b of the entity `key` of patch a lying in side_a."""
    pa, sa, pb, sb, orient = iface
    ta = discretize.tangential_dirs(d, sa)
    tb = discretize.tangential_dirs(d, sb)
    swap = (d == 3) and bool(orient & 4)
    out = [(sb // 2, sb % 2)]
    for (a, end) in key:
        if a == sa // 2:
            continue
        c = ta.index(a)            # tangential coordinate on side a
        cb = (1 - c) if swap else c  # matching coordinate on side b
        flip = bool(orient & (1 << cb))
        out.append((tb[cb], end ^ int(flip)))
    return tuple(sorted(out))


def decompose(problem, num):
    """Pieces of one level: list of dicts with kind ('interior'|'interface'),
    patch (interior only) and dofs (global indices, increasing)."""
    d = problem["dim"]
    shapes = num["shapes"]
    # union-find over (patch, entity key)
    parent = {}

    def find(x):
        while parent.setdefault(x, x) != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    def union(x, y):
        rx, ry = find(x), find(y)
        if rx != ry:
            parent[max(rx, ry)] = min(rx, ry)

    # every entity contained in an interface side is identified across it
    for iface in problem["interfaces"]:
        pa, sa, pb, sb, _o = iface
        a = sa // 2
        others = [t for t in range(d) if t != a]
        # all entities of patch a inside side sa: fix (a, end) plus any subset
        # of the other directions at either end
        for mask in range(3 ** len(others)):
            key = [(a, sa % 2)]
            m = mask
            for t in others:
                c = m % 3
                m //= 3
                if c < 2:
                    key.append((t, c))
            key = tuple(sorted(key))
            union((pa, key), (pb, _map_key(key, iface, d)))

    interior = []
    groups = {}
    for k, shape in enumerate(shapes):
        l2g = num["loc2glob"][k]
        multi = discretize.unflatten(np.arange(len(l2g)), shape)
        inner = np.ones(len(l2g), dtype=bool)
        for a, n in enumerate(shape):
            inner &= (multi[a] >= 1) & (multi[a] <= n - 2)
        interior.append(dict(kind="interior", patch=k, dofs=np.sort(l2g[inner])))
        for f in np.nonzero(~inner & (l2g >= 0))[0]:
            key = _entity_key([multi[a][f] for a in range(d)], shape)
            root = find((k, key))
            groups.setdefault(root, set()).add(int(l2g[f]))
    iface_pieces = [dict(kind="interface", patch=-1, dofs=np.array(sorted(s), dtype=np.int64))
                    for s in groups.values()]
    iface_pieces.sort(key=lambda pc: pc["dofs"][0])
    return [pc for pc in interior if len(pc["dofs"]) > 0] + iface_pieces
