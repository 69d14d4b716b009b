"""Seeded synthetic multi-patch Poisson problems.

This module only generates inputs (patch layouts, knot vectors, geometry
control points, interface pairings, right-hand sides and initial guesses).
It holds none of the solver's arithmetic and imports neither the library
binding nor the oracle, so both can be fed from it.

The paper's own domains (L-shape, Yeti footprint, Fichera corner) are read from
geometry files that are not published; the generators below build domains of
the same kind: grids of multilinear patches with jittered interior vertices,
uniform knot vectors, conforming or non-matching (SIPG) discretisations.

Problem dict (the layout the binding marshals into `mgiga_problem`):
  dim, degree, knots[k][a], geo_degree, geo_knots[k][a], geo_ctrl[k] (x-fastest),
  interfaces [(patch_a, side_a, patch_b, side_b, orient)], coupling
  ('conforming' | 'sipg'), sipg_penalty (C in eta = C / h), source
  ('sinprod': f = d pi^2 prod sin(pi x_a)).
"""
import itertools

import numpy as np


def uniform_knots(n, p):
    """Open uniform knot vector with n intervals on [0, 1] (knot i is i/n)."""
    inner = [i / n for i in range(1, n)]
    return np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1))


def _corner_index(bits):
    """Control point index of a multilinear patch corner (x-fastest)."""
    return sum(b << a for a, b in enumerate(bits))


def grid_problem(cells, n, p, coupling, box=None, jitter=0.0, seed=0,
                 jitter_boundary_tangential=False, penalty_factor=5.0,
                 flip_patches=(), transpose_patches=(), active=None):
    """Grid of cells[0] x ... multilinear patches covering the box [0, box_a].

    n: intervals per direction, an int or a callable (patch grid multi-index,
       direction) -> int.
    jitter: interior vertices move by U[-jitter, jitter]^d (seeded); with
       jitter_boundary_tangential, boundary vertices that are not corners move
       along the boundary only, so the domain stays the box.
    flip_patches: patch ids whose first parameter direction is reversed;
    transpose_patches: patch ids whose first two parameter directions are
       swapped.  Both exercise the interface orientation bits.
    active: optional set of cell multi-indices to keep (a non-rectangular
       arrangement); vertices on the boundary of the kept cells are not jittered.
    Patch ids are row-major over the (kept) cell grid (first direction fastest).
    """
    d = len(cells)
    box = tuple(float(b) for b in (box if box is not None else cells))
    rng = np.random.default_rng(seed)
    vshape = tuple(c + 1 for c in cells)
    verts = {}
    for vidx in itertools.product(*[range(s) for s in reversed(vshape)]):
        vidx = tuple(reversed(vidx))  # first index fastest
        x = np.array([box[a] * vidx[a] / cells[a] for a in range(d)])
        verts[vidx] = x
    keep = None if active is None else set(tuple(c) for c in active)

    def interior_vertex(vidx):
        # a vertex inside the domain: every cell around it is kept
        for off in itertools.product(*[(-1, 0)] * d):
            c = tuple(vidx[a] + off[a] for a in range(d))
            if any(c[a] < 0 or c[a] >= cells[a] for a in range(d)) or (keep is not None and c not in keep):
                return False
        return True

    for vidx in sorted(verts, key=lambda v: tuple(reversed(v))):
        on_bnd = [vidx[a] in (0, cells[a]) for a in range(d)]
        if keep is not None:
            if interior_vertex(vidx):
                verts[vidx] = verts[vidx] + rng.uniform(-jitter, jitter, size=d)
            continue
        if not any(on_bnd):
            verts[vidx] = verts[vidx] + rng.uniform(-jitter, jitter, size=d)
        elif jitter_boundary_tangential and not all(on_bnd):
            delta = rng.uniform(-jitter, jitter, size=d)
            for a in range(d):
                if on_bnd[a]:
                    delta[a] = 0.0
            verts[vidx] = verts[vidx] + delta

    knots, geo_knots, geo_ctrl, corner_vertex = [], [], [], []
    cell_list = [tuple(reversed(c)) for c in itertools.product(*[range(c) for c in reversed(cells)])]
    if keep is not None:
        cell_list = [c for c in cell_list if c in keep]
    for pid, cidx in enumerate(cell_list):
        perm = list(range(d))
        if pid in transpose_patches:
            perm[0], perm[1] = perm[1], perm[0]
        flip = [False] * d
        if pid in flip_patches:
            flip[0] = True
        # local direction a runs along global direction perm[a]
        cmap = {}
        ctrl = np.zeros((2 ** d, d))
        for bits in itertools.product(*[range(2)] * d):
            bits = tuple(reversed(bits))
            gbits = [0] * d
            for a in range(d):
                gbits[perm[a]] = bits[a] ^ int(flip[a])
            v = tuple(cidx[a] + gbits[a] for a in range(d))
            cmap[bits] = v
            ctrl[_corner_index(bits)] = verts[v]
        nk = []
        for a in range(d):
            na = n(cidx, perm[a]) if callable(n) else n
            nk.append(uniform_knots(na, p))
        knots.append(nk)
        geo_knots.append([np.array([0.0, 0.0, 1.0, 1.0]) for _ in range(d)])
        geo_ctrl.append(ctrl)
        corner_vertex.append(cmap)

    interfaces = []
    K = len(cell_list)
    for ka in range(K):
        for kb in range(ka + 1, K):
            shared = set(corner_vertex[ka].values()) & set(corner_vertex[kb].values())
            if len(shared) != 2 ** (d - 1):
                continue
            sa = _side_of(corner_vertex[ka], shared, d)
            sb = _side_of(corner_vertex[kb], shared, d)
            interfaces.append((ka, sa, kb, sb, _orientation(corner_vertex[ka], sa,
                                                            corner_vertex[kb], sb, d)))
    return dict(dim=d, degree=p, knots=knots, geo_degree=1, geo_knots=geo_knots,
                geo_ctrl=geo_ctrl, interfaces=interfaces, coupling=coupling,
                sipg_penalty=penalty_factor * (p + 1) ** 2, source="sinprod")


def _side_of(cmap, shared, d):
    bits = [b for b, v in cmap.items() if v in shared]
    for a in range(d):
        vals = {b[a] for b in bits}
        if len(vals) == 1:
            return 2 * a + vals.pop()
    raise ValueError("vertices do not form a side")


def _side_corner(side, tbits, d):
    """Local corner bits of the side corner with tangential bits tbits."""
    a = side // 2
    tdirs = [t for t in range(d) if t != a]
    bits = [0] * d
    bits[a] = side % 2
    for m, t in enumerate(tdirs):
        bits[t] = tbits[m]
    return tuple(bits)


def _orientation(cmap_a, sa, cmap_b, sb, d):
    """Orientation bits of the interface, as defined in the problem layout."""
    m = d - 1
    inv_b = {}
    for tb in itertools.product(*[range(2)] * m):
        inv_b[cmap_b[_side_corner(sb, tb, d)]] = tb
    origin_b = inv_b[cmap_a[_side_corner(sa, (0,) * m, d)]]
    orient = 0
    for c in range(m):
        if origin_b[c]:
            orient |= 1 << c
    if m == 2:
        e0 = inv_b[cmap_a[_side_corner(sa, (1, 0), d)]]
        if e0[0] == origin_b[0]:
            orient |= 4
    return orient


# ----------------------------------------------------------------------------
# source terms and right-hand sides
# ----------------------------------------------------------------------------

def source_sinprod(x):
    """f = d pi^2 prod_a sin(pi x_a), i.e. -Laplace of prod_a sin(pi x_a)."""
    x = np.atleast_2d(x)
    d = x.shape[1]
    return d * np.pi ** 2 * np.prod(np.sin(np.pi * x), axis=1)


def exact_sinprod(x):
    x = np.atleast_2d(x)
    return np.prod(np.sin(np.pi * x), axis=1)


def random_vector(ndof, seed, kind="uniform"):
    """Seeded vector: U[-1, 1] ('uniform') or N(0, 1) ('normal')."""
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return rng.uniform(-1.0, 1.0, size=ndof)
    return rng.standard_normal(ndof)


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------

def unit_square_2x2(n=32, p=2):
    """Unit square as 2x2 conforming identity-geometry patches (p=2, n=32:
    4,225 unknowns); solved with the V-cycle and SCMS (tau=1, delta=.12),
    4 levels, initial guess seeded U[-1, 1] (seed 101)."""
    prob = grid_problem((2, 2), n, p, "conforming", box=(1.0, 1.0))
    opts = dict(levels=4, smoother="scms", tau=1.0, delta=0.12, nu=1, seed_u0=101)
    return prob, opts


def sipg_3x3(p, scale=1, smoother="scms"):
    """[0,3]^2 as 3x3 SIPG patches, interior vertices jittered U[-.1, .1]^2,
    64 (even i+j) / 96 (odd) intervals times `scale`, penalty 5 (p+1)^2 / h.

    scale=1 is 60-66k unknowns, scale=3 is 0.52-0.54M unknowns.
    SCMS: tau=.25, delta=.2; hybrid: tau=.25, delta=.1; PCG.
    """
    def n_of(cidx, a):
        return (64 if (cidx[0] + cidx[1]) % 2 == 0 else 96) * scale
    prob = grid_problem((3, 3), n_of, p, "sipg", box=(3.0, 3.0), jitter=0.1,
                        seed=201 + (p - 2))
    delta = 0.2 if smoother == "scms" else 0.1
    opts = dict(levels=0, smoother=smoother, tau=0.25, delta=delta, nu=1)
    return prob, opts


def with_patch_degrees(prob, degrees):
    """The same patches (same interval counts) with spline degree degrees[k] on patch k: knot
    vectors rebuilt per patch, `degree` the largest, the SIPG penalty factor 5 (p + 1)^2 taken
    with that largest degree."""
    out = dict(prob)
    out["degrees"] = [int(x) for x in degrees]
    out["degree"] = max(out["degrees"])
    out["knots"] = [[uniform_knots(len(np.unique(t)) - 1, pk) for t in kn]
                    for kn, pk in zip(prob["knots"], out["degrees"])]
    out["sipg_penalty"] = 5.0 * (out["degree"] + 1) ** 2
    return out


def lshape(p, r, nonmatching=True, smoother="scms"):
    """The L-shaped domain of the paper's experiments (Sec. 2: three quadrilaterals whose
    geometry maps are the identity or a translation): [0,2]^2 without (1,2]^2, patches [0,1]^2,
    [1,2]x[0,1], [0,1]x[1,2].  Patch 0 has 2^r intervals per direction.  nonmatching (the SIPG
    setting of Sec. 5, Table SCMS2): patch 0 carries S_{p,h}, patch 1 S_{p+1,2h}, patch 2
    S_{p,2h}; else all three S_{p,h} with SIPG coupling.  f from u = sin(pi x) sin(pi y), which
    vanishes on the whole boundary.  Options: the subspace-corrected mass smoother with the
    table's damping .9 and scaling .12 (smoother="hybrid": .25 / .1), PCG; levels: coarsen until
    the coarse patches have 2 intervals (the paper's coarsest grid has one element per patch)."""
    cells = [(0, 0), (1, 0), (0, 1)]
    n_of = {0: 2 ** r, 1: 2 ** (r - 1) if nonmatching else 2 ** r, 2: 2 ** (r - 1) if nonmatching else 2 ** r}

    def n(cidx, a):
        return n_of[cells.index(tuple(cidx))]
    prob = grid_problem((2, 2), n, p, "sipg", box=(2.0, 2.0), jitter=0.0, active=cells)
    if nonmatching:
        prob = with_patch_degrees(prob, [p, p + 1, p])
    opts = (dict(levels=0, smoother="scms", tau=0.9, delta=0.12) if smoother == "scms"
            else dict(levels=0, smoother="hybrid", tau=0.25, delta=0.1))
    return prob, opts


def cube_2x2x2(p, coupling, n=48):
    """[0,1]^3 as 2x2x2 trilinear patches: centre vertex jittered U[-.05,.05]^3,
    boundary non-corner vertices jittered tangentially; hybrid smoother
    (tau=.25, delta=.12), PCG."""
    prob = grid_problem((2, 2, 2), n, p, coupling, box=(1.0, 1.0, 1.0), jitter=0.05,
                        seed=301 + (p - 3), jitter_boundary_tangential=True)
    opts = dict(levels=0, smoother="hybrid", tau=0.25, delta=0.12, nu=1)
    return prob, opts


def batched_problem(seed):
    """One problem of the batched layout (seeded): K ~ U{1..16} unit-square
    patches in ceil(sqrt(K)) columns filled row-major (the last row may be
    partial), intervals per direction log-uniform in [16, 256] rounded to the
    nearest c 2^j with c in {4..7} (so the hierarchy has >= 2 levels with >= 4
    intervals on the coarsest), p ~ U{2..5}, conforming or SIPG with
    probability 1/2, vertices inside the domain jittered U[-.1, .1]^2, hybrid
    smoother (tau .25, delta .1), PCG; the right-hand side is i.i.d. N(0, 1)
    load coefficients (seed + 1000).  Returns (problem, options, rhs seed)."""
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 17))
    cols = int(np.ceil(np.sqrt(K)))
    rows = (K + cols - 1) // cols
    active = [(i % cols, i // cols) for i in range(K)]
    n_raw = float(np.exp(rng.uniform(np.log(16.0), np.log(256.0))))
    cands = [c * 2 ** j for c in range(4, 8) for j in range(0, 7) if 16 <= c * 2 ** j <= 256]
    n = int(min(cands, key=lambda v: (abs(v - n_raw), v)))
    p = int(rng.integers(2, 6))
    coupling = "conforming" if rng.uniform() < 0.5 else "sipg"
    prob = grid_problem((cols, rows), n, p, coupling, box=(float(cols), float(rows)), jitter=0.1,
                        seed=seed, active=active)
    opts = dict(levels=0, smoother="hybrid", tau=0.25, delta=0.1, nu=1)
    return prob, opts, seed + 1000


def serving_stream(n_requests, seed=501, max_patch_dof=1e6):
    """Requests of the serving layout (seeded): 2D with probability .7, else 3D;
    1-27 unit patches in a near-square (near-cubic) arrangement filled row-major;
    per-patch DoF log-uniform in [1e3, max_patch_dof] (intervals per direction
    rounded to the nearest c 2^j, c in {4..7}, >= 2 levels); p ~ U{2..6};
    conforming or SIPG with probability 1/2; vertices inside the domain jittered
    (.1 in 2D, .05 in 3D); hybrid smoother; half of the requests reuse an earlier
    operator.  Yields (key, problem, options, rhs seed); the right-hand side is
    i.i.d. N(0, 1) load coefficients."""
    rng = np.random.default_rng(seed)
    ops = []
    for i in range(n_requests):
        if ops and rng.uniform() < 0.5:
            key, prob, opts = ops[int(rng.integers(len(ops)))]
        else:
            d = 2 if rng.uniform() < 0.7 else 3
            K = int(rng.integers(1, 28))
            side = int(np.ceil(K ** (1.0 / d) - 1e-9))
            cells = (side,) * d
            active = [tuple((j // side ** a) % side for a in range(d)) for j in range(K)]
            p = int(rng.integers(2, 7))
            dof = float(np.exp(rng.uniform(np.log(1e3), np.log(max_patch_dof))))
            n_raw = max(dof ** (1.0 / d) - p, 8.0)
            min_n = 8 if d == 2 else 12  # two levels with >= 2 (2D) / 3 (3D) intervals per half
            cands = [c * 2 ** j for c in range(4, 8) for j in range(0, 9) if c * 2 ** j >= min_n]
            n = int(min(cands, key=lambda v: (abs(v - n_raw), v)))
            coupling = "conforming" if rng.uniform() < 0.5 else "sipg"
            prob = grid_problem(cells, n, p, coupling, box=tuple(float(c) for c in cells),
                                jitter=0.1 if d == 2 else 0.05, seed=seed * 1000 + i, active=active)
            opts = dict(levels=0, smoother="hybrid", tau=0.25, delta=0.1 if d == 2 else 0.12, nu=1)
            key = f"op{i}"
            ops.append((key, prob, opts))
        yield key, prob, opts, seed * 1000 + 500 + i
