"""Multi-patch discretisation: DoF numbering, Galerkin and SIPG assembly -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Sec. 2 (conforming space V^c, Eq. igaspace0 / model:discr) and Sec. 3
(non-conforming space V^n, SIPG form Eq. model:discr2).

A problem is a dict:
  dim, degree              d in {2, 3}, spline degree p (all patches/directions)
  knots[k][a]              open knot vector of patch k in direction a
  geo_degree, geo_knots[k][a], geo_ctrl[k]
                           geometry spline of patch k (control points x-fastest)
  interfaces               list of (patch_a, side_a, patch_b, side_b, orient)
  coupling                 'conforming' or 'sipg'
  sipg_penalty             C; the penalty is eta = C / h_I (see sipg_eta)
Sides: 2*a + 0 is xi_a = 0, 2*a + 1 is xi_a = 1.  A patch side that is not
listed in an interface lies on the boundary and carries the homogeneous
Dirichlet condition, imposed strongly (Sec. 3).  orient: bit 2 swaps the two
tangential coordinates (3D), then bit m flips tangential coordinate m of side_b
(s -> 1 - s).  Tangential directions of a side are the other directions in
increasing order.

Local (patch) DoF index: flat = i_0 + N_0 (i_1 + N_1 i_2), xi_0 fastest.
Global DoF order: patches in id order, local flat order within a patch,
Dirichlet DoFs skipped, and in the conforming case a DoF already numbered
through a lower-id patch is skipped.
"""
import numpy as np
import scipy.sparse as sp

from . import bspline, geometry


# ----------------------------------------------------------------------------
# index helpers
# ----------------------------------------------------------------------------

def shape_of(knots_k, p):
    """Number of basis functions per direction (N_0, ..., N_{d-1})."""
    return tuple(bspline.num_basis(t, p) for t in knots_k)


def degree_of(problem, k):
    """Spline degree of patch k (the same in every direction): problem["degrees"][k] when the
    problem lists one per patch (the non-matching setting of the SIPG experiments of Sec. 5,
    Table SCMS2: one third of the patches carry S_{p,h}, one third S_{p+1,2h} and one third
    S_{p,2h}), else problem["degree"]."""
    dk = problem.get("degrees")
    return int(problem["degree"] if dk is None else dk[k])


def max_degree(problem):
    """Largest patch degree (the reach of the patch band, the modulus of the colouring)."""
    dk = problem.get("degrees")
    return int(problem["degree"] if dk is None else max(dk))


def unflatten(flat, shape):
    """Multi-index (i_0, ..., i_{d-1}) of local flat index (xi_0 fastest)."""
    out = []
    for n in shape:
        out.append(flat % n)
        flat = flat // n
    return tuple(out)


def flatten(multi, shape):
    flat = np.zeros_like(np.asarray(multi[0]))
    stride = 1
    for a, n in enumerate(shape):
        flat = flat + np.asarray(multi[a]) * stride
        stride *= n
    return flat


def tangential_dirs(d, side):
    return [a for a in range(d) if a != side // 2]


def interface_sides(problem):
    """Per patch, the set of sides that are listed in an interface."""
    sides = [set() for _ in problem["knots"]]
    for (pa, sa, pb, sb, _o) in problem["interfaces"]:
        sides[pa].add(sa)
        sides[pb].add(sb)
    return sides


def side_dofs(shape, side, layer=0):
    """Flat indices of the DoFs in layer `layer` from side `side`.

    Returned with their tangential multi-index (first tangential dir fastest).
    """
    d = len(shape)
    a = side // 2
    idx_n = layer if side % 2 == 0 else shape[a] - 1 - layer
    tdirs = tangential_dirs(d, side)
    tshape = [shape[t] for t in tdirs]
    grids = np.meshgrid(*[np.arange(n) for n in reversed(tshape)], indexing="ij")
    tmulti = [g.ravel() for g in reversed(grids)]  # first tangential fastest
    multi = [None] * d
    multi[a] = np.full_like(tmulti[0], idx_n)
    for m, t in enumerate(tdirs):
        multi[t] = tmulti[m]
    return flatten(multi, shape), tmulti


def map_tangential(tmulti_a, orient, tshape_b):
    """Tangential multi-index on side b of the DoF matching tmulti_a on side a.

    Used for fully matching interfaces (Assumption 2): the knot vector of side
    b, after the orientation map, equals that of side a, so flipping a
    coordinate reverses the basis index.
    """
    m = len(tmulti_a)
    if m == 2 and (orient & 4):
        tb = [tmulti_a[1], tmulti_a[0]]
    else:
        tb = list(tmulti_a)
    for c in range(m):
        if orient & (1 << c):
            tb[c] = tshape_b[c] - 1 - tb[c]
    return tb


def map_param(s_a, orient):
    """Interface parameter on side b of the point with parameter s_a on side a.

    s_a: (npts, m) tangential coordinates on side a.  Same map as
    map_tangential, applied to coordinates in [0, 1].
    """
    s = np.array(s_a, dtype=np.float64, copy=True)
    if s.shape[1] == 2 and (orient & 4):
        s = s[:, ::-1].copy()
    for c in range(s.shape[1]):
        if orient & (1 << c):
            s[:, c] = 1.0 - s[:, c]
    return s


# ----------------------------------------------------------------------------
# DoF numbering (Sec. 2, Eq. igaspace0 and Fig. dof; Sec. 3, Eq. igaspace)
# ----------------------------------------------------------------------------

class _UnionFind:
    def __init__(self, n):
        self.parent = np.arange(n)

    def find(self, x):
        root = x
        while self.parent[root] != root:
            root = self.parent[root]
        while self.parent[x] != root:
            self.parent[x], x = root, self.parent[x]
        return root

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra != rb:
            if ra < rb:
                self.parent[rb] = ra
            else:
                self.parent[ra] = rb


def dirichlet_local(problem, shapes):
    """Per patch, boolean mask of local DoFs with nonzero trace on a boundary side."""
    d = problem["dim"]
    isides = interface_sides(problem)
    out = []
    for k, shape in enumerate(shapes):
        mask = np.zeros(int(np.prod(shape)), dtype=bool)
        for s in range(2 * d):
            if s not in isides[k]:
                flat, _ = side_dofs(shape, s)
                mask[flat] = True
        out.append(mask)
    return out


def numbering(problem, knots):
    """Global DoF numbering for the patch knot vectors `knots` (one level).

    Returns a dict with
      shapes    per patch (N_0, ..., N_{d-1})
      offsets   start of each patch block in the concatenated local layout
      loc2glob  per patch int array, -1 for Dirichlet DoFs
      ndof      number of global unknowns
      owner     per global DoF, (patch, flat) of the copy that numbered it
    Conforming: copies of one DoF on matching interfaces share a number; a
    class of copies is Dirichlet if any copy has a nonzero trace on a
    boundary side.
    """
    shapes = [shape_of(kn, degree_of(problem, k)) for k, kn in enumerate(knots)]
    sizes = [int(np.prod(s)) for s in shapes]
    offsets = np.concatenate(([0], np.cumsum(sizes)))
    dir_local = dirichlet_local(problem, shapes)
    total = int(offsets[-1])
    conforming = problem["coupling"] == "conforming"

    uf = _UnionFind(total)
    if conforming:
        for (pa, sa, pb, sb, orient) in problem["interfaces"]:
            fa, ta = side_dofs(shapes[pa], sa)
            tdir_b = tangential_dirs(problem["dim"], sb)
            tshape_b = [shapes[pb][t] for t in tdir_b]
            tb = map_tangential(ta, orient, tshape_b)
            multi_b = [None] * problem["dim"]
            ab = sb // 2
            multi_b[ab] = np.full_like(tb[0], 0 if sb % 2 == 0 else shapes[pb][ab] - 1)
            for m, t in enumerate(tdir_b):
                multi_b[t] = tb[m]
            fb = flatten(multi_b, shapes[pb])
            for x, y in zip(fa + offsets[pa], fb + offsets[pb]):
                uf.union(int(x), int(y))

    roots = np.array([uf.find(i) for i in range(total)]) if conforming else np.arange(total)
    all_dir = np.concatenate(dir_local)
    root_dir = np.zeros(total, dtype=bool)
    np.logical_or.at(root_dir, roots, all_dir)

    glob_of_root = -np.ones(total, dtype=np.int64)
    loc2glob = []
    owner = []
    nxt = 0
    for k in range(len(shapes)):
        l2g = -np.ones(sizes[k], dtype=np.int64)
        for f in range(sizes[k]):
            r = roots[offsets[k] + f]
            if root_dir[r]:
                continue
            if glob_of_root[r] < 0:
                glob_of_root[r] = nxt
                owner.append((k, f))
                nxt += 1
            l2g[f] = glob_of_root[r]
        loc2glob.append(l2g)
    return dict(shapes=shapes, offsets=offsets, loc2glob=loc2glob, ndof=nxt,
                owner=owner, dirichlet=dir_local)


# ----------------------------------------------------------------------------
# Element quadrature on one patch
# ----------------------------------------------------------------------------

def _direction_data(t, p, nq):
    """Per direction: element spans, local basis values/derivatives at Gauss points."""
    x, w, elem = bspline.element_quadrature(t, nq)
    ne = elem.max() + 1
    z = bspline.breakpoints(t)
    mids = 0.5 * (z[:-1] + z[1:])
    spans = bspline.find_span(t, p, mids)
    B = bspline.basis(t, p, x)
    D = bspline.basis_deriv(t, p, x)
    vals = np.zeros((ne, nq, p + 1))
    ders = np.zeros((ne, nq, p + 1))
    for e in range(ne):
        cols = np.arange(spans[e] - p, spans[e] + 1)
        rows = np.arange(e * nq, (e + 1) * nq)
        vals[e] = B[np.ix_(rows, cols)]
        ders[e] = D[np.ix_(rows, cols)]
    return dict(x=x, w=w.reshape(ne, nq), ne=ne, spans=spans, vals=vals, ders=ders)


def _outer(mats):
    """Tensor product over directions of per-direction (q, l) arrays.

    mats[0] carries a leading element axis: (E, q, l).  Output axes
    (E, Q, L) with Q = q_0 + nq q_1 + ..., L = l_0 + (p+1) l_1 + ...
    """
    d = len(mats)
    out = mats[0]  # (E, q0, l0)
    for a in range(1, d):
        m = mats[a]  # (q_a, l_a)
        # out: (E, Qprev, Lprev) -> (E, q_a, Qprev, l_a, Lprev)
        out = out[:, None, :, None, :] * m[None, :, None, :, None]
        E = out.shape[0]
        out = out.reshape(E, out.shape[1] * out.shape[2], out.shape[3] * out.shape[4])
    return out


def _patch_elements(problem, k, knots_k):
    """Iterate over element rows of patch k, yielding quadrature data.

    Yields (outer, dd, J, X, W): outer = element multi-index of directions
    1..d-1, dd = per-direction data, J/X geometry at the points of that row of
    elements (E0, Q, d, d)/(E0, Q, d), W = tensor weights (E0, Q).
    """
    d = problem["dim"]
    p = degree_of(problem, k)
    nq = p + 1
    dd = [_direction_data(t, p, nq) for t in knots_k]
    X, J = geometry.eval_grid(problem["geo_degree"], problem["geo_knots"][k],
                              problem["geo_ctrl"][k], [dd[a]["x"] for a in range(d)])
    # X: (npts_{d-1}, ..., npts_0, d)
    E0 = dd[0]["ne"]
    outer_shape = [dd[a]["ne"] for a in range(1, d)]
    for outer in np.ndindex(*outer_shape):
        # select quad rows of the outer elements; reorder to (E0, Q)
        sl = []
        for a in reversed(range(1, d)):
            e = outer[a - 1]
            sl.append(slice(e * nq, (e + 1) * nq))
        Xs = X[tuple(sl)]  # (nq_{d-1}, ..., nq_1, npts_0, d)
        Js = J[tuple(sl)]
        Xs = Xs.reshape(Xs.shape[:-2] + (E0, nq, d))
        Js = Js.reshape(Js.shape[:-3] + (E0, nq, d, d))
        # move E0 to the front, then the point axes (q_{d-1}, ..., q_1, q_0)
        Xs = np.moveaxis(Xs, d - 1, 0).reshape(E0, nq ** d, d)
        Js = np.moveaxis(Js, d - 1, 0).reshape(E0, nq ** d, d, d)
        wt = dd[0]["w"]  # (E0, nq)
        for a in range(1, d):
            wa = dd[a]["w"][outer[a - 1]]  # (nq,)
            wt = (wt[:, None, :] * wa[None, :, None]).reshape(E0, -1)
        yield outer, dd, Js, Xs, wt


def _local_rows(dd, outer, p, shape):
    """Local flat indices (E0, L) of the basis functions active on each element."""
    d = len(shape)
    E0 = dd[0]["ne"]
    l = np.arange(p + 1)
    # multi-index per direction
    idx = [(dd[0]["spans"][:, None] - p + l[None, :])]  # (E0, p+1)
    for a in range(1, d):
        idx.append(dd[a]["spans"][outer[a - 1]] - p + l)  # (p+1,)
    flat = idx[0]  # (E0, l0)
    stride = shape[0]
    for a in range(1, d):
        flat = (flat[:, None, :] + stride * idx[a][None, :, None]).reshape(E0, -1)
        stride *= shape[a]
    return flat


def patch_stiffness(problem, k, knots_k):
    """Stiffness matrix of patch k on its local DoFs (before Dirichlet elimination).

    K_ij = (grad B_i, grad B_j)_{L2(Omega_k)} = sum_q w_q |det J| (J^{-T} grad^ B_i).(J^{-T} grad^ B_j)
    with p+1 Gauss points per element and direction (Sec. 2, Eq. model with
    the gradient form of Eq. model:discr).  Returned as scipy CSR.
    """
    d = problem["dim"]
    p = degree_of(problem, k)
    shape = shape_of(knots_k, p)
    n = int(np.prod(shape))
    acc = _Accumulator(n)
    for outer, dd, Js, Xs, wt in _patch_elements(problem, k, knots_k):
        detJ = np.linalg.det(Js)
        Jinv = np.linalg.inv(Js)
        C = np.einsum("eqab,eqcb->eqac", Jinv, Jinv) * (np.abs(detJ) * wt)[:, :, None, None]
        grads = []
        for a in range(d):
            mats = []
            for b in range(d):
                src = dd[b]["ders"] if a == b else dd[b]["vals"]
                mats.append(src if b == 0 else src[outer[b - 1]])
            grads.append(_outer(mats))  # (E0, Q, L)
        G = np.stack(grads, axis=-1)  # (E0, Q, L, d)
        H = np.einsum("eqab,eqlb->eqla", C, G)  # C symmetric
        E0, Q, L, _ = G.shape
        Gm = G.transpose(0, 2, 1, 3).reshape(E0, L, Q * d)
        Hm = H.transpose(0, 1, 3, 2).reshape(E0, Q * d, L)
        Ke = np.matmul(Gm, Hm)  # (E0, L, L)
        flat = _local_rows(dd, outer, p, shape)
        acc.add(np.repeat(flat, L, axis=1).ravel(), np.tile(flat, (1, L)).ravel(),
                Ke.ravel())
    return acc.result()


def patch_mass(problem, k, knots_k):
    """Mass matrix M_ij = (B_i, B_j)_{L2(Omega_k)} of patch k (scipy CSR)."""
    d = problem["dim"]
    p = degree_of(problem, k)
    shape = shape_of(knots_k, p)
    n = int(np.prod(shape))
    acc = _Accumulator(n)
    for outer, dd, Js, Xs, wt in _patch_elements(problem, k, knots_k):
        c = np.abs(np.linalg.det(Js)) * wt
        mats = [dd[0]["vals"]] + [dd[b]["vals"][outer[b - 1]] for b in range(1, d)]
        V = _outer(mats)  # (E0, Q, L)
        Me = np.einsum("eql,eq,eqm->elm", V, c, V)
        flat = _local_rows(dd, outer, p, shape)
        L = V.shape[2]
        acc.add(np.repeat(flat, L, axis=1).ravel(), np.tile(flat, (1, L)).ravel(),
                Me.ravel())
    return acc.result()


def patch_load(problem, k, knots_k, f):
    """Load vector f_i = (f, B_i)_{L2(Omega_k)} on the local DoFs of patch k.

    f: vectorised callable of physical points (npts, d) -> (npts,).
    """
    d = problem["dim"]
    p = degree_of(problem, k)
    shape = shape_of(knots_k, p)
    n = int(np.prod(shape))
    out = np.zeros(n)
    for outer, dd, Js, Xs, wt in _patch_elements(problem, k, knots_k):
        E0, Q, _ = Xs.shape
        fv = f(Xs.reshape(-1, d)).reshape(E0, Q)
        c = np.abs(np.linalg.det(Js)) * wt * fv
        mats = [dd[0]["vals"]] + [dd[b]["vals"][outer[b - 1]] for b in range(1, d)]
        V = _outer(mats)
        Fe = np.einsum("eql,eq->el", V, c)
        flat = _local_rows(dd, outer, p, shape)
        np.add.at(out, flat.ravel(), Fe.ravel())
    return out


class _Accumulator:
    """Sums (row, col, value) triples into a CSR matrix in bounded memory."""

    def __init__(self, n):
        self.n = n
        self.total = sp.csr_matrix((n, n))
        self.parts = []
        self.count = 0

    def add(self, rows, cols, vals):
        self.parts.append((rows, cols, vals))
        self.count += len(vals)
        if self.count > 4_000_000:
            self.flush()

    def flush(self):
        if self.parts:
            r = np.concatenate([x[0] for x in self.parts])
            c = np.concatenate([x[1] for x in self.parts])
            v = np.concatenate([x[2] for x in self.parts])
            self.total = self.total + _sum_coo(r, c, v, self.n)
            self.parts, self.count = [], 0

    def result(self):
        self.flush()
        out = self.total.tocsr()
        out.sum_duplicates()
        return out


def _sum_coo(rows, cols, vals, n):
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def param_matrices_1d(t, p):
    """1D stiffness and mass on the parameter domain (0,1) (dense, N x N).

    K^_ij = (B_i', B_j')_{L2(0,1)}, M^_ij = (B_i, B_j)_{L2(0,1)}: the pencil
    of the subspace-corrected mass smoother on patch interiors (Sec. 5; the
    same pencil as the eigenfunctions of the Appendix, Lemma 5 proof).
    """
    x, w, elem = bspline.element_quadrature(t, p + 1)
    B = bspline.basis(t, p, x)
    D = bspline.basis_deriv(t, p, x)
    K = (D * w[:, None]).T @ D
    M = (B * w[:, None]).T @ B
    return K, M


# ----------------------------------------------------------------------------
# SIPG interface terms (Sec. 3, Eq. model:discr2)
# ----------------------------------------------------------------------------

def grid_size(knots_k):
    """h of a patch: the largest knot span over all directions."""
    return max(np.max(np.diff(bspline.breakpoints(t))) for t in knots_k)


def sipg_eta(problem, fine_knots, pa, pb):
    """Penalty eta = C / h_I on interface (pa, pb) with h_I = min(h_a, h_b).

    h is the finest-level parameter-domain grid size of each side; the
    penalty stays frozen on coarser levels (Sec. 3, Eq. a:galerkin: the
    chosen parameter is sigma p^2 / h_L on every level).
    """
    h = min(grid_size(fine_knots[pa]), grid_size(fine_knots[pb]))
    return problem["sipg_penalty"] / h


def _merge_points(a, b, tol=1e-12):
    z = np.sort(np.concatenate((a, b)))
    keep = np.concatenate(([True], np.diff(z) > tol))
    return z[keep]


def _side_eval(problem, k, knots_k, side, s_pts):
    """Basis values and physical gradients at side points of patch k.

    s_pts: (npts, m) tangential coordinates.  Only the two layers of DoFs next
    to the side have nonzero value or normal derivative there (open knot
    vectors).  Returns flats (nloc,), V (npts, nloc), G (npts, nloc, d), the
    outward unit normal n (npts, d) and dS (npts,) with dS = |det J| |J^{-T} e_a|
    per unit tangential parameter measure (Nanson's formula).
    """
    d = problem["dim"]
    p = degree_of(problem, k)
    shape = shape_of(knots_k, p)
    a = side // 2
    tdirs = tangential_dirs(d, side)
    npts = s_pts.shape[0]
    xi = np.zeros((npts, d))
    xi[:, a] = 0.0 if side % 2 == 0 else 1.0
    for m, t in enumerate(tdirs):
        xi[:, t] = s_pts[:, m]
    X, J = geometry.eval_points(problem["geo_degree"], problem["geo_knots"][k],
                                problem["geo_ctrl"][k], xi)
    vals = [bspline.basis(knots_k[b], p, xi[:, b]) for b in range(d)]
    ders = [bspline.basis_deriv(knots_k[b], p, xi[:, b]) for b in range(d)]
    f0, _ = side_dofs(shape, side, 0)
    f1, _ = side_dofs(shape, side, 1)
    flats = np.concatenate((f0, f1))
    multi = unflatten(flats, shape)
    V = np.ones((npts, len(flats)))
    Gh = np.ones((npts, len(flats), d))
    for b in range(d):
        vb = vals[b][:, multi[b]]
        db = ders[b][:, multi[b]]
        V *= vb
        for c in range(d):
            Gh[:, :, c] *= db if c == b else vb
    Jinv = np.linalg.inv(J)
    G = np.einsum("qba,qlb->qla", Jinv, Gh)  # J^{-T} grad^
    sign = -1.0 if side % 2 == 0 else 1.0
    co = Jinv[:, a, :]  # row a of J^{-1} = J^{-T} e_a
    nrm = np.linalg.norm(co, axis=1)
    n = sign * co / nrm[:, None]
    dS = np.abs(np.linalg.det(J)) * nrm
    return flats, V, G, n, dS


def interface_matrix(problem, knots, fine_knots, iface):
    """SIPG terms of one interface on the two layers of DoFs of each side.

    For (u, v) in V^n the interface contributes
      -(u, v)_B - (v, u)_B + eta (u, v)_J,
      (u, v)_B = ([[u]], {grad v}.n)_I,  (u, v)_J = ([[u]], [[v]])_I,
    [[u]] = u_a - u_b, {w} = (w_a + w_b)/2, n the outward normal of patch a
    (Sec. 3, Eq. model:discr2).  Quadrature: p+1 Gauss points on every cell of
    the union of both sides' breakpoints, in the parameter of side a, p the
    larger of the two patches' degrees.
    Returns (flats_a, flats_b, M) with M over [flats_a, flats_b].
    """
    pa, sa, pb, sb, orient = iface
    d = problem["dim"]
    p = max(degree_of(problem, pa), degree_of(problem, pb))  # points per cell: exact for both sides
    eta = sipg_eta(problem, fine_knots, pa, pb)
    tdir_a = tangential_dirs(d, sa)
    tdir_b = tangential_dirs(d, sb)
    m = d - 1
    # breakpoints in side-a parameter for each tangential coordinate
    zb_dirs = [bspline.breakpoints(knots[pb][t]) for t in tdir_b]
    if m == 2 and (orient & 4):
        zb_dirs = zb_dirs[::-1]
    pts_1d, wts_1d = [], []
    xg, wg = bspline.gauss_legendre(p + 1)
    for c in range(m):
        za = bspline.breakpoints(knots[pa][tdir_a[c]])
        zb = zb_dirs[c]
        # bit of the matching coordinate of side b (swapped in 3D if bit 2)
        bit = (1 << (1 - c)) if (m == 2 and (orient & 4)) else (1 << c)
        if orient & bit:
            zb = 1.0 - zb[::-1]
        z = _merge_points(za, zb)
        xs = (z[:-1, None] + np.diff(z)[:, None] * xg[None, :]).ravel()
        ws = (np.diff(z)[:, None] * wg[None, :]).ravel()
        pts_1d.append(xs)
        wts_1d.append(ws)
    if m == 1:
        s_a = pts_1d[0][:, None]
        w = wts_1d[0]
    else:
        g1, g0 = np.meshgrid(pts_1d[1], pts_1d[0], indexing="ij")
        w1, w0 = np.meshgrid(wts_1d[1], wts_1d[0], indexing="ij")
        s_a = np.stack((g0.ravel(), g1.ravel()), axis=1)
        w = (w0 * w1).ravel()
    s_b = map_param(s_a, orient)
    fa, Va, Ga, na, dS = _side_eval(problem, pa, knots[pa], sa, s_a)
    fb, Vb, Gb, _nb, _ = _side_eval(problem, pb, knots[pb], sb, s_b)
    wq = w * dS
    jump = np.concatenate((Va, -Vb), axis=1)
    dn = 0.5 * np.concatenate((np.einsum("qla,qa->ql", Ga, na),
                               np.einsum("qla,qa->ql", Gb, na)), axis=1)
    JD = (jump * wq[:, None]).T @ dn
    JJ = (jump * wq[:, None]).T @ jump
    M = -JD.T - JD + eta * JJ
    return fa, fb, M


# ----------------------------------------------------------------------------
# Global system
# ----------------------------------------------------------------------------

def assemble_global(problem, knots, num, fine_knots=None):
    """Global matrix A (Eq. linear:system:0 or linear:system) for one level.

    Conforming: sum of patch stiffness matrices through the shared numbering.
    SIPG: patch stiffness plus the interface terms of every interface.
    fine_knots: knots of the finest level (frozen penalty); default `knots`.
    """
    if fine_knots is None:
        fine_knots = knots
    rows, cols, vals = [], [], []
    for k in range(len(knots)):
        Kk = patch_stiffness(problem, k, knots[k]).tocoo()
        l2g = num["loc2glob"][k]
        r, c = l2g[Kk.row], l2g[Kk.col]
        keep = (r >= 0) & (c >= 0)
        rows.append(r[keep]); cols.append(c[keep]); vals.append(Kk.data[keep])
    if problem["coupling"] == "sipg":
        for iface in problem["interfaces"]:
            pa, _sa, pb, _sb, _o = iface
            fa, fb, M = interface_matrix(problem, knots, fine_knots, iface)
            g = np.concatenate((num["loc2glob"][pa][fa], num["loc2glob"][pb][fb]))
            rr, cc = np.meshgrid(g, g, indexing="ij")
            keep = (rr >= 0) & (cc >= 0)
            rows.append(rr[keep]); cols.append(cc[keep]); vals.append(M[keep])
    n = num["ndof"]
    A = _sum_coo(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)
    A.eliminate_zeros()  # interface blocks hold exact zeros where supports do not meet
    return A


def assemble_load(problem, knots, num, f):
    """Global load vector (f, phi_i) on the finest level."""
    out = np.zeros(num["ndof"])
    for k in range(len(knots)):
        fk = patch_load(problem, k, knots[k], f)
        l2g = num["loc2glob"][k]
        keep = l2g >= 0
        np.add.at(out, l2g[keep], fk[keep])
    return out


def local_to_global_vector(num, local_vecs):
    """Global coefficient vector from per-patch local coefficients (owner copies)."""
    out = np.zeros(num["ndof"])
    for g, (k, f) in enumerate(num["owner"]):
        out[g] = local_vecs[k][f]
    return out


def global_to_local_vectors(num, u):
    """Per-patch local coefficients (0 at Dirichlet DoFs) of a global vector."""
    out = []
    for k, l2g in enumerate(num["loc2glob"]):
        v = np.zeros(len(l2g))
        keep = l2g >= 0
        v[keep] = u[l2g[keep]]
        out.append(v)
    return out


def evaluate(problem, knots, local_coeffs, k, xi):
    """Value of the discrete function on patch k at parameter points xi (npts, d)."""
    d = problem["dim"]
    p = degree_of(problem, k)
    shape = shape_of(knots[k], p)
    vals = [bspline.basis(knots[k][a], p, xi[:, a]) for a in range(d)]
    c = np.asarray(local_coeffs).reshape(tuple(reversed(shape)))
    out = np.zeros(len(xi))
    for q in range(len(xi)):
        w = np.ones(())
        for a in reversed(range(d)):
            w = np.multiply.outer(w, vals[a][q])
        out[q] = np.sum(w * c)
    return out
