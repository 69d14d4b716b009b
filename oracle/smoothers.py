"""Smoothers: subspace-corrected mass smoother and Gauss-Seidel -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

SCMS (Sec. 5, Eq. Ldef):  L^{-1} = tau sum_T P_T L_T^{-1} P_T^T.
  Interface pieces: L_T = P_T^T A P_T, applied by a dense Cholesky solve.
  Patch interiors: the paper takes the subspace-corrected mass smoother of
  Hofreither and Takacs (2017) with scaling 1/(delta h^2) without restating
  it.  Reading used here: L_T is the parameter-domain operator
      sum_a  M^_{d-1} x .. x K^_a x .. x M^_0  +  sigma M^_{d-1} x .. x M^_0,
      sigma = 1 / (delta h_l^2),
  restricted to the interior indices 1..N-2 of every direction, h_l the
  largest knot span of the patch on level l.  The oracle assembles this
  Kronecker matrix and solves with it by a sparse LU (the definition); the
  library applies it by fast diagonalisation.

Gauss-Seidel (Sec. 4): forward sweep u += L^{-1}(f - A u) with L the lower
triangle of A, backward sweep with L^T.  The DoFs are taken in a fixed
multicolour order (reading: see colouring()); the oracle writes the sweep as
the triangular solve on the permuted matrix.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import discretize


# ----------------------------------------------------------------------------
# subspace-corrected mass smoother
# ----------------------------------------------------------------------------

def interior_operator(knots_k, p, delta):
    """L_T of a patch interior as a sparse matrix (interior flat order)."""
    mats = []
    for t in knots_k:
        K, M = discretize.param_matrices_1d(t, p)
        mats.append((sp.csr_matrix(K[1:-1, 1:-1]), sp.csr_matrix(M[1:-1, 1:-1])))
    h = discretize.grid_size(knots_k)
    sigma = 1.0 / (delta * h * h)
    d = len(knots_k)

    def kron_all(choose):
        # flat index has direction 0 fastest: kron(m_{d-1}, ..., m_0)
        out = choose[d - 1]
        for a in range(d - 2, -1, -1):
            out = sp.kron(out, choose[a], format="csr")
        return out

    L = sigma * kron_all([mats[a][1] for a in range(d)])
    for b in range(d):
        L = L + kron_all([mats[a][0] if a == b else mats[a][1] for a in range(d)])
    return L.tocsc(), sigma


def interior_eigen(knots_k, p, delta):
    """The interior operator L_T of a patch in its eigenbasis (Sec. 5, Eq. Ldef).

    L_T (interior_operator above) is a Kronecker sum of the 1D parameter-domain
    pencils (K^_a, M^_a) restricted to the interior indices, plus sigma times
    the Kronecker product of the M^_a.  With the generalised eigenpairs
    K^_a U_a = M^_a U_a diag(lam_a), U_a^T M^_a U_a = I (LAPACK through
    scipy.linalg.eigh, a library routine), it is
        L_T = (M^ U)_{d-1} x .. x (M^ U)_0 diag(sigma + sum_a lam_a) (..)^T,
    so L_T^{-1} = (U_{d-1} x .. x U_0) diag(1 / (sigma + sum_a lam_a)) (..)^T.
    Returns (U_a list, lam_a list, sigma).  Used where a sparse LU of the
    Kronecker matrix is too slow (large patches); pinned against that LU on
    small patches.
    """
    Us, lams = [], []
    for t in knots_k:
        K, M = discretize.param_matrices_1d(t, p)
        lam, U = sla.eigh(K[1:-1, 1:-1], M[1:-1, 1:-1])
        Us.append(U)
        lams.append(lam)
    h = discretize.grid_size(knots_k)
    return Us, lams, 1.0 / (delta * h * h)


def interior_solve_eigen(knots_k, p, delta):
    """x -> L_T^{-1} x on one patch interior (interior flat order, direction 0
    fastest) by the eigenbasis of interior_eigen: the transforms are applied
    one direction at a time to the array of shape (n_{d-1}, .., n_0)."""
    Us, lams, sigma = interior_eigen(knots_k, p, delta)
    d = len(Us)
    shape = tuple(len(lams[a]) for a in range(d - 1, -1, -1))
    den = np.full(shape, sigma)
    for a in range(d):
        ax = d - 1 - a  # array axis of direction a
        den = den + lams[a].reshape([-1 if i == ax else 1 for i in range(d)])

    def apply(x):
        X = x.reshape(shape)
        for a in range(d):  # X <- U_a^T along direction a
            X = np.moveaxis(np.tensordot(Us[a].T, X, axes=([1], [d - 1 - a])), 0, d - 1 - a)
        X = X / den
        for a in range(d):  # X <- U_a along direction a
            X = np.moveaxis(np.tensordot(Us[a], X, axes=([1], [d - 1 - a])), 0, d - 1 - a)
        return X.reshape(-1)

    return apply


def interior_dofs(num, k):
    """Global DoFs of the interior of patch k (indices 1..N-2 in every
    direction) in interior flat order (direction 0 fastest)."""
    shape = num["shapes"][k]
    multi = discretize.unflatten(np.arange(int(np.prod(shape))), shape)
    inner = np.ones(len(multi[0]), dtype=bool)
    for a, n in enumerate(shape):
        inner &= (multi[a] >= 1) & (multi[a] <= n - 2)
    return num["loc2glob"][k][inner]


class SCMS:
    """Subspace-corrected mass smoother of one level (Sec. 5, Eq. Ldef)."""

    def __init__(self, problem, knots, num, A, pieces, tau, delta):
        self.tau = tau
        self.pieces = pieces
        self.solvers = []
        for pc in pieces:
            if pc["kind"] == "interior":
                k = pc["patch"]
                L, _sigma = interior_operator(knots[k], discretize.degree_of(problem, k), delta)
                # interior DoFs of patch k in interior flat order
                shape = num["shapes"][k]
                multi = discretize.unflatten(np.arange(int(np.prod(shape))), shape)
                inner = np.ones(len(multi[0]), dtype=bool)
                for a, n in enumerate(shape):
                    inner &= (multi[a] >= 1) & (multi[a] <= n - 2)
                order = num["loc2glob"][k][inner]
                self.solvers.append(("lu", order, spla.splu(L)))
            else:
                dofs = pc["dofs"]
                LT = A[dofs][:, dofs].toarray()
                self.solvers.append(("chol", dofs, sla.cho_factor(LT, lower=True)))

    def apply(self, r):
        """tau sum_T P_T L_T^{-1} P_T^T r."""
        z = np.zeros_like(r)
        for kind, dofs, fac in self.solvers:
            if kind == "lu":
                z[dofs] = fac.solve(r[dofs])
            else:
                z[dofs] = sla.cho_solve(fac, r[dofs])
        return self.tau * z


# ----------------------------------------------------------------------------
# multicolour ordering for Gauss-Seidel
# ----------------------------------------------------------------------------

def patch_parity(problem):
    """Checkerboard parity of the patches (breadth-first 2-colouring).

    Patches are visited in id order; an unvisited patch gets parity 0 and
    its breadth-first search gives neighbours (ascending id) the opposite
    parity.  On a patch grid this is the checkerboard.
    """
    K = len(problem["knots"])
    nbrs = [set() for _ in range(K)]
    for (pa, _sa, pb, _sb, _o) in problem["interfaces"]:
        nbrs[pa].add(pb)
        nbrs[pb].add(pa)
    par = [-1] * K
    for s in range(K):
        if par[s] >= 0:
            continue
        par[s] = 0
        queue = [s]
        while queue:
            cur = queue.pop(0)
            for nb in sorted(nbrs[cur]):
                if par[nb] < 0:
                    par[nb] = 1 - par[cur]
                    queue.append(nb)
    return par


def structural_pattern(problem, knots, num):
    """Couplings of the global DoFs that decide the colouring (integer work).

    Two DoFs couple if some patch k holds copies of both whose local indices
    differ by at most p_k (that patch's degree) in every direction, or (SIPG)
    if they lie in the two
    layers next to the two sides of an interface and their tangential
    supports overlap on a set of positive measure.  Returned as a boolean CSR
    matrix (symmetric, diagonal included).
    """
    from . import bspline
    d = problem["dim"]
    rows, cols = [], []
    for k, shape in enumerate(num["shapes"]):
        p = discretize.degree_of(problem, k)
        l2g = num["loc2glob"][k]
        n = len(l2g)
        multi = discretize.unflatten(np.arange(n), shape)
        offs = np.array(np.meshgrid(*[np.arange(-p, p + 1)] * d, indexing="ij")).reshape(d, -1)
        for o in offs.T:
            nb = [multi[a] + o[a] for a in range(d)]
            ok = np.ones(n, dtype=bool)
            for a in range(d):
                ok &= (nb[a] >= 0) & (nb[a] < shape[a])
            src = np.nonzero(ok)[0]
            dst = discretize.flatten([nb[a][ok] for a in range(d)], shape)
            g1, g2 = l2g[src], l2g[dst]
            keep = (g1 >= 0) & (g2 >= 0)
            rows.append(g1[keep]); cols.append(g2[keep])
    if problem["coupling"] == "sipg":
        for (pa, sa, pb, sb, orient) in problem["interfaces"]:
            ta = discretize.tangential_dirs(d, sa)
            tb = discretize.tangential_dirs(d, sb)
            swap = (d == 3) and bool(orient & 4)
            fa = np.concatenate([discretize.side_dofs(num["shapes"][pa], sa, l)[0] for l in (0, 1)])
            fb = np.concatenate([discretize.side_dofs(num["shapes"][pb], sb, l)[0] for l in (0, 1)])
            ma = discretize.unflatten(fa, num["shapes"][pa])
            mb = discretize.unflatten(fb, num["shapes"][pb])
            ok = np.ones((len(fa), len(fb)), dtype=bool)
            p_a, p_b = discretize.degree_of(problem, pa), discretize.degree_of(problem, pb)
            for c in range(d - 1):
                cb = (1 - c) if swap else c
                tka = knots[pa][ta[c]]
                tkb = knots[pb][tb[cb]]
                lo_a, hi_a = tka[ma[ta[c]]], tka[ma[ta[c]] + p_a + 1]
                lo_b, hi_b = tkb[mb[tb[cb]]], tkb[mb[tb[cb]] + p_b + 1]
                if orient & (1 << cb):
                    lo_b, hi_b = 1.0 - hi_b, 1.0 - lo_b
                lo = np.maximum(lo_a[:, None], lo_b[None, :])
                hi = np.minimum(hi_a[:, None], hi_b[None, :])
                ok &= hi - lo > 1e-12
            ia, ib = np.nonzero(ok)
            g1 = num["loc2glob"][pa][fa[ia]]
            g2 = num["loc2glob"][pb][fb[ib]]
            keep = (g1 >= 0) & (g2 >= 0)
            rows += [g1[keep], g2[keep]]
            cols += [g2[keep], g1[keep]]
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    n = num["ndof"]
    S = sp.csr_matrix((np.ones(len(r), dtype=bool), (r, c)), shape=(n, n))
    S.sum_duplicates()
    return S


def colouring(problem, knots, num):
    """Multicolour ordering of the global DoFs for Gauss-Seidel (integer work).

    Base colour of a DoF, from the copy that numbered it (patch k, local
    multi-index i):  par(k) (p+1)^d + sum_a (i_a mod (p+1)) (p+1)^a, p the
    largest patch degree (with per-patch degrees, a patch of lower degree
    couples over fewer indices, so its base colours still never couple).
    A DoF is moved if it couples with a DoF of lower global index and the
    same base colour, if it couples with a DoF owned by another patch of the
    same parity, or if it has copies in several patches (a conforming
    interface DoF).  Moved DoFs are visited in increasing global order and
    each takes the smallest colour >= 2 (p+1)^d not used by a moved DoF of
    lower index that couples with it.  (The last two rules keep the DoFs on
    base colours inside one patch and patches of one parity uncoupled, so
    patches can be swept side by side.)  Returns the colour of every DoF.
    """
    d = problem["dim"]
    p = discretize.max_degree(problem)  # patches of lower degree reach less: still a valid colouring
    par = patch_parity(problem)
    base = np.zeros(num["ndof"], dtype=np.int64)
    for g, (k, f) in enumerate(num["owner"]):
        multi = discretize.unflatten(f, num["shapes"][k])
        c = par[k] * (p + 1) ** d
        for a in range(d):
            c += (multi[a] % (p + 1)) * (p + 1) ** a
        base[g] = c
    S = structural_pattern(problem, knots, num).tocoo()
    owner_patch = np.array([k for (k, f) in num["owner"]], dtype=np.int64)
    par_arr = np.array(par)
    clash = (S.col < S.row) & (base[S.row] == base[S.col])
    po, qo = owner_patch[S.row], owner_patch[S.col]
    cross = (po != qo) & (par_arr[po] == par_arr[qo])
    moved = np.zeros(num["ndof"], dtype=bool)
    moved[S.row[clash | cross]] = True
    copies = np.zeros(num["ndof"], dtype=np.int64)
    for l2g in num["loc2glob"]:
        np.add.at(copies, l2g[l2g >= 0], 1)
    moved |= copies > 1
    colour = base.copy()
    first_extra = 2 * (p + 1) ** d
    Scsr = S.tocsr()
    for i in np.nonzero(moved)[0]:
        nb = Scsr.indices[Scsr.indptr[i]:Scsr.indptr[i + 1]]
        used = {int(colour[j]) for j in nb if moved[j] and j < i}
        c = first_extra
        while c in used:
            c += 1
        colour[i] = c
    return colour


def gs_order(colour):
    """Visiting order of the forward sweep: by colour, then by global index."""
    return np.lexsort((np.arange(len(colour)), colour))


class GaussSeidel:
    """Forward/backward Gauss-Seidel sweeps in a fixed order (Sec. 4)."""

    def __init__(self, A, order):
        self.A = A.tocsr()
        self.order = order
        Ap = self.A[order][:, order]
        self.Lp = sp.tril(Ap, format="csr")
        self.Up = sp.triu(Ap, format="csr")

    def forward(self, f, u):
        """u + L^{-1}(f - A u), L the lower triangle of A in the sweep order."""
        r = (f - self.A @ u)[self.order]
        z = spla.spsolve_triangular(self.Lp, r, lower=True)
        out = u.copy()
        out[self.order] += z
        return out

    def backward(self, f, u):
        """u + L^{-T}(f - A u)."""
        r = (f - self.A @ u)[self.order]
        z = spla.spsolve_triangular(self.Up, r, lower=False)
        out = u.copy()
        out[self.order] += z
        return out
