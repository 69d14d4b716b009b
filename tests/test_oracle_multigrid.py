"""Pins of the oracle's hierarchy, pieces, smoothers and cycle (Sec. 3-6)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import discretize, hierarchy, pieces, smoothers, mg
from paper_1902_01818_gb300 import workloads as W
from oracle_helpers import full_numbering


def _nm(cidx, a):
    return 4 if (cidx[0] + cidx[1]) % 2 == 0 else 8


@pytest.mark.parametrize("coupling", ["conforming", "sipg"])
def test_galerkin_equals_rediscretisation_affine(coupling):
    # Eq. a:galerkin: with the penalty frozen at h_L the coarse form is the fine form
    n = 8 if coupling == "conforming" else _nm
    prob = W.grid_problem((2, 2), n, 2, coupling, box=(2.0, 1.0), flip_patches=(1,))
    h = hierarchy.build(prob, levels=3)
    for l in range(2):
        Ar = hierarchy.rediscretize(prob, h, l)
        d = (Ar - h["A"][l]).toarray()
        assert np.max(np.abs(d)) <= 1e-12 * abs(Ar).max()


def test_prolongation_preserves_mass():
    prob = W.grid_problem((2, 1), 8, 3, "conforming", jitter=0.0)
    h = hierarchy.build(prob, levels=2)
    kn = h["knots"]
    Ms = []
    for l in range(2):
        num = h["num"][l]
        rows, cols, vals = [], [], []
        for k in range(2):
            Mk = discretize.patch_mass(prob, k, kn[l][k]).tocoo()
            g = num["loc2glob"][k]
            keep = (g[Mk.row] >= 0) & (g[Mk.col] >= 0)
            rows.append(g[Mk.row][keep]); cols.append(g[Mk.col][keep]); vals.append(Mk.data[keep])
        Ms.append(sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(num["ndof"], num["ndof"])))
    P = h["P"][1]
    assert np.max(np.abs((P.T @ Ms[1] @ P - Ms[0]).toarray())) <= 1e-15 * 10


def test_auto_levels_of_the_workloads():
    assert hierarchy.auto_levels(W.sipg_3x3(2)[0]) == 6
    assert hierarchy.auto_levels(W.sipg_3x3(2, scale=3)[0]) == 6  # 288 -> 9 is odd
    assert hierarchy.auto_levels(W.cube_2x2x2(3, "sipg")[0]) == 5


@pytest.mark.parametrize("coupling", ["conforming", "sipg"])
def test_pieces_partition_the_dofs_2d(coupling):
    prob = W.grid_problem((2, 2), 4, 2, coupling, flip_patches=(3,))
    num = discretize.numbering(prob, prob["knots"])
    pcs = pieces.decompose(prob, num)
    allx = np.concatenate([pc["dofs"] for pc in pcs])
    assert np.array_equal(np.sort(allx), np.arange(num["ndof"]))
    kinds = [pc["kind"] for pc in pcs]
    assert kinds.count("interior") == 4 and kinds.count("interface") == 5
    sizes = sorted(len(pc["dofs"]) for pc in pcs if pc["kind"] == "interface")
    # conforming: 4 edges of N-2 = 4 DoFs, centre vertex 1; SIPG: edges 2(N-2), vertex 4
    assert sizes == ([1, 4, 4, 4, 4] if coupling == "conforming" else [4, 8, 8, 8, 8])


@pytest.mark.parametrize("coupling", ["conforming", "sipg"])
def test_pieces_partition_the_dofs_3d(coupling):
    prob = W.grid_problem((2, 2, 2), 3, 2, coupling, flip_patches=(5,), transpose_patches=(6,))
    num = discretize.numbering(prob, prob["knots"])
    pcs = pieces.decompose(prob, num)
    allx = np.concatenate([pc["dofs"] for pc in pcs])
    assert np.array_equal(np.sort(allx), np.arange(num["ndof"]))
    kinds = [pc["kind"] for pc in pcs]
    # 8 interiors, 12 interior faces, 6 interior edges, 1 centre vertex
    assert kinds.count("interior") == 8 and kinds.count("interface") == 19
    sizes = sorted(len(pc["dofs"]) for pc in pcs if pc["kind"] == "interface")
    m = 3 + 2 - 2  # N - 2 tangential interior DoFs
    if coupling == "conforming":
        assert sizes == [1] + [m] * 6 + [m * m] * 12
    else:
        assert sizes == [8] + [4 * m] * 6 + [2 * m * m] * 12


@pytest.mark.parametrize("coupling,d", [("conforming", 2), ("sipg", 2), ("conforming", 3), ("sipg", 3)])
def test_colouring_is_valid(coupling, d):
    cells = (3, 3) if d == 2 else (2, 2, 2)
    n = (lambda c, a: 3 if sum(c) % 2 == 0 else 4) if coupling == "sipg" else 3
    prob = W.grid_problem(cells, n, 2, coupling, jitter=0.05, seed=2)
    num = discretize.numbering(prob, prob["knots"])
    col = smoothers.colouring(prob, prob["knots"], num)
    A = discretize.assemble_global(prob, prob["knots"], num).tocoo()
    off = A.row != A.col
    assert not np.any(col[A.row[off]] == col[A.col[off]])
    S = smoothers.structural_pattern(prob, prob["knots"], num).tocoo()
    off = S.row != S.col
    assert not np.any(col[S.row[off]] == col[S.col[off]])
    # the numeric pattern is contained in the structural one
    Sd = set(zip(S.row.tolist(), S.col.tolist()))
    assert all((r, c) in Sd for r, c in zip(A.row.tolist(), A.col.tolist()))


@pytest.mark.parametrize("coupling,d", [("conforming", 2), ("sipg", 2), ("conforming", 3), ("sipg", 3)])
def test_base_colours_keep_same_parity_patches_uncoupled(coupling, d):
    # DoFs on base colours (< 2 (p+1)^d) never couple with a DoF owned by
    # another patch of the same parity; on patch grids with SIPG nothing moves
    cells = (3, 3) if d == 2 else (2, 2, 2)
    n = (lambda c, a: 3 if sum(c) % 2 == 0 else 4) if coupling == "sipg" else 3
    p = 2
    prob = W.grid_problem(cells, n, p, coupling, jitter=0.05, seed=2)
    num = discretize.numbering(prob, prob["knots"])
    col = smoothers.colouring(prob, prob["knots"], num)
    par = smoothers.patch_parity(prob)
    own = np.array([k for (k, f) in num["owner"]])
    S = smoothers.structural_pattern(prob, prob["knots"], num).tocoo()
    nb = 2 * (p + 1) ** d
    both_base = (col[S.row] < nb) & (col[S.col] < nb)
    other = own[S.row] != own[S.col]
    same_par = np.array(par)[own[S.row]] == np.array(par)[own[S.col]]
    assert not np.any(both_base & other & same_par)
    if coupling == "sipg":
        assert col.max() < nb


def test_colouring_conflicts_get_extra_colours():
    # a non-bipartite patch graph (3 patches around a vertex cannot be
    # 2-coloured) is emulated by a 2x2 conforming grid: the shared centre
    # vertex DoF couples DoFs of the diagonal patches, which share a parity
    prob = W.grid_problem((2, 2), 2, 1, "conforming")
    num = discretize.numbering(prob, prob["knots"])
    col = smoothers.colouring(prob, prob["knots"], num)
    S = smoothers.structural_pattern(prob, prob["knots"], num).tocoo()
    off = S.row != S.col
    assert not np.any(col[S.row[off]] == col[S.col[off]])


def test_gauss_seidel_equals_pointwise_sweep():
    prob = W.grid_problem((2, 2), _nm, 2, "sipg", jitter=0.1, seed=1)
    num = discretize.numbering(prob, prob["knots"])
    A = discretize.assemble_global(prob, prob["knots"], num)
    col = smoothers.colouring(prob, prob["knots"], num)
    order = smoothers.gs_order(col)
    gs = smoothers.GaussSeidel(A, order)
    rng = np.random.default_rng(0)
    f, u = rng.standard_normal(num["ndof"]), rng.standard_normal(num["ndof"])
    Ad = A.toarray()
    ref = u.copy()
    for i in order:  # textbook pointwise update, current values
        ref[i] += (f[i] - Ad[i] @ ref) / Ad[i, i]
    assert np.max(np.abs(gs.forward(f, u) - ref)) <= 1e-12 * np.max(np.abs(ref))
    ref = u.copy()
    for i in order[::-1]:
        ref[i] += (f[i] - Ad[i] @ ref) / Ad[i, i]
    assert np.max(np.abs(gs.backward(f, u) - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_interior_operator_brute_force():
    # L_T entries from the definition: sum over directions of products of 1D
    # stiffness/mass entries plus sigma times the mass product
    p, n, delta = 2, 4, 0.3
    kn = [W.uniform_knots(n, p), W.uniform_knots(2 * n, p)]
    L, sigma = smoothers.interior_operator(kn, p, delta)
    assert abs(sigma - 1.0 / (delta * (1.0 / n) ** 2)) <= 1e-12
    (K0, M0), (K1, M1) = [discretize.param_matrices_1d(t, p) for t in kn]
    n0, n1 = K0.shape[0] - 2, K1.shape[0] - 2
    Ld = L.toarray()
    for r in range(n0 * n1):
        i0, i1 = r % n0 + 1, r // n0 + 1
        for c in range(n0 * n1):
            j0, j1 = c % n0 + 1, c // n0 + 1
            ref = K0[i0, j0] * M1[i1, j1] + M0[i0, j0] * K1[i1, j1] + sigma * M0[i0, j0] * M1[i1, j1]
            assert abs(Ld[r, c] - ref) <= 1e-12 * abs(Ld).max()


def test_scms_is_damped_block_jacobi_over_pieces():
    prob = W.grid_problem((2, 2), 4, 2, "sipg", jitter=0.1, seed=3)
    M = mg.Multigrid(prob, levels=2, smoother="scms", tau=0.7, delta=0.2)
    sm = M.scms[1]
    n = M.ndof
    A = M.A.toarray()
    Z = np.zeros((n, n))
    for pc in M.pieces[1]:
        dofs = pc["dofs"]
        if pc["kind"] == "interface":
            Z[np.ix_(dofs, dofs)] = np.linalg.inv(A[np.ix_(dofs, dofs)])
        else:
            k = pc["patch"]
            L, _ = smoothers.interior_operator(M.h["knots"][1][k], 2, 0.2)
            shape = M.h["num"][1]["shapes"][k]
            multi = discretize.unflatten(np.arange(int(np.prod(shape))), shape)
            inner = (multi[0] >= 1) & (multi[0] <= shape[0] - 2) & (multi[1] >= 1) & (multi[1] <= shape[1] - 2)
            order = M.h["num"][1]["loc2glob"][k][inner]
            Z[np.ix_(order, order)] = np.linalg.inv(L.toarray())
    r = np.random.default_rng(1).standard_normal(n)
    assert np.max(np.abs(sm.apply(r) - 0.7 * Z @ r)) <= 1e-12 * np.max(np.abs(Z @ r))


@pytest.mark.parametrize("smoother", ["scms", "hybrid", "gs"])
@pytest.mark.parametrize("coupling", ["conforming", "sipg"])
def test_cycle_converges_and_preconditioner_is_symmetric(smoother, coupling):
    n = 4 if coupling == "conforming" else _nm
    prob = W.grid_problem((2, 2), n, 2, coupling, jitter=0.1, seed=8)
    tau = 1.0 if coupling == "conforming" else 0.5
    M = mg.Multigrid(prob, levels=3, smoother=smoother, tau=tau, delta=0.2)
    E = M.error_propagation()
    rho = max(abs(np.linalg.eigvals(E)))
    assert rho < 1.0, rho
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(M.ndof), rng.standard_normal(M.ndof)
    bx, by = M.precondition(x), M.precondition(y)
    assert abs(y @ bx - x @ by) <= 1e-12 * np.linalg.norm(bx) * np.linalg.norm(y)


def _energy_norm(E, A):
    w, V = np.linalg.eigh(A)
    Ah = V @ np.diag(np.sqrt(w)) @ V.T
    Aih = V @ np.diag(1 / np.sqrt(w)) @ V.T
    return np.linalg.norm(Ah @ E @ Aih, 2)


def test_hybrid_no_worse_than_scms_in_energy_norm():
    # Sec. 6: ||W~||_A <= ||W||_A (Gauss-Seidel is an A-contraction)
    prob = W.grid_problem((2, 2), _nm, 2, "sipg", jitter=0.1, seed=8)
    Ms = mg.Multigrid(prob, levels=3, smoother="scms", tau=0.5, delta=0.2)
    Mh = mg.Multigrid(prob, levels=3, smoother="hybrid", tau=0.5, delta=0.2)
    A = Ms.A.toarray()
    assert _energy_norm(Mh.error_propagation(), A) <= _energy_norm(Ms.error_propagation(), A) + 1e-12


def test_pcg_reaches_the_stopping_rule_and_the_discrete_solution():
    prob = W.grid_problem((2, 2), _nm, 3, "sipg", jitter=0.1, seed=8)
    M = mg.Multigrid(prob, smoother="scms", tau=0.5, delta=0.2)
    num = M.h["num"][-1]
    f = discretize.assemble_load(prob, prob["knots"], num, W.source_sinprod)
    u, it, hist = M.solve_pcg(f)
    assert np.linalg.norm(f - M.A @ u) / np.linalg.norm(f) <= 1e-8
    ex = spla.spsolve(M.A.tocsc(), f)
    assert np.linalg.norm(u - ex) <= 1e-6 * np.linalg.norm(ex)
    u2, it2, _ = M.solve_pcg(f, max_iter=3)
    assert it2 == 3


def test_coarse_solve_inverts_a0():
    prob = W.grid_problem((2, 2), 4, 2, "conforming", jitter=0.1, seed=1)
    M = mg.Multigrid(prob, levels=2)
    A0 = M.h["A"][0].toarray()
    f = np.random.default_rng(0).standard_normal(A0.shape[0])
    assert np.max(np.abs(A0 @ M.coarse_solve(f) - f)) <= 1e-12 * np.max(np.abs(f))


@pytest.mark.parametrize("d,p", [(2, 2), (2, 4), (3, 2)])
def test_couplings_within_a_slow_residue_run_stay_on_one_slow_index(d, p):
    """A base colour fixes every index modulo p + 1, the slow one outermost, so the
    colours with one residue of the slowest index form a consecutive run.  Two
    coupled DoFs of one patch whose colours lie in the same run have the same slow
    index: during such a run a row never reads a value that another slow index
    (another slab, hence another CTA of the patch-parallel sweep) updates in it."""
    cells = (3, 3) if d == 2 else (2, 2, 2)
    n = (lambda c, a: 6 if sum(c) % 2 == 0 else 8) if d == 2 else 4
    prob = W.grid_problem(cells, n, p, "sipg", jitter=0.05, seed=7)
    num = discretize.numbering(prob, prob["knots"])
    col = smoothers.colouring(prob, prob["knots"], num)
    B = (p + 1) ** d
    run_len = B // (p + 1)
    S = smoothers.structural_pattern(prob, prob["knots"], num).tocoo()
    owner = num["owner"]
    shapes = num["shapes"]
    checked = 0
    for r, c in zip(S.row.tolist(), S.col.tolist()):
        if r == c or col[r] >= 2 * B or col[c] >= 2 * B:
            continue
        (kr, fr), (kc, fc) = owner[r], owner[c]
        if kr != kc or col[r] // B != col[c] // B:
            continue
        if (col[r] % B) // run_len != (col[c] % B) // run_len:
            continue
        slow_r = discretize.unflatten(fr, shapes[kr])[d - 1]
        slow_c = discretize.unflatten(fc, shapes[kc])[d - 1]
        assert slow_r == slow_c, (r, c)
        checked += 1
    assert checked > 0


def _smoother_error_ops(M, l):
    """Dense error propagation of the pre- and post-smoothing steps on level l,
    built from the oracle's single smoother applications (each pinned above):
    S_pre = (I - W A)^nu (I - G_f A), S_post = (I - G_b A)(I - W A)^nu for the
    hybrid smoother (Algorithm 2), without the Gauss-Seidel factors for SCMS."""
    A = M.h["A"][l].toarray()
    n = A.shape[0]
    I = np.eye(n)
    W = np.column_stack([M.scms[l].apply(I[:, j]) for j in range(n)])
    S = np.linalg.matrix_power(I - W @ A, M.nu)
    if M.smoother == "hybrid":
        z = np.zeros(n)
        Gf = np.column_stack([M.gs[l].forward(I[:, j], z) for j in range(n)])
        Gb = np.column_stack([M.gs[l].backward(I[:, j], z) for j in range(n)])
        return S @ (I - Gf @ A), (I - Gb @ A) @ S
    return S, S


@pytest.mark.parametrize("smoother,nu", [("hybrid", 1), ("hybrid", 2), ("scms", 2)])
def test_w_cycle_matches_the_textbook_recursion(smoother, nu):
    """mu = 2 (W-cycle, Sec. 4): the error propagation of the cycle satisfies the
    two-grid recursion E_l = S_post (I - P_l (I - E_{l-1}^mu) A_{l-1}^{-1} P_l^T A_l)
    S_pre with E_0 = 0 (exact coarse solve); evaluated here with dense matrices
    on three levels, so that level 1 is visited twice per cycle on level 2.
    A second visit that reuses a stale residual, or a single visit, fails it."""
    prob = W.grid_problem((2, 2), _nm, 2, "sipg", jitter=0.1, seed=8)
    M = mg.Multigrid(prob, levels=3, smoother=smoother, tau=0.5, delta=0.2, nu=nu, mu=2)
    E = None
    for l in range(1, 3):
        A = M.h["A"][l].toarray()
        P = M.h["P"][l].toarray()
        Ac = M.h["A"][l - 1].toarray()
        n = A.shape[0]
        Ec = np.zeros_like(Ac) if E is None else E
        mu = 2 if l > 1 else 1  # with an exact coarse solve a second visit changes nothing
        coarse = (np.eye(Ac.shape[0]) - np.linalg.matrix_power(Ec, mu)) @ np.linalg.inv(Ac)
        S_pre, S_post = _smoother_error_ops(M, l)
        E = S_post @ (np.eye(n) - P @ coarse @ P.T @ A) @ S_pre
    Eo = M.error_propagation()
    assert np.max(np.abs(Eo - E)) <= 1e-10 * max(1.0, np.max(np.abs(E)))
    # and with mu = 1 the recursion differs: the pin separates V- and W-cycles
    Mv = mg.Multigrid(prob, levels=3, smoother=smoother, tau=0.5, delta=0.2, nu=nu, mu=1)
    assert np.max(np.abs(Mv.error_propagation() - E)) > 1e-6


@pytest.mark.parametrize("coupling", ["conforming", "sipg"])
def test_w_cycle_converges_and_preconditioner_is_symmetric(coupling):
    n = 4 if coupling == "conforming" else _nm
    prob = W.grid_problem((2, 2), n, 2, coupling, jitter=0.1, seed=8)
    tau = 1.0 if coupling == "conforming" else 0.5
    M = mg.Multigrid(prob, levels=3, smoother="hybrid", tau=tau, delta=0.2, mu=2, nu=2)
    rho = max(abs(np.linalg.eigvals(M.error_propagation())))
    Mv = mg.Multigrid(prob, levels=3, smoother="hybrid", tau=tau, delta=0.2, mu=1, nu=2)
    rho_v = max(abs(np.linalg.eigvals(Mv.error_propagation())))
    assert rho < 1.0 and rho <= rho_v + 1e-12, (rho, rho_v)  # more coarse work contracts no worse
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(M.ndof), rng.standard_normal(M.ndof)
    bx, by = M.precondition(x), M.precondition(y)
    assert abs(y @ bx - x @ by) <= 1e-12 * np.linalg.norm(bx) * np.linalg.norm(y)


def test_two_level_w_cycle_equals_v_cycle():
    """On two levels the coarse solve is exact, so after the first coarse
    correction P^T (f - A u) = 0 (Galerkin A_0 = P^T A P) and a second one adds
    nothing: the W- and V-cycles coincide."""
    prob = W.grid_problem((2, 2), _nm, 3, "sipg", jitter=0.1, seed=5)
    Mw = mg.Multigrid(prob, levels=2, smoother="hybrid", tau=0.5, delta=0.2, mu=2)
    Mv = mg.Multigrid(prob, levels=2, smoother="hybrid", tau=0.5, delta=0.2, mu=1)
    r = np.random.default_rng(4).standard_normal(Mw.ndof)
    bw, bv = Mw.precondition(r), Mv.precondition(r)
    assert np.max(np.abs(bw - bv)) <= 1e-12 * np.max(np.abs(bv))


@pytest.mark.parametrize("d,p", [(1, 3), (2, 1), (2, 2), (2, 4), (2, 6), (3, 2), (3, 3)])
def test_interior_eigen_solve_equals_sparse_lu(d, p):
    """The eigenbasis form of L_T^{-1} (used at sizes where the sparse LU is too
    slow) against the sparse LU of the assembled Kronecker operator, on patches
    with a different interval count in every direction (a transposed direction
    or a wrong eigenvalue sum fails)."""
    nint = [5, 7, 6][:d] if d > 1 else [9]
    cells = (1,) * max(d, 2) if d > 1 else (1, 1)
    prob = W.grid_problem(cells, lambda c, a: nint[a] if a < len(nint) else 4, p, "sipg", jitter=0.0)
    kn = prob["knots"][0][:d]
    L, _ = smoothers.interior_operator(kn, p, 0.12)
    ap = smoothers.interior_solve_eigen(kn, p, 0.12)
    x = np.random.default_rng(d * 10 + p).standard_normal(L.shape[0])
    ref = spla.spsolve(L, x)
    assert np.max(np.abs(ap(x) - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("coupling", ["conforming", "sipg"])
@pytest.mark.parametrize("smoother,tau,delta", [("scms", 0.25, 0.12), ("hybrid", 0.25, 0.1)])
def test_pcg_iterations_bounded_under_refinement(coupling, smoother, tau, delta):
    """Sec. 4 and 5 (Tables GS1, SCMS1): with one more level per refinement and the coarsest grid
    fixed, the cycle-preconditioned CG needs a number of iterations bounded in the grid size.  On a
    jittered 2x2 patch grid, p = 2, 16 / 32 / 64 intervals per patch: the counts vary by at most 4
    and the last refinement adds at most one.  Checked by planting a coarse-grid correction scaled
    by 1/2 (restriction 0.5 P^T) in the oracle: the counts then grow with every refinement."""
    counts = []
    for n, levels in ((16, 4), (32, 5), (64, 6)):
        prob = W.grid_problem((2, 2), n, 2, coupling, jitter=0.1, seed=1, flip_patches=(3,))
        M = mg.Multigrid(prob, levels=levels, smoother=smoother, tau=tau, delta=delta)
        f = discretize.assemble_load(prob, prob["knots"], M.h["num"][-1], W.source_sinprod)
        counts.append(M.solve_pcg(f)[1])
    assert max(counts) - min(counts) <= 4 and counts[2] <= counts[1] + 1, counts
