"""Multigrid cycle, PCG and the error propagation operator -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Algorithm 1 (Sec. 4): nu pre-smoothing steps u += L^{-1}(f - A u), coarse
correction (direct solve on level 0, mu recursive calls otherwise), nu
post-smoothing steps with L^{-T}.  Algorithm 2 (Sec. 6): the hybrid smoother,
a forward Gauss-Seidel sweep before the nu SCMS pre-smoothing steps and a
backward sweep after the nu SCMS post-smoothing steps.  The SCMS operator is
symmetric, so L^{-T} = L^{-1} for it.

The method is used directly (u <- MG(L, f, u)) or as preconditioner of CG
with one cycle and zero initial guess per application (Sec. 4, "PCG").
Stopping rule: ||A u - f||_2 / ||f||_2 <= 1e-8 (Sec. 4).
"""
import numpy as np
import scipy.linalg as sla

from . import hierarchy, pieces as pieces_mod, smoothers


class Multigrid:
    """Hierarchy plus smoothers for one problem.

    smoother: 'scms' | 'gs' | 'hybrid'; tau, delta: SCMS damping and scaling;
    nu: smoothing steps; mu: 1 (V-cycle) or 2 (W-cycle).
    """

    def __init__(self, problem, levels=None, smoother="scms", tau=1.0, delta=0.12,
                 nu=1, mu=1):
        self.problem = problem
        self.h = hierarchy.build(problem, levels)
        self.smoother = smoother
        self.nu, self.mu = nu, mu
        L = self.h["levels"]
        self.scms = [None] * L
        self.gs = [None] * L
        self.pieces = [None] * L
        for l in range(1, L):
            if smoother in ("scms", "hybrid"):
                pcs = pieces_mod.decompose(problem, self.h["num"][l])
                self.pieces[l] = pcs
                self.scms[l] = smoothers.SCMS(problem, self.h["knots"][l], self.h["num"][l],
                                              self.h["A"][l], pcs, tau, delta)
            if smoother in ("gs", "hybrid"):
                col = smoothers.colouring(problem, self.h["knots"][l], self.h["num"][l])
                self.gs[l] = smoothers.GaussSeidel(self.h["A"][l], smoothers.gs_order(col))
        A0 = self.h["A"][0].toarray()
        self.coarse = sla.cho_factor(A0, lower=True) if A0.shape[0] > 0 else None

    @property
    def A(self):
        return self.h["A"][-1]

    @property
    def ndof(self):
        return self.h["num"][-1]["ndof"]

    def coarse_solve(self, f):
        """A_0^{-1} f by the Cholesky factorisation of A_0."""
        if self.coarse is None:
            return np.zeros_like(f)
        return sla.cho_solve(self.coarse, f)

    def _pre(self, l, f, u):
        A = self.h["A"][l]
        if self.smoother == "gs":
            for _ in range(self.nu):
                u = self.gs[l].forward(f, u)
            return u
        if self.smoother == "hybrid":
            u = self.gs[l].forward(f, u)
        for _ in range(self.nu):
            u = u + self.scms[l].apply(f - A @ u)
        return u

    def _post(self, l, f, u):
        A = self.h["A"][l]
        if self.smoother == "gs":
            for _ in range(self.nu):
                u = self.gs[l].backward(f, u)
            return u
        for _ in range(self.nu):
            u = u + self.scms[l].apply(f - A @ u)
        if self.smoother == "hybrid":
            u = self.gs[l].backward(f, u)
        return u

    def cycle(self, l, f, u):
        """MULTIGRID(l, f, u) of Algorithm 1 / Algorithm 2."""
        if l == 0:
            return self.coarse_solve(f)
        A, P = self.h["A"][l], self.h["P"][l]
        u = self._pre(l, f, u)
        if l == 1:
            u = u + P @ self.coarse_solve(P.T @ (f - A @ u))
        else:
            for _ in range(self.mu):
                u = u + P @ self.cycle(l - 1, P.T @ (f - A @ u), np.zeros(P.shape[1]))
        u = self._post(l, f, u)
        return u

    def precondition(self, r):
        """B r: one cycle on the finest level with zero initial guess."""
        return self.cycle(self.h["levels"] - 1, r, np.zeros_like(r))

    # ------------------------------------------------------------------
    def solve_direct(self, f, u0=None, tol=1e-8, max_iter=1000):
        """u <- MG(L, f, u) until ||f - A u|| / ||f|| <= tol.

        Returns (u, iterations, relative residual history).
        """
        A = self.A
        u = np.zeros_like(f) if u0 is None else u0.copy()
        nf = np.linalg.norm(f)
        hist = [np.linalg.norm(f - A @ u) / nf]
        it = 0
        while hist[-1] > tol and it < max_iter:
            u = self.cycle(self.h["levels"] - 1, f, u)
            it += 1
            hist.append(np.linalg.norm(f - A @ u) / nf)
        return u, it, hist

    def solve_pcg(self, f, u0=None, tol=1e-8, max_iter=1000):
        """Preconditioned CG with B = one cycle (Sec. 4).

        Standard PCG: q = A p, alpha = (r, z)/(p, q), u += alpha p,
        r -= alpha q; stop when the recursive residual satisfies the rule and
        the true residual confirms it; z = B r, beta = (r, z)_new/(r, z)_old,
        p = z + beta p.  Returns (u, iterations, relative residual history).
        max_iter bounds the number of updates of u; the iterate after exactly
        k updates is returned when max_iter = k.
        """
        A = self.A
        u = np.zeros_like(f) if u0 is None else u0.copy()
        nf = np.linalg.norm(f)
        r = f - A @ u
        hist = [np.linalg.norm(r) / nf]
        if hist[-1] <= tol:
            return u, 0, hist
        z = self.precondition(r)
        p = z.copy()
        rz = r @ z
        it = 0
        while it < max_iter:
            q = A @ p
            alpha = rz / (p @ q)
            u = u + alpha * p
            r = r - alpha * q
            it += 1
            rel = np.linalg.norm(r) / nf
            hist.append(rel)
            if rel <= tol:
                true_rel = np.linalg.norm(f - A @ u) / nf
                if true_rel <= tol:
                    hist[-1] = true_rel
                    break
            z = self.precondition(r)
            rz_new = r @ z
            beta = rz_new / rz
            rz = rz_new
            p = z + beta * p
        return u, it, hist

    # ------------------------------------------------------------------
    def error_propagation(self):
        """Dense E = I - B A of one cycle with zero initial guess (tiny grids)."""
        n = self.ndof
        A = self.A.toarray()
        E = np.zeros((n, n))
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            E[:, j] = e - self.precondition(A[:, j])
        return E

    def preconditioner_matrix(self):
        n = self.ndof
        B = np.zeros((n, n))
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            B[:, j] = self.precondition(e)
        return B
