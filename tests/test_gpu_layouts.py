"""FP64 parity of the PCG iterates on the parity layouts at their stated sizes.

* the 2D SIPG 3x3 layout at 64/96 intervals (59-66k unknowns, 6 levels),
  p = 2..6;
* the 3D cube (2x2x2 patches) at 12 intervals, p = 3..5, conforming and SIPG
  (20-33k unknowns, 3 levels).

Hybrid smoother, automatic levels, V-cycle-preconditioned CG (Sec. 4), plain
FP64.  The oracle's load vector (Gauss quadrature of f = d pi^2 prod sin) is
the right-hand side of both sides.  Bars (the plain FP64 path): the iterates
after k = 1, 3, 6 iterations within 1e-10 relative (2-norm), the iteration
counts to the 1e-8 stopping rule within +-1, the residual histories within
1e-6 relative plus 1e-10 of ||f|| entry by entry (the confirmed true
residual last).  The oracle
runs in spawned worker processes started at collection (oracle_pool.py).
"""
import numpy as np
import pytest

import oracle_pool
from lib_fixture import binding

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", list(oracle_pool.LAYOUTS))
def test_pcg_iterates_on_parity_layout(name):
    spec = oracle_pool.LAYOUTS[name]
    prob, opts = oracle_pool.problem_of(spec)
    ref = oracle_pool.result(name)
    mgb = binding()
    f = ref["f"]
    for k in oracle_pool.ITERATES:
        lk = mgb.Solver(prob, levels=0, smoother=opts["smoother"], tau=opts["tau"], delta=opts["delta"],
                        precision="fp64", max_iter=k)
        assert lk.ndof() == ref["ndof"]
        u, it, rel, st = lk.solve(f, tol=1e-300, allow_noconv=True)
        lk.close()
        uo = ref["iterates"][k]
        err = np.linalg.norm(u - uo) / np.linalg.norm(uo)
        assert it == k and err <= 1e-10, (k, err)
    lib = mgb.Solver(prob, levels=0, smoother=opts["smoother"], tau=opts["tau"], delta=opts["delta"],
                     precision="fp64")
    u, it, rel, st = lib.solve(f, tol=1e-8)
    h = lib.residual_history()
    lib.close()
    assert abs(it - ref["it"]) <= 1, (it, ref["it"])
    assert rel <= 1e-8
    hist = np.asarray(ref["hist"])
    m = min(len(h), len(hist)) - 1  # the last entries: confirmed true residual vs recursive one
    dev = np.abs(np.asarray(h[:m]) - hist[:m])
    bound = 1e-6 * np.abs(hist[:m]) + 1e-10  # as in test_gpu_parity: the drift of two FP64 recursions
    assert np.all(dev <= bound), [(i, h[i], hist[i]) for i in np.nonzero(dev > bound)[0]]
    # the solutions of the two stopped solves agree to the accuracy the stopping rule allows
    assert np.linalg.norm(u - ref["u"]) <= 1e-6 * np.linalg.norm(ref["u"])
