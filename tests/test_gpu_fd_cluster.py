"""The fast diagonalisation of 2D patch interiors by one thread-block cluster per patch (FP32 path).

With MGIGA_FD_CLUSTER=1 the interior part of the subspace-corrected mass smoother (Sec. 5, Eq. Ldef)
on every 2D level of the FP32 arithmetic where it fits runs as fd_cluster_2d: the CTAs of a cluster
own column slices of the intermediates and exchange one of them through distributed shared memory.
Each smoother application is compared with the oracle's (sparse LU of L_T, dense Cholesky of the
interface pieces) at the FP32 bound of test_gpu_mixed (1e-5 relative to the correction), on

* the small mixed-precision layouts (interiors of 2..14 rows: clusters of 16, slices of 4 columns);
* the benchmark layout at 64/96 intervals, p = 3 (interiors up to 97 x 97), with clusters of 8 and
  16 (slices of 16 and 8 columns) and the automatic choice;
* two patches of 148 x 148 interior unknowns with clusters of 8 (slices of 20 columns: the widest
  shape, two groups over the contraction index to fit shared memory);

and without it (the default: one CTA per small patch, batched steps above).
The two paths sum in different orders, so their results differ in the last bits wherever the
cluster kernel ran -- checked, so that a silent fallback cannot pass for it.
"""
import numpy as np
import pytest

from oracle import mg as omg
from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

pytestmark = pytest.mark.gpu


def _nm(c, a):
    return 4 if sum(c) % 2 == 0 else 8


CASES = {
    # name: (problem factory, levels (0: automatic), options, levels to check (from the finest))
    "conf2d_p2": (lambda: W.grid_problem((2, 2), 8, 2, "conforming", jitter=0.1, seed=1, flip_patches=(3,)),
                  3, dict(tau=1.0, delta=0.12), 2),
    "sipg2d_p3": (lambda: W.grid_problem((3, 3), _nm, 3, "sipg", jitter=0.1, seed=2, flip_patches=(1,),
                                         transpose_patches=(4,)), 3, dict(tau=0.25, delta=0.1), 2),
    "bench_p3": (lambda: W.sipg_3x3(3, scale=1, smoother="hybrid")[0], 4, dict(tau=0.25, delta=0.1), 3),
    "wide_p2": (lambda: W.grid_problem((2, 1), 148, 2, "sipg", jitter=0.05, seed=7, flip_patches=(1,)),
                3, dict(tau=0.25, delta=0.1), 1),
}

_orc = {}


def _oracle(name):
    if name not in _orc:
        fac, levels, opt, _ = CASES[name]
        prob = fac()
        _orc[name] = (prob, omg.Multigrid(prob, levels=levels, smoother="hybrid", **opt))
    return _orc[name]


def _smooth_all(name, precision, monkeypatch, env):
    fac, levels, opt, ncheck = CASES[name]
    prob, orc = _oracle(name)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    lib = binding().Solver(prob, levels=levels, smoother="hybrid", precision=precision, **opt)
    for k in env:
        monkeypatch.delenv(k)
    rng = np.random.default_rng(21)
    out = {}
    for l in range(levels - 1, levels - 1 - ncheck, -1):
        A = orc.h["A"][l]
        n = A.shape[0]
        u, f = rng.standard_normal(n), rng.standard_normal(n)
        ref = u + orc.scms[l].apply(f - A @ u)
        got = lib.apply("smooth", l, f, u)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref - u), (l, env)
        out[l] = got
    lib.close()
    return out


ON = {"MGIGA_FD_CLUSTER": "1"}
SHAPES = {
    "conf2d_p2": [ON],
    "sipg2d_p3": [ON],
    "bench_p3": [ON, dict(ON, MGIGA_FD_CLUSTER_CS="8"), dict(ON, MGIGA_FD_CLUSTER_CS="16")],
    "wide_p2": [dict(ON, MGIGA_FD_CLUSTER_CS="8")],
}


@pytest.mark.parametrize("precision", ["fp32", "tf32"])
@pytest.mark.parametrize("name,env", [(n, e) for n in CASES for e in SHAPES[n]])
def test_cluster_fast_diagonalisation_against_oracle(name, env, precision, monkeypatch):
    got = _smooth_all(name, precision, monkeypatch, env)
    off = _smooth_all(name, precision, monkeypatch, {})
    # the cluster kernel ran where it applies: another summation order than the path without it
    # (the coarsest smoothed level of the small layouts has interiors of 2 rows, where the two
    # orders may coincide; the finest checked level always has more)
    top = max(got)
    assert not np.array_equal(got[top], off[top]), (name, env)
