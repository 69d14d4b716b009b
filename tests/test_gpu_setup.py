"""The level operators assembled on the GPU (element stiffness by sum
factorisation, Galerkin products one direction at a time; Sec. 2, Sec. 3
Eq. a:galerkin) against the host set-up (MGIGA_HOST_SETUP=1) and against the
oracle's assembled matrices.  In 3D the device stiffness kernel is enabled
with MGIGA_GPU_STIFFNESS_3D=1 (by default the host assembles the 3D finest
level and the GPU forms its Galerkin products).

Both set-ups compute the same sums in different orders, so the products A_l u
agree to a few rounding units of |A| |u| on every level (bound 1e-13 of
max |A u|); the oracle comparison uses the oracle's A_l (Galerkin products of
its own assembly) at the parity bar of the residual tests (1e-12).
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
    "conf2d_p2": (lambda: W.grid_problem((2, 2), 8, 2, "conforming", jitter=0.1, seed=1, flip_patches=(3,)), 3),
    "sipg2d_p3": (lambda: W.grid_problem((3, 3), _nm, 3, "sipg", jitter=0.1, seed=2, flip_patches=(1,),
                                         transpose_patches=(4,)), 3),
    "sipg2d_p1": (lambda: W.grid_problem((2, 2), _nm, 1, "sipg", jitter=0.1, seed=3), 3),
    "sipg2d_p6": (lambda: W.grid_problem((2, 2), (lambda c, a: 8 if sum(c) % 2 == 0 else 12), 6, "sipg",
                                         jitter=0.1, seed=5), 2),
    "conf3d_p2": (lambda: W.grid_problem((2, 2, 2), 4, 2, "conforming", jitter=0.05, seed=3,
                                         jitter_boundary_tangential=True, flip_patches=(5,)), 2),
    "sipg3d_p3": (lambda: W.grid_problem((2, 1, 2), _nm, 3, "sipg", jitter=0.05, seed=4, flip_patches=(1,),
                                         transpose_patches=(2,)), 2),
    "conf3d_p5": (lambda: W.grid_problem((2, 1, 1), 6, 5, "conforming", jitter=0.05, seed=6,
                                         jitter_boundary_tangential=True), 2),
}


def _pair(prob, levels, monkeypatch):
    mgb = binding()
    # 3D: the device stiffness kernel is not the default (slower than the host at 48 intervals); test it
    monkeypatch.setenv("MGIGA_GPU_STIFFNESS_3D", "1")
    gpu = mgb.Solver(prob, levels=levels, smoother="hybrid", tau=0.25, delta=0.12)
    monkeypatch.delenv("MGIGA_GPU_STIFFNESS_3D")
    monkeypatch.setenv("MGIGA_HOST_SETUP", "1")
    host = mgb.Solver(prob, levels=levels, smoother="hybrid", tau=0.25, delta=0.12)
    monkeypatch.delenv("MGIGA_HOST_SETUP")
    return gpu, host


@pytest.mark.parametrize("name", list(CASES))
def test_gpu_operators_match_host_and_oracle(name, monkeypatch):
    fac, levels = CASES[name]
    prob = fac()
    gpu, host = _pair(prob, levels, monkeypatch)
    orc = omg.Multigrid(prob, levels=levels, smoother="scms", tau=0.25, delta=0.12)
    rng = np.random.default_rng(7)
    for l in range(levels):
        A = orc.h["A"][l]
        u = rng.standard_normal(A.shape[0])
        g, h = gpu.apply("matvec", l, u), host.apply("matvec", l, u)
        ref = A @ u
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(g - h)) <= 1e-13 * scale, (l, np.max(np.abs(g - h)) / scale)
        assert np.max(np.abs(g - ref)) <= 1e-12 * scale, (l, np.max(np.abs(g - ref)) / scale)
    gpu.close()
    host.close()


@pytest.mark.parametrize("p", [2, 6])
def test_gpu_operators_benchmark_layout(p, monkeypatch):
    """The benchmark layout (192/288 intervals): every level's operator from the
    GPU set-up against the host set-up."""
    prob, opts = W.sipg_3x3(p, scale=3, smoother="hybrid")
    gpu, host = _pair(prob, 0, monkeypatch)
    rng = np.random.default_rng(8)
    for l in range(gpu.levels):
        u = rng.standard_normal(gpu.ndof(l))
        g, h = gpu.apply("matvec", l, u), host.apply("matvec", l, u)
        assert np.max(np.abs(g - h)) <= 1e-13 * np.max(np.abs(h)), l
    gpu.close()
    host.close()


@pytest.mark.parametrize("coupling", ["conforming", "sipg"])
def test_gpu_operators_cube(coupling, monkeypatch):
    """The 3D cube at its full size (48 intervals, p = 3)."""
    prob, opts = W.cube_2x2x2(3, coupling)
    gpu, host = _pair(prob, 0, monkeypatch)
    rng = np.random.default_rng(9)
    for l in range(gpu.levels):
        u = rng.standard_normal(gpu.ndof(l))
        g, h = gpu.apply("matvec", l, u), host.apply("matvec", l, u)
        assert np.max(np.abs(g - h)) <= 1e-13 * np.max(np.abs(h)), l
    gpu.close()
    host.close()
