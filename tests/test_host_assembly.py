"""The library's host set-up on the CPU against the oracle (test-only shim over
host_problem.cpp, host_assembly.cpp, host_hierarchy.cpp and host_spline.cpp,
compiled here with g++): every level's operator -- the finest by quadrature,
the coarser ones by Galerkin products -- equals the oracle's independently
assembled matrix in the global DoF order, for conforming and SIPG coupling in
2D and 3D with flipped and transposed patches and non-matching interfaces."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest
import scipy.sparse as sps

from oracle import hierarchy
from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1902_01818_gb300", "csrc")
OUT = os.path.join(HERE, "_build")


def _nm(c, a):
    return 4 if sum(c) % 2 == 0 else 8


CASES = {
    "conf2d_p2": (lambda: W.grid_problem((2, 2), 8, 2, "conforming", jitter=0.1, seed=1, flip_patches=(3,)), 3),
    "sipg2d_p3": (lambda: W.grid_problem((3, 3), _nm, 3, "sipg", jitter=0.1, seed=2, flip_patches=(1,),
                                         transpose_patches=(4,)), 3),
    "sipg2d_p1": (lambda: W.grid_problem((2, 2), _nm, 1, "sipg", jitter=0.1, seed=3), 3),
    "conf3d_p2": (lambda: W.grid_problem((2, 2, 2), 4, 2, "conforming", jitter=0.05, seed=3,
                                         jitter_boundary_tangential=True, flip_patches=(5,)), 2),
    "sipg3d_p2": (lambda: W.grid_problem((2, 1, 2), _nm, 2, "sipg", jitter=0.05, seed=4, flip_patches=(1,),
                                         transpose_patches=(2,)), 2),
    "sipg2d_p6": (lambda: W.grid_problem((2, 2), lambda c, a: 8 if sum(c) % 2 == 0 else 10, 6, "sipg",
                                         jitter=0.1, seed=8, flip_patches=(2,)), 2),
    "sipg3d_p4": (lambda: W.grid_problem((2, 2, 2), 2, 4, "sipg", jitter=0.05, seed=9, transpose_patches=(1,),
                                         jitter_boundary_tangential=True), 2),
    "conf3d_p4": (lambda: W.grid_problem((2, 2, 2), 2, 4, "conforming", jitter=0.05, seed=10, flip_patches=(3,),
                                         jitter_boundary_tangential=True), 2),
    "lshape_conf_p3": (lambda: W.grid_problem((2, 2), 4, 3, "conforming", jitter=0.1, seed=5,
                                              active=[(0, 0), (1, 0), (0, 1)]), 2),
    "lshape_sipg_p2": (lambda: W.grid_problem((2, 2), _nm, 2, "sipg", jitter=0.1, seed=6,
                                              active=[(0, 0), (1, 0), (0, 1)]), 2),
    # one degree per patch (Sec. 5, Table SCMS2): S_{p,h} / S_{p+1,2h} / S_{p,2h} on the L-shape,
    # and mixed degrees on jittered, flipped / transposed 2D and 3D grids
    "lshape_nonmatching_p3": (lambda: W.lshape(3, 4)[0], 3),
    "mixed2d_1232": (lambda: W.with_patch_degrees(W.grid_problem((2, 2), _nm, 3, "sipg", jitter=0.1, seed=31,
                                                                 flip_patches=(1,), transpose_patches=(2,)),
                                                  [1, 2, 3, 2]), 3),
    "mixed3d_23": (lambda: W.with_patch_degrees(W.grid_problem((2, 1, 2), lambda c, a: 2 if sum(c) % 2 == 0 else 4, 3,
                                                               "sipg", jitter=0.05, seed=32, flip_patches=(1,)),
                                                [2, 3, 3, 2]), 2),
}


@pytest.fixture(scope="module")
def ha():
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libhostassembly.so")
    srcs = [os.path.join(CSRC, f) for f in ("host_spline.cpp", "host_assembly.cpp", "host_hierarchy.cpp",
                                            "host_problem.cpp")]
    subprocess.run(["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", "-I", CSRC, *srcs,
                    os.path.join(HERE, "host_assembly_shim.cpp"), "-o", so], check=True)
    lib = C.CDLL(so)
    lib.ha_build.restype = C.c_void_p
    lib.ha_build.argtypes = [C.c_void_p, C.c_int]
    lib.ha_error.restype = C.c_char_p
    for name in ("ha_levels", "ha_ndof"):
        getattr(lib, name).restype = C.c_int
    lib.ha_levels.argtypes = [C.c_void_p]
    lib.ha_ndof.argtypes = [C.c_void_p, C.c_int]
    lib.ha_count.restype = C.c_longlong
    lib.ha_count.argtypes = [C.c_void_p, C.c_int]
    lib.ha_coo.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.ha_free.argtypes = [C.c_void_p]
    return lib


def _operators(ha, prob, levels):
    cp, keep = binding().marshal_problem(prob)
    h = ha.ha_build(C.byref(cp), levels)
    assert h, ha.ha_error().decode()
    out = []
    for l in range(ha.ha_levels(h)):
        n, m = ha.ha_ndof(h, l), ha.ha_count(h, l)
        r, c, v = np.zeros(m, np.int32), np.zeros(m, np.int32), np.zeros(m)
        ha.ha_coo(h, l, r.ctypes.data, c.ctypes.data, v.ctypes.data)
        out.append(sps.coo_matrix((v, (r, c)), shape=(n, n)).tocsr())
    ha.ha_free(h)
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_every_level_operator_equals_the_oracle(ha, name):
    fac, levels = CASES[name]
    prob = fac()
    lib_A = _operators(ha, prob, levels)
    orc = hierarchy.build(prob, levels)
    assert len(lib_A) == orc["levels"]
    for l, A in enumerate(lib_A):
        R = orc["A"][l].tocsr()
        assert A.shape == R.shape, l
        scale = abs(R).max()
        assert abs(A - R).max() <= 1e-12 * scale, (l, abs(A - R).max() / scale)


def test_invalid_problem_is_reported(ha):
    prob = W.grid_problem((2, 1), 4, 2, "sipg")
    cp, keep = binding().marshal_problem(dict(prob, sipg_penalty=0.0))
    assert not ha.ha_build(C.byref(cp), 2)
    assert b"penalty" in ha.ha_error()
