"""CPU tests of the C-ABI library: exports, host-side integer maps against the
oracle (bit-exact), host-side load vector, argument validation.  No GPU call."""
import os
import re

import numpy as np
import pytest

from oracle import discretize, hierarchy, pieces as opieces, smoothers
from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mgiga.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mgiga_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    mg = binding()
    names = _declared()
    assert "mgiga_solve" in names and "mgiga_vcycle_d" in names
    for n in names:
        assert hasattr(mg._lib, n), n
    assert sorted(names) == sorted(mg.EXPORTED)


def _cases():
    def nm(c, a):
        return 4 if sum(c) % 2 == 0 else 8
    return [
        ("conf2d", W.grid_problem((2, 2), 8, 2, "conforming", jitter=0.1, seed=1, flip_patches=(3,)), 3),
        ("sipg2d", W.grid_problem((3, 3), nm, 3, "sipg", jitter=0.1, seed=2, flip_patches=(1,),
                                  transpose_patches=(4,)), 3),
        ("conf3d", W.grid_problem((2, 2, 2), 4, 2, "conforming", jitter=0.05, seed=3, flip_patches=(5,),
                                  transpose_patches=(6,)), 2),
        ("sipg3d", W.grid_problem((2, 1, 2), nm, 2, "sipg", jitter=0.05, seed=4, flip_patches=(1,),
                                  transpose_patches=(2,)), 2),
        ("lshape_like", W.grid_problem((2, 2), 4, 1, "conforming"), 2),
        # one degree per patch (Sec. 5, Table SCMS2): the L-shape S_{p,h} / S_{p+1,2h} / S_{p,2h}
        ("lshape_nonmatching", W.lshape(2, 5)[0], 3),
        ("mixed2d", W.with_patch_degrees(W.grid_problem((2, 2), nm, 3, "sipg", jitter=0.1, seed=31,
                                                        flip_patches=(1,)), [1, 2, 3, 2]), 3),
        ("mixed3d", W.with_patch_degrees(W.grid_problem((2, 1, 1), lambda c, a: 4 if c[0] == 0 else 6, 3, "sipg",
                                                        jitter=0.05, seed=32), [2, 3]), 2),
    ]


@pytest.mark.parametrize("name,prob,levels", _cases(), ids=[c[0] for c in _cases()])
def test_numbering_pieces_colours_bit_exact(name, prob, levels):
    mg = binding()
    s = mg.Solver(prob, levels=levels, smoother="hybrid", assemble=False)
    h = hierarchy.build(prob, levels)
    for l in range(levels):
        num = h["num"][l]
        patch, local = s.dof_map(l)
        own = np.array(num["owner"], dtype=np.int64).reshape(-1, 2)
        assert s.ndof(l) == num["ndof"]
        assert np.array_equal(patch, own[:, 0]) and np.array_equal(local, own[:, 1])
        if l == 0:
            continue
        pcs = opieces.decompose(prob, num)
        ref = np.full(num["ndof"], -1)
        for i, pc in enumerate(pcs):
            ref[pc["dofs"]] = i
        got, npcs = s.pieces(l)
        assert npcs == len(pcs) and np.array_equal(got, ref)
        col = smoothers.colouring(prob, h["knots"][l], num)
        assert np.array_equal(s.colours(l), col)
    s.close()


@pytest.mark.parametrize("coupling,d", [("conforming", 2), ("sipg", 2), ("sipg", 3)])
def test_load_vector_matches_oracle(coupling, d):
    mg = binding()
    if d == 2:
        prob = W.grid_problem((2, 2), 6, 3, coupling, jitter=0.1, seed=5)
    else:
        prob = W.grid_problem((2, 1, 1), 3, 2, coupling, jitter=0.05, seed=6)
    s = mg.Solver(prob, levels=1, assemble=False)
    got = s.load_sinprod()
    num = discretize.numbering(prob, prob["knots"])
    ref = discretize.assemble_load(prob, prob["knots"], num, W.source_sinprod)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    s.close()


def test_invalid_problems_return_status():
    mg = binding()
    prob = W.grid_problem((2, 1), 4, 2, "sipg")
    bad = dict(prob, degree=9)
    with pytest.raises(mg.MgigaError) as e:
        mg.Solver(bad, assemble=False)
    assert e.value.status == mg.EINVAL and "degree" in str(e.value)
    bad = dict(prob, sipg_penalty=0.0)
    with pytest.raises(mg.MgigaError) as e:
        mg.Solver(bad, assemble=False)
    assert e.value.status == mg.EINVAL
    bad = dict(prob, interfaces=[(0, 1, 0, 0, 0)])
    with pytest.raises(mg.MgigaError) as e:
        mg.Solver(bad, assemble=False)
    assert e.value.status == mg.EINVAL
    # odd interval counts cannot be coarsened
    odd = W.grid_problem((2, 1), 5, 2, "sipg")
    with pytest.raises(mg.MgigaError) as e:
        mg.Solver(odd, levels=2, assemble=False)
    assert e.value.status == mg.EINVAL
    with pytest.raises(mg.MgigaError) as e:
        mg.Solver(prob, levels=2, gs_cluster=3, assemble=False)
    assert e.value.status == mg.EINVAL
    mg.Solver(prob, levels=2, gs_cluster=8, assemble=False).close()
    s = mg.Solver(prob, levels=2, assemble=False)
    with pytest.raises(mg.MgigaError) as e:
        s.vcycle(np.zeros(s.ndof()))
    assert e.value.status == mg.ESTATE
    s.close()
    s = mg.Solver(prob, levels=2, smoother="hybrid", assemble=False)
    for stage in ("band", "residual", "gs", "fd"):  # no operators before the set-up
        with pytest.raises(mg.MgigaError) as e:
            s.stage_work(stage, 1)
        assert e.value.status == mg.ESTATE
    s.close()


def test_budget_refusal_before_any_host_or_device_work():
    """An HBM budget below the FP64 operators of all levels is refused by
    mgiga_assemble at once (MGIGA_ENOMEM), before the host assembly and without
    touching a GPU; the handle stays destroyable."""
    import time
    mg = binding()
    prob = W.grid_problem((2, 2), 16, 3, "sipg", jitter=0.1, seed=3)
    s = mg.Solver(prob, levels=2, precision="fp32", hbm_budget=1 << 16, assemble=False)
    t0 = time.perf_counter()
    with pytest.raises(mg.MgigaError) as e:
        s.assemble()
    assert e.value.status == mg.ENOMEM and "FP64 operators alone" in s.last_error()
    assert time.perf_counter() - t0 < 1.0
    s.close()


def test_residual_history_is_empty_before_a_solve():
    mg = binding()
    prob = W.grid_problem((2, 1), 4, 2, "sipg")
    s = mg.Solver(prob, levels=2, assemble=False)
    assert s.residual_history().size == 0
    s.close()


def test_patch_degrees_validated():
    """One degree per patch: `degree` must be their largest, and conforming coupling needs equal
    degrees on both sides of an interface (a continuous space across it)."""
    mg = binding()
    prob = W.with_patch_degrees(W.grid_problem((2, 1), 4, 3, "conforming"), [2, 3])
    with pytest.raises(mg.MgigaError) as e:
        mg.Solver(prob, levels=2, assemble=False)
    assert e.value.status == mg.EINVAL and "same degree" in str(e.value)
    prob = W.with_patch_degrees(W.grid_problem((2, 1), 4, 3, "sipg"), [2, 3])
    prob["degree"] = 4
    with pytest.raises(mg.MgigaError) as e:
        mg.Solver(prob, levels=2, assemble=False)
    assert e.value.status == mg.EINVAL and "largest" in str(e.value)
