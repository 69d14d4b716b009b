"""The allocation-free residual entry point (mgiga_residual_noalloc_d).

Callers that may not allocate device memory while they run (a request loop
inside an HBM budget it has already reserved, code that cannot take the
device-wide synchronisation of cudaMalloc/cudaFree) use this entry point: its
scratch is a fixed device array inside the library.  This file runs last so
that a failure here leaves every other test already run; it passes alone and
after the others.
"""
import numpy as np
import pytest

from paper_1902_01818_gb300 import workloads as W
from lib_fixture import binding

pytestmark = pytest.mark.gpu


def _nm(c, a):
    return 4 if sum(c) % 2 == 0 else 8


@pytest.mark.parametrize("coupling", ["sipg", "conforming"])
def test_noalloc_residual_matches_residual_entry_point_twice(coupling):
    import torch
    mg = binding()
    n = _nm if coupling == "sipg" else 8
    prob = W.grid_problem((3, 2), n, 3, coupling, jitter=0.1, seed=12, flip_patches=(2,))
    s = mg.Solver(prob, levels=2, smoother="scms", tau=0.5, delta=0.2)
    rng = np.random.default_rng(7)
    for call in range(2):  # two calls in a row share (and reuse) the fixed scratch
        for level in (1, 0):
            nd = s.ndof(level)
            f = torch.from_numpy(rng.standard_normal(nd)).cuda()
            u = torch.from_numpy(rng.standard_normal(nd)).cuda()
            ref = torch.zeros_like(f)
            got = torch.full_like(f, float("nan"))
            s.apply_d("residual", level, f, u, ref)
            s.residual_noalloc_d(level, f, u, got)
            ref, got = ref.cpu().numpy(), got.cpu().numpy()
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), (call, level)
    s.close()


def test_noalloc_residual_rejects_levels_beyond_the_scratch():
    import torch
    mg = binding()
    # 2 x 1 patches of 770 x 770 B-splines: 1.19M local coefficients on the
    # finest level, more than the fixed scratch holds (the coarsest level is tiny)
    prob = W.grid_problem((2, 1), 768, 2, "sipg")
    s = mg.Solver(prob, levels=0, smoother="gs")
    top = s.levels - 1
    nd = s.ndof(top)
    f = torch.zeros(nd, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MgigaError) as e:
        s.residual_noalloc_d(top, f, f, torch.zeros_like(f))
    assert e.value.status == mg.EINVAL and "fixed scratch holds" in str(e.value)
    s.close()
