"""The oracle against its own stored results (tests/golden/oracle_regression.json,
written by tests/golden/make_oracle_regression.py, which calls only oracle/):
a change of the oracle's arithmetic shows up here and has to be justified by
the passage of the paper it follows, and the fixture regenerated."""
import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_oracle_regression",
                                               os.path.join(HERE, "golden", "make_oracle_regression.py"))
gen = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(gen)
with open(os.path.join(HERE, "golden", "oracle_regression.json")) as fh:
    GOLDEN = json.load(fh)


@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_oracle_matches_its_stored_solves(name):
    ref, got = GOLDEN[name], gen.solve_case(name)
    assert got["ndof"] == ref["ndof"] and got["iterations"] == ref["iterations"]
    assert got["final_relres"] == pytest.approx(ref["final_relres"], rel=1e-5)
    assert got["u_norm"] == pytest.approx(ref["u_norm"], rel=1e-10)
    assert np.allclose(got["u_head"], ref["u_head"], rtol=1e-9, atol=1e-12)
