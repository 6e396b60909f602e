"""The FP64 oracle against its own stored record (tests/golden/oracle_solve_rect64.json,
written by tests/golden/make_oracle_regression.py): a later change to the oracle's
arithmetic shows up here and has to be justified by the paper and re-recorded."""
import json
import os
import sys

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)

import make_oracle_regression as mk  # noqa: E402


def test_oracle_solve_matches_its_record():
    with open(os.path.join(GOLDEN, "oracle_solve_rect64.json")) as f:
        rec = json.load(f)
    got = mk.run(rec["case"])
    assert np.allclose(got["loss"], rec["loss"], rtol=1e-9, atol=0)
    assert got["l2"] == rec["l2"] and got["pvb"] == rec["pvb"]
    assert got["mask_pixels"] == rec["mask_pixels"]
    assert np.allclose([got["phi_sum"], got["phi_sq_sum"]], [rec["phi_sum"], rec["phi_sq_sum"]], rtol=1e-9)
    for name, stored in rec["variants"].items():
        got = mk.run(rec["case"], mk.VARIANTS[name])
        assert np.allclose(got["loss"], stored["loss"], rtol=1e-9, atol=0), name
        assert got["l2"] == stored["l2"] and got["pvb"] == stored["pvb"], name
        assert got["mask_pixels"] == stored["mask_pixels"], name
        assert np.allclose([got["phi_sum"], got["phi_sq_sum"]], [stored["phi_sum"], stored["phi_sq_sum"]],
                           rtol=1e-9), name
