"""Writes oracle_solve_rect64.json: the FP64 oracle's loss, L2 and PVBand history of a
small solve (64^2 rectangle clip, K = 6, k = 9, 8 iterations, dose corners, re-initialisation
every 5). It calls only oracle/ and the seeded input generators. The stored values are a
regression record of the oracle itself (any later change to its arithmetic shows up in
tests/test_oracle_regression.py), not a pin against the paper.

    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import resist, solve  # noqa: E402

CASE = dict(n=64, K=6, k=9, seed=2, iters=8, beta=7.5, dt=0.5, lam=0.1, reinit_every=5)
# the same clip through the solve's options: WENO5 upwinding, and the CG direction (with
# the paper's CFL number and a long re-initialisation period, where its directions differ
# from the plain velocity's)
VARIANTS = {"default": {}, "weno5": {"weno": True},
            "cg": {"optimizer": "cg", "dt": 0.85, "reinit_every": 20}}


def run(case=CASE, variant=None):
    o = synth.optics(case["n"], case["K"], case["k"])
    Zt = synth.rect_clip(case["seed"], n=case["n"], nrect=(2, 3), short=(8, 14), long=(10, 30), gap=6, border=8)
    kw = dict(resist=resist.ResistParams(beta=case["beta"]), dt=case["dt"], lam=case["lam"], iters=case["iters"],
              reinit_every=case["reinit_every"])
    kw.update(variant or {})
    p = solve.SolveParams(**kw)
    out = solve.ilt_solve(Zt, o.H, o.w, p)
    return {"loss": [float(x) for x in out.loss], "l2": [int(x) for x in out.l2], "pvb": [int(x) for x in out.pvb],
            "mask_pixels": int(out.mask.sum()), "phi_sum": float(out.phi.sum()),
            "phi_sq_sum": float((out.phi ** 2).sum())}


if __name__ == "__main__":
    rec = {"note": "FP64 oracle regression record (not a paper value); written by make_oracle_regression.py",
           "case": CASE, **run(),
           "variants": {name: run(CASE, v) for name, v in VARIANTS.items() if v}}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_solve_rect64.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print(path)
