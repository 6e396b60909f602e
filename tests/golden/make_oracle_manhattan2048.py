"""Writes oracle_solve_manhattan2048.npz: the FP64 oracle's DSO solve of the full-size
workload (2048^2 Manhattan clip of seed 1000, K = 24 SOCS kernels of 35 x 35, dose corners
+/-2%, alpha = 1, beta = 7.5, dt = 0.5, lambda = 0.1) for 6 iterations with
re-initialisation every 5, so that the record covers the initial TSDF, five steps, one
re-initialisation and a step after it. It calls only oracle/ and the seeded input
generators.

Stored: the optics the solve used (H as complex64, w as float32: the GPU path is given the
same arrays, so eigenvector phases and degenerate splits of the synthetic TCC cannot differ
between machines), the target (packed bits), the per-iteration L_DSO, L2 and PVBand, the
final mask (packed bits), and two scalars of the first iteration that bound how an aerial
image error moves the loss: max |I| and sum |dL/dI| of the target's own image.

    python tests/golden/make_oracle_manhattan2048.py     # about 10 minutes on one core
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import levelset, litho, resist, sdf, solve  # noqa: E402

CASE = dict(n=2048, K=24, k=35, seed=1000, iters=6, beta=7.5, dt=0.5, lam=0.1, reinit_every=5)
PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_solve_manhattan2048.npz")


def main():
    t0 = time.time()
    c = CASE
    o = synth.optics(c["n"], c["K"], c["k"])
    H32 = o.H.astype(np.complex64)
    w32 = o.w.astype(np.float32)
    H, w = H32.astype(np.complex128), w32.astype(np.float64)
    Zt = synth.manhattan_clip(c["seed"])
    rp = resist.ResistParams(beta=c["beta"])
    p = solve.SolveParams(resist=rp, dt=c["dt"], lam=c["lam"], iters=c["iters"], reinit_every=c["reinit_every"])
    out = solve.ilt_solve(Zt, H, w, p)
    # first-iteration image and dL/dI of the target's own mask (the TSDF keeps the mask)
    M0 = levelset.mask_from_phi(sdf.tsdf(Zt))
    I0 = litho.aerial(M0, H, w)
    R0 = resist.resist(I0, Zt, rp).R
    np.savez_compressed(
        PATH, case=np.array(repr(c)), H=H32, w=w32, target_bits=np.packbits(Zt.ravel()),
        loss=np.array(out.loss, dtype=np.float64), l2=np.array(out.l2, dtype=np.int64),
        pvb=np.array(out.pvb, dtype=np.int64), mask_bits=np.packbits(out.mask.astype(np.uint8).ravel()),
        I0_max=np.float64(np.abs(I0).max()), R0_abs_sum=np.float64(np.abs(R0).sum()))
    print(PATH, f"{time.time() - t0:.0f} s", out.loss, out.l2, out.pvb)


if __name__ == "__main__":
    main()
