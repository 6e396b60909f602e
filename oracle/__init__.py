"""FP64 CPU oracle for the level-set ILT hot path of DevelSet (arXiv 2303.12529).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct
definition of what the CUDA library computes; it exists to check that library
against the paper. Only the test suite, the smoke check and the benchmark's
CPU-baseline / reference arm may import it. The CUDA library never calls it,
and nothing here imports the CUDA library: the two share no code. The only
common dependency is the seeded input generator package ``synth``, which holds
none of the method's arithmetic.

Everything is NumPy float64. Library primitives used as single steps: the 2-D
FFT (numpy.fft), einsum contractions, sort/search, and elementwise ufuncs.

Modules
-------
litho     Sec. II-B SOCS imaging (circular convolution, full-size FFT) and the
          gradient of Eq. (ilt_gradient) / (pvb_gradient).
resist    Sec. II-B constant-threshold resist, Sec. III-A sigmoid resist,
          L_ilt, L_pvb (Sec. III-A) and the binary L2 / PVBand metrics (Sec. II-C).
levelset  Eqs. (numerical-settings), (curva_numer) curvature term; Godunov
          upwind transport for Eq. (dso_evolution); mask extraction Eq. (phi2mask).
sdf       Eqs. (sdf), (tsdf): exact squared Euclidean distance transform and
          the truncated signed distance function.
solve     The DSO loop (Sec. III-A, III-C): T iterations of image, loss,
          velocity, level-set update, with periodic re-initialisation; the
          optional WENO5 upwinding, defocused inner corner and CG direction.
cg        Polak-Ribiere (PR+) conjugate-gradient direction for the front
          velocity (Sec. III-C names CG without a formula).
modulation  Sec. III-B modulation labels: candidate maps H(phi_gt + dh) and the
          approximated Heaviside H_eps.
dsn       Sec. III-B level-set branch of DevelSet-Net: convolutions, pooling,
          upsampling, their gradients, the MSE and AHF losses, Adam, and the
          resampling between a clip's grid and a coarser network grid.
shots     Sec. II-C.3 shot count: minimum rectangle partition by exhaustive
          search (tiny masks).

Pins: every function is checked in ``tests/test_oracle_*.py`` against closed
forms, invariants and brute force (see each test's docstring). No function of
this package is "parity unpinned".
"""
from . import litho, resist, levelset, sdf, solve  # noqa: F401  (cg, modulation, dsn, shots: import directly)
