"""Python binding of libdevelset, the GB300 level-set ILT library.

Argument marshalling only: every function forwards to the C entry point of
the same name in ``libdevelset.so`` (declared in ``include/develset.h``);
PyTorch supplies device memory and the current CUDA stream. There is no
fallback: if the library is not built, importing this package fails.

Build it with ``python paper_2303_12529_gb300/build.py`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdevelset.so")

DEVEL_OK = 0
DEVEL_EINVAL = -1
DEVEL_ECUDA = -2
DEVEL_ENOMEM = -3
DEVEL_ETIMEOUT = -4
DEVEL_ENAN = -5
DEVEL_UPWIND_GODUNOV1 = 0
DEVEL_UPWIND_WENO5 = 1
DEVEL_OPT_STEEPEST = 0
DEVEL_OPT_CG = 1
DEVEL_MOD_MAX_CANDIDATES = 64
DEVEL_PREC_FP32 = 0
DEVEL_PREC_BF16X3 = 1

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is not built; run `python paper_2303_12529_gb300/build.py` (needs nvcc)")

_lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float


class DevelError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class devel_resist_params(ctypes.Structure):
    _fields_ = [("sigma_z", _F), ("I_th", _F), ("alpha", _F), ("beta", _F),
                ("dose_in", _F), ("dose_out", _F)]


class devel_ilt_params(ctypes.Structure):
    _fields_ = [("resist", devel_resist_params), ("dt", _F), ("lambda_", _F), ("d_lo", _F),
                ("d_hi", _F), ("iters", _I), ("reinit_every", _I), ("start_iter", _I), ("use_graph", _I),
                ("upwind", _I), ("optimizer", _I)]


class devel_clip(ctypes.Structure):
    _fields_ = [("optics", _P), ("target", _P), ("phi", _P), ("phi_given", _I), ("m", _P),
                ("mask_out", _P), ("loss_hist", _P), ("l2_hist", _P), ("pvb_hist", _P),
                ("optics_defocus", _P)]


def _sig(name, argtypes, restype=_I):
    f = getattr(_lib, name)
    f.argtypes = argtypes
    f.restype = restype
    return f


_lib.devel_last_error.restype = ctypes.c_char_p
_lib.devel_last_error.argtypes = []
_sig("devel_version", [])
_sig("devel_optics_create", [_I, _I, _I, _P, _P, _I, ctypes.POINTER(_P)])
_sig("devel_optics_destroy", [_P])
_sig("devel_optics_n", [_P])
_sig("devel_optics_check", [_P, _P])
_sig("devel_litho_forward", [_P, _P, _P, _P])
_sig("devel_resist_loss", [_P, _P, _P, ctypes.POINTER(devel_resist_params), _P, _P, _P, _P])
_sig("devel_litho_adjoint", [_P, _P, _P, _P, _P, _P])
_sig("devel_levelset_step", [_I, _P, _P, _P, _P, _F, _F, _P, _P, _P])
_sig("devel_reinit_sdf", [_I, _P, _P, _P, _F, _F, _P])
_sig("devel_reinit_sdf_batch", [_I, _I, _P, _P, _P, _F, _F, _P])
_sig("devel_levelset_step_weno5", [_I, _P, _P, _P, _P, _F, _F, _P, _P, _P])
_sig("devel_cg_direction", [_P, _P, _P, _P, _I, _P, _P, _P, _P])
_sig("devel_modulation_candidates", [_I, _P, _I, _P, _P, _P])
_sig("devel_ahf_loss", [_P, _P, _P, _F, _P, _P, _P])
_sig("devel_modulation_search", [ctypes.POINTER(devel_ilt_params), _I, ctypes.POINTER(_P), _P, _P, _P, _P, _P, _P,
                                 _I, _P, _P, _P])
_sig("devel_shot_count", [_I, _P, ctypes.POINTER(ctypes.c_longlong)])
_sig("devel_dsn_create", [_I, _I, _I, ctypes.POINTER(_P)])
_sig("devel_dsn_destroy", [_P])
_sig("devel_dsn_param_count", [_P], ctypes.c_longlong)
_sig("devel_dsn_init", [_P, ctypes.c_ulonglong])
_sig("devel_dsn_set_params", [_P, _P])
_sig("devel_dsn_get_params", [_P, _P])
_sig("devel_dsn_grads", [_P, _P])
_sig("devel_dsn_forward", [_P, _I, _P, _F, _P, _P])
_sig("devel_dsn_train_step", [_P, _I, _P, _P, _F, _F, _P, _P])
_sig("devel_dsn_forward_ahf", [_P, _I, _P, _F, _F, _P, _P])
_sig("devel_dsn_train_step_ahf", [_P, _I, _P, _P, _F, _F, _F, _P, _P])
_sig("devel_ilt_solve", [ctypes.POINTER(devel_ilt_params), _I, ctypes.POINTER(devel_clip), _P, _P])
_sig("devel_batch_create", [_P, _I, ctypes.POINTER(_P)])
_sig("devel_batch_destroy", [_P])
_sig("devel_ilt_solve_batch", [ctypes.POINTER(devel_ilt_params), _P, _I, _P, _P, _I, _P, _P, _P, _P, _P, _I, _P,
                               _P])
_sig("devel_phi_downsample", [_I, _I, _I, _P, _P, _P])
_sig("devel_phi_upsample", [_I, _I, _I, _P, _P, _P])

_sig("devel_reinit_sdf_static", [_I, _P, _P, _F, _F, _P])
_sig("devel_profile_start", [_I])
_sig("devel_profile_stop", [])
_sig("devel_profile_collect", [])
_sig("devel_profile_kinds", [])
_sig("devel_profile_select", [ctypes.c_ulonglong])
_sig("devel_optics_autotune", [_P, _P])
_sig("devel_selftest_bounded_wait", [_P, _P])
_sig("devel_optics_config", [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)])
_sig("devel_profile_query", [_I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_I),
                             ctypes.POINTER(ctypes.c_double)])

# every symbol the header declares (checked by the CPU test suite)
EXPORTED = ("devel_last_error", "devel_version", "devel_optics_create", "devel_optics_destroy",
            "devel_optics_n", "devel_optics_check", "devel_litho_forward", "devel_resist_loss", "devel_litho_adjoint",
            "devel_levelset_step", "devel_reinit_sdf", "devel_ilt_solve", "devel_profile_start",
            "devel_profile_stop", "devel_profile_kinds", "devel_profile_query", "devel_profile_collect",
            "devel_reinit_sdf_static", "devel_profile_select", "devel_optics_autotune", "devel_optics_config",
            "devel_selftest_bounded_wait", "devel_levelset_step_weno5", "devel_cg_direction",
            "devel_modulation_candidates", "devel_ahf_loss", "devel_shot_count", "devel_dsn_create", "devel_dsn_destroy",
            "devel_dsn_param_count", "devel_dsn_init", "devel_dsn_set_params", "devel_dsn_get_params",
            "devel_dsn_grads", "devel_dsn_forward", "devel_dsn_train_step", "devel_dsn_forward_ahf",
            "devel_dsn_train_step_ahf", "devel_phi_downsample", "devel_phi_upsample", "devel_modulation_search",
            "devel_batch_create", "devel_batch_destroy", "devel_ilt_solve_batch", "devel_reinit_sdf_batch")
REINIT_STATIC_MAX_N = 2048


def _check(rc: int):
    if rc != DEVEL_OK:
        raise DevelError(rc, _lib.devel_last_error().decode(errors="replace"))


def devel_last_error() -> str:
    return _lib.devel_last_error().decode(errors="replace")


def devel_version() -> int:
    return _lib.devel_version()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


class Optics:
    """Owner of a ``devel_optics*`` handle (destroyed with the object)."""

    def __init__(self, handle: int, n: int, K: int, k: int, precision: int):
        self.handle = handle
        self.n, self.K, self.k, self.precision = n, K, k, precision

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(_lib.devel_optics_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def devel_optics_create(n: int, H: np.ndarray, w: np.ndarray, precision: int = DEVEL_PREC_FP32) -> Optics:
    """H: complex [K, k, k] kernel spectra on the centred window; w: [K] weights."""
    H = np.asarray(H)
    K, k, k2 = H.shape
    if k != k2:
        raise ValueError("H must be [K, k, k]")
    Hf = np.ascontiguousarray(np.stack([H.real, H.imag], axis=-1), dtype=np.float32)
    wf = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
    if wf.shape != (K,):
        raise ValueError("w must be [K]")
    out = _P()
    _check(_lib.devel_optics_create(n, K, k, Hf.ctypes.data, wf.ctypes.data, precision, ctypes.byref(out)))
    return Optics(out.value, n, K, k, precision)


def devel_optics_check(optics: Optics, stream=None):
    """Synchronise and raise DevelError if a bounded device wait of this handle gave up."""
    _check(_lib.devel_optics_check(optics.handle, _stream(stream)))


def devel_optics_autotune(optics: Optics, stream=None):
    """Pick the tile shapes of the handle's tensor-core kernels by timing them."""
    _check(_lib.devel_optics_autotune(optics.handle, _stream(stream)))


def devel_optics_config(optics: Optics) -> dict:
    bn, split = _I(), _I()
    _check(_lib.devel_optics_config(optics.handle, ctypes.byref(bn), ctypes.byref(split)))
    return {"expand_tile_n": bn.value, "reduce_split": split.value}


def devel_selftest_bounded_wait(optics: Optics, stream=None):
    """Diagnostic: a device wait on a barrier nothing signals gives up (about 1 s) and
    leaves DEVEL_ETIMEOUT for the next devel_optics_check."""
    _check(_lib.devel_selftest_bounded_wait(optics.handle, _stream(stream)))


def devel_optics_destroy(optics: Optics):
    optics.close()


def devel_litho_forward(optics: Optics, mask, intensity, stream=None):
    import torch
    N = optics.n * optics.n
    _check(_lib.devel_litho_forward(optics.handle, _ptr(mask, torch.float32, N, "mask"),
                                    _ptr(intensity, torch.float32, N, "intensity"), _stream(stream)))


def resist_params(sigma_z=50.0, I_th=0.225, alpha=1.0, beta=0.0, dose_in=0.98, dose_out=1.02):
    return devel_resist_params(sigma_z, I_th, alpha, beta, dose_in, dose_out)


def devel_resist_loss(optics: Optics, intensity, target, params: devel_resist_params, dLdI,
                      loss_out, counts_out, stream=None):
    import torch
    N = optics.n * optics.n
    _check(_lib.devel_resist_loss(optics.handle, _ptr(intensity, torch.float32, N, "intensity"),
                                  _ptr(target, torch.uint8, N, "target"), ctypes.byref(params),
                                  _ptr(dLdI, torch.float32, N, "dLdI"),
                                  _ptr(loss_out, torch.float64, 4, "loss_out"),
                                  _ptr(counts_out, torch.int64, 2, "counts_out"), _stream(stream)))


def devel_litho_adjoint(optics: Optics, mask, dLdI, dLdM, vmax, stream=None):
    import torch
    N = optics.n * optics.n
    _check(_lib.devel_litho_adjoint(optics.handle, _ptr(mask, torch.float32, N, "mask"),
                                    _ptr(dLdI, torch.float32, N, "dLdI"),
                                    _ptr(dLdM, torch.float32, N, "dLdM"),
                                    _ptr(vmax, torch.float64, 1, "vmax"), _stream(stream)))


def devel_levelset_step(n: int, phi, V, vmax, m, dt: float, lam: float, phi_out, mask_out,
                        stream=None, weno5: bool = False):
    import torch
    N = n * n
    fn = _lib.devel_levelset_step_weno5 if weno5 else _lib.devel_levelset_step
    _check(fn(n, _ptr(phi, torch.float32, N, "phi"),
                                    _ptr(V, torch.float32, N, "V"),
                                    _ptr(vmax, torch.float64, 1, "vmax"),
                                    _ptr(m, torch.float32, N, "m"), dt, lam,
                                    _ptr(phi_out, torch.float32, N, "phi_out"),
                                    _ptr(mask_out, torch.uint8, N, "mask_out"), _stream(stream)))


def devel_cg_direction(optics: Optics, V, Vprev, D, restart: bool, vmax, beta=None, status=None,
                       stream=None):
    """D = V + beta D (PR+ beta; restart: D = V), Vprev = V, vmax = max|D|."""
    import torch
    N = optics.n * optics.n
    _check(_lib.devel_cg_direction(optics.handle, _ptr(V, torch.float32, N, "V"),
                                   _ptr(Vprev, torch.float32, N, "Vprev"), _ptr(D, torch.float32, N, "D"),
                                   int(bool(restart)), _ptr(beta, torch.float64, 1, "beta"),
                                   _ptr(vmax, torch.float64, 1, "vmax"), _ptr(status, torch.int32, 1, "status"),
                                   _stream(stream)))


def devel_modulation_candidates(n: int, phi_gt, dh, m_out, stream=None):
    """m_out[j] = H(phi_gt + dh[j]) (Sec. III-B); m_out float32 [len(dh) * n * n]."""
    import torch
    N = n * n
    dh_host = (ctypes.c_float * len(dh))(*[float(d) for d in dh])
    _check(_lib.devel_modulation_candidates(n, _ptr(phi_gt, torch.float32, N, "phi_gt"), len(dh),
                                            ctypes.cast(dh_host, _P), _ptr(m_out, torch.float32, N * len(dh), "m_out"),
                                            _stream(stream)))


def devel_ahf_loss(optics: Optics, phi_m, m_gt, eps: float, loss_out, grad_out=None, stream=None):
    import torch
    N = optics.n * optics.n
    _check(_lib.devel_ahf_loss(optics.handle, _ptr(phi_m, torch.float32, N, "phi_m"),
                               _ptr(m_gt, torch.float32, N, "m_gt"), float(eps),
                               _ptr(loss_out, torch.float64, 1, "loss_out"),
                               _ptr(grad_out, torch.float32, N, "grad_out"), _stream(stream)))


def modulation_search(handles, target, phi_gt, dh, params: "devel_ilt_params", stream=None):
    """The label search of Sec. III-B through devel_modulation_search (candidate maps
    H(phi_gt + dh_j), one DSO solve per candidate on handle j, the device argmin of the
    final L_DSO). Returns (index, final losses as a host array, candidate maps
    [len(dh), n*n])."""
    import torch
    n = handles[0].n
    N = n * n
    dev = target.device
    J = len(dh)
    cands = torch.empty(J * N, dtype=torch.float32, device=dev)
    phi_work = torch.empty(J * N, dtype=torch.float32, device=dev)
    H = params.iters + 1
    ldh = (H + 1) // 2 * 2                                   # rows 16-byte aligned
    hist = torch.zeros(J, ldh, dtype=torch.float64, device=dev)
    best = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    harr = (_P * J)(*[h.handle for h in handles])
    dh_host = (ctypes.c_float * J)(*[float(d) for d in dh])
    _check(_lib.devel_modulation_search(ctypes.byref(params), J, harr, _ptr(target, torch.uint8, N, "target"),
                                        _ptr(phi_gt, torch.float32, N, "phi_gt"), ctypes.cast(dh_host, _P),
                                        _ptr(cands, torch.float32, J * N, "m_out"),
                                        _ptr(phi_work, torch.float32, J * N, "phi_work"),
                                        _ptr(hist, torch.float64, J * ldh, "loss_hist"), ldh,
                                        _ptr(best, torch.int32, 1, "best"), _ptr(st, torch.int32, 1, "status"),
                                        _stream(stream)))
    if int(st.item()) != 0:
        raise DevelError(int(st.item()), "modulation_search: a candidate solve reported a non-finite loss")
    return int(best.item()), hist[:, H - 1].cpu().numpy(), cands.view(J, N)


def devel_shot_count(mask) -> int:
    """Minimum rectangle partition of a square host mask (numpy uint8 [n, n])."""
    import numpy as np
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    assert m.ndim == 2 and m.shape[0] == m.shape[1]
    out = ctypes.c_longlong()
    _check(_lib.devel_shot_count(m.shape[0], m.ctypes.data, ctypes.byref(out)))
    return int(out.value)


class Dsn:
    """Owner of a ``devel_dsn*`` (the DSN level-set branch, Sec. III-B)."""

    def __init__(self, side: int, batch: int, width: int = 32, seed: int = 0):
        h = _P()
        _check(_lib.devel_dsn_create(side, batch, width, ctypes.byref(h)))
        self.handle, self.side, self.batch, self.width = h.value, side, batch, width
        _check(_lib.devel_dsn_init(self.handle, seed))

    def close(self):
        if self.handle:
            _lib.devel_dsn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def param_count(self) -> int:
        return int(_lib.devel_dsn_param_count(self.handle))

    def get_params(self):
        import numpy as np
        out = np.empty(self.param_count, dtype=np.float32)
        _check(_lib.devel_dsn_get_params(self.handle, out.ctypes.data))
        return out

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.param_count
        _check(_lib.devel_dsn_set_params(self.handle, p.ctypes.data))

    def grads(self):
        import numpy as np
        out = np.empty(self.param_count, dtype=np.float32)
        _check(_lib.devel_dsn_grads(self.handle, out.ctypes.data))
        return out

    def forward(self, nb: int, tsdf, phi0, band: float = 16.0, stream=None):
        import torch
        N = nb * self.side * self.side
        _check(_lib.devel_dsn_forward(self.handle, nb, _ptr(tsdf, torch.float32, N, "tsdf"), float(band),
                                      _ptr(phi0, torch.float32, N, "phi0"), _stream(stream)))

    def forward_ahf(self, nb: int, tsdf, m_out, eps: float = 0.03, band: float = 16.0, stream=None):
        import torch
        N = nb * self.side * self.side
        _check(_lib.devel_dsn_forward_ahf(self.handle, nb, _ptr(tsdf, torch.float32, N, "tsdf"), float(band),
                                          float(eps), _ptr(m_out, torch.float32, N, "m_out"), _stream(stream)))

    def train_step_ahf(self, nb: int, tsdf, m_gt, lr: float, loss_out=None, eps: float = 0.03, band: float = 16.0,
                       stream=None):
        import torch
        N = nb * self.side * self.side
        _check(_lib.devel_dsn_train_step_ahf(self.handle, nb, _ptr(tsdf, torch.float32, N, "tsdf"),
                                             _ptr(m_gt, torch.float32, N, "m_gt"), float(band), float(eps),
                                             float(lr), _ptr(loss_out, torch.float64, 1, "loss_out"),
                                             _stream(stream)))

    def train_step(self, nb: int, tsdf, phi_gt, lr: float, loss_out=None, band: float = 16.0, stream=None):
        import torch
        N = nb * self.side * self.side
        _check(_lib.devel_dsn_train_step(self.handle, nb, _ptr(tsdf, torch.float32, N, "tsdf"),
                                         _ptr(phi_gt, torch.float32, N, "phi_gt"), float(band), float(lr),
                                         _ptr(loss_out, torch.float64, 1, "loss_out"), _stream(stream)))


def devel_reinit_sdf(n: int, mask, phi, d2, d_lo: float = -100.0, d_hi: float = 900.0, stream=None):
    import torch
    N = n * n
    _check(_lib.devel_reinit_sdf(n, _ptr(mask, torch.uint8, N, "mask"), _ptr(phi, torch.float32, N, "phi"),
                                 _ptr(d2, torch.int32, N, "d2"), d_lo, d_hi, _stream(stream)))


def devel_reinit_sdf_batch(n: int, nb: int, mask, phi, d2, d_lo: float = -100.0, d_hi: float = 900.0,
                           stream=None):
    """devel_reinit_sdf of nb masks stored back to back (arrays of nb * n * n elements)."""
    import torch
    N = nb * n * n
    _check(_lib.devel_reinit_sdf_batch(n, nb, _ptr(mask, torch.uint8, N, "mask"), _ptr(phi, torch.float32, N, "phi"),
                                       _ptr(d2, torch.int32, N, "d2"), d_lo, d_hi, _stream(stream)))


def devel_reinit_sdf_static(n: int, mask, phi, d_lo: float = -100.0, d_hi: float = 900.0, stream=None):
    """devel_reinit_sdf without the scratch argument: the library's static
    device array (n <= 2048) serves as scratch; nothing is allocated."""
    import torch
    N = n * n
    _check(_lib.devel_reinit_sdf_static(n, _ptr(mask, torch.uint8, N, "mask"),
                                        _ptr(phi, torch.float32, N, "phi"), d_lo, d_hi, _stream(stream)))


def devel_phi_downsample(n: int, f: int, fine, coarse, stream=None):
    """fine: float [nb, n*n] (or [n*n]) -> coarse: float [nb, (n/f)^2], the f x f block
    means divided by f (distances in coarse pixels)."""
    import torch
    N, m = n * n, n // f if f > 0 else 0
    nb = fine.numel() // N if N else 0
    _check(_lib.devel_phi_downsample(n, f, nb, _ptr(fine, torch.float32, nb * N, "fine"),
                                     _ptr(coarse, torch.float32, nb * m * m, "coarse"), _stream(stream)))


def devel_phi_upsample(n: int, f: int, coarse, fine, stream=None):
    """coarse: float [nb, (n/f)^2] -> fine: float [nb, n*n], f times the bilinear
    interpolation at the fine pixel centres."""
    import torch
    N, m = n * n, n // f if f > 0 else 0
    nb = fine.numel() // N if N else 0
    _check(_lib.devel_phi_upsample(n, f, nb, _ptr(coarse, torch.float32, nb * m * m, "coarse"),
                                   _ptr(fine, torch.float32, nb * N, "fine"), _stream(stream)))


def ilt_params(resist: devel_resist_params = None, dt=0.5, lam=0.1, d_lo=-100.0, d_hi=900.0, iters=20,
               reinit_every=5, start_iter=0, use_graph=True, upwind=0, optimizer=0) -> devel_ilt_params:
    """upwind: DEVEL_UPWIND_GODUNOV1 (0) or DEVEL_UPWIND_WENO5 (1);
    optimizer: DEVEL_OPT_STEEPEST (0) or DEVEL_OPT_CG (1)."""
    return devel_ilt_params(resist if resist is not None else resist_params(), dt, lam, d_lo, d_hi,
                            iters, reinit_every, start_iter, int(bool(use_graph)), int(upwind), int(optimizer))


@dataclass
class Clip:
    """One clip of a devel_ilt_solve call (tensors stay owned by the caller)."""
    optics: Optics
    target: object           # uint8 [n*n]
    phi: object              # float32 [n*n], in/out
    phi_given: bool = False
    m: object = None         # float32 [n*n] or None
    mask_out: object = None  # uint8 [n*n] or None
    loss_hist: object = None  # float64 [iters+1] or None
    l2_hist: object = None   # int64 [iters+1] or None
    pvb_hist: object = None  # int64 [iters+1] or None
    optics_defocus: Optics = None  # defocused system of the inner process corner, or None


def devel_ilt_solve(params: devel_ilt_params, clips, status, stream=None):
    import torch
    arr = (devel_clip * len(clips))()
    H = params.iters + 1
    for i, c in enumerate(clips):
        N = c.optics.n * c.optics.n
        arr[i] = devel_clip(c.optics.handle, _ptr(c.target, torch.uint8, N, "target"),
                            _ptr(c.phi, torch.float32, N, "phi"), int(bool(c.phi_given)),
                            _ptr(c.m, torch.float32, N, "m"), _ptr(c.mask_out, torch.uint8, N, "mask_out"),
                            _ptr(c.loss_hist, torch.float64, H, "loss_hist"),
                            _ptr(c.l2_hist, torch.int64, H, "l2_hist"),
                            _ptr(c.pvb_hist, torch.int64, H, "pvb_hist"),
                            c.optics_defocus.handle if c.optics_defocus is not None else None)
    _check(_lib.devel_ilt_solve(ctypes.byref(params), len(clips), arr, _ptr(status, torch.int32, 1, "status"),
                                _stream(stream)))


class Batch:
    """Owner of a ``devel_batch*``: the workspace of up to ``capacity`` clips on one
    compensated-BF16 optics handle (kept alive by this object)."""

    def __init__(self, optics: Optics, capacity: int):
        out = _P()
        _check(_lib.devel_batch_create(optics.handle, int(capacity), ctypes.byref(out)))
        self.handle = out.value
        self.optics = optics
        self.capacity = int(capacity)

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(_lib.devel_batch_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def devel_ilt_solve_batch(params: devel_ilt_params, batch: Batch, target, phi, status, phi_given: bool = False,
                          m=None, mask_out=None, loss_hist=None, l2_hist=None, pvb_hist=None, stream=None):
    """The solve of ``nclips = target.shape[0]`` clips with every stage launched once over
    the batch. target uint8 [nclips, n*n]; phi float32 [nclips, n*n] in/out; m float32
    [nclips, n*n] or None; mask_out uint8 [nclips, n*n] or None; histories [nclips, ldh]
    (float64 / int64 / int64, ldh >= iters + 1) or None; status int32 [1]."""
    import torch
    B = int(target.shape[0]) if target.dim() == 2 else 1
    N = batch.optics.n * batch.optics.n
    hists = [h for h in (loss_hist, l2_hist, pvb_hist) if h is not None]
    ldh = int(hists[0].shape[-1]) if hists else 0
    _check(_lib.devel_ilt_solve_batch(ctypes.byref(params), batch.handle, B, _ptr(target, torch.uint8, B * N, "target"),
                                      _ptr(phi, torch.float32, B * N, "phi"), int(bool(phi_given)),
                                      _ptr(m, torch.float32, B * N, "m"),
                                      _ptr(mask_out, torch.uint8, B * N, "mask_out"),
                                      _ptr(loss_hist, torch.float64, B * ldh, "loss_hist"),
                                      _ptr(l2_hist, torch.int64, B * ldh, "l2_hist"),
                                      _ptr(pvb_hist, torch.int64, B * ldh, "pvb_hist"), ldh,
                                      _ptr(status, torch.int32, 1, "status"), _stream(stream)))


def devel_profile_start(capacity: int = 1 << 16):
    _check(_lib.devel_profile_start(capacity))


def devel_profile_kind_names() -> list:
    """Kernel class names, indexed by kind."""
    names = []
    for k in range(_lib.devel_profile_kinds()):
        name = ctypes.c_char_p()
        cnt = _I()
        ms = ctypes.c_double()
        _check(_lib.devel_profile_query(k, ctypes.byref(name), ctypes.byref(cnt), ctypes.byref(ms)))
        names.append(name.value.decode())
    return names


def devel_profile_select(kinds=None):
    """Limit the events of the next profiles to the named kernel classes (None: all)."""
    if kinds is None:
        mask = (1 << 64) - 1
    else:
        names = devel_profile_kind_names()
        mask = 0
        for kname in kinds:
            mask |= 1 << names.index(kname)
    _check(_lib.devel_profile_select(mask))


def devel_profile_collect():
    """Accumulate the events recorded so far (after each graph replay, or once)."""
    _check(_lib.devel_profile_collect())


def devel_profile_stop(collect: bool = True) -> dict:
    """Close the profile (collecting first unless collect=False); returns
    {kernel: (launches, total_ms)} for kernels that ran."""
    if collect:
        _check(_lib.devel_profile_collect())
    _check(_lib.devel_profile_stop())
    out = {}
    for k in range(_lib.devel_profile_kinds()):
        name = ctypes.c_char_p()
        cnt = _I()
        ms = ctypes.c_double()
        _check(_lib.devel_profile_query(k, ctypes.byref(name), ctypes.byref(cnt), ctypes.byref(ms)))
        if cnt.value:
            out[name.value.decode()] = (cnt.value, ms.value)
    return out
