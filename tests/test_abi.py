"""The C ABI library loads on the CPU and exports every symbol its header
declares; argument checks reject bad input before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "develset.h")
LIB = os.path.join(ROOT, "paper_2303_12529_gb300", "libdevelset.so")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(devel_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_hot_path():
    names = declared_functions()
    for f in ("devel_litho_forward", "devel_litho_adjoint", "devel_levelset_step",
              "devel_reinit_sdf", "devel_ilt_solve", "devel_optics_create", "devel_resist_loss"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    import paper_2303_12529_gb300 as dv
    assert sorted(dv.EXPORTED) == declared_functions()
    assert dv.devel_version() >> 16 == 1


def test_modulation_search_checks_its_arguments(lib):
    """devel_modulation_search refuses a missing parameter block, a candidate count
    outside [1, DEVEL_MOD_MAX_CANDIDATES] and a missing handle list before any launch."""
    import paper_2303_12529_gb300 as dv
    f = dv._lib.devel_modulation_search
    P = dv.ilt_params(iters=3)
    null = (dv._P * 1)(None)
    assert f(None, 1, null, None, None, None, None, None, None, 4, None, None, None) == dv.DEVEL_EINVAL
    for ncand in (0, dv.DEVEL_MOD_MAX_CANDIDATES + 1):
        rc = f(ctypes.byref(P), ncand, null, None, None, None, None, None, None, 4, None, None, None)
        assert rc == dv.DEVEL_EINVAL and "ncand" in dv.devel_last_error()
    assert f(ctypes.byref(P), 1, null, None, None, None, None, None, None, 4, None, None, None) == dv.DEVEL_EINVAL


def test_binding_constants_match_the_header():
    """The binding's copies of the header's limits and codes are the header's values."""
    import paper_2303_12529_gb300 as dv
    txt = open(HEADER).read()
    defs = dict(re.findall(r"#define\s+(DEVEL_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", txt))
    assert int(defs["DEVEL_REINIT_STATIC_MAX_N"]) == dv.REINIT_STATIC_MAX_N
    assert int(defs["DEVEL_MOD_MAX_CANDIDATES"]) == dv.DEVEL_MOD_MAX_CANDIDATES
    for name in ("DEVEL_OK", "DEVEL_EINVAL", "DEVEL_ECUDA", "DEVEL_ENOMEM", "DEVEL_ETIMEOUT", "DEVEL_ENAN",
                 "DEVEL_PREC_FP32", "DEVEL_PREC_BF16X3", "DEVEL_UPWIND_GODUNOV1", "DEVEL_UPWIND_WENO5",
                 "DEVEL_OPT_STEEPEST", "DEVEL_OPT_CG"):
        assert int(defs[name]) == getattr(dv, name), name


def test_argument_checks_need_no_device(lib):
    import paper_2303_12529_gb300 as dv
    H = np.zeros((2, 5, 5), np.complex64)
    w = np.ones(2, np.float32)
    with pytest.raises(dv.DevelError) as e:
        dv.devel_optics_create(64, H[:, :4, :4], w[:2])  # even window
    assert e.value.code == dv.DEVEL_EINVAL and "odd" in str(e.value)
    with pytest.raises(dv.DevelError) as e:
        dv.devel_optics_create(8, H, w)  # n too small
    assert e.value.code == dv.DEVEL_EINVAL
    with pytest.raises(dv.DevelError) as e:
        dv.devel_optics_create(64, H, -w)  # negative weights
    assert e.value.code == dv.DEVEL_EINVAL
    lib.devel_reinit_sdf.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_float, ctypes.c_float, ctypes.c_void_p]
    assert lib.devel_reinit_sdf(0, None, None, None, 0.0, 1.0, None) == dv.DEVEL_EINVAL
    # misaligned pointers and an inverted clamp are refused before any launch
    # (the addresses are never dereferenced)
    assert lib.devel_reinit_sdf(16, 17, 32, 48, 0.0, 1.0, None) == dv.DEVEL_EINVAL
    assert lib.devel_reinit_sdf(16, 16, 32, 48, 2.0, 1.0, None) == dv.DEVEL_EINVAL
    assert "d_lo" in dv.devel_last_error()
    lib.devel_reinit_sdf_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_void_p]
    assert lib.devel_reinit_sdf_batch(16, 0, 16, 32, 48, 0.0, 1.0, None) == dv.DEVEL_EINVAL      # no clips
    assert lib.devel_reinit_sdf_batch(16, 65536, 16, 32, 48, 0.0, 1.0, None) == dv.DEVEL_EINVAL  # grid limit
    assert lib.devel_reinit_sdf_batch(16, 2, 17, 32, 48, 0.0, 1.0, None) == dv.DEVEL_EINVAL      # misaligned
    assert lib.devel_reinit_sdf_batch(16, 2, 16, 32, 48, 2.0, 1.0, None) == dv.DEVEL_EINVAL      # inverted clamp
    # the CG direction refuses a missing handle and aliased arrays before any launch
    lib.devel_cg_direction.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int] + [ctypes.c_void_p] * 4
    assert lib.devel_cg_direction(None, 16, 32, 48, 0, None, 64, None, None) == dv.DEVEL_EINVAL
    assert "optics" in dv.devel_last_error()
    # resampling: sides that the factor does not divide, a zero factor, a negative batch
    # and misaligned pointers are refused; an empty batch is a no-op
    for fn in (lib.devel_phi_downsample, lib.devel_phi_upsample):
        fn.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 3
        assert fn(64, 3, 1, 16, 32, None) == dv.DEVEL_EINVAL
        assert fn(64, 0, 1, 16, 32, None) == dv.DEVEL_EINVAL
        assert fn(64, 4, -1, 16, 32, None) == dv.DEVEL_EINVAL
        assert fn(64, 4, 1, 17, 32, None) == dv.DEVEL_EINVAL
        assert fn(64, 4, 1, None, 32, None) == dv.DEVEL_EINVAL
        assert fn(64, 4, 0, None, None, None) == dv.DEVEL_OK


def test_ilt_params_layout_matches_the_header():
    """The ctypes mirror of devel_ilt_params has the header's fields in order (the
    new optimizer field last)."""
    import paper_2303_12529_gb300 as dv
    names = [f[0] for f in dv.devel_ilt_params._fields_]
    assert names[-2:] == ["upwind", "optimizer"]
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\} devel_ilt_params;", txt, flags=re.S).group(1)
    fields = re.findall(r"\b(\w+)\s*(?:,\s*(\w+))?\s*;", body)
    flat = [x for pair in fields for x in pair if x]
    assert flat[-2:] == ["upwind", "optimizer"]


def test_new_entry_points_refuse_bad_arguments_without_a_device(lib):
    import paper_2303_12529_gb300 as dv
    c = ctypes
    lib.devel_modulation_candidates.argtypes = [c.c_int, c.c_void_p, c.c_int, c.c_void_p, c.c_void_p, c.c_void_p]
    dh = (c.c_float * 2)(1.0, float("nan"))
    assert lib.devel_modulation_candidates(64, 16, 0, dh, 32, None) == dv.DEVEL_EINVAL        # no candidates
    assert lib.devel_modulation_candidates(64, 16, 65, dh, 32, None) == dv.DEVEL_EINVAL       # too many
    assert lib.devel_modulation_candidates(64, 16, 2, dh, 32, None) == dv.DEVEL_EINVAL        # NaN shift
    assert "finite" in dv.devel_last_error()
    lib.devel_ahf_loss.argtypes = [c.c_void_p, c.c_void_p, c.c_void_p, c.c_float, c.c_void_p, c.c_void_p, c.c_void_p]
    assert lib.devel_ahf_loss(None, 16, 32, 0.03, 48, None, None) == dv.DEVEL_EINVAL
    h = c.c_void_p()
    lib.devel_dsn_create.argtypes = [c.c_int, c.c_int, c.c_int, c.POINTER(c.c_void_p)]
    assert lib.devel_dsn_create(40, 2, 4, c.byref(h)) == dv.DEVEL_EINVAL                      # side % 16
    assert lib.devel_dsn_create(32, 0, 4, c.byref(h)) == dv.DEVEL_EINVAL                      # batch
    assert h.value is None
    lib.devel_shot_count.argtypes = [c.c_int, c.c_void_p, c.c_void_p]
    assert lib.devel_shot_count(0, None, None) == dv.DEVEL_EINVAL
    # the shot count is host code: it runs here
    assert dv.devel_shot_count(np.eye(5, dtype=np.uint8)) == 5
    # the batched solve: a missing handle, batch or params is refused before any device call
    lib.devel_batch_create.argtypes = [c.c_void_p, c.c_int, c.POINTER(c.c_void_p)]
    assert lib.devel_batch_create(None, 4, c.byref(h)) == dv.DEVEL_EINVAL
    assert h.value is None
    assert lib.devel_batch_create(None, 4, None) == dv.DEVEL_EINVAL
    lib.devel_batch_destroy.argtypes = [c.c_void_p]
    assert lib.devel_batch_destroy(None) == dv.DEVEL_OK
    p = dv.ilt_params(iters=4)
    lib.devel_ilt_solve_batch.argtypes = [c.POINTER(dv.devel_ilt_params)] + [c.c_void_p, c.c_int, c.c_void_p,
                                          c.c_void_p, c.c_int] + [c.c_void_p] * 5 + [c.c_int, c.c_void_p, c.c_void_p]
    assert lib.devel_ilt_solve_batch(c.byref(p), None, 1, 16, 16, 0, None, None, None, None, None, 0, 16,
                                     None) == dv.DEVEL_EINVAL
    assert "batch is NULL" in dv.devel_last_error()
    assert lib.devel_ilt_solve_batch(None, None, 1, 16, 16, 0, None, None, None, None, None, 0, 16,
                                     None) == dv.DEVEL_EINVAL


def test_last_error_is_per_thread(lib):
    """devel_last_error() is thread-local: two threads failing in different calls each read
    their own message (no device needed: the checks refuse the arguments first)."""
    import threading
    import paper_2303_12529_gb300 as dv
    for fn in (lib.devel_phi_downsample, lib.devel_phi_upsample):
        fn.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 3
    lib.devel_last_error.restype = ctypes.c_char_p
    out = {}
    go = threading.Barrier(2)

    def fail(name, call):
        rc = call()
        go.wait()                      # both have failed before either reads
        out[name] = (rc, lib.devel_last_error().decode())

    t1 = threading.Thread(target=fail, args=("a", lambda: lib.devel_phi_downsample(64, 3, 1, 16, 32, None)))
    t2 = threading.Thread(target=fail, args=("b", lambda: lib.devel_phi_upsample(64, 4, -2, 16, 32, None)))
    t1.start(); t2.start(); t1.join(); t2.join()
    assert out["a"][0] == dv.DEVEL_EINVAL and "devel_phi_downsample" in out["a"][1] and "f=3" in out["a"][1]
    assert out["b"][0] == dv.DEVEL_EINVAL and "devel_phi_upsample" in out["b"][1] and "nb=-2" in out["b"][1]
