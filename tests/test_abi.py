"""The C-ABI library loads and exports every symbol declared in include/hydro.h; host-side parameter
validation (no GPU needed: these calls return before touching CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1306_6883_gb300 import build, hydro
    build.build()
    return hydro.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("hydro.h")
    assert "hydro_init" in names and "hydro_step" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1306_6883_gb300 import hydro
    assert set(names) <= set(hydro.SIGNATURES), set(names) - set(hydro.SIGNATURES)


def test_defaults_and_layout(lib):
    from paper_1306_6883_gb300 import hydro as H
    p = H.default_params(100, 60)
    assert (p.ng, p.limiter, p.use_flattening, p.riemann_maxiter) == (4, 2, 1, 32)
    assert p.cvisc == 0.1 and p.riemann_tol == 1e-14 and p.gamma == 1.4 and p.cfl == 0.8
    pitch = H.state_pitch(p)
    assert pitch >= 108 and pitch * 8 % 128 == 0
    assert H.state_bytes(p) == 4 * pitch * 68 * 8
    p32 = H.default_params(100, 60, H.HYDRO_FP32)
    assert H.state_pitch(p32) * 4 % 128 == 0 and p32.riemann_tol == 1e-6
    assert p.recover_ke_frac == 0.999 and p32.recover_ke_frac == 0.999
    # the binding mirrors the library's struct byte for byte
    assert lib.hydro_params_size() == ctypes.sizeof(H.HydroParams)


@pytest.mark.parametrize("field,value", [("nx", 0), ("ny", -3), ("ng", 3), ("gamma", 1.0), ("cfl", 0.0),
                                         ("limiter", 3), ("riemann_maxiter", 0), ("small_pres", 0.0),
                                         ("precision", 2), ("bc_xlo", 1), ("use_learned_guess", 1),
                                         ("bc_xlo", 3), ("bc_xhi", 3), ("bc_yhi", 4), ("bc_ylo", -1),
                                         ("grav", float("nan")), ("grav", float("inf")), ("split", 2),
                                         ("split", -1), ("recover_ke_frac", -0.5),
                                         ("recover_ke_frac", float("nan")), ("recover_ke_frac", float("inf"))])
def test_invalid_parameters_are_rejected_before_any_allocation(lib, field, value):
    from paper_1306_6883_gb300 import hydro as H
    p = H.default_params(16, 16)
    setattr(p, field, value)
    assert H.state_pitch(p) == 0
    ctx = ctypes.c_void_p()
    st = lib.hydro_init(ctypes.byref(p), ctypes.c_void_p(256), ctypes.c_void_p(512), None, ctypes.byref(ctx))
    assert st == H.HYDRO_EINVAL and not ctx.value


@pytest.mark.parametrize("bc", [("reflect",) * 4, ("periodic", "periodic", "hydrostatic", "hydrostatic"),
                                ("reflect", "outflow", "hydrostatic", "reflect")])
def test_reflecting_and_hydrostatic_sides_are_accepted(lib, bc):
    from paper_1306_6883_gb300 import hydro as H
    p = H.default_params(16, 16, bc=bc, grav=-1.0)
    assert H.state_pitch(p) > 0
    p = H.default_params(3, 3, bc=bc)  # a mirrored ghost cell's source must lie inside the domain
    assert H.state_pitch(p) == 0


def test_null_and_misaligned_buffers_are_rejected(lib):
    from paper_1306_6883_gb300 import hydro as H
    p = H.default_params(16, 16)
    ctx = ctypes.c_void_p()
    assert lib.hydro_init(ctypes.byref(p), None, ctypes.c_void_p(512), None, ctypes.byref(ctx)) == H.HYDRO_EINVAL
    assert lib.hydro_init(ctypes.byref(p), ctypes.c_void_p(264), ctypes.c_void_p(512), None,
                          ctypes.byref(ctx)) == H.HYDRO_EINVAL
    assert lib.hydro_init(ctypes.byref(p), ctypes.c_void_p(512), ctypes.c_void_p(512), None,
                          ctypes.byref(ctx)) == H.HYDRO_EINVAL
    assert lib.hydro_step(None, ctypes.c_double(0.1)) == H.HYDRO_EINVAL


def test_oracle_library_builds_and_loads():
    import oracle
    assert oracle.num_threads() >= 1


@pytest.mark.parametrize("extra", [dict(use_learned_guess=1, precision=1)])
def test_split_variant_rejects_what_it_does_not_implement(lib, extra):
    from paper_1306_6883_gb300 import hydro as H
    p = H.default_params(16, 16, split=1)
    assert H.state_pitch(p) > 0
    for k, v in extra.items():
        setattr(p, k, v)
    assert H.state_pitch(p) == 0


@pytest.mark.parametrize("extra", [dict(use_learned_guess=1, precision=1), dict(riemann_solver=2)])
def test_hllc_rejects_what_it_does_not_implement(lib, extra):
    from paper_1306_6883_gb300 import hydro as H
    p = H.default_params(16, 16, riemann_solver="hllc")
    assert H.state_pitch(p) > 0 and p.riemann_solver == 1
    for k, v in extra.items():
        setattr(p, k, v)
    assert H.state_pitch(p) == 0


@pytest.mark.parametrize("extra", [dict(use_learned_guess=1, precision=1), dict(reconstruction=2)])
def test_ppm_rejects_what_it_does_not_implement(lib, extra):
    from paper_1306_6883_gb300 import hydro as H
    p = H.default_params(16, 16, reconstruction="ppm")
    assert H.state_pitch(p) > 0 and p.reconstruction == 1
    for k, v in extra.items():
        setattr(p, k, v)
    assert H.state_pitch(p) == 0


def test_ensembles_take_the_two_shock_unsplit_step_only(lib):
    from paper_1306_6883_gb300 import hydro as H
    for kw in (dict(riemann_solver="hllc"), dict(split=1), dict(reconstruction="ppm")):
        p = H.default_params(16, 16, H.HYDRO_FP32, **kw)
        arr = (H.HydroParams * 1)(p)
        ptrs = (ctypes.c_void_p * 1)(256)
        alt = (ctypes.c_void_p * 1)(512)
        b = ctypes.c_void_p()
        assert lib.hydro_batch_create(1, arr, ptrs, alt, None, ctypes.byref(b)) == H.HYDRO_EINVAL
        assert not b.value
