"""Thin ctypes binding of libhydro.so (include/hydro.h): argument marshalling only.

Every step of the path runs in the library's CUDA kernels.  PyTorch provides device memory and the
stream.  There is no CPU fallback: loading fails loudly if the library is missing.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhydro.so")

(HYDRO_OK, HYDRO_EINVAL, HYDRO_ENOMEM, HYDRO_ECUDA, HYDRO_ENONFINITE, HYDRO_ENEGATIVE, HYDRO_ENONCONV,
 HYDRO_ETIMEOUT, HYDRO_ERANGE) = range(9)
STATUS_NAMES = ["HYDRO_OK", "HYDRO_EINVAL", "HYDRO_ENOMEM", "HYDRO_ECUDA", "HYDRO_ENONFINITE", "HYDRO_ENEGATIVE",
                "HYDRO_ENONCONV", "HYDRO_ETIMEOUT", "HYDRO_ERANGE"]
NOALLOC_MAX_ROWS = 16384
HYDRO_FP64, HYDRO_FP32 = 0, 1
BC = {"outflow": 0, "periodic": 1, "reflect": 2, "hydrostatic": 3}
RIEMANN = {"two-shock": 0, "hllc": 1}
RECON = {"plm": 0, "ppm": 1}


class HydroParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("ng", ctypes.c_int),
        ("xmin", ctypes.c_double), ("xmax", ctypes.c_double), ("ymin", ctypes.c_double), ("ymax", ctypes.c_double),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("bc_xlo", ctypes.c_int), ("bc_xhi", ctypes.c_int), ("bc_ylo", ctypes.c_int), ("bc_yhi", ctypes.c_int),
        ("limiter", ctypes.c_int), ("use_flattening", ctypes.c_int), ("cvisc", ctypes.c_double),
        ("riemann_maxiter", ctypes.c_int), ("riemann_tol", ctypes.c_double),
        ("small_dens", ctypes.c_double), ("small_pres", ctypes.c_double),
        ("precision", ctypes.c_int), ("use_learned_guess", ctypes.c_int),
        ("grav", ctypes.c_double), ("split", ctypes.c_int), ("riemann_solver", ctypes.c_int),
        ("reconstruction", ctypes.c_int), ("recover_ke_frac", ctypes.c_double),
    ]


class HydroError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}" if msg else name)


_LIB = None
_VP = ctypes.c_void_p
_PP = ctypes.POINTER(HydroParams)

# name -> (restype, argtypes); the same names as the C ABI
SIGNATURES = {
    "hydro_default_params": (ctypes.c_int, [_PP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "hydro_params_size": (ctypes.c_size_t, []),
    "hydro_state_pitch": (ctypes.c_size_t, [_PP]),
    "hydro_state_bytes": (ctypes.c_size_t, [_PP]),
    "hydro_init": (ctypes.c_int, [_PP, _VP, _VP, _VP, ctypes.POINTER(_VP)]),
    "hydro_destroy": (None, [_VP]),
    "hydro_state": (_VP, [_VP]),
    "hydro_fill_ghost": (ctypes.c_int, [_VP]),
    "hydro_cfl_dt": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "hydro_step": (ctypes.c_int, [_VP, ctypes.c_double]),
    "hydro_advance": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double]),
    "hydro_cfl_dt_async": (ctypes.c_int, [_VP, ctypes.c_double]),
    "hydro_step_device_dt": (ctypes.c_int, [_VP]),
    "hydro_step_fused": (ctypes.c_int, [_VP, ctypes.c_double]),
    "hydro_get_time": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "hydro_conserved_totals": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "hydro_sync_status": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_ulonglong)]),
    "hydro_conserved_totals_noalloc": (ctypes.c_int, [_PP, _VP, _VP, ctypes.POINTER(ctypes.c_double)]),
    "hydro_upload": (ctypes.c_int, [_VP, _VP]),
    "hydro_download": (ctypes.c_int, [_VP, _VP]),
    "hydro_step_host": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double]),
    "hydro_step_host_chained": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double]),
    "hydro_mlp_create": (ctypes.c_int, [ctypes.c_ulonglong, _VP, ctypes.POINTER(_VP)]),
    "hydro_mlp_destroy": (None, [_VP]),
    "hydro_mlp_set_weights": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "hydro_mlp_get_weights": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "hydro_mlp_set_gate": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double]),
    "hydro_mlp_gradient": (ctypes.c_int, [_VP, _VP, ctypes.c_longlong, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_double)]),
    "hydro_mlp_train": (ctypes.c_int, [_VP, _VP, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_double)]),
    "hydro_mlp_predict": (ctypes.c_int, [_VP, _VP, ctypes.c_longlong, ctypes.c_int, _VP]),
    "hydro_mlp_iterations": (ctypes.c_int, [_VP, _VP, ctypes.c_longlong, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_longlong)]),
    "hydro_mlp_device_blob": (_VP, [_VP]),
    "hydro_mlp_last_error": (ctypes.c_char_p, [_VP]),
    "hydro_set_riemann_model": (ctypes.c_int, [_VP, _VP]),
    "hydro_set_harvest": (ctypes.c_int, [_VP, _VP, ctypes.c_ulonglong, ctypes.c_double, _VP]),
    "hydro_set_harvest_gate": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double]),
    "hydro_batch_create": (ctypes.c_int, [ctypes.c_int, _PP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP,
                                          ctypes.POINTER(_VP)]),
    "hydro_batch_destroy": (None, [_VP]),
    "hydro_batch_set_riemann_model": (ctypes.c_int, [_VP, _VP]),
    "hydro_batch_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "hydro_batch_num_classes": (ctypes.c_int, [_VP]),
    "hydro_batch_class_info": (ctypes.c_int, [_VP, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 6),
    "hydro_batch_run": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "hydro_batch_state": (_VP, [_VP, ctypes.c_int]),
    "hydro_batch_get_time": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_longlong)]),
    "hydro_batch_sync_status": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_ulonglong)]),
    "hydro_batch_conserved_totals": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "hydro_batch_last_error": (ctypes.c_char_p, [_VP]),
    "hydro_last_error": (ctypes.c_char_p, [_VP]),
    "hydro_build_info": (ctypes.c_char_p, []),
    "hydro_tma_enabled": (ctypes.c_int, [_VP]),
    "hydro_test_drop_tile_copies": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_uint]),
}


def load(path=LIB_PATH):
    """Load libhydro.so (build it first with paper_1306_6883_gb300.build.build())."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(path):
            raise ImportError(f"CUDA library {path} is missing: run __graft_entry__.build() (no CPU fallback exists)")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if L.hydro_params_size() != ctypes.sizeof(HydroParams):
            raise ImportError(f"{path}: hydro_params is {L.hydro_params_size()} bytes in the library and "
                              f"{ctypes.sizeof(HydroParams)} in this binding (stale build)")
        _LIB = L
    return _LIB


def default_params(nx, ny, precision=HYDRO_FP64, **overrides):
    p = HydroParams()
    _check(load().hydro_default_params(ctypes.byref(p), nx, ny, precision), None, "hydro_default_params")
    for k, v in overrides.items():
        if k == "bc":
            p.bc_xlo, p.bc_xhi, p.bc_ylo, p.bc_yhi = (BC[b] if isinstance(b, str) else b for b in v)
        elif k == "riemann_solver" and isinstance(v, str):
            p.riemann_solver = RIEMANN[v]
        elif k == "reconstruction" and isinstance(v, str):
            p.reconstruction = RECON[v]
        else:
            setattr(p, k, v)
    return p


def state_pitch(p):
    return load().hydro_state_pitch(ctypes.byref(p))


def state_bytes(p):
    return load().hydro_state_bytes(ctypes.byref(p))


def _check(status, ctx, what):
    if status != HYDRO_OK:
        msg = load().hydro_last_error(ctx).decode() if ctx else ""
        raise HydroError(status, f"{what}: {msg}")


def hydro_init(p, d_state_ptr, d_state_alt_ptr, stream_ptr):
    ctx = _VP()
    _check(load().hydro_init(ctypes.byref(p), _VP(d_state_ptr), _VP(d_state_alt_ptr), _VP(stream_ptr),
                             ctypes.byref(ctx)), None, "hydro_init")
    return ctx


def hydro_destroy(ctx):
    load().hydro_destroy(ctx)


def hydro_state(ctx):
    return load().hydro_state(ctx)


def hydro_fill_ghost(ctx):
    _check(load().hydro_fill_ghost(ctx), ctx, "hydro_fill_ghost")


def hydro_cfl_dt(ctx):
    dt = ctypes.c_double()
    _check(load().hydro_cfl_dt(ctx, ctypes.byref(dt)), ctx, "hydro_cfl_dt")
    return dt.value


def hydro_step(ctx, dt):
    _check(load().hydro_step(ctx, float(dt)), ctx, "hydro_step")


def hydro_advance(ctx, nsteps, tmax=0.0):
    _check(load().hydro_advance(ctx, int(nsteps), float(tmax)), ctx, "hydro_advance")


def hydro_cfl_dt_async(ctx, tmax=0.0):
    _check(load().hydro_cfl_dt_async(ctx, float(tmax)), ctx, "hydro_cfl_dt_async")


def hydro_step_device_dt(ctx):
    _check(load().hydro_step_device_dt(ctx), ctx, "hydro_step_device_dt")


def hydro_step_fused(ctx, tmax=0.0):
    _check(load().hydro_step_fused(ctx, float(tmax)), ctx, "hydro_step_fused")


def hydro_get_time(ctx):
    t, n = ctypes.c_double(), ctypes.c_longlong()
    _check(load().hydro_get_time(ctx, ctypes.byref(t), ctypes.byref(n)), ctx, "hydro_get_time")
    return t.value, n.value


def hydro_conserved_totals(ctx):
    out = (ctypes.c_double * 4)()
    _check(load().hydro_conserved_totals(ctx, out), ctx, "hydro_conserved_totals")
    return list(out)


def hydro_conserved_totals_noalloc(p, d_state_ptr, stream_ptr):
    """Totals of a state without any allocation (file-scope device scratch; see include/hydro.h)."""
    out = (ctypes.c_double * 4)()
    _check(load().hydro_conserved_totals_noalloc(ctypes.byref(p), _VP(d_state_ptr), _VP(stream_ptr), out), None,
           "hydro_conserved_totals_noalloc")
    return list(out)


def hydro_sync_status(ctx, raise_on_error=True):
    stats = (ctypes.c_ulonglong * 3)()
    st = load().hydro_sync_status(ctx, stats)
    if raise_on_error:
        _check(st, ctx, "hydro_sync_status")
    return st, list(stats)


def hydro_upload(ctx, host_ptr):
    _check(load().hydro_upload(ctx, _VP(host_ptr)), ctx, "hydro_upload")


def hydro_download(ctx, host_ptr):
    _check(load().hydro_download(ctx, _VP(host_ptr)), ctx, "hydro_download")


def hydro_step_host(ctx, host_in_ptr, host_out_ptr, tmax=0.0):
    _check(load().hydro_step_host(ctx, _VP(host_in_ptr), _VP(host_out_ptr), tmax), ctx, "hydro_step_host")


def hydro_step_host_chained(ctx, host_in_ptr, host_out_ptr, tmax=0.0):
    _check(load().hydro_step_host_chained(ctx, _VP(host_in_ptr), _VP(host_out_ptr), tmax), ctx,
           "hydro_step_host_chained")


def hydro_build_info():
    return load().hydro_build_info().decode()


def hydro_tma_enabled(ctx):
    return bool(load().hydro_tma_enabled(ctx))


def hydro_test_drop_tile_copies(ctx, drop, polls=0):
    _check(load().hydro_test_drop_tile_copies(ctx, int(drop), int(polls)), ctx, "hydro_test_drop_tile_copies")


# ---------------------------------------------------------------------------------------------------- ensembles
def _bcheck(status, b, what):
    if status != HYDRO_OK:
        msg = load().hydro_batch_last_error(b).decode() if b else ""
        raise HydroError(status, f"{what}: {msg}")


def hydro_batch_create(params_list, states, states_alt, stream_ptr):
    n = len(params_list)
    arr = (HydroParams * n)(*params_list)
    s0 = (_VP * n)(*[_VP(p) for p in states])
    s1 = (_VP * n)(*[_VP(p) for p in states_alt])
    b = _VP()
    _bcheck(load().hydro_batch_create(n, arr, s0, s1, _VP(stream_ptr), ctypes.byref(b)), None, "hydro_batch_create")
    return b


def hydro_batch_destroy(b):
    load().hydro_batch_destroy(b)


def hydro_batch_set_riemann_model(b, m):
    _bcheck(load().hydro_batch_set_riemann_model(b, m), b, "hydro_batch_set_riemann_model")


def hydro_batch_autotune(b, reps=3):
    n = load().hydro_batch_num_classes(b)
    out = (ctypes.c_int * max(n, 1))()
    _bcheck(load().hydro_batch_autotune(b, int(reps), out), b, "hydro_batch_autotune")
    return list(out)[:n]


def hydro_batch_classes(b):
    out = []
    for k in range(load().hydro_batch_num_classes(b)):
        v = [ctypes.c_int() for _ in range(6)]
        _bcheck(load().hydro_batch_class_info(b, k, *[ctypes.byref(x) for x in v]), b, "hydro_batch_class_info")
        nx, ny, members, tx, ty, threads = (x.value for x in v)
        out.append(dict(nx=nx, ny=ny, members=members, tile=(tx, ty), threads=threads))
    return out


def hydro_batch_run(b, nsteps, use_graph=True):
    _bcheck(load().hydro_batch_run(b, int(nsteps), 1 if use_graph else 0), b, "hydro_batch_run")


def hydro_batch_state(b, member):
    return load().hydro_batch_state(b, int(member))


def hydro_batch_get_time(b, member):
    t, n = ctypes.c_double(), ctypes.c_longlong()
    _bcheck(load().hydro_batch_get_time(b, int(member), ctypes.byref(t), ctypes.byref(n)), b, "hydro_batch_get_time")
    return t.value, n.value


def hydro_batch_sync_status(b, raise_on_error=True):
    stats = (ctypes.c_ulonglong * 3)()
    st = load().hydro_batch_sync_status(b, stats)
    if raise_on_error:
        _bcheck(st, b, "hydro_batch_sync_status")
    return st, list(stats)


def hydro_batch_conserved_totals(b, member):
    out = (ctypes.c_double * 4)()
    _bcheck(load().hydro_batch_conserved_totals(b, int(member), out), b, "hydro_batch_conserved_totals")
    return list(out)


# ---------------------------------------------------------------------------------------------------- learned proposal
MLP_NPARAM = 4673
_FP = ctypes.POINTER(ctypes.c_float)


def _mcheck(status, m, what):
    if status != HYDRO_OK:
        msg = load().hydro_mlp_last_error(m).decode() if m else ""
        raise HydroError(status, f"{what}: {msg}")


def hydro_mlp_create(seed, stream_ptr):
    m = _VP()
    _mcheck(load().hydro_mlp_create(int(seed), _VP(stream_ptr), ctypes.byref(m)), None, "hydro_mlp_create")
    return m


def hydro_mlp_destroy(m):
    load().hydro_mlp_destroy(m)


def hydro_mlp_set_weights(m, theta):
    import numpy as np
    a = np.ascontiguousarray(theta, dtype=np.float32)
    assert a.size == MLP_NPARAM
    _mcheck(load().hydro_mlp_set_weights(m, a.ctypes.data_as(_FP)), m, "hydro_mlp_set_weights")


def hydro_mlp_get_weights(m):
    import numpy as np
    a = np.zeros(MLP_NPARAM, dtype=np.float32)
    _mcheck(load().hydro_mlp_get_weights(m, a.ctypes.data_as(_FP)), m, "hydro_mlp_get_weights")
    return a


def hydro_mlp_set_gate(m, gate_dp, gate_du):
    _mcheck(load().hydro_mlp_set_gate(m, float(gate_dp), float(gate_du)), m, "hydro_mlp_set_gate")


def hydro_mlp_gradient(m, d_samples_ptr, n):
    import numpy as np
    g = np.zeros(MLP_NPARAM, dtype=np.float32)
    loss = ctypes.c_double()
    _mcheck(load().hydro_mlp_gradient(m, _VP(d_samples_ptr), int(n), g.ctypes.data_as(_FP), ctypes.byref(loss)), m,
            "hydro_mlp_gradient")
    return g, loss.value


def hydro_mlp_train(m, d_samples_ptr, n, steps, batch, lr, seed):
    loss = ctypes.c_double()
    _mcheck(load().hydro_mlp_train(m, _VP(d_samples_ptr), int(n), int(steps), int(batch), float(lr), int(seed),
                                   ctypes.byref(loss)), m, "hydro_mlp_train")
    return loss.value


def hydro_mlp_predict(m, d_samples_ptr, n, use_tensor_cores, d_out_ptr):
    _mcheck(load().hydro_mlp_predict(m, _VP(d_samples_ptr), int(n), 1 if use_tensor_cores else 0, _VP(d_out_ptr)),
            m, "hydro_mlp_predict")


def hydro_mlp_iterations(m, d_samples_ptr, n, learned, gamma=1.4, tol=1e-6, maxiter=16):
    mean, nonconv = ctypes.c_double(), ctypes.c_longlong()
    _mcheck(load().hydro_mlp_iterations(m, _VP(d_samples_ptr), int(n), 1 if learned else 0, float(gamma), float(tol),
                                        int(maxiter), ctypes.byref(mean), ctypes.byref(nonconv)), m,
            "hydro_mlp_iterations")
    return mean.value, nonconv.value


def hydro_set_riemann_model(ctx, m):
    _check(load().hydro_set_riemann_model(ctx, m), ctx, "hydro_set_riemann_model")


def hydro_set_harvest(ctx, d_buf_ptr, capacity, rate, d_count_ptr):
    _check(load().hydro_set_harvest(ctx, _VP(d_buf_ptr) if d_buf_ptr else None, int(capacity), float(rate),
                                    _VP(d_count_ptr) if d_count_ptr else None), ctx, "hydro_set_harvest")


def hydro_set_harvest_gate(ctx, gate_dp, gate_du):
    _check(load().hydro_set_harvest_gate(ctx, float(gate_dp), float(gate_du)), ctx, "hydro_set_harvest_gate")
