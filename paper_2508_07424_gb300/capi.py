"""ctypes bindings of include/pff_rve.h: argument marshalling only, same names as the C ABI."""
import ctypes as C
import os

from .build import LIB

RVE_OK, RVE_EINVAL, RVE_ENOMEM, RVE_ESTATE, RVE_ENOCONV = 0, -1, -2, -3, -4
RVE_ENOROOT, RVE_ETIMEOUT, RVE_ENOTFRACTURED, RVE_ECUDA, RVE_EBREAKDOWN = -5, -6, -7, -8, -9
RVE_SPLIT_NONE, RVE_SPLIT_SPECTRAL = 0, 1
RVE_STEP_STAGNATED, RVE_STEP_CUTBACK, RVE_STEP_UNCONVERGED = 1, 2, 4
RVE_FP64, RVE_FP32R = 0, 1
RVE_CRACK_NONE, RVE_CRACK_CTE, RVE_CRACK_CPFE = 0, 1, 2
RVE_SOLVER_STAGGERED, RVE_SOLVER_NEWTON = 0, 1
(RVE_FIELD_PHI, RVE_FIELD_H, RVE_FIELD_PSI_INI, RVE_FIELD_EPS, RVE_FIELD_SIGMA, RVE_FIELD_FLUCT1,
 RVE_FIELD_PSI1, RVE_FIELD_PHI_TRIAL) = range(8)


class rve_config(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("ell", C.c_double), ("k_res", C.c_double),
                ("split", C.c_int), ("precision", C.c_int), ("history", C.c_int), ("f", C.c_double * 6),
                ("tol_mech", C.c_double), ("tol_dmg", C.c_double), ("tol_root", C.c_double),
                ("tol_stag", C.c_double), ("max_mech_iters", C.c_int), ("max_dmg_iters", C.c_int),
                ("max_root_evals", C.c_int), ("max_stag_iters", C.c_int), ("anderson_m", C.c_int),
                ("fracture_ratio", C.c_double), ("stream", C.c_void_p), ("solver", C.c_int)]


class rve_micro(C.Structure):
    _fields_ = [("grain_id", C.POINTER(C.c_int32)), ("n_grains", C.c_int), ("C_cubic", C.POINTER(C.c_double)),
                ("R", C.POINTER(C.c_double)), ("Gc", C.POINTER(C.c_double)), ("cleave_n", C.POINTER(C.c_double)),
                ("beta", C.POINTER(C.c_double)), ("crack_kind", C.c_int), ("crack_row", C.c_int),
                ("crack_x0", C.c_int), ("crack_len", C.c_int), ("crack_phi_M", C.c_double),
                ("crack_stiffness", C.c_double)]


class rve_step_result(C.Structure):
    _fields_ = [("n", C.c_int), ("E", C.c_double), ("Sigma", C.c_double), ("D", C.c_double),
                ("Emec", C.c_double), ("T", C.c_double), ("Gamma", C.c_double), ("tau", C.c_double),
                ("mech_iters", C.c_int), ("dmg_iters", C.c_int), ("root_evals", C.c_int),
                ("stag_iters", C.c_int), ("fractured", C.c_int), ("stag_err", C.c_double), ("flags", C.c_int),
                ("G_inst", C.c_double)]


class rve_scalars(C.Structure):
    _fields_ = [("n", C.c_int), ("E", C.c_double), ("tau", C.c_double), ("T", C.c_double),
                ("Sigma", C.c_double), ("Sigma_max", C.c_double), ("tau0", C.c_double), ("fractured", C.c_int),
                ("D", C.c_double), ("Gamma", C.c_double)]


class rve_request_result(C.Structure):
    _fields_ = [("id", C.c_long), ("status", C.c_int), ("fractured", C.c_int), ("n_done", C.c_int),
                ("toughness", C.c_double), ("E_last", C.c_double), ("Sigma_last", C.c_double),
                ("T_last", C.c_double), ("Sigma_max", C.c_double), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_end", C.c_double), ("voxel_updates", C.c_long)]


rve_handle = C.c_void_p
rve_server = C.c_void_p
_dp = C.POINTER(C.c_double)

_SIGS = {
    "rve_config_default": (None, [C.POINTER(rve_config)]),
    "rve_config_validate": (C.c_int, [C.POINTER(rve_config)]),
    "rve_fp64_fma_rate": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "rve_create": (C.c_int, [C.POINTER(rve_config), C.POINTER(rve_handle)]),
    "set_microstructure": (C.c_int, [rve_handle, C.POINTER(rve_micro)]),
    "step_dissipation": (C.c_int, [rve_handle, C.c_double, C.POINTER(rve_step_result)]),
    "rve_step_batch": (C.c_int, [C.POINTER(rve_handle), C.c_int, C.POINTER(C.c_double), C.POINTER(rve_step_result)]),
    "rve_batch_group_create": (C.c_int, [C.POINTER(C.c_void_p)]),
    "rve_step_in_group": (C.c_int, [rve_handle, C.c_void_p, C.c_double, C.POINTER(rve_step_result)]),
    "rve_batch_group_destroy": (C.c_int, [C.c_void_p]),
    "effective_toughness": (C.c_int, [rve_handle, _dp]),
    "effective_toughness_functional": (C.c_int, [rve_handle, _dp]),
    "rve_get_field": (C.c_int, [rve_handle, C.c_int, _dp, C.c_size_t]),
    "rve_set_field": (C.c_int, [rve_handle, C.c_int, _dp, C.c_size_t]),
    "rve_get_scalars": (C.c_int, [rve_handle, C.POINTER(rve_scalars)]),
    "rve_set_scalars": (C.c_int, [rve_handle, C.POINTER(rve_scalars)]),
    "rve_mech_solve": (C.c_int, [rve_handle, C.POINTER(C.c_int)]),
    "rve_damage_solve": (C.c_int, [rve_handle, C.c_double, _dp, C.POINTER(C.c_int)]),
    "rve_dissipation": (C.c_int, [rve_handle, _dp, _dp, _dp]),
    "rve_save": (C.c_int, [rve_handle, C.c_void_p, C.POINTER(C.c_size_t)]),
    "rve_load": (C.c_int, [rve_handle, C.c_void_p, C.c_size_t]),
    "rve_timing_enable": (C.c_int, [rve_handle, C.c_int]),
    "rve_timing_get": (C.c_int, [rve_handle, C.c_int, _dp, C.POINTER(C.c_long), _dp]),
    "rve_timing_get_flops": (C.c_int, [rve_handle, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_long),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "rve_launch_count": (C.c_long, [rve_handle]),
    "rve_tile_config": (C.c_int, [rve_handle, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "rve_destroy": (C.c_int, [rve_handle]),
    "rve_strerror": (C.c_char_p, [C.c_int]),
    "rve_footprint_bytes": (C.c_size_t, [C.POINTER(rve_config)]),
    "rve_server_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(rve_server)]),
    "rve_server_submit": (C.c_int, [rve_server, C.c_long, C.POINTER(rve_config), C.POINTER(rve_micro), C.c_int,
                                    C.c_double]),
    "rve_server_wait": (C.c_int, [rve_server, C.POINTER(rve_request_result), C.c_int, C.c_double,
                                  C.POINTER(C.c_int)]),
    "rve_server_stats": (C.c_int, [rve_server, C.POINTER(C.c_int), C.POINTER(C.c_size_t), C.POINTER(C.c_long)]),
    "rve_server_destroy": (C.c_int, [rve_server]),
    "rve_server_set_batching": (C.c_int, [rve_server, C.c_int]),
    "rve_dissipation_noalloc": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
}

EXPORTED = tuple(_SIGS)
_lib = None


def lib():
    """Load libpff_gb300.so (raises if it has not been built: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_2508_07424_gb300.build.build()")
        L = C.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class RveError(RuntimeError):
    def __init__(self, code, what):
        msg = lib().rve_strerror(code)
        super().__init__(f"{what}: {msg.decode() if msg else code} ({code})")
        self.code = code


def check(code, what):
    if code != RVE_OK:
        raise RveError(code, what)
    return code


def __getattr__(name):
    if name in _SIGS:
        return getattr(lib(), name)
    raise AttributeError(name)
