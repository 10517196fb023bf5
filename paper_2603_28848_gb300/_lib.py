"""ctypes declarations of the C ABI in include/best.h (argument marshalling only)."""
import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_uint32, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbest.so")

MAX_LEGS = 6
BEST_OK = 0
STATUS_NAMES = {0: "BEST_OK", 1: "BEST_ERR_INVALID", 2: "BEST_ERR_CUDA", 3: "BEST_ERR_OOM",
                4: "BEST_ERR_NUMERIC", 5: "BEST_ERR_TIMEOUT"}


class best_grid(ctypes.Structure):
    _fields_ = [("n", c_int32), ("log_spaced", c_int32), ("q_min", c_double), ("q_max", c_double)]


MAX_MASS_KNOTS = 8


class best_species(ctypes.Structure):
    _fields_ = [("stat", c_int32), ("n_mass_knots", c_int32), ("mass0", c_double), ("mass1", c_double),
                ("mass_t", c_double * MAX_MASS_KNOTS), ("mass_m", c_double * MAX_MASS_KNOTS)]


class best_process(ctypes.Structure):
    _fields_ = [("n_in", c_int32), ("n_out", c_int32), ("species", c_int32 * MAX_LEGS),
                ("coupling", c_double), ("sigma_E", c_double), ("neval", c_int64),
                ("neval_per_point", POINTER(c_int64)), ("nitn", c_int32), ("nbins", c_int32),
                ("alpha", c_double), ("width_mode", c_int32), ("pad_", c_int32), ("width", c_double),
                ("width_rel_lo", c_double), ("width_rel_hi", c_double), ("width_factor", c_double),
                ("width_min", c_double), ("width_max", c_double), ("strat", c_int32),
                ("strat_max_hcubes", c_int32), ("strat_beta", c_double), ("me_coef", c_double * 4),
                ("budget", c_int32), ("sides", c_int32), ("neval_min", c_int64), ("neval_max", c_int64)]


class best_config(ctypes.Structure):
    _fields_ = [("grid", best_grid), ("n_species", c_int32), ("n_processes", c_int32),
                ("species", POINTER(best_species)), ("processes", POINTER(best_process)),
                ("precision", c_int32), ("tail_points", c_int32), ("seed", c_uint64),
                ("e_cut", c_double), ("expansion", c_int32), ("pad_", c_int32),
                ("a0", c_double), ("t0", c_double), ("eps_dt", c_double),
                ("point_lo", c_int32), ("point_hi", c_int32)]


class BestError(RuntimeError):
    pass


# Every exported symbol with its argument and result types.
SIGNATURES = {
    "best_collision_init": ([POINTER(best_config), POINTER(c_void_p)], c_int32),
    "best_collision_eval": ([c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p], c_int32),
    "best_step_euler": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "best_step_heun": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "best_collision_eval_log": ([c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p], c_int32),
    "best_step_stage": ([c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                         c_void_p], c_int32),
    "best_evolve": ([c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_double, c_void_p], c_int32),
    "best_autotune": ([c_void_p, c_void_p, c_double, POINTER(c_int32), c_void_p], c_int32),
    "best_collision_vjp": ([c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                            c_void_p], c_int32),
    "best_collision_jvp": ([c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "best_step_implicit_euler": ([c_void_p, c_void_p, c_double, c_double, c_int32, c_double, c_int32, c_int32,
                                  c_double, c_void_p, c_void_p], c_int32),
    "best_get_budgets": ([c_void_p, c_void_p, c_void_p], c_int32),
    "best_launch_shape": ([c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)], c_int32),
    "best_moments": ([c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p], c_int32),
    "best_get_strata": ([c_void_p, c_int32, POINTER(c_int32), POINTER(c_int32), c_void_p], c_int32),
    "best_get_widths": ([c_void_p, c_void_p, c_void_p], c_int32),
    "best_species_masses": ([c_void_p, c_double, c_void_p], c_int32),
    "best_set_widths": ([c_void_p, c_void_p], c_int32),
    "best_state_size": ([c_void_p], c_int64),
    "best_save_state": ([c_void_p, c_void_p, c_int64], c_int32),
    "best_load_state": ([c_void_p, c_void_p, c_int64], c_int32),
    "best_num_tasks": ([c_void_p], c_int32),
    "best_num_side_integrals": ([c_void_p], c_int32),
    "best_sweep_samples": ([c_void_p, c_int32], c_int64),
    "best_partition_groups": ([c_void_p, c_int32, c_void_p], c_int32),
    "best_chunk_bounds": ([c_int64, c_int32, c_void_p, c_int32, c_void_p], c_int32),
    "best_get_task_results": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "best_map_stride": ([c_void_p], c_int64),
    "best_get_maps": ([c_void_p, c_void_p], c_int32),
    "best_set_maps": ([c_void_p, c_void_p], c_int32),
    "best_get_call_counter": ([c_void_p, POINTER(c_uint32)], c_int32),
    "best_set_call_counter": ([c_void_p, c_uint32], c_int32),
    "best_check": ([c_void_p, c_void_p], c_int32),
    "best_last_launch_count": ([c_void_p], c_int32),
    "best_profile_enable": ([c_void_p, c_int32], c_int32),
    "best_profile_read": ([c_void_p, POINTER(c_double), POINTER(c_int64)], c_int32),
    "best_last_error": ([c_void_p], c_char_p),
    "best_collision_destroy": ([c_void_p], None),
    "best_vegas_iteration_noalloc": ([POINTER(best_config), c_int32, c_void_p, c_double, c_void_p, c_uint32,
                                      c_uint32, c_void_p, c_void_p], c_int32),
}

_lib = None


def load(path=LIB_PATH):
    """Load libbest.so; raises if it has not been built (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise BestError(f"{path} is missing: build it with paper_2603_28848_gb300.build()")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(status, ctx=None):
    if status != BEST_OK:
        msg = load().best_last_error(ctx).decode()
        raise BestError(f"{STATUS_NAMES.get(status, status)}: {msg}")
