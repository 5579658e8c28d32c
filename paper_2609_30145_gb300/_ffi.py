"""ctypes declarations of the C ABI in include/sed.h (argument marshalling only).

The shared library is ``_build/libsed.so`` next to this file; it is built by
``paper_2609_30145_gb300.build.build()``.  Loading fails loudly when it is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsed.so")

SED_OK, SED_EINVAL, SED_ENOMEM, SED_ECUDA, SED_ERANGE, SED_ENONFINITE, SED_EBUSY, SED_ETIMEOUT, \
    SED_EUNSUPPORTED = range(9)
PREC_FP32, PREC_FP32_SIMT, PREC_BF16, PREC_FP8 = 0, 1, 2, 3
DUST_POWER_LAW, DUST_KC13 = 0, 1
LSF_R_FWHM, LSF_R_SIGMA, LSF_FWHM_AA, LSF_SIGMA_AA, LSF_SIGMA_KMS, LSF_FWHM_KMS = range(6)
ROW_BAD_THETA, ROW_BAD_Z, ROW_BAD_TMAX, ROW_NONFINITE, ROW_DEVICE_TIMEOUT = 1, 2, 4, 16, 32
KEYS = ("sfh", "logzsol", "afe", "logmass", "zred", "tau_pow", "alpha_pow", "diffuse_tau_kc",
        "diffuse_dust_index", "gas_logz", "gas_logu", "sigma_gal",
        "log_err_scale_phot", "log_f_calib_phot", "log_f_data_phot", "log_jitter_phot",
        "log_err_scale_spec", "log_f_calib_spec", "log_f_data_spec", "log_jitter_spec", "frac_obrun",
        "sigma_gas", "dust_bins", "igm_factor")
FLOOR_ERR_SCALE, FLOOR_F_CALIB, FLOOR_F_DATA, FLOOR_JITTER = 1, 2, 4, 8
SFH_STEP, SFH_LINEAR = 0, 1
FESC_NONE, FESC_RUNAWAY_BC, FESC_PICKET = 0, 1, 2
NKEYS = len(KEYS)
GRID_COPY_FP32, GRID_COPY_FP32_SIMT, GRID_COPY_BF16, GRID_COPY_FP8 = 1, 2, 4, 8
CALIB_MARGINAL, CALIB_OPTIMISED = 0, 1
GAS_SIGMA_TIED, GAS_SIGMA_FIXED, GAS_SIGMA_SAMPLED = 0, 1, 2
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024

P = C.c_void_p


class GridDesc(C.Structure):
    _fields_ = [("n_age", C.c_int), ("n_feh", C.c_int), ("n_afe", C.c_int), ("n_lam", C.c_int),
                ("log_age_yr", P), ("feh", P), ("afe", P), ("lam_aa", P), ("flux", P),
                ("sigma_lib_kms", P), ("neb_n_logu", C.c_int), ("neb_n_logz", C.c_int),
                ("neb_logu", P), ("neb_logz", P), ("neb_log10_lnu_per_q", P), ("precision_mask", C.c_uint),
                ("neb_n_line", C.c_int), ("neb_line_lam_aa", P), ("neb_log10_line_per_q", P),
                ("neb_n_age", C.c_int), ("neb_log_age_yr", P)]


class ModelDesc(C.Structure):
    _fields_ = [("grid", C.c_int32), ("n_sfh", C.c_int), ("zf", C.c_double), ("zmode", C.c_int),
                ("use_afe", C.c_int), ("use_nebular", C.c_int), ("dust_law", C.c_int),
                ("bc_edge_log_age_yr", C.c_double), ("H0", C.c_double), ("Om0", C.c_double),
                ("n_filt", C.c_int), ("filt_len", P), ("filt_lam_aa", P), ("filt_trans", P),
                ("phot_d", P), ("phot_sigma", P), ("phot_mask", P),
                ("n_pix", C.c_int), ("spec_lam_aa", P), ("spec_d", P), ("spec_sigma", P),
                ("spec_mask", P), ("lsf_mode", C.c_int), ("lsf_value", P),
                ("sigma_gal_kms", C.c_double), ("z_ref", C.c_double),
                ("sample_sigma_gal", C.c_int), ("sigma_gal_max_kms", C.c_double),
                ("calib_n", C.c_int), ("calib_sigma", P),
                ("noise_floor_phot", C.c_int), ("noise_floor_spec", C.c_int), ("sfh_scheme", C.c_int),
                ("phot_upper", P), ("fesc_geometry", C.c_int),
                ("fixed", C.c_int * NKEYS), ("fixed_val", C.c_double * NKEYS), ("calib_mode", C.c_int),
                ("use_lines", C.c_int), ("gas_sigma_mode", C.c_int), ("sigma_gas_kms", C.c_double),
                ("sigma_gas_max_kms", C.c_double), ("n_lcat", C.c_int), ("lcat_len", P), ("lcat_line", P),
                ("lcat_d", P), ("lcat_sigma", P), ("lcat_mask", P), ("lcat_upper", P), ("dust_n_bin", C.c_int),
                ("dust_bin_M", P), ("dust_bin_law", P), ("use_igm", C.c_int)]


class StageStats(C.Structure):
    _fields_ = [("ms_prep", C.c_float), ("ms_contract", C.c_float), ("ms_epilogue", C.c_float),
                ("nnz_w", C.c_double), ("dense_k", C.c_double), ("issued_flop", C.c_double), ("n_rows", C.c_int),
                ("n_lam", C.c_int), ("ldn", C.c_int), ("precision", C.c_int), ("is_grad", C.c_int),
                ("ms_dw", C.c_float), ("ms_prep_bwd", C.c_float)]


class ServerDesc(C.Structure):
    _fields_ = [("grid", C.c_int32), ("model_layout", C.c_int32), ("precision", C.c_int),
                ("max_launch_rows", C.c_int), ("n_slots", C.c_int), ("fit_budget_bytes", C.c_size_t)]


class ServerStats(C.Structure):
    _fields_ = [("calls", C.c_uint64), ("launches", C.c_uint64), ("rows", C.c_uint64),
                ("fits_open", C.c_int), ("fit_bytes", C.c_size_t)]


class NssDesc(C.Structure):
    _fields_ = [("n_live", C.c_int), ("n_replace", C.c_int), ("n_slice_steps", C.c_int), ("max_iter", C.c_int),
                ("stop_dlnz", C.c_double), ("slice_width", C.c_double), ("seed", C.c_uint64),
                ("precision", C.c_int), ("lo", P), ("hi", P)]


class NssResult(C.Structure):
    _fields_ = [("lnz", C.c_double), ("info_h", C.c_double), ("n_iter", C.c_int), ("n_dead", C.c_int),
                ("converged", C.c_int), ("n_like", C.c_int64), ("n_rows", C.c_int64)]


# exported symbols and their signatures (name -> (restype, argtypes))
SIGNATURES = {
    "sed_create": (C.c_int, [C.POINTER(P), C.c_int, C.c_size_t]),
    "sed_destroy": (C.c_int, [P]),
    "sed_status_string": (C.c_char_p, [C.c_int]),
    "sed_last_error": (C.c_char_p, [P]),
    "sed_memory_used": (C.c_int, [P, C.POINTER(C.c_size_t)]),
    "sed_last_host_path": (C.c_int, [P, C.POINTER(C.c_int)]),
    "sed_load_grid": (C.c_int, [P, C.POINTER(GridDesc), C.POINTER(C.c_int32)]),
    "sed_create_model": (C.c_int, [P, C.POINTER(ModelDesc), C.POINTER(C.c_int32)]),
    "sed_model_layout": (C.c_int, [P, C.c_int32, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "sed_set_data": (C.c_int, [P, C.c_int32, P, P, P, P]),
    "sed_destroy_model": (C.c_int, [P, C.c_int32]),
    "sed_forward": (C.c_int, [P, C.c_int32, P, C.c_int, C.c_int, P, P, C.c_int, P]),
    "sed_loglike": (C.c_int, [P, C.c_int32, P, C.c_int, C.c_int, P, P, C.c_int, P]),
    "sed_line_fluxes": (C.c_int, [P, C.c_int32, P, C.c_int, C.c_int, P, C.c_int, P]),
    "sed_loglike_grad": (C.c_int, [P, C.c_int32, P, C.c_int, C.c_int, P, P, P, C.c_int, P]),
    "sed_loglike_host": (C.c_int, [P, C.c_int32, P, C.c_int, C.c_int, P, P, C.c_int, P]),
    "sed_loglike_noalloc": (C.c_int, [P, C.c_int32, P, C.c_int, C.c_int, P, P, C.c_int, P]),
    "sed_set_profiling": (C.c_int, [P, C.c_int]),
    "sed_server_create": (C.c_int, [P, C.POINTER(ServerDesc), C.POINTER(P)]),
    "sed_server_destroy": (C.c_int, [P]),
    "sed_server_open_fit": (C.c_int, [P, C.c_int32, C.c_int, C.POINTER(C.c_int)]),
    "sed_server_close_fit": (C.c_int, [P, C.c_int]),
    "sed_server_fit_theta": (P, [P, C.c_int]),
    "sed_server_submit": (C.c_int, [P, C.c_int, P, C.c_int, C.c_int, C.POINTER(C.c_uint64)]),
    "sed_server_submit_device": (C.c_int, [P, C.c_int, C.c_int, C.POINTER(C.c_uint64)]),
    "sed_server_wait": (C.c_int, [P, C.c_uint64, P, P, C.c_int, C.POINTER(C.c_double)]),
    "sed_server_get_stats": (C.c_int, [P, C.POINTER(ServerStats)]),
    "sed_last_stats": (C.c_int, [P, P, C.POINTER(StageStats)]),
    "sed_nss_run": (C.c_int, [P, C.c_int32, C.POINTER(NssDesc), P, P, P, P, C.c_int, C.POINTER(NssResult), P]),
}

_lib = None


def load():
    """Load libsed.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                              "(run paper_2609_30145_gb300.build.build())")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib
