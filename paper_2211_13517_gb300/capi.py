"""ctypes binding of libfdas.so -- argument marshalling only.

Every function here has the name of the C entry point it calls (see
include/fdas.h for the semantics).  No step of the search runs in Python:
the binding converts arguments, calls the library and turns a non-OK status
into an exception.  If the library is missing, `lib()` raises; there is no
fallback.

`Plan` is a small convenience wrapper that takes torch tensors (device memory
and streams only) and calls the same entry points.

With FDAS_CHECKED=1 in the environment when the library is first loaded,
`lib()` loads the checked build (libfdas_checked.so, built by
build.build(checked=True)) instead: the same entry points with device bounds
checks and workspace canaries (include/fdas.h, "Checked build").
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_int32, c_int64,
                    c_uint16, c_uint32, c_void_p, c_float)

import numpy as np

from .build import LIB, LIB_CHECKED

FDAS_OK = 0
FDAS_ERR_ARG = 1
FDAS_ERR_CUDA = 2
FDAS_ERR_OOM = 3
FDAS_ERR_CAND_OVERFLOW = 4
FDAS_ERR_NONFINITE = 5
FDAS_ERR_TIMEOUT = 6
FDAS_ERR_UNSUPPORTED = 7
FDAS_ERR_CAND_STORE_FULL = 8
FDAS_ERR_BOUNDS = 9
STATUS_NAMES = {0: "FDAS_OK", 1: "FDAS_ERR_ARG", 2: "FDAS_ERR_CUDA", 3: "FDAS_ERR_OOM",
                4: "FDAS_ERR_CAND_OVERFLOW", 5: "FDAS_ERR_NONFINITE",
                6: "FDAS_ERR_TIMEOUT", 7: "FDAS_ERR_UNSUPPORTED",
                8: "FDAS_ERR_CAND_STORE_FULL", 9: "FDAS_ERR_BOUNDS"}
# statuses fdas_search / fdas_threshold return (not raise): the call ran and
# *n_found holds the true number of crossings
COUNT_STATUSES = (FDAS_ERR_CAND_OVERFLOW, FDAS_ERR_CAND_STORE_FULL)

FDAS_FP32, FDAS_BF16, FDAS_FP16 = 0, 1, 2
FDAS_THRESH_GAMMA_TAIL, FDAS_THRESH_MEAN_PLUS_KSIGMA = 0, 1
FDAS_NORM_MEDIAN, FDAS_NORM_NONE = 0, 1
FDAS_CORR_AUTO, FDAS_CORR_FFT, FDAS_CORR_TENSOR, FDAS_CORR_TENSOR_SPLIT = 0, 1, 2, 3
FDAS_HARM_TOP, FDAS_HARM_FUNDAMENTAL = 0, 1
FDAS_TORDER_DEFAULT, FDAS_TORDER_Z, FDAS_TORDER_PAIRED = 0, 1, 2

EXPORTED = ["fdas_opts_default", "fdas_plan_create", "fdas_plan_destroy",
            "fdas_plan_get_info", "fdas_search", "fdas_search_async", "fdas_spectrum",
            "fdas_power_plane",
            "fdas_correlation_plane",
            "fdas_harmonic_sums", "fdas_threshold", "fdas_template_bank",
            "fdas_spectrum_static", "fdas_fourier_power", "fdas_fourier_power_backward",
            "fdas_refine", "fdas_profile_enable", "fdas_profile_read",
            "fdas_selftest_wait_timeout", "fdas_last_error", "fdas_version",
            "fdas_checked_build",
            "fdas_dedisp_plan_create", "fdas_dedisp_plan_destroy", "fdas_dedisp_get_info",
            "fdas_dedisp_delays", "fdas_dedisperse", "fdas_dedisperse_u8"]


class fdas_opts(Structure):
    _fields_ = [("precision", c_int32), ("threshold_sigma", c_double),
                ("threshold_mode", c_int32), ("norm_mode", c_int32),
                ("norm_block", c_int32), ("max_candidates", c_int64),
                ("autotune", c_int32), ("use_graph", c_int32),
                ("correlator", c_int32), ("harmonic_mode", c_int32),
                ("interbin", c_int32), ("template_order", c_int32)]


class fdas_series(Structure):
    _fields_ = [("data", c_void_p), ("n_samples", c_int64), ("decimation", c_int32),
                ("trial_id", c_uint32)]


class fdas_candidate(Structure):
    _fields_ = [("trial_id", c_uint32), ("ir", c_uint32), ("iz", c_uint16),
                ("harm", c_uint16), ("power", c_float), ("sigma", c_float)]


CANDIDATE_DTYPE = np.dtype([("trial_id", np.uint32), ("ir", np.uint32), ("iz", np.uint16),
                            ("harm", np.uint16), ("power", np.float32), ("sigma", np.float32)])


class fdas_plan_info(Structure):
    _fields_ = [("n_samples", c_int64), ("n_r", c_int64),
                ("n_z", c_int32), ("iz0", c_int32), ("m_max", c_int32), ("m_overlap", c_int32),
                ("seg_len", c_int32), ("valid_per_seg", c_int32), ("n_seg", c_int32),
                ("n_harm", c_int32), ("n_stages", c_int32), ("precision", c_int32),
                ("norm_block", c_int32), ("threshold_mode", c_int32),
                ("tsamp", c_double), ("z_max", c_double), ("z_step", c_double),
                ("threshold_sigma", c_double), ("stage_factor", c_double * 6),
                ("workspace_bytes", c_int64), ("z_chunks", c_int32), ("use_graph", c_int32),
                ("tuned_ms", c_double), ("correlator", c_int32), ("harmonic_mode", c_int32),
                ("interbin", c_int32), ("template_order", c_int32), ("plane_cols", c_int64)]


class fdas_seed(Structure):
    _fields_ = [("r", c_double), ("z", c_double), ("trial_id", c_uint32), ("reserved", c_uint32)]


class fdas_refined(Structure):
    _fields_ = [("r", c_double), ("z", c_double), ("power", c_float), ("dpdr", c_float),
                ("dpdz", c_float), ("steps", c_int32), ("trial_id", c_uint32),
                ("reserved", c_uint32)]


SEED_DTYPE = np.dtype([("r", np.float64), ("z", np.float64), ("trial_id", np.uint32),
                       ("reserved", np.uint32)])
REFINED_DTYPE = np.dtype([("r", np.float64), ("z", np.float64), ("power", np.float32),
                          ("dpdr", np.float32), ("dpdz", np.float32), ("steps", np.int32),
                          ("trial_id", np.uint32), ("reserved", np.uint32)])


class fdas_profile(Structure):
    _fields_ = [("trials", c_int64), ("launches", c_int64 * 4), ("timed", c_int64 * 4),
                ("ms", c_double * 4)]


FDAS_PROF_SPECTRUM, FDAS_PROF_CORRELATE, FDAS_PROF_HARMONIC, FDAS_PROF_FINISH = 0, 1, 2, 3
PROFILE_GROUPS = ["spectrum", "correlate", "harmonic", "finish"]   # index = FDAS_PROF_*


class fdas_dedisp_info(Structure):
    _fields_ = [("n_chan", c_int32), ("n_dm", c_int32), ("n_t", c_int64), ("n_out", c_int64),
                ("f_top_mhz", c_double), ("df_mhz", c_double), ("tsamp", c_double),
                ("dm_lo", c_double), ("dm_step", c_double), ("max_delay", c_int32),
                ("tile_span", c_int32), ("workspace_bytes", c_int64)]


class FdasError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib_path() -> str:
    """The library lib() loads: the checked build when FDAS_CHECKED=1."""
    return LIB_CHECKED if os.environ.get("FDAS_CHECKED") == "1" else LIB


def lib() -> ctypes.CDLL:
    """Load libfdas.so (built in-tree by build.build()), or libfdas_checked.so
    with FDAS_CHECKED=1; raise if absent."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} is not built ({path}); run "
                               "paper_2211_13517_gb300.build.build("
                               f"{'checked=True' if path == LIB_CHECKED else ''}) first")
        L = ctypes.CDLL(path)
        L.fdas_opts_default.argtypes = [POINTER(fdas_opts)]
        L.fdas_opts_default.restype = None
        L.fdas_plan_create.argtypes = [POINTER(c_void_p), c_int64, c_double, c_double,
                                       c_double, c_int32, c_int32, POINTER(fdas_opts)]
        L.fdas_plan_create.restype = c_int32
        L.fdas_dedisp_plan_create.argtypes = [POINTER(c_void_p), c_int32, c_int64, c_double,
                                              c_double, c_double, c_double, c_double, c_int32,
                                              c_int64]
        L.fdas_dedisp_plan_create.restype = c_int32
        L.fdas_dedisp_plan_destroy.argtypes = [c_void_p]
        L.fdas_dedisp_plan_destroy.restype = None
        L.fdas_dedisp_get_info.argtypes = [c_void_p, POINTER(fdas_dedisp_info)]
        L.fdas_dedisp_get_info.restype = c_int32
        L.fdas_dedisp_delays.argtypes = [c_void_p, c_void_p]
        L.fdas_dedisp_delays.restype = c_int32
        L.fdas_dedisperse.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
        L.fdas_dedisperse.restype = c_int32
        L.fdas_dedisperse_u8.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
        L.fdas_dedisperse_u8.restype = c_int32
        L.fdas_plan_destroy.argtypes = [c_void_p]
        L.fdas_plan_destroy.restype = None
        L.fdas_plan_get_info.argtypes = [c_void_p, POINTER(fdas_plan_info)]
        L.fdas_plan_get_info.restype = c_int32
        L.fdas_search.argtypes = [c_void_p, POINTER(fdas_series), c_int32, c_void_p, c_int64,
                                  POINTER(c_int64), c_void_p]
        L.fdas_search.restype = c_int32
        L.fdas_search_async.argtypes = [c_void_p, POINTER(fdas_series), c_int32, c_void_p, c_int64,
                                        c_void_p, c_void_p, c_void_p]
        L.fdas_search_async.restype = c_int32
        L.fdas_spectrum.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.fdas_spectrum.restype = c_int32
        L.fdas_power_plane.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.fdas_power_plane.restype = c_int32
        L.fdas_correlation_plane.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
        L.fdas_correlation_plane.restype = c_int32
        L.fdas_harmonic_sums.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
        L.fdas_harmonic_sums.restype = c_int32
        L.fdas_threshold.argtypes = [c_void_p, c_void_p, c_void_p, c_uint32, c_void_p, c_int64,
                                     POINTER(c_int64), c_void_p]
        L.fdas_threshold.restype = c_int32
        L.fdas_template_bank.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.fdas_template_bank.restype = c_int32
        L.fdas_spectrum_static.argtypes = [c_void_p, c_int64, c_int32, c_int32, c_int32,
                                           c_void_p, c_void_p, c_void_p]
        L.fdas_spectrum_static.restype = c_int32
        L.fdas_fourier_power.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_void_p,
                                         c_void_p, c_void_p]
        L.fdas_fourier_power.restype = c_int32
        L.fdas_fourier_power_backward.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_void_p,
                                                  c_void_p, c_void_p, c_void_p]
        L.fdas_fourier_power_backward.restype = c_int32
        L.fdas_refine.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p,
                                  c_void_p]
        L.fdas_refine.restype = c_int32
        L.fdas_selftest_wait_timeout.argtypes = [c_void_p, c_int64, c_void_p]
        L.fdas_selftest_wait_timeout.restype = c_int32
        L.fdas_profile_enable.argtypes = [c_void_p, c_int32]
        L.fdas_profile_enable.restype = c_int32
        L.fdas_profile_read.argtypes = [c_void_p, POINTER(fdas_profile)]
        L.fdas_profile_read.restype = c_int32
        L.fdas_last_error.argtypes = []
        L.fdas_last_error.restype = c_char_p
        L.fdas_version.argtypes = []
        L.fdas_version.restype = c_char_p
        L.fdas_checked_build.argtypes = []
        L.fdas_checked_build.restype = c_int32
        _lib = L
    return _lib


def _check(status: int, where: str, allow=()):
    if status != FDAS_OK and status not in allow:
        raise FdasError(status, where, fdas_last_error())
    return status


# ----------------------------------------------------------------------------
# the C entry points, same names
# ----------------------------------------------------------------------------
def fdas_opts_default() -> fdas_opts:
    o = fdas_opts()
    lib().fdas_opts_default(ctypes.byref(o))
    return o


def fdas_plan_create(n_samples, tsamp, z_max, z_step, seg_len, n_harm, opts=None) -> c_void_p:
    h = c_void_p()
    _check(lib().fdas_plan_create(ctypes.byref(h), n_samples, tsamp, z_max, z_step, seg_len,
                                  n_harm, ctypes.byref(opts) if opts is not None else None),
           "fdas_plan_create")
    return h


def fdas_plan_destroy(plan) -> None:
    lib().fdas_plan_destroy(plan)


def fdas_plan_get_info(plan) -> fdas_plan_info:
    info = fdas_plan_info()
    _check(lib().fdas_plan_get_info(plan, ctypes.byref(info)), "fdas_plan_get_info")
    return info


def fdas_dedisp_plan_create(n_chan, n_t, f_top_mhz, df_mhz, tsamp, dm_lo, dm_step, n_dm,
                            n_out) -> c_void_p:
    h = c_void_p()
    _check(lib().fdas_dedisp_plan_create(ctypes.byref(h), n_chan, n_t, f_top_mhz, df_mhz, tsamp,
                                         dm_lo, dm_step, n_dm, n_out), "fdas_dedisp_plan_create")
    return h


def fdas_dedisp_plan_destroy(plan) -> None:
    lib().fdas_dedisp_plan_destroy(plan)


def fdas_dedisp_get_info(plan) -> fdas_dedisp_info:
    info = fdas_dedisp_info()
    _check(lib().fdas_dedisp_get_info(plan, ctypes.byref(info)), "fdas_dedisp_get_info")
    return info


def fdas_dedisp_delays(plan, delays_ptr) -> None:
    _check(lib().fdas_dedisp_delays(plan, delays_ptr), "fdas_dedisp_delays")


def fdas_dedisperse(plan, filterbank_ptr, out_ptr, stream=None) -> None:
    _check(lib().fdas_dedisperse(plan, filterbank_ptr, out_ptr, stream), "fdas_dedisperse")


def fdas_dedisperse_u8(plan, filterbank_ptr, out_ptr, stream=None) -> None:
    _check(lib().fdas_dedisperse_u8(plan, filterbank_ptr, out_ptr, stream), "fdas_dedisperse_u8")


def fdas_search(plan, batch, n_series, cands_ptr, capacity, stream=None):
    """Returns (status, n_found); FDAS_ERR_CAND_OVERFLOW and
    FDAS_ERR_CAND_STORE_FULL are returned, not raised."""
    n = c_int64(0)
    st = lib().fdas_search(plan, batch, n_series, cands_ptr, capacity, ctypes.byref(n), stream)
    _check(st, "fdas_search", allow=COUNT_STATUSES)
    return st, n.value


def fdas_search_async(plan, batch, n_series, cands_ptr, capacity, n_found_ptr, status_ptr,
                      stream=None):
    """Queues the search on `stream`; *n_found_ptr and *status_ptr (device or
    page-locked host) receive the results when the stream reaches them."""
    _check(lib().fdas_search_async(plan, batch, n_series, cands_ptr, capacity, n_found_ptr,
                                   status_ptr, stream), "fdas_search_async")


def fdas_spectrum(plan, series_ptr, spectrum_ptr, medians_ptr=None, stream=None):
    _check(lib().fdas_spectrum(plan, series_ptr, spectrum_ptr, medians_ptr, stream), "fdas_spectrum")


def fdas_power_plane(plan, spectrum_ptr, plane_ptr, stats_ptr=None, stream=None):
    _check(lib().fdas_power_plane(plan, spectrum_ptr, plane_ptr, stats_ptr, stream),
           "fdas_power_plane")


def fdas_correlation_plane(plan, spectrum_ptr, corr_ptr, stream=None):
    _check(lib().fdas_correlation_plane(plan, spectrum_ptr, corr_ptr, stream),
           "fdas_correlation_plane")


def fdas_harmonic_sums(plan, plane_ptr, sums_ptr, stream=None):
    _check(lib().fdas_harmonic_sums(plan, plane_ptr, sums_ptr, stream), "fdas_harmonic_sums")


def fdas_threshold(plan, plane_ptr, stats_ptr, trial_id, cands_ptr, capacity, stream=None):
    n = c_int64(0)
    st = lib().fdas_threshold(plan, plane_ptr, stats_ptr, trial_id, cands_ptr, capacity,
                              ctypes.byref(n), stream)
    _check(st, "fdas_threshold", allow=COUNT_STATUSES)
    return st, n.value


def fdas_template_bank(plan, taps_ptr=None, energy_ptr=None, bank_ptr=None, stream=None):
    _check(lib().fdas_template_bank(plan, taps_ptr, energy_ptr, bank_ptr, stream),
           "fdas_template_bank")


def fdas_spectrum_static(series_ptr, n_samples, precision, norm_mode, norm_block,
                         spectrum_ptr, medians_ptr=None, stream=None):
    _check(lib().fdas_spectrum_static(series_ptr, n_samples, precision, norm_mode, norm_block,
                                      spectrum_ptr, medians_ptr, stream), "fdas_spectrum_static")


def fdas_fourier_power(plan, spectrum_ptr, rz_ptr, n, power_ptr, grad_ptr=None, stream=None):
    _check(lib().fdas_fourier_power(plan, spectrum_ptr, rz_ptr, n, power_ptr, grad_ptr, stream),
           "fdas_fourier_power")


def fdas_fourier_power_backward(plan, spectrum_ptr, rz_ptr, n, grad_power_ptr,
                                grad_spectrum_ptr=None, grad_rz_ptr=None, stream=None):
    _check(lib().fdas_fourier_power_backward(plan, spectrum_ptr, rz_ptr, n, grad_power_ptr,
                                             grad_spectrum_ptr, grad_rz_ptr, stream),
           "fdas_fourier_power_backward")


def fdas_refine(plan, spectrum_ptr, seeds_ptr, n, n_steps, out_ptr, stream=None):
    _check(lib().fdas_refine(plan, spectrum_ptr, seeds_ptr, n, n_steps, out_ptr, stream),
           "fdas_refine")


def fdas_selftest_wait_timeout(plan, limit_cycles, stream=None) -> int:
    """Status of the bounded-wait check: FDAS_ERR_TIMEOUT when the wait gave
    up as it should (returned, not raised), FDAS_OK if it did not."""
    st = lib().fdas_selftest_wait_timeout(plan, limit_cycles, stream)
    _check(st, "fdas_selftest_wait_timeout", allow=(FDAS_ERR_TIMEOUT,))
    return st


def fdas_profile_enable(plan, on: bool) -> None:
    _check(lib().fdas_profile_enable(plan, 1 if on else 0), "fdas_profile_enable")


def fdas_profile_read(plan) -> fdas_profile:
    out = fdas_profile()
    _check(lib().fdas_profile_read(plan, ctypes.byref(out)), "fdas_profile_read")
    return out


def fdas_last_error() -> str:
    return lib().fdas_last_error().decode()


def fdas_version() -> str:
    return lib().fdas_version().decode()


def fdas_checked_build() -> bool:
    return lib().fdas_checked_build() == 1


# ----------------------------------------------------------------------------
# torch convenience wrapper (device memory and streams only)
# ----------------------------------------------------------------------------
def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream)


class Plan:
    """Owns an fdas_plan; methods take torch tensors and call the C ABI."""

    def __init__(self, n_samples, tsamp=64e-6, z_max=96.0, z_step=1.0, seg_len=8192,
                 n_harm=16, precision=FDAS_FP32, threshold_sigma=6.0,
                 threshold_mode=FDAS_THRESH_GAMMA_TAIL, norm_mode=FDAS_NORM_MEDIAN,
                 norm_block=2048, max_candidates=1 << 20, autotune=False, use_graph=False,
                 correlator=None, harmonic_mode=FDAS_HARM_TOP, interbin=False,
                 template_order=FDAS_TORDER_DEFAULT):
        o = fdas_opts_default()
        o.precision = precision
        o.threshold_sigma = threshold_sigma
        o.threshold_mode = threshold_mode
        o.norm_mode = norm_mode
        o.norm_block = norm_block
        o.max_candidates = max_candidates
        o.autotune = 1 if autotune else 0
        o.use_graph = 1 if use_graph else 0
        if correlator is not None:
            o.correlator = correlator
        o.harmonic_mode = harmonic_mode
        o.interbin = 1 if interbin else 0
        o.template_order = template_order
        self.handle = fdas_plan_create(n_samples, tsamp, z_max, z_step, seg_len, n_harm, o)
        self.info = fdas_plan_get_info(self.handle)

    def close(self):
        if self.handle:
            fdas_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # dtypes of the plan's storage
    @property
    def spec_dtype(self):
        import torch
        return {FDAS_FP32: torch.float32, FDAS_BF16: torch.bfloat16,
                FDAS_FP16: torch.float16}[self.info.precision]

    def search(self, series, trial_ids=None, capacity=1 << 16, stream=None, out=None):
        """series: list of 1-D float32 tensors (device or host).  Returns
        (status, numpy structured array of the first min(n, capacity)
        candidates -- none with FDAS_ERR_CAND_STORE_FULL --, n_found)."""
        n = len(series)
        batch = (fdas_series * max(n, 1))()
        for i, x in enumerate(series):
            batch[i].data = x.data_ptr()
            batch[i].n_samples = x.numel()
            batch[i].decimation = 1
            batch[i].trial_id = i if trial_ids is None else int(trial_ids[i])
        if out is None:
            out = np.zeros(capacity, dtype=CANDIDATE_DTYPE)
        st, nf = fdas_search(self.handle, batch, n, out.ctypes.data_as(c_void_p), out.shape[0],
                             _stream_ptr(stream))
        k = 0 if st == FDAS_ERR_CAND_STORE_FULL else min(nf, out.shape[0])
        return st, out[:k], nf

    def search_async(self, series, cands, n_found, status, trial_ids=None, stream=None):
        """Stream-ordered search.  cands: uint8 tensor of capacity x 20 bytes
        (device or pinned host); n_found: int64 tensor of 1, status: int32
        tensor of 1 (device or pinned host).  Returns at once; after the
        stream is synchronised, cands holds the first min(n_found, capacity)
        records (none with FDAS_ERR_CAND_STORE_FULL) and status the code
        fdas_search would have returned.  The series and the output tensors
        must stay alive until then."""
        n = len(series)
        batch = (fdas_series * max(n, 1))()
        for i, x in enumerate(series):
            batch[i].data = x.data_ptr()
            batch[i].n_samples = x.numel()
            batch[i].decimation = 1
            batch[i].trial_id = i if trial_ids is None else int(trial_ids[i])
        capacity = cands.numel() // CANDIDATE_DTYPE.itemsize
        fdas_search_async(self.handle, batch, n, c_void_p(cands.data_ptr()), capacity,
                          c_void_p(n_found.data_ptr()), c_void_p(status.data_ptr()),
                          _stream_ptr(stream))

    @staticmethod
    def candidates(cands, n):
        """The first n records of a candidate buffer (a tensor of bytes) as a
        numpy structured array."""
        raw = cands[:n * CANDIDATE_DTYPE.itemsize].cpu().numpy()
        return raw.view(CANDIDATE_DTYPE)

    def profile(self, on=None):
        """Enable/disable tracing (resetting it) or, with no argument, read it
        as a dict {group: (launches, timed intervals, ms)}."""
        if on is not None:
            fdas_profile_enable(self.handle, on)
            return None
        p = fdas_profile_read(self.handle)
        return {"trials": p.trials, **{g: (p.launches[i], p.timed[i], p.ms[i])
                                         for i, g in enumerate(PROFILE_GROUPS)}}

    def spectrum(self, x, stream=None, medians=False):
        import torch
        nr = self.info.n_r
        spec = torch.empty(2 * nr, dtype=self.spec_dtype, device=x.device)
        med = None
        if medians:
            med = torch.empty(max(1, nr // min(self.info.norm_block, nr)), dtype=torch.float32,
                              device=x.device)
        fdas_spectrum(self.handle, c_void_p(x.data_ptr()), c_void_p(spec.data_ptr()),
                      c_void_p(med.data_ptr()) if med is not None else None, _stream_ptr(stream))
        return (spec, med) if medians else spec

    def power_plane(self, spec, stream=None):
        import torch
        plane = torch.empty((self.info.n_z, self.info.plane_cols), dtype=self.spec_dtype,
                            device=spec.device)
        stats = torch.empty(2, dtype=torch.float64, device=spec.device)
        fdas_power_plane(self.handle, c_void_p(spec.data_ptr()), c_void_p(plane.data_ptr()),
                         c_void_p(stats.data_ptr()), _stream_ptr(stream))
        return plane, stats

    def correlation_plane(self, spec, stream=None):
        """Complex F[n_z][N_r] as a (n_z, 2 N_r) tensor of (re, im) pairs."""
        import torch
        corr = torch.empty((self.info.n_z, 2 * self.info.n_r), dtype=self.spec_dtype,
                           device=spec.device)
        fdas_correlation_plane(self.handle, c_void_p(spec.data_ptr()), c_void_p(corr.data_ptr()),
                               _stream_ptr(stream))
        return corr

    def harmonic_sums(self, plane, stream=None):
        import torch
        out = torch.empty((self.info.n_stages, self.info.n_z, self.info.plane_cols),
                          dtype=torch.float32, device=plane.device)
        fdas_harmonic_sums(self.handle, c_void_p(plane.data_ptr()), c_void_p(out.data_ptr()),
                           _stream_ptr(stream))
        return out

    def threshold(self, plane, stats, trial_id=0, capacity=1 << 16, stream=None):
        out = np.zeros(capacity, dtype=CANDIDATE_DTYPE)
        st, nf = fdas_threshold(self.handle, c_void_p(plane.data_ptr()),
                                c_void_p(stats.data_ptr()), trial_id,
                                out.ctypes.data_as(c_void_p), capacity, _stream_ptr(stream))
        k = 0 if st == FDAS_ERR_CAND_STORE_FULL else min(nf, capacity)
        return st, out[:k], nf

    # -- refinement (spectrum: complex64 device tensor of N_r bins) ------------
    def fourier_power(self, spectrum, rz, stream=None):
        """(P float32[n], grad float32[n, 2]) at rz (float64 device tensor [n, 2])."""
        import torch
        sp = torch.view_as_real(spectrum.contiguous())
        rz = rz.contiguous()
        n = rz.shape[0]
        P = torch.empty(n, dtype=torch.float32, device=rz.device)
        g = torch.empty((n, 2), dtype=torch.float32, device=rz.device)
        fdas_fourier_power(self.handle, c_void_p(sp.data_ptr()), c_void_p(rz.data_ptr()), n,
                           c_void_p(P.data_ptr()), c_void_p(g.data_ptr()), _stream_ptr(stream))
        return P, g

    def refine(self, spectrum, seeds, n_steps=50, stream=None):
        """seeds: numpy SEED_DTYPE array (host); returns a REFINED_DTYPE array."""
        import torch
        sp = torch.view_as_real(spectrum.contiguous())
        seeds = np.ascontiguousarray(seeds, dtype=SEED_DTYPE)
        out = np.zeros(seeds.shape[0], dtype=REFINED_DTYPE)
        fdas_refine(self.handle, c_void_p(sp.data_ptr()), seeds.ctypes.data_as(c_void_p),
                    seeds.shape[0], n_steps, out.ctypes.data_as(c_void_p), _stream_ptr(stream))
        return out

    def template_bank(self):
        """(taps list per z of complex128 arrays, energies)."""
        info = self.info
        m = [8 + int(np.ceil(abs(i - info.iz0) * info.z_step / 2.0 - 1e-9))
             for i in range(info.n_z)]
        n_taps = sum(2 * mm + 1 for mm in m)
        taps = np.zeros(2 * n_taps, dtype=np.float64)
        energy = np.zeros(info.n_z, dtype=np.float64)
        fdas_template_bank(self.handle, taps.ctypes.data_as(c_void_p),
                           energy.ctypes.data_as(c_void_p), None, None)
        c = taps[0::2] + 1j * taps[1::2]
        out, acc = [], 0
        for mm in m:
            out.append(c[acc:acc + 2 * mm + 1])
            acc += 2 * mm + 1
        return out, energy


def _fourier_power_function():
    import torch

    class FourierPower(torch.autograd.Function):
        """P(r, z) of a complex64 spectrum at float64 points rz [n, 2]; the
        backward pass runs the library's backward kernel."""

        @staticmethod
        def forward(ctx, plan, spectrum, rz):
            P, _ = plan.fourier_power(spectrum, rz)
            ctx.plan = plan
            ctx.save_for_backward(spectrum, rz)
            return P

        @staticmethod
        def backward(ctx, gP):
            spectrum, rz = ctx.saved_tensors
            plan = ctx.plan
            gP = gP.contiguous().to(torch.float32)
            g_spec = g_rz = None
            want_s, want_rz = ctx.needs_input_grad[1], ctx.needs_input_grad[2]
            sp = torch.view_as_real(spectrum.contiguous())
            if want_s:
                g_spec = torch.zeros_like(spectrum)
            if want_rz:
                g_rz = torch.empty_like(rz)
            fdas_fourier_power_backward(
                plan.handle, c_void_p(sp.data_ptr()), c_void_p(rz.contiguous().data_ptr()),
                rz.shape[0], c_void_p(gP.data_ptr()),
                c_void_p(torch.view_as_real(g_spec).data_ptr()) if want_s else None,
                c_void_p(g_rz.data_ptr()) if want_rz else None, _stream_ptr(None))
            return None, g_spec, g_rz

    return FourierPower


_FP = None


def FourierPower():
    """The torch.autograd.Function for P(r, z) (built on first use)."""
    global _FP
    if _FP is None:
        _FP = _fourier_power_function()
    return _FP


class DedispPlan:
    """Owns an fdas_dedisp_plan: incoherent dedispersion of a filterbank
    (device float32 or uint8 [n_chan][n_t]) into n_dm DM-trial series of
    n_out samples."""

    def __init__(self, n_chan, n_t, f_top_mhz, df_mhz, tsamp, dm_lo, dm_step, n_dm, n_out):
        self.handle = fdas_dedisp_plan_create(n_chan, n_t, f_top_mhz, df_mhz, tsamp, dm_lo,
                                              dm_step, n_dm, n_out)
        self.info = fdas_dedisp_get_info(self.handle)

    def close(self):
        if self.handle:
            fdas_dedisp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def delays(self):
        d = np.zeros((self.info.n_dm, self.info.n_chan), dtype=np.int32)
        fdas_dedisp_delays(self.handle, d.ctypes.data_as(c_void_p))
        return d

    def dedisperse(self, filterbank, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.info.n_dm, self.info.n_out), dtype=torch.float32,
                              device=filterbank.device)
        fn = fdas_dedisperse_u8 if filterbank.dtype == torch.uint8 else fdas_dedisperse
        fn(self.handle, c_void_p(filterbank.data_ptr()), c_void_p(out.data_ptr()),
           _stream_ptr(stream))
        return out
