"""ctypes binding of libsrs.so (include/srs.h): argument marshalling only.

Every step of the search runs in the library's CUDA kernels; this module
converts numpy arrays (host) or torch CUDA tensors (device) into pointers and
sizes, calls the C entry point of the same name, and raises SrsError on a
non-zero status.  There is no CPU path: if the library cannot be built or
loaded, the first call raises.
"""
import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

SRS_OK = 0
STATUS = {0: "SRS_OK", -1: "SRS_ERR_ARG", -2: "SRS_ERR_OOM", -3: "SRS_ERR_CUDA", -4: "SRS_ERR_TIMEOUT",
          -5: "SRS_ERR_UNSUPPORTED", -6: "SRS_ERR_DOMAIN"}
SRS_F32, SRS_F64 = 0, 1
SRS_PLAIN_FP64, SRS_MIXED = 0, 1

# Entry points declared in include/srs.h (checked by the tests).
EXPORTS = ("srs_create", "srs_destroy", "srs_last_error", "srs_plan", "srs_search", "srs_search_async", "srs_sync",
           "srs_segment_spectra", "srs_segment_spectra_cufft", "srs_time_map", "srs_segment_spectra_static", "srs_make_strain",
           "srs_patches", "srs_mlp_forward", "srs_mlp_grad", "srs_mlp_train", "srs_score_map", "srs_refine",
           "srs_search_proposed", "srs_power_cube", "srs_stack_slide", "srs_slide_search", "srs_selftest_wait",
           "srs_nsigma_threshold", "srs_detection_noncentrality", "srs_detection_probability",
           "srs_cube_whiten")
SRS_SLIDE_FIRST, SRS_SLIDE_LAST = 1, 2
SRS_WEIGHT_EQUAL, SRS_WEIGHT_AMPLITUDE = 0, 1
MLP_INPUTS, MLP_HIDDEN, MLP_PARAMS = 297, 64, 19137


class SrsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("fs", ctypes.c_double), ("t_coh", ctypes.c_double), ("f_lo", ctypes.c_double),
                ("f_hi", ctypes.c_double), ("f_ref", ctypes.c_double), ("eps", ctypes.c_double),
                ("sigma", ctypes.c_double), ("top_k", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("cut_segments", ctypes.c_int32), ("io_on_device", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("deterministic", ctypes.c_int32)]


class _PlanInfo(ctypes.Structure):
    _fields_ = [("n_s", ctypes.c_int64), ("n_seg_total", ctypes.c_int32), ("n_bins", ctypes.c_int32),
                ("n_fine", ctypes.c_int32), ("w", ctypes.c_int32), ("beta_es", ctypes.c_double),
                ("sigma", ctypes.c_double), ("n_spectra", ctypes.c_int64), ("chunk", ctypes.c_int32),
                ("n_items", ctypes.c_int32)]


class Candidate(ctypes.Structure):
    _fields_ = [("value", ctypes.c_float), ("template_idx", ctypes.c_int32), ("bin", ctypes.c_int32)]


class _Report(ctypes.Structure):
    _fields_ = [("device_ms", ctypes.c_double), ("spectra_per_s", ctypes.c_double),
                ("n_spectra", ctypes.c_int64), ("w", ctypes.c_int32), ("n_fine", ctypes.c_int32),
                ("sigma", ctypes.c_double), ("beta_es", ctypes.c_double), ("chunk", ctypes.c_int32),
                ("n_items", ctypes.c_int32), ("kernel_launches", ctypes.c_int32), ("spread_ms", ctypes.c_double),
                ("cta_threads", ctypes.c_int32), ("staging", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("fft_ms", ctypes.c_double), ("slide_ms", ctypes.c_double), ("slide_reads", ctypes.c_int64)]


class _Bank(ctypes.Structure):
    _fields_ = [("beta_min", ctypes.c_double), ("beta_max", ctypes.c_double), ("n_beta", ctypes.c_int32)]


class _SlideGrid(ctypes.Structure):
    _fields_ = [("f0", ctypes.c_double), ("mc", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("n_rows", ctypes.c_int32), ("n_t0", ctypes.c_int32), ("weighting", ctypes.c_int32),
                ("s_eff", ctypes.c_void_p), ("whiten", ctypes.c_int32)]


class _Injection(ctypes.Structure):
    _fields_ = [("mc", ctypes.c_double), ("f0", ctypes.c_double), ("amp", ctypes.c_double),
                ("phi0", ctypes.c_double)]


class _TrainCfg(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class _ProposalParams(ctypes.Structure):
    _fields_ = [("score_threshold", ctypes.c_float), ("nms_templates", ctypes.c_int32),
                ("nms_bins", ctypes.c_int32), ("fine_rows", ctypes.c_int32), ("component_top", ctypes.c_int32),
                ("nms_by_nsigma", ctypes.c_int32), ("template_budget", ctypes.c_int32)]


class _ProposalReport(ctypes.Structure):
    _fields_ = [("device_ms", ctypes.c_double), ("coarse_spectra", ctypes.c_int64),
                ("proposed_coarse", ctypes.c_int32), ("fine_cells", ctypes.c_int32),
                ("fine_segment_bins", ctypes.c_int64), ("fine_templates", ctypes.c_int32)]


CAND_DTYPE = np.dtype([("value", np.float32), ("template_idx", np.int32), ("bin", np.int32)])


@dataclass
class Params:
    """srs_params (include/srs.h).  Defaults are the paper's search: 30 s
    segments, 40-60 Hz band, chirp masses quoted at 40 Hz, eps = 1e-6."""
    fs: float = 256.0
    t_coh: float = 30.0
    f_lo: float = 40.0
    f_hi: float = 60.0
    f_ref: float = 40.0
    eps: float = 1e-6
    sigma: float = 0.0
    top_k: int = 32
    precision: int = SRS_MIXED
    cut_segments: int = 1
    io_on_device: int = 0
    chunk: int = 0
    deterministic: int = 1

    def c(self):
        return _Params(self.fs, self.t_coh, self.f_lo, self.f_hi, self.f_ref, self.eps, self.sigma,
                       self.top_k, self.precision, self.cut_segments, self.io_on_device, self.chunk,
                       self.deterministic)


_LIB = None


def lib():
    """Load libsrs.so, building it first if it is missing or stale."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.srs_create.restype = i32
        L.srs_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
        L.srs_destroy.restype = None
        L.srs_destroy.argtypes = [vp]
        L.srs_last_error.restype = ctypes.c_char_p
        L.srs_last_error.argtypes = [vp]
        L.srs_plan.restype = i32
        L.srs_plan.argtypes = [ctypes.POINTER(_Params), vp, i32, i64, ctypes.POINTER(_PlanInfo), vp, vp]
        L.srs_search.restype = i32
        L.srs_search.argtypes = [vp, vp, i64, i32, vp, i32, ctypes.POINTER(_Params), vp, vp,
                                 ctypes.POINTER(i32), ctypes.POINTER(_Report)]
        L.srs_search_async.restype = i32
        L.srs_search_async.argtypes = [vp, vp, i64, i32, vp, i32, ctypes.POINTER(_Params), vp, vp,
                                       ctypes.POINTER(i32)]
        L.srs_sync.restype = i32
        L.srs_sync.argtypes = [vp, ctypes.POINTER(_Report)]
        for fn in (L.srs_segment_spectra, L.srs_segment_spectra_cufft):
            fn.restype = i32
            fn.argtypes = [vp, vp, i64, i32, vp, i32, i32, i32, ctypes.POINTER(_Params), vp,
                           ctypes.POINTER(_Report)]
        L.srs_cube_whiten.restype = i32
        L.srs_cube_whiten.argtypes = [vp, vp, i32, i32, i32, vp, i32, vp, vp]
        L.srs_nsigma_threshold.restype = i32
        L.srs_nsigma_threshold.argtypes = [vp, i32, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
        L.srs_detection_noncentrality.restype = i32
        L.srs_detection_noncentrality.argtypes = [vp, i32, ctypes.c_double, ctypes.c_double,
                                                  ctypes.POINTER(ctypes.c_double)]
        L.srs_detection_probability.restype = i32
        L.srs_detection_probability.argtypes = [vp, vp, i32, vp, i32, vp]
        L.srs_selftest_wait.restype = i32
        L.srs_selftest_wait.argtypes = [vp]
        L.srs_power_cube.restype = i32
        L.srs_power_cube.argtypes = [vp, vp, i64, i32, ctypes.POINTER(_Bank), i32, i32, ctypes.POINTER(_Params), vp,
                                     ctypes.POINTER(_Report)]
        L.srs_stack_slide.restype = i32
        L.srs_stack_slide.argtypes = [vp, vp, i32, i32, i32, ctypes.POINTER(_Bank), ctypes.POINTER(_SlideGrid),
                                      ctypes.POINTER(_Params), i32, vp, vp, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(_Report)]
        L.srs_slide_search.restype = i32
        L.srs_slide_search.argtypes = [vp, vp, i64, i32, ctypes.POINTER(_Bank), ctypes.POINTER(_SlideGrid),
                                       ctypes.POINTER(_Params), i64, vp, vp, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(_Report)]
        L.srs_time_map.restype = i32
        L.srs_time_map.argtypes = [vp, vp, i32, vp, vp, i32, ctypes.POINTER(_Params), i64, vp, vp]
        f32p = ctypes.POINTER(ctypes.c_float)
        L.srs_make_strain.restype = i32
        L.srs_make_strain.argtypes = [vp, vp, i64, ctypes.c_double, ctypes.c_uint64, i32, vp, i32, ctypes.c_double]
        L.srs_patches.restype = i32
        L.srs_patches.argtypes = [vp, vp, i32, i32, vp, vp, i32, vp, i32]
        L.srs_mlp_forward.restype = i32
        L.srs_mlp_forward.argtypes = [vp, vp, i32, vp, vp, i32]
        L.srs_mlp_grad.restype = i32
        L.srs_mlp_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp, i32]
        L.srs_mlp_train.restype = i32
        L.srs_mlp_train.argtypes = [vp, vp, vp, i32, ctypes.POINTER(_TrainCfg), vp, vp]
        L.srs_score_map.restype = i32
        L.srs_score_map.argtypes = [vp, vp, i32, i32, vp, vp]
        L.srs_refine.restype = i32
        L.srs_refine.argtypes = [vp, vp, i64, i32, vp, i32, ctypes.POINTER(_Params), vp, vp, i32, vp,
                                 ctypes.POINTER(_Report)]
        L.srs_search_proposed.restype = i32
        L.srs_search_proposed.argtypes = [vp, vp, i64, i32, vp, i32, vp, i32, ctypes.POINTER(_Params), vp,
                                          ctypes.POINTER(_ProposalParams), i32, vp, vp, vp, ctypes.POINTER(i32),
                                          vp, ctypes.POINTER(i32), ctypes.POINTER(_ProposalReport)]
        L.srs_segment_spectra_static.restype = i32
        L.srs_segment_spectra_static.argtypes = [vp, vp, i64, i32, vp, i32, i32, i32, ctypes.POINTER(_Params),
                                                 vp, ctypes.c_char_p, ctypes.c_size_t]
        _LIB = L
    return _LIB


def nsigma_threshold(n_seg, p_fa, weights=None):
    """srs_nsigma_threshold: n_sigma^th at false-alarm probability p_fa for a
    track of n_seg segments, equal weights or the given positive weights."""
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if w is not None and w.size != n_seg:
        raise ValueError("weights must have n_seg entries")
    out = ctypes.c_double(0.0)
    st = lib().srs_nsigma_threshold(w.ctypes.data if w is not None else None, int(n_seg), float(p_fa),
                                    ctypes.byref(out))
    if st != SRS_OK:
        raise SrsError(st, "srs_nsigma_threshold rejected its arguments")
    return out.value


def detection_noncentrality(n_seg, p_fa, p_det, weights=None):
    """srs_detection_noncentrality: the total non-centrality a signal needs
    to cross the p_fa threshold with probability p_det (equal weights, or the
    given positive weights with the signal split in proportion to them)."""
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if w is not None and w.size != n_seg:
        raise ValueError("weights must have n_seg entries")
    out = ctypes.c_double(0.0)
    st = lib().srs_detection_noncentrality(w.ctypes.data if w is not None else None, int(n_seg), float(p_fa),
                                           float(p_det), ctypes.byref(out))
    if st != SRS_OK:
        raise SrsError(st, "srs_detection_noncentrality rejected its arguments")
    return out.value


def detection_probability(n_seg, p_fa, lambdas=None, weights=None):
    """srs_detection_probability: P(n_sigma > n_sigma^th(p_fa)) for a signal
    with per-segment non-centralities `lambdas` (None: no signal), equal
    weights or the given positive weights.  p_fa may be a scalar or a sequence
    (the points of a ROC curve); the result has the same shape."""
    pf = np.ascontiguousarray(np.atleast_1d(p_fa), dtype=np.float64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    lam = None if lambdas is None else np.ascontiguousarray(lambdas, dtype=np.float64)
    for a, name in ((w, "weights"), (lam, "lambdas")):
        if a is not None and a.size != n_seg:
            raise ValueError(f"{name} must have n_seg entries")
    out = np.zeros(pf.size, dtype=np.float64)
    st = lib().srs_detection_probability(w.ctypes.data if w is not None else None,
                                         lam.ctypes.data if lam is not None else None, int(n_seg),
                                         pf.ctypes.data, int(pf.size), out.ctypes.data)
    if st != SRS_OK:
        raise SrsError(st, "srs_detection_probability rejected its arguments")
    return float(out[0]) if np.ndim(p_fa) == 0 else out


def _report_dict(r):
    return {k: getattr(r, k) for k, _ in _Report._fields_}


def srs_plan(params, mc, n_samples):
    """Host planner: returns (info dict, beta[m], nseg[m]).  No GPU needed."""
    mc = np.ascontiguousarray(mc, dtype=np.float64)
    info = _PlanInfo()
    beta = np.zeros(mc.size)
    nseg = np.zeros(mc.size, dtype=np.int32)
    p = params.c()
    st = lib().srs_plan(ctypes.byref(p), mc.ctypes.data, mc.size, int(n_samples), ctypes.byref(info),
                        beta.ctypes.data, nseg.ctypes.data)
    if st != SRS_OK:
        raise SrsError(st, "srs_plan rejected the parameters")
    return {k: getattr(info, k) for k, _ in _PlanInfo._fields_}, beta, nseg


def _is_torch_cuda(x):
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def _dtype_code(x):
    if _is_torch_cuda(x):
        import torch
        if x.dtype == torch.float64:
            return SRS_F64
        if x.dtype == torch.float32:
            return SRS_F32
        raise TypeError("strain must be float32 or float64")
    if x.dtype == np.float64:
        return SRS_F64
    if x.dtype == np.float32:
        return SRS_F32
    raise TypeError("strain must be float32 or float64")

def _dev_in(x, device, name, dtypes=None, ndim=None):
    """A torch CUDA input of a Context call: on the context's device and
    contiguous (the library reads it as a flat array), of one of `dtypes` and
    with `ndim` dimensions when given."""
    if x.device.index != device:
        raise ValueError("%s is on %s; the context runs on cuda:%d" % (name, x.device, device))
    if not x.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtypes is not None and x.dtype not in dtypes:
        raise TypeError("%s must be of dtype %s" % (name, " or ".join(str(d) for d in dtypes)))
    if ndim is not None and x.dim() != ndim:
        raise ValueError("%s must have %d dimensions" % (name, ndim))


def _dev_out(x, shape, dtype, device, name):
    """A caller-supplied torch CUDA output: exactly the shape and dtype the
    library writes, contiguous, on the context's device (None: not wanted)."""
    if x is None:
        return
    if (not _is_torch_cuda(x) or x.dtype != dtype or tuple(x.shape) != tuple(shape) or not x.is_contiguous()
            or x.device.index != device):
        raise ValueError("%s must be a contiguous %s CUDA tensor of shape %s on cuda:%d"
                         % (name, dtype, tuple(shape), device))


def _host_out(x, shape, dtype, name):
    """A caller-supplied numpy output: exactly the shape and dtype the library
    writes, C-contiguous and writeable (None: not wanted)."""
    if x is None:
        return
    if (not isinstance(x, np.ndarray) or x.dtype != dtype or x.shape != tuple(shape)
            or not x.flags["C_CONTIGUOUS"] or not x.flags["WRITEABLE"]):
        raise ValueError("%s must be a writeable C-contiguous %s array of shape %s" % (name, dtype, tuple(shape)))


class Context:
    """srs_ctx: one CUDA device, one stream, a reusable device workspace."""

    def __init__(self, device=0, stream=None):
        self._lib = lib()
        self._h = ctypes.c_void_p()
        st = self._lib.srs_create(ctypes.byref(self._h), int(device), stream)
        if st != SRS_OK:
            raise SrsError(st, "srs_create failed (no CUDA device?)")
        self.device = int(device)

    def close(self):
        if self._h:
            self._lib.srs_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != SRS_OK:
            raise SrsError(st, self._lib.srs_last_error(self._h).decode())

    def _check_dev_search_out(self, out, map_shape, top_k):
        """The device outputs of a search: {"map": float32 [templates, n_bins]
        or None, "cands": int32 [top_k, 3]} on this context's device."""
        import torch
        if out.get("cands") is None:
            raise ValueError("out['cands'] is required")
        _dev_out(out.get("map"), map_shape, torch.float32, self.device, "out['map']")
        _dev_out(out["cands"], (top_k, 3), torch.int32, self.device, "out['cands']")

    def search(self, strain, mc, params, stat_map=True, out=None):
        """srs_search.  Host numpy strain (params.io_on_device = 0) returns numpy
        results; a torch CUDA tensor (io_on_device = 1) returns torch tensors on
        its device.  Returns (candidates structured array / dict of tensors,
        map or None, report dict)."""
        mc = np.ascontiguousarray(mc, dtype=np.float64)
        dt = _dtype_code(strain)
        p = params.c()
        n_cands = ctypes.c_int32(0)
        rep = _Report()
        if _is_torch_cuda(strain):
            import torch
            _dev_in(strain, self.device, "strain")
            p.io_on_device = 1
            n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
            if out is None:
                out = {"map": torch.empty((mc.size, n_bins), dtype=torch.float32, device=strain.device)
                       if stat_map else None,
                       "cands": torch.empty((params.top_k, 3), dtype=torch.int32, device=strain.device)}
            else:
                self._check_dev_search_out(out, (mc.size, n_bins), params.top_k)
            mp = out["map"].data_ptr() if out.get("map") is not None else None
            st = self._lib.srs_search(self._h, strain.data_ptr(), strain.numel(), dt, mc.ctypes.data, mc.size,
                                      ctypes.byref(p), mp, out["cands"].data_ptr(), ctypes.byref(n_cands),
                                      ctypes.byref(rep))
            self._check(st)
            return out, _report_dict(rep)
        strain = np.ascontiguousarray(strain)
        p.io_on_device = 0
        n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
        m = np.empty((mc.size, n_bins), dtype=np.float32) if stat_map else None
        c = np.zeros(params.top_k, dtype=CAND_DTYPE)
        st = self._lib.srs_search(self._h, strain.ctypes.data, strain.size, dt, mc.ctypes.data, mc.size,
                                  ctypes.byref(p), m.ctypes.data if m is not None else None, c.ctypes.data,
                                  ctypes.byref(n_cands), ctypes.byref(rep))
        self._check(st)
        return c[:n_cands.value], m, _report_dict(rep)

    def search_async(self, strain, mc, params, out):
        """srs_search_async: enqueue a search and return at once; results and
        device status become final at sync().  A torch CUDA strain fills the
        device tensors of `out` ({"map": float32 [templates, n_bins] or None,
        "cands": int32 [top_k, 3]}); a numpy strain (pinned memory for
        overlap) fills the numpy arrays of `out` ({"map": float32 or None,
        "cands": CAND_DTYPE [top_k]}).  Keep strain and out alive and unchanged
        until sync()."""
        mc = np.ascontiguousarray(mc, dtype=np.float64)
        p = params.c()
        n_cands = ctypes.c_int32(0)
        n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
        if _is_torch_cuda(strain):
            _dev_in(strain, self.device, "strain")
            self._check_dev_search_out(out, (mc.size, n_bins), params.top_k)
            p.io_on_device = 1
            mp = out["map"].data_ptr() if out.get("map") is not None else None
            st = self._lib.srs_search_async(self._h, strain.data_ptr(), strain.numel(), _dtype_code(strain),
                                            mc.ctypes.data, mc.size, ctypes.byref(p), mp, out["cands"].data_ptr(),
                                            ctypes.byref(n_cands))
        else:
            if not (isinstance(strain, np.ndarray) and strain.flags["C_CONTIGUOUS"]):
                raise ValueError("a host strain must be a C-contiguous numpy array (kept alive until sync)")
            p.io_on_device = 0
            c = out["cands"]
            if (not isinstance(c, np.ndarray) or c.dtype != CAND_DTYPE or c.size < params.top_k
                    or not c.flags["C_CONTIGUOUS"] or not c.flags["WRITEABLE"]):
                raise ValueError("out['cands'] must be a contiguous CAND_DTYPE array of top_k entries")
            m = out.get("map")
            _host_out(m, (mc.size, n_bins), np.float32, "out['map']")
            st = self._lib.srs_search_async(self._h, strain.ctypes.data, strain.size, _dtype_code(strain),
                                            mc.ctypes.data, mc.size, ctypes.byref(p),
                                            m.ctypes.data if m is not None else None, c.ctypes.data,
                                            ctypes.byref(n_cands))
        self._check(st)
        return int(n_cands.value)

    def sync(self):
        """srs_sync: wait for the queued asynchronous searches; their averaged
        timing and the last one's sizes as a report dict."""
        rep = _Report()
        self._check(self._lib.srs_sync(self._h, ctypes.byref(rep)))
        return _report_dict(rep)

    def segment_spectra(self, strain, mc, seg_begin, seg_end, params, via_cufft=False):
        """srs_segment_spectra: complex128 [templates, seg_end - seg_begin, n_bins]
        (numpy for host strain, torch for a CUDA tensor).  via_cufft=True calls
        srs_segment_spectra_cufft, the unfused comparison (spread grids in HBM,
        cuFFT transforms, deconvolution)."""
        fn = self._lib.srs_segment_spectra_cufft if via_cufft else self._lib.srs_segment_spectra
        mc = np.ascontiguousarray(mc, dtype=np.float64)
        dt = _dtype_code(strain)
        p = params.c()
        rep = _Report()
        n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
        shape = (mc.size, seg_end - seg_begin, n_bins)
        if _is_torch_cuda(strain):
            import torch
            _dev_in(strain, self.device, "strain")
            p.io_on_device = 1
            F = torch.empty(shape, dtype=torch.complex128, device=strain.device)
            st = fn(self._h, strain.data_ptr(), strain.numel(), dt, mc.ctypes.data, mc.size, int(seg_begin),
                    int(seg_end), ctypes.byref(p), F.data_ptr(), ctypes.byref(rep))
            self._check(st)
            return F, _report_dict(rep)
        strain = np.ascontiguousarray(strain)
        p.io_on_device = 0
        F = np.empty(shape, dtype=np.complex128)
        st = fn(self._h, strain.ctypes.data, strain.size, dt, mc.ctypes.data, mc.size, int(seg_begin),
                int(seg_end), ctypes.byref(p), F.ctypes.data, ctypes.byref(rep))
        self._check(st)
        return F, _report_dict(rep)

    def selftest_wait(self):
        """srs_selftest_wait: the bounded staging wait's give-up path; raises
        SrsError (SRS_ERR_TIMEOUT) as a search whose wait gave up would."""
        self._check(self._lib.srs_selftest_wait(self._h))

    # ----- two-stage search: power cube + stack-slide ----------------------
    @staticmethod
    def _bank(bank):
        return _Bank(float(bank[0]), float(bank[1]), int(bank[2]))

    @staticmethod
    def _grid(rows_mc, rows_c, n_t0, f0, weighting=0, s_eff=None, whiten=False):
        mc = np.ascontiguousarray(rows_mc, dtype=np.float64)
        c = np.ascontiguousarray(rows_c, dtype=np.float64)
        if mc.shape != c.shape:
            raise ValueError("rows_mc and rows_c must have the same length")
        se = None if s_eff is None else np.ascontiguousarray(s_eff, dtype=np.float32)
        g = _SlideGrid(float(f0), mc.ctypes.data, c.ctypes.data, mc.size, int(n_t0), int(weighting),
                       se.ctypes.data if se is not None else None, 1 if whiten else 0)
        return g, (mc, c, se)   # keep the arrays alive with the struct

    def power_cube(self, strain, bank, seg_begin, seg_end, params):
        """srs_power_cube: float32 [n_beta, n_bins, seg_end - seg_begin] powers of
        every segment under each bank entry (bank = (beta_min, beta_max, n_beta));
        numpy for host strain, torch for a CUDA tensor."""
        dt = _dtype_code(strain)
        p = params.c()
        rep = _Report()
        n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
        shape = (int(bank[2]), n_bins, seg_end - seg_begin)
        b = self._bank(bank)
        if _is_torch_cuda(strain):
            import torch
            _dev_in(strain, self.device, "strain")
            p.io_on_device = 1
            out = torch.empty(shape, dtype=torch.float32, device=strain.device)
            st = self._lib.srs_power_cube(self._h, strain.data_ptr(), strain.numel(), dt, ctypes.byref(b),
                                          int(seg_begin), int(seg_end), ctypes.byref(p), out.data_ptr(),
                                          ctypes.byref(rep))
        else:
            strain = np.ascontiguousarray(strain)
            p.io_on_device = 0
            out = np.empty(shape, dtype=np.float32)
            st = self._lib.srs_power_cube(self._h, strain.ctypes.data, strain.size, dt, ctypes.byref(b),
                                          int(seg_begin), int(seg_end), ctypes.byref(p), out.ctypes.data,
                                          ctypes.byref(rep))
        self._check(st)
        return out, _report_dict(rep)

    def stack_slide(self, cube, seg_begin, n_seg_total, bank, rows_mc, rows_c, n_t0, params, f0=None,
                    first=True, last=True, want_map=True, weighting=0, s_eff=None, whiten=False):
        """srs_stack_slide over a cube chunk [n_beta, n_bins, chunk segments]
        holding segments [seg_begin, seg_begin + chunk).  With last=True returns
        (candidates, n_sigma map [rows, n_t0] or None, report); otherwise
        (None, None, report).  numpy cube: host I/O; torch CUDA cube: device I/O."""
        f0 = params.f_lo if f0 is None else f0
        g, keep = self._grid(rows_mc, rows_c, n_t0, f0, weighting, s_eff, whiten)
        b = self._bank(bank)
        p = params.c()
        rep = _Report()
        n_cands = ctypes.c_int32(0)
        flags = (SRS_SLIDE_FIRST if first else 0) | (SRS_SLIDE_LAST if last else 0)
        n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
        if tuple(cube.shape[:2]) != (int(bank[2]), n_bins) or len(cube.shape) != 3:
            raise ValueError("cube must be [n_beta, n_bins, segments]")
        if _is_torch_cuda(cube) and (cube.dtype != __import__("torch").float32 or not cube.is_contiguous()):
            raise ValueError("a device cube must be a contiguous float32 tensor")
        if _is_torch_cuda(cube):
            _dev_in(cube, self.device, "cube")
        seg_end = int(seg_begin) + int(cube.shape[2])
        R = keep[0].size
        if _is_torch_cuda(cube):
            import torch
            p.io_on_device = 1
            m = torch.empty((R, int(n_t0)), dtype=torch.float32, device=cube.device) if (last and want_map) else None
            c = torch.empty((params.top_k, 3), dtype=torch.int32, device=cube.device) if last else None
            st = self._lib.srs_stack_slide(self._h, cube.data_ptr(), int(seg_begin), seg_end, int(n_seg_total),
                                           ctypes.byref(b), ctypes.byref(g), ctypes.byref(p), flags,
                                           m.data_ptr() if m is not None else None,
                                           c.data_ptr() if c is not None else None, ctypes.byref(n_cands),
                                           ctypes.byref(rep))
            self._check(st)
            return (c[:n_cands.value] if c is not None else None), m, _report_dict(rep)
        cube = np.ascontiguousarray(cube, dtype=np.float32)
        p.io_on_device = 0
        m = np.empty((R, int(n_t0)), dtype=np.float32) if (last and want_map) else None
        c = np.zeros(params.top_k, dtype=CAND_DTYPE) if last else None
        st = self._lib.srs_stack_slide(self._h, cube.ctypes.data, int(seg_begin), seg_end, int(n_seg_total),
                                       ctypes.byref(b), ctypes.byref(g), ctypes.byref(p), flags,
                                       m.ctypes.data if m is not None else None,
                                       c.ctypes.data if c is not None else None, ctypes.byref(n_cands),
                                       ctypes.byref(rep))
        self._check(st)
        return (c[:n_cands.value] if c is not None else None), m, _report_dict(rep)

    def cube_whiten(self, cube, s_eff=None):
        """srs_cube_whiten on a torch CUDA cube [n_beta, n_bins, n_seg] in place:
        returns (s_eff [n_beta, n_bins], mu [n_seg], sigma [n_seg]) as tensors;
        the PSD is estimated from the cube unless s_eff is given."""
        import torch
        if not (_is_torch_cuda(cube) and cube.dtype == torch.float32 and cube.is_contiguous() and cube.dim() == 3):
            raise ValueError("cube must be a contiguous float32 CUDA tensor [n_beta, n_bins, n_seg]")
        _dev_in(cube, self.device, "cube")
        K, B, N = (int(v) for v in cube.shape)
        est = s_eff is None
        S = torch.empty((K, B), dtype=torch.float32, device=cube.device) if est else \
            torch.as_tensor(s_eff, dtype=torch.float32, device=cube.device).contiguous()
        mu = torch.empty(N, dtype=torch.float32, device=cube.device)
        sg = torch.empty(N, dtype=torch.float32, device=cube.device)
        self._check(self._lib.srs_cube_whiten(self._h, cube.data_ptr(), K, B, N, S.data_ptr(), 1 if est else 0,
                                              mu.data_ptr(), sg.data_ptr()))
        return S, mu, sg

    def slide_search(self, strain, bank, rows_mc, rows_c, n_t0, params, f0=None, cube_budget_bytes=0,
                     want_map=True, out=None, weighting=0, s_eff=None, whiten=False):
        """srs_slide_search: power cube + stack-slide over the whole strain.
        Host numpy strain returns (candidates, map or None, report); a torch
        CUDA strain returns ({"map", "cands"} tensors, report)."""
        f0 = params.f_lo if f0 is None else f0
        g, keep = self._grid(rows_mc, rows_c, n_t0, f0, weighting, s_eff, whiten)
        b = self._bank(bank)
        dt = _dtype_code(strain)
        p = params.c()
        rep = _Report()
        n_cands = ctypes.c_int32(0)
        R = keep[0].size
        if _is_torch_cuda(strain):
            import torch
            _dev_in(strain, self.device, "strain")
            p.io_on_device = 1
            if out is None:
                out = {"map": torch.empty((R, int(n_t0)), dtype=torch.float32, device=strain.device)
                       if want_map else None,
                       "cands": torch.empty((params.top_k, 3), dtype=torch.int32, device=strain.device)}
            else:
                self._check_dev_search_out(out, (R, int(n_t0)), params.top_k)
            mp = out["map"].data_ptr() if out.get("map") is not None else None
            st = self._lib.srs_slide_search(self._h, strain.data_ptr(), strain.numel(), dt, ctypes.byref(b),
                                            ctypes.byref(g), ctypes.byref(p), int(cube_budget_bytes), mp,
                                            out["cands"].data_ptr(), ctypes.byref(n_cands), ctypes.byref(rep))
            self._check(st)
            return out, _report_dict(rep)
        strain = np.ascontiguousarray(strain)
        p.io_on_device = 0
        m = np.empty((R, int(n_t0)), dtype=np.float32) if want_map else None
        c = np.zeros(params.top_k, dtype=CAND_DTYPE)
        st = self._lib.srs_slide_search(self._h, strain.ctypes.data, strain.size, dt, ctypes.byref(b),
                                        ctypes.byref(g), ctypes.byref(p), int(cube_budget_bytes),
                                        m.ctypes.data if m is not None else None, c.ctypes.data,
                                        ctypes.byref(n_cands), ctypes.byref(rep))
        self._check(st)
        return c[:n_cands.value], m, _report_dict(rep)

    # ----- learned proposal -----------------------------------------------
    def make_strain(self, n, fs, seed, injections=(), f_hi=60.0, noise=True, out=None):
        """srs_make_strain: float32 CUDA tensor [n] of seeded noise plus 0PN
        chirps (dicts with mc, f0, amp and optional phi0)."""
        import torch
        if out is None:
            out = torch.empty(int(n), dtype=torch.float32, device="cuda:%d" % self.device)
        else:
            _dev_out(out, (int(n),), torch.float32, self.device, "out")
        arr = (_Injection * max(1, len(injections)))()
        for k, inj in enumerate(injections):
            arr[k] = _Injection(inj["mc"], inj["f0"], inj["amp"], inj.get("phi0", 0.0))
        st = self._lib.srs_make_strain(self._h, out.data_ptr(), int(n), float(fs), int(seed) & (2 ** 64 - 1),
                                       1 if noise else 0, ctypes.cast(arr, ctypes.c_void_p), len(injections),
                                       float(f_hi))
        self._check(st)
        return out

    def patches(self, stat_map, cells):
        """srs_patches for (m, b) cells of a map: numpy map -> numpy [n, 297];
        torch CUDA map -> torch CUDA [n, 297]."""
        cells = np.asarray(cells, dtype=np.int32).reshape(-1, 2)
        n = cells.shape[0]
        if _is_torch_cuda(stat_map):
            import torch
            _dev_in(stat_map, self.device, "stat_map", (torch.float32,), 2)
            M, NB = stat_map.shape
            cm = torch.from_numpy(np.ascontiguousarray(cells[:, 0])).to(stat_map.device)
            cb = torch.from_numpy(np.ascontiguousarray(cells[:, 1])).to(stat_map.device)
            out = torch.empty((n, MLP_INPUTS), dtype=torch.float32, device=stat_map.device)
            torch.cuda.synchronize()
            st = self._lib.srs_patches(self._h, stat_map.data_ptr(), M, NB, cm.data_ptr(), cb.data_ptr(), n,
                                       out.data_ptr(), 1)
            self._check(st)
            return out
        stat_map = np.ascontiguousarray(stat_map, dtype=np.float32)
        M, NB = stat_map.shape
        cm = np.ascontiguousarray(cells[:, 0]); cb = np.ascontiguousarray(cells[:, 1])
        out = np.empty((n, MLP_INPUTS), dtype=np.float32)
        st = self._lib.srs_patches(self._h, stat_map.ctypes.data, M, NB, cm.ctypes.data, cb.ctypes.data, n,
                                   out.ctypes.data, 0)
        self._check(st)
        return out

    def mlp_forward(self, X, params):
        """srs_mlp_forward: logits of inputs X [n, 297] (numpy or torch CUDA)."""
        params = np.ascontiguousarray(params, dtype=np.float32)
        if _is_torch_cuda(X):
            import torch
            _dev_in(X, self.device, "X", (torch.float32,), 2)
            if X.shape[1] != MLP_INPUTS:
                raise ValueError("X must be [n, %d]" % MLP_INPUTS)
            out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
            st = self._lib.srs_mlp_forward(self._h, X.data_ptr(), X.shape[0], params.ctypes.data, out.data_ptr(), 1)
            self._check(st)
            return out
        X = np.ascontiguousarray(X, dtype=np.float32)
        out = np.empty(X.shape[0], dtype=np.float32)
        st = self._lib.srs_mlp_forward(self._h, X.ctypes.data, X.shape[0], params.ctypes.data, out.ctypes.data, 0)
        self._check(st)
        return out

    def mlp_grad(self, X, y, params):
        """srs_mlp_grad: (gradient [19137], mean loss) over host X [n, 297], y [n]."""
        params = np.ascontiguousarray(params, dtype=np.float32)
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        st = self._lib.srs_mlp_grad(self._h, X.ctypes.data, y.ctypes.data, X.shape[0], params.ctypes.data,
                                    g.ctypes.data, ctypes.byref(loss), 0)
        self._check(st)
        return g, loss.value

    def mlp_train(self, X, y, params, epochs=20, batch=256, lr=1e-3, seed=0, beta1=0.9, beta2=0.999, eps=1e-8):
        """srs_mlp_train on a CUDA training set X [n, 297], y [n]; returns
        (trained FP32 parameters, mean loss of each epoch)."""
        import torch
        if not (_is_torch_cuda(X) and _is_torch_cuda(y)):
            raise TypeError("X and y must be CUDA tensors")
        _dev_in(X, self.device, "X", (torch.float32,), 2)
        _dev_in(y, self.device, "y", (torch.float32,), 1)
        if X.shape[1] != MLP_INPUTS or y.shape[0] != X.shape[0]:
            raise ValueError("X must be [n, %d] and y [n]" % MLP_INPUTS)
        p = np.array(params, dtype=np.float32)
        losses = np.zeros(epochs, dtype=np.float32)
        cfg = _TrainCfg(int(epochs), int(batch), float(lr), float(beta1), float(beta2), float(eps),
                        int(seed) & (2 ** 64 - 1))
        st = self._lib.srs_mlp_train(self._h, X.data_ptr(), y.data_ptr(), X.shape[0], ctypes.byref(cfg),
                                     p.ctypes.data, losses.ctypes.data)
        self._check(st)
        return p, losses

    def score_map(self, stat_map, params):
        """srs_score_map: logits of every cell of a CUDA map [templates, bins]."""
        import torch
        params = np.ascontiguousarray(params, dtype=np.float32)
        if not _is_torch_cuda(stat_map):
            raise TypeError("stat_map must be a CUDA tensor")
        _dev_in(stat_map, self.device, "stat_map", (torch.float32,), 2)
        M, NB = stat_map.shape
        out = torch.empty((M, NB), dtype=torch.float32, device=stat_map.device)
        st = self._lib.srs_score_map(self._h, stat_map.data_ptr(), M, NB, params.ctypes.data, out.data_ptr())
        self._check(st)
        return out

    def refine(self, strain, mc, params, cells):
        """srs_refine: n_sigma (numpy) of listed (m, b) cells by direct sums."""
        mc = np.ascontiguousarray(mc, dtype=np.float64)
        cells = np.asarray(cells, dtype=np.int32).reshape(-1, 2)
        cm = np.ascontiguousarray(cells[:, 0]); cb = np.ascontiguousarray(cells[:, 1])
        ns = np.empty(cells.shape[0], dtype=np.float32)
        p = params.c()
        rep = _Report()
        if _is_torch_cuda(strain):
            _dev_in(strain, self.device, "strain")
            p.io_on_device = 1
            ptr, n = strain.data_ptr(), strain.numel()
        else:
            strain = np.ascontiguousarray(strain)
            p.io_on_device = 0
            ptr, n = strain.ctypes.data, strain.size
        st = self._lib.srs_refine(self._h, ptr, n, _dtype_code(strain), mc.ctypes.data, mc.size, ctypes.byref(p),
                                  cm.ctypes.data, cb.ctypes.data, cells.shape[0], ns.ctypes.data,
                                  ctypes.byref(rep))
        self._check(st)
        return ns, _report_dict(rep)

    def search_proposed(self, strain, coarse_mc, fine_mc, params, mlp_params, threshold, max_cells=1 << 20,
                        nms=(0, 0), fine_rows=1, component_top=0, nms_by_nsigma=False, template_budget=0):
        """srs_search_proposed: returns dict(cells [n, 2], nsigma [n], cands,
        report).  nms = (templates, bins) half-window of the non-maximum
        suppression ((0, 0): off); fine_rows = coarse rows either side whose
        fine templates a proposal covers; component_top > 0: each connected
        group of above-threshold cells proposes its component_top cells of
        highest coarse n_sigma; nms_by_nsigma: the suppression window
        compares coarse n_sigma instead of scores; template_budget > 0: only
        the template_budget fine templates with the highest best proposing
        score are refined."""
        cmc = np.ascontiguousarray(coarse_mc, dtype=np.float64)
        fmc = np.ascontiguousarray(fine_mc, dtype=np.float64)
        mp = np.ascontiguousarray(mlp_params, dtype=np.float32)
        cm = np.empty(max_cells, dtype=np.int32); cb = np.empty(max_cells, dtype=np.int32)
        ns = np.empty(max_cells, dtype=np.float32)
        nout = ctypes.c_int32(0); nc = ctypes.c_int32(0)
        cands = np.zeros(max(1, params.top_k), dtype=CAND_DTYPE)
        rep = _ProposalReport()
        p = params.c()
        if _is_torch_cuda(strain):
            _dev_in(strain, self.device, "strain")
            p.io_on_device = 1
            ptr, n = strain.data_ptr(), strain.numel()
        else:
            strain = np.ascontiguousarray(strain)
            p.io_on_device = 0
            ptr, n = strain.ctypes.data, strain.size
        if int(template_budget) < 0:
            raise ValueError("template_budget must be >= 0")
        pp = _ProposalParams(float(threshold), int(nms[0]), int(nms[1]), int(fine_rows), int(component_top),
                             int(bool(nms_by_nsigma)), int(template_budget))
        st = self._lib.srs_search_proposed(self._h, ptr, n, _dtype_code(strain), cmc.ctypes.data, cmc.size,
                                           fmc.ctypes.data, fmc.size, ctypes.byref(p), mp.ctypes.data,
                                           ctypes.byref(pp), max_cells, cm.ctypes.data, cb.ctypes.data,
                                           ns.ctypes.data, ctypes.byref(nout), cands.ctypes.data,
                                           ctypes.byref(nc), ctypes.byref(rep))
        self._check(st)
        k = min(nout.value, max_cells)
        return {"cells": np.stack([cm[:k], cb[:k]], axis=1), "nsigma": ns[:k], "n_cells": nout.value,
                "cands": cands[:nc.value], "report": {f: getattr(rep, f) for f, _ in _ProposalReport._fields_}}

    def time_map(self, mc, items, params, n_samples):
        """srs_time_map: (psi, theta) float64 [len(items), n_s] for (m, i) items."""
        mc = np.ascontiguousarray(mc, dtype=np.float64)
        items = np.asarray(items, dtype=np.int32).reshape(-1, 2)
        im = np.ascontiguousarray(items[:, 0]); ii = np.ascontiguousarray(items[:, 1])
        n_s = int(round(params.t_coh * params.fs))
        psi = np.empty((items.shape[0], n_s)); th = np.empty((items.shape[0], n_s))
        p = params.c()
        st = self._lib.srs_time_map(self._h, mc.ctypes.data, mc.size, im.ctypes.data, ii.ctypes.data,
                                    items.shape[0], ctypes.byref(p), int(n_samples), psi.ctypes.data,
                                    th.ctypes.data)
        self._check(st)
        return psi, th


def segment_spectra_static(strain, mc, seg_begin, seg_end, params, F=None, stream=None):
    """srs_segment_spectra_static: the mixed-form segment spectra for callers
    that cannot let the library allocate device memory.  `strain` is a torch
    CUDA tensor (float32 or float64); F, if given, a complex128 CUDA tensor
    [templates, seg_end - seg_begin, n_bins] that receives the result; stream
    a torch.cuda.Stream (default: the current stream).  Returns F."""
    import torch
    if not _is_torch_cuda(strain):
        raise TypeError("strain must be a CUDA tensor")
    if not strain.is_contiguous():
        raise ValueError("strain must be contiguous")
    mc = np.ascontiguousarray(mc, dtype=np.float64)
    n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
    shape = (mc.size, int(seg_end) - int(seg_begin), n_bins)
    if F is None:
        F = torch.empty(shape, dtype=torch.complex128, device=strain.device)
    elif (not _is_torch_cuda(F) or F.dtype != torch.complex128 or tuple(F.shape) != shape
          or not F.is_contiguous() or F.device != strain.device):
        raise ValueError("F must be a contiguous complex128 tensor of shape %s on %s" % (shape, strain.device))
    s = stream if stream is not None else torch.cuda.current_stream(strain.device)
    p = params.c()
    p.io_on_device = 1
    buf = ctypes.create_string_buffer(256)
    with torch.cuda.device(strain.device):
        st = lib().srs_segment_spectra_static(ctypes.c_void_p(s.cuda_stream), strain.data_ptr(), strain.numel(),
                                              _dtype_code(strain), mc.ctypes.data, mc.size, int(seg_begin),
                                              int(seg_end), ctypes.byref(p), F.data_ptr(), buf, 256)
    if st != SRS_OK:
        raise SrsError(st, buf.value.decode())
    return F
