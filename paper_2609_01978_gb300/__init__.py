"""Python binding of libfzp.so (argument marshalling only).

libfzp evaluates the Fresnel diffraction integral (Eq. 1-2) of a full-aperture
Fresnel zone plate onto a focal-plane region of interest by stripe-processed
chirp-z transforms (Sec. 2.6, Fig. 2, Fig. 18) on a GB300 GPU.  Every step of
the computation runs in the library's CUDA kernels; this module only converts
Python arguments into the C structures of ``include/fzp.h`` and passes device
pointers (``torch`` tensors, used for device memory and streams) through.

There is no CPU fallback: if the compiled library is missing, importing the
binding raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfzp.so")

FZP_OK, FZP_E_INVALID, FZP_E_OOM, FZP_E_CUDA, FZP_E_TIMEOUT, FZP_E_UNSUPPORTED = range(6)
FORM_AUTO, FORM_BLUESTEIN, FORM_DENSE, FORM_SACZT = 0, 1, 2, 3
PREC_FP64, PREC_FP32, PREC_SPLIT_BF16, PREC_BF16, PREC_AUTO_1E4 = 0, 1, 2, 3, 4
CONV_AUTO, CONV_SINGLE, CONV_PARTITIONED = 0, 1, 2

_STATUS = {0: "FZP_OK", 1: "FZP_E_INVALID", 2: "FZP_E_OOM", 3: "FZP_E_CUDA", 4: "FZP_E_TIMEOUT",
           5: "FZP_E_UNSUPPORTED"}


class FzpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Deform(ctypes.Structure):
    _fields_ = [("amp", ctypes.c_double), ("period", ctypes.c_double), ("theta", ctypes.c_double),
                ("taper", ctypes.c_double), ("n_ridges", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ridge_px", ctypes.c_double * 3), ("ridge_py", ctypes.c_double * 3),
                ("ridge_alpha", ctypes.c_double * 3), ("ridge_h", ctypes.c_double * 3),
                ("ridge_width", ctypes.c_double * 3)]


class Params(ctypes.Structure):
    _fields_ = [("D", ctypes.c_double), ("f", ctypes.c_double), ("lam", ctypes.c_double),
                ("dx", ctypes.c_double), ("N", ctypes.c_int64), ("M", ctypes.c_int32),
                ("form", ctypes.c_int32), ("pitch", ctypes.c_double), ("precision", ctypes.c_int32),
                ("stripe_rows", ctypes.c_int32), ("deform", ctypes.POINTER(Deform)),
                ("promote", ctypes.c_int32), ("row_batch", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("centre_open", ctypes.c_int32), ("roi_origin", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("exact_radii", ctypes.c_int32), ("conv", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("c", ctypes.c_int64), ("total_zones", ctypes.c_int64),
                ("n_thresholds", ctypes.c_int64), ("dx", ctypes.c_double), ("R", ctypes.c_double),
                ("kappa", ctypes.c_double), ("x0", ctypes.c_double), ("M", ctypes.c_int32),
                ("form", ctypes.c_int32), ("precision", ctypes.c_int32), ("stripe_rows", ctypes.c_int32),
                ("fft_length", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("promote", ctypes.c_int32), ("row_batch", ctypes.c_int32), ("chunk_rows", ctypes.c_int64),
                ("cluster", ctypes.c_int32), ("fft_inner", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("passes", ctypes.c_int32), ("centre_open", ctypes.c_int32),
                ("conv", ctypes.c_int32), ("s_R", ctypes.c_int64)]


class Metrics(ctypes.Structure):
    _fields_ = [("fwhm_x", ctypes.c_double), ("fwhm_y", ctypes.c_double), ("de_lobe", ctypes.c_double),
                ("de_roi", ctypes.c_double), ("p_in", ctypes.c_double), ("p_in_disc", ctypes.c_double),
                ("peak", ctypes.c_double), ("strehl", ctypes.c_double), ("mtf_half_cut", ctypes.c_double),
                ("mtf16", ctypes.c_double * 16), ("aperture_count", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "mtf16"}
        d["mtf16"] = list(self.mtf16)
        return d


class Profile(ctypes.Structure):
    _fields_ = [("dominant_ms", ctypes.c_double), ("dominant_launches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("dominant_name", ctypes.c_char * 48)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libfzp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2609_01978_gb300/build.py (or "
                              "__graft_entry__.build()) first; there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        sig = {
            "fzp_plan": [ctypes.POINTER(Params), ctypes.POINTER(vp)],
            "fzp_plan_info_get": [vp, ctypes.POINTER(PlanInfo)],
            "fzp_plan_query": [ctypes.POINTER(Params), ctypes.POINTER(PlanInfo)],
            "fzp_zone_thresholds": [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_int64), i64,
                                    ctypes.POINTER(ctypes.c_int64)],
            "fzp_plan_destroy": [vp],
            "fzp_propagate_roi": [vp, i64, i64, vp, i32, vp],
            "fzp_intensity": [vp, vp, vp, vp],
            "fzp_metrics": [vp, vp, vp, ctypes.POINTER(Metrics)],
            "fzp_aperture_mask": [vp, i64, i64, vp, vp],
            "fzp_metrics_noalloc": [ctypes.POINTER(Params), vp, vp, ctypes.POINTER(Metrics)],
            "fzp_selftest_wait_timeout": [ctypes.c_uint32, vp],
            "fzp_profile_enable": [vp, i32],
            "fzp_batch_plan": [ctypes.POINTER(Params), i32, ctypes.POINTER(vp)],
            "fzp_batch_propagate": [vp, ctypes.POINTER(vp), vp],
            "fzp_batch_info": [vp, i32, ctypes.POINTER(PlanInfo)],
            "fzp_batch_metrics": [vp, i32, vp, vp, ctypes.POINTER(Metrics)],
            "fzp_batch_destroy": [vp],
            "fzp_batch_kernels": [vp, ctypes.POINTER(ctypes.c_int64)],
            "fzp_batch_intensity": [vp, i32, vp, vp, vp],
            "fzp_surrogate_create": [i32, i32, i32, i32, i32, ctypes.c_uint64, ctypes.POINTER(vp)],
            "fzp_surrogate_params": [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t, i32],
            "fzp_surrogate_infer": [vp, vp, i32, vp, vp],
            "fzp_surrogate_grad": [vp, vp, vp, i32, vp, vp, vp],
            "fzp_surrogate_train_step": [vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, vp, vp],
            "fzp_surrogate_destroy": [vp],
            "fzp_profile_read": [vp, ctypes.POINTER(Profile)],
            "fzp_report_write": [vp, vp, ctypes.c_double, ctypes.c_char_p, ctypes.c_char_p, vp,
                                 ctypes.POINTER(Metrics)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.fzp_last_error.restype = ctypes.c_char_p
        L.fzp_last_error.argtypes = []
        L.fzp_surrogate_param_count.argtypes = [vp]
        L.fzp_surrogate_param_count.restype = ctypes.c_size_t
        L.fzp_version.restype = ctypes.c_char_p
        L.fzp_version.argtypes = []
        _lib = L
    return _lib


def _check(st: int):
    if st != FZP_OK:
        raise FzpError(st, lib().fzp_last_error().decode())


def _ptr(x) -> Optional[int]:
    """Device pointer of a torch tensor, or an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _origin(x0):
    """(roi_origin, x0, y0) of fzp_params: None keeps the ROI centred on the focus."""
    return (0, 0.0, 0.0) if x0 is None else (1, float(x0), float(x0))


def make_deform(amp=0.0, period=1e-2, theta=0.0, taper=0.0, ridges=()) -> Deform:
    d = Deform()
    d.amp, d.period, d.theta, d.taper = amp, period, theta, taper
    d.n_ridges = len(ridges)
    for k, (px, py, al, h, w) in enumerate(ridges):
        d.ridge_px[k], d.ridge_py[k], d.ridge_alpha[k], d.ridge_h[k], d.ridge_width[k] = px, py, al, h, w
    return d


class Plan:
    """fzp_plan / fzp_propagate_roi / fzp_metrics / fzp_plan_destroy."""

    def __init__(self, D: float, f: float, lam: float, M: int, pitch: float, dx: float = 0.0, N: int = 0,
                 form: int = FORM_AUTO, precision: int = PREC_FP32, stripe_rows: int = 0,
                 deform: Optional[Deform] = None, promote: int = 0, row_batch: int = 0, cluster: int = 0,
                 levels: int = 0, centre_open: int = 0, x0: Optional[float] = None, exact_radii: int = 0,
                 conv: int = CONV_AUTO):
        """x0: first ROI coordinate on both axes (None: the ROI centred on the focus);
        exact_radii: the zone radii of Eq. 3 (FORM_SACZT only); conv: the
        Bluestein row convolution (CONV_SINGLE, CONV_PARTITIONED, CONV_AUTO)."""
        self._deform = deform
        org, ox, oy = _origin(x0)
        p = Params(D=D, f=f, lam=lam, dx=dx, N=N, M=M, form=form, pitch=pitch, precision=precision,
                   stripe_rows=stripe_rows, deform=ctypes.pointer(deform) if deform is not None else None,
                   promote=promote, row_batch=row_batch, cluster=cluster, levels=levels,
                   centre_open=centre_open, roi_origin=org, x0=ox, y0=oy, exact_radii=exact_radii, conv=conv)
        h = ctypes.c_void_p()
        _check(lib().fzp_plan(ctypes.byref(p), ctypes.byref(h)))
        self._h = h
        self.M = M

    @property
    def info(self) -> dict:
        inf = PlanInfo()
        _check(lib().fzp_plan_info_get(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in inf._fields_}

    def propagate_roi(self, row_begin: int, row_end: int, field, accumulate: bool = False, stream=None):
        _check(lib().fzp_propagate_roi(self._h, row_begin, row_end, _ptr(field), int(accumulate), _stream(stream)))

    def intensity(self, field, out, stream=None):
        _check(lib().fzp_intensity(self._h, _ptr(field), _ptr(out), _stream(stream)))

    def metrics(self, field, stream=None) -> dict:
        m = Metrics()
        _check(lib().fzp_metrics(self._h, _ptr(field), _stream(stream), ctypes.byref(m)))
        return m.as_dict()

    def report(self, field, run_dir: str, tag: str, t_propagate_s: float = 0.0, stream=None) -> dict:
        """fzp_report_write: metrics of `field`, then result_<tag>.npy (I),
        report_<tag>.txt and result_<tag>.json in `run_dir` (Fig. 18 run outputs)."""
        m = Metrics()
        _check(lib().fzp_report_write(self._h, _ptr(field), float(t_propagate_s), run_dir.encode(), tag.encode(),
                                      _stream(stream), ctypes.byref(m)))
        return m.as_dict()

    def aperture_mask(self, row_begin: int, row_end: int, out, stream=None):
        _check(lib().fzp_aperture_mask(self._h, row_begin, row_end, _ptr(out), _stream(stream)))

    def profile(self, enable: bool = True):
        _check(lib().fzp_profile_enable(self._h, int(enable)))

    def profile_read(self) -> dict:
        p = Profile()
        _check(lib().fzp_profile_read(self._h, ctypes.byref(p)))
        return {"dominant_ms": p.dominant_ms, "dominant_launches": p.dominant_launches,
                "kernel_launches": p.kernel_launches, "dominant_name": p.dominant_name.decode()}

    def close(self):
        if getattr(self, "_h", None):
            lib().fzp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """fzp_batch_plan / fzp_batch_propagate: many apertures replayed as one CUDA graph.

    `problems` is a list of dicts with the keyword arguments of Plan."""

    def __init__(self, problems):
        n = len(problems)
        arr = (Params * n)()
        self._keep = []
        for k, pr in enumerate(problems):
            d = pr.get("deform")
            self._keep.append(d)
            org, ox, oy = _origin(pr.get("x0"))
            arr[k] = Params(D=pr["D"], f=pr["f"], lam=pr["lam"], dx=pr.get("dx", 0.0), N=pr.get("N", 0), M=pr["M"],
                            form=pr.get("form", FORM_AUTO), pitch=pr["pitch"],
                            precision=pr.get("precision", PREC_AUTO_1E4), stripe_rows=pr.get("stripe_rows", 0),
                            deform=ctypes.pointer(d) if d is not None else None, promote=pr.get("promote", 0),
                            row_batch=pr.get("row_batch", 0), cluster=pr.get("cluster", 0),
                            levels=pr.get("levels", 0), centre_open=pr.get("centre_open", 0),
                            roi_origin=org, x0=ox, y0=oy, conv=pr.get("conv", CONV_AUTO))
        h = ctypes.c_void_p()
        _check(lib().fzp_batch_plan(arr, n, ctypes.byref(h)))
        self._h = h
        self.n = n

    def info(self, i: int) -> dict:
        inf = PlanInfo()
        _check(lib().fzp_batch_info(self._h, i, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in inf._fields_}

    def propagate(self, fields, stream=None):
        ptrs = (ctypes.c_void_p * self.n)(*[_ptr(f) for f in fields])
        _check(lib().fzp_batch_propagate(self._h, ptrs, _stream(stream)))

    def intensity(self, i: int, field, out, stream=None):
        """fzp_batch_intensity: I = |U|^2 of instance i into `out` (float64 M x M)."""
        _check(lib().fzp_batch_intensity(self._h, i, _ptr(field), _ptr(out), _stream(stream)))

    @property
    def kernels(self) -> int:
        """Kernel launches of one replay of the captured graph."""
        n = ctypes.c_int64()
        _check(lib().fzp_batch_kernels(self._h, ctypes.byref(n)))
        return n.value

    def metrics(self, i: int, field, stream=None) -> dict:
        m = Metrics()
        _check(lib().fzp_batch_metrics(self._h, i, _ptr(field), _stream(stream), ctypes.byref(m)))
        return m.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib().fzp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SurrogateNet:
    """fzp_surrogate_*: MLP n_in -> hidden x layers (SiLU) -> n_out, BF16 tensor-core
    products with FP32 accumulation, FP32 masters, AdamW -- all in libfzp kernels."""

    def __init__(self, n_in=8, hidden=512, layers=3, n_out=4114, max_batch=256, seed=0):
        h = ctypes.c_void_p()
        _check(lib().fzp_surrogate_create(n_in, hidden, layers, n_out, max_batch, seed, ctypes.byref(h)))
        self._h = h
        self.n_in, self.n_out, self.max_batch = n_in, n_out, max_batch
        self.sizes = [n_in] + [hidden] * layers + [n_out]

    @property
    def param_count(self) -> int:
        return int(lib().fzp_surrogate_param_count(self._h))

    def get_params(self):
        import numpy as np
        buf = np.zeros(self.param_count, dtype=np.float32)
        _check(lib().fzp_surrogate_params(self._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), buf.size, 0))
        return buf

    def set_params(self, vec):
        import numpy as np
        buf = np.ascontiguousarray(vec, dtype=np.float32)
        assert buf.size == self.param_count
        _check(lib().fzp_surrogate_params(self._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), buf.size, 1))

    def infer(self, x, y, stream=None):
        _check(lib().fzp_surrogate_infer(self._h, _ptr(x), x.shape[0], _ptr(y), _stream(stream)))

    def grad(self, x, y, grad_out=None, loss_out=None, stream=None):
        _check(lib().fzp_surrogate_grad(self._h, _ptr(x), _ptr(y), x.shape[0], _ptr(grad_out), _ptr(loss_out),
                                        _stream(stream)))

    def train_step(self, x, y, lr, weight_decay=0.0, loss_out=None, stream=None):
        _check(lib().fzp_surrogate_train_step(self._h, _ptr(x), _ptr(y), x.shape[0], lr, weight_decay,
                                              _ptr(loss_out), _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().fzp_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _params(D, f, lam, M, pitch, dx=0.0, N=0, form=FORM_AUTO, precision=PREC_FP32, stripe_rows=0, promote=0,
            row_batch=0, cluster=0, levels=0, centre_open=0, x0=None, exact_radii=0, conv=0) -> Params:
    org, ox, oy = _origin(x0)
    return Params(D=D, f=f, lam=lam, dx=dx, N=N, M=M, form=form, pitch=pitch, precision=precision,
                  stripe_rows=stripe_rows, deform=None, promote=promote, row_batch=row_batch, cluster=cluster,
                  levels=levels, centre_open=centre_open, roi_origin=org, x0=ox, y0=oy, exact_radii=exact_radii,
                  conv=conv)


def plan_query(**kw) -> dict:
    """fzp_plan_query: the plan description fzp_plan would produce (keyword
    arguments of Plan, without deform), from host code alone -- no GPU needed."""
    p = _params(**kw)
    inf = PlanInfo()
    _check(lib().fzp_plan_query(ctypes.byref(p), ctypes.byref(inf)))
    return {k: getattr(inf, k) for k, _ in inf._fields_}


def zone_thresholds(**kw):
    """fzp_zone_thresholds: the host-built zone-threshold table S_m (numpy int64)."""
    import numpy as np
    p = _params(**kw)
    n = ctypes.c_int64()
    _check(lib().fzp_zone_thresholds(ctypes.byref(p), None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.int64)
    _check(lib().fzp_zone_thresholds(ctypes.byref(p), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     out.size, ctypes.byref(n)))
    return out


def metrics_noalloc(field, D: float, f: float, lam: float, M: int, pitch: float, dx: float = 0.0, N: int = 0,
                    levels: int = 0, centre_open: int = 0, stream=None) -> dict:
    """fzp_metrics_noalloc: the metric extractor without a plan and without any
    device allocation (scratch in a static device array; M <= 512).  `levels`
    enters through the default dx (Fig. 18 Stage 1); the aperture count does
    not depend on the plate's levels or centre configuration.

    `field` is a torch tensor (complex128, contiguous, M*M elements, on the
    current CUDA device) or a raw device address (int) that the caller vouches
    for; a tensor that does not fit the call is refused here, before the
    kernels read M*M samples from it."""
    if not isinstance(field, int):
        import torch
        if not (field.is_cuda and field.dtype == torch.complex128 and field.is_contiguous()
                and field.numel() == M * M):
            raise ValueError("metrics_noalloc: field must be a contiguous complex128 CUDA tensor of M*M "
                             f"= {M * M} elements (got {tuple(field.shape)} {field.dtype} on {field.device})")
        if field.device.index != torch.cuda.current_device():
            raise ValueError(f"metrics_noalloc: field is on {field.device}, the current device is "
                             f"cuda:{torch.cuda.current_device()}")
    p = Params(D=D, f=f, lam=lam, dx=dx, N=N, M=M, form=0, pitch=pitch, precision=0, stripe_rows=0, deform=None,
               levels=levels, centre_open=centre_open)
    m = Metrics()
    _check(lib().fzp_metrics_noalloc(ctypes.byref(p), _ptr(field), _stream(stream), ctypes.byref(m)))
    return m.as_dict()


def selftest_wait_timeout(limit_us: int, stream=None) -> None:
    """fzp_selftest_wait_timeout: one bounded device wait that runs out; raises
    FzpError with status FZP_E_TIMEOUT, the expected outcome."""
    _check(lib().fzp_selftest_wait_timeout(int(limit_us), _stream(stream)))


def version() -> str:
    return lib().fzp_version().decode()
