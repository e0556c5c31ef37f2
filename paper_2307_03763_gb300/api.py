"""Thin Python binding of libgb (``include/gb.h``): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module checks
tensor dtypes, devices and shapes, passes raw device pointers and the current
CUDA stream, and turns nonzero status codes into exceptions.  There is no CPU
fallback: if ``libgb.so`` is missing the import of the library raises.

Tensors: theta float64 (n, 8) in the order (f0, fdot, beta, lambda, A, iota,
psi, phi0); data complex128; weights 1/S float64; all on one CUDA device.
"""
import ctypes
import os

import torch

from . import build as _build

GB_OK, GB_EINVAL, GB_ECUDA, GB_ETIMEOUT, GB_ENOMEM = 0, -1, -2, -3, -4
GB_FP64, GB_MIXED = 0, 1
# bound on the relative template error of the mixed path, |h_mixed - h_fp64| <= EPS |h| in the
# window's noise-weighted norm, used by mh_certified (measured maximum and margin in gb.h)
MIXED_EPS = 1e-5
PRECISIONS = {"fp64": GB_FP64, "mixed": GB_MIXED, GB_FP64: GB_FP64, GB_MIXED: GB_MIXED}


class GBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libgb error %d: %s" % (code, msg))
        self.code = code


class Window(ctypes.Structure):
    _fields_ = [("k0", ctypes.c_int64), ("data_off", ctypes.c_int64), ("cand_off", ctypes.c_int64),
                ("W", ctypes.c_int32), ("N", ctypes.c_int32), ("n_cand", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Obs(ctypes.Structure):
    _fields_ = [("T_obs", ctypes.c_double), ("arm_L", ctypes.c_double), ("orbit_model", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class GAParams(ctypes.Structure):
    _fields_ = [("tournament", ctypes.c_int32), ("reserved", ctypes.c_int32), ("p_cross", ctypes.c_double),
                ("p_mut", ctypes.c_double), ("mut_scale", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("item", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("ms", ctypes.c_double), ("ms_default", ctypes.c_double)]


_LIB = None
_P = ctypes.c_void_p
_I32, _I64 = ctypes.c_int32, ctypes.c_int64

_SIGNATURES = {
    "gb_ctx_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(Obs), ctypes.c_int]),
    "gb_ctx_destroy": (ctypes.c_int, [_P]),
    "gb_last_error": (ctypes.c_char_p, [_P]),
    "gb_ctx_check": (ctypes.c_int, [_P]),
    "gb_launch_count": (ctypes.c_uint64, [_P]),
    "gb_ctx_set_time_budget": (ctypes.c_int, [_P, ctypes.c_double]),
    "gb_ctx_set_kernel_events": (ctypes.c_int, [_P, _P, _P]),
    "gb_waveform": (ctypes.c_int, [_P, ctypes.c_int, _P, _I64, _I32, _P, _P, _P, _P]),
    "gb_loglik": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(Window), _I32, _P, _P, _P, _P, _I64, _P, _I64,
                                 _P, _P, _P, _P]),
    "gb_loglik_aet": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(Window), _I32, _P, _P, _P, _P, _P, _P, _I64,
                                     _P, _I64, _P, _P, _P, _P]),
    "gb_loglik_phase_aet": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(Window), _I32, _P, _P, _P, _P, _P, _P,
                                           _I64, _P, _I64, _P, _P, _P, _P, _P]),
    "gb_loglik_grad_aet": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(Window), _I32, _P, _P, _P, _P, _P, _P,
                                          _I64, _P, _I64, _P, _P, _P]),
    "gb_waveform_aet": (ctypes.c_int, [_P, ctypes.c_int, _P, _I64, _I32, _P, _P, _P, _P, _P]),
    "gb_loglik_phase": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(Window), _I32, _P, _P, _P, _P, _I64, _P,
                                       _I64, _P, _P, _P, _P, _P]),
    "gb_loglik_grad": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(Window), _I32, _P, _P, _P, _P, _I64, _P,
                                      _I64, _P, _P, _P]),
    "gb_mh_independence": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P, _P, _I32, _P, _P, _P]),
    "gb_snr_multi": (ctypes.c_int, [_P, ctypes.POINTER(Window), _I32, _P, _P, _P, _P, _I64, _P, _I64, _I32, _P, _P,
                                    _P, _P]),
    "gb_loglik_rows": (ctypes.c_int, [_P, ctypes.POINTER(Window), _I32, _P, _P, _P, _P, _I64, _P, _I64, _P, _P, _P,
                                      _P, _P, _P, _P]),
    "gb_mh_certified": (ctypes.c_int, [_P, ctypes.POINTER(Window), _I32, _P, _P, _P, _P, _I64, _P, _P, _P, _P, _I32,
                                       ctypes.c_double, _I32, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gb_loglik_mixed_noalloc": (ctypes.c_int, [ctypes.POINTER(Obs), ctypes.POINTER(Window), _I32, _P, _P, _P, _P,
                                               _I64, _P, _I64, _P, _P, _P, _P, _P, ctypes.c_char_p, _I32]),
    "gb_ga_step": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P, _P, _P, ctypes.c_uint64, _P, _P,
                                  ctypes.POINTER(GAParams), _P, _P, _P, _P]),
    "gb_gauss_refit": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, _P, _P, _P]),
    "gb_noise_median": (ctypes.c_int, [_P, ctypes.POINTER(Window), _I32, _P, _P, _I64, _I32, _P, _P, _P, _P]),
    "gb_kde_build": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P, _I32, ctypes.c_double, _P, _P, _P]),
    "gb_kde_draw": (ctypes.c_int, [_P, _I32, _I32, _P, _I32, _P, _P, ctypes.c_uint64, _P, _P, _P, _P, _P, _P]),
    "gb_philox4x32": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint32, _P, _P]),
    "gb_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(Window), _I32, _P, _P, _P, _P, _I64, _P, _I64,
                                   _P, _I32, ctypes.POINTER(Tuning), _P]),
    "gb_draw_gaussian": (ctypes.c_int, [_P, _I32, _I32, _P, _P, ctypes.c_uint64, _P, _P, _P, _P, _P, _P]),
}


def library_path():
    return _build.LIB


def lib():
    """Load libgb.so (built in-tree by ``build.build()``); raise if it is missing."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libgb.so is not built (%s); run paper_2307_03763_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _need(t, dtype, device, name, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if t.device != device:
        raise ValueError("%s must be on %s, got %s" % (name, device, t.device))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))


def windows_array(windows):
    """ctypes array of gb_window_t from a sequence of (k0, W, N, data_off, cand_off, n_cand)."""
    arr = (Window * max(1, len(windows)))()
    for i, (k0, W, N, doff, coff, nc) in enumerate(windows):
        arr[i] = Window(int(k0), int(doff), int(coff), int(W), int(N), int(nc), 0)
    return arr


class Context:
    """A libgb context on one CUDA device (owns the orbit and twiddle tables)."""

    def __init__(self, T_obs, arm_L=2.5e9, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libgb needs a CUDA device; none is available")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.T_obs = float(T_obs)
        self.arm_L = float(arm_L)
        h = ctypes.c_void_p()
        obs = Obs(self.T_obs, self.arm_L, 0, 0)
        rc = lib().gb_ctx_create(ctypes.byref(h), ctypes.byref(obs), self.device.index)
        if rc != GB_OK:
            raise GBError(rc, "gb_ctx_create failed")
        self._h = h
        self._win_cache = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().gb_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != GB_OK:
            raise GBError(rc, lib().gb_last_error(self._h).decode())

    def set_time_budget(self, seconds):
        """Work budget of the persistent mixed-precision kernels (0: none)."""
        self._check(lib().gb_ctx_set_time_budget(self._h, float(seconds)))

    def set_kernel_events(self, start, end):
        """Record two torch.cuda.Event objects (timing enabled, recorded at
        least once so that they exist) around the next mixed-precision
        likelihood kernels; None for both clears them."""
        if (start is None) != (end is None):
            raise ValueError("give both events or neither")
        h = [None if e is None else ctypes.c_void_p(e.cuda_event) for e in (start, end)]
        if start is not None and not (h[0].value and h[1].value):
            raise ValueError("record each event once before passing it")
        self._check(lib().gb_ctx_set_kernel_events(self._h, h[0], h[1]))

    def launch_count(self):
        """Kernels launched by this context's calls so far."""
        return int(lib().gb_launch_count(self._h))

    def check(self):
        """Synchronise and raise if a kernel met a non-finite parameter."""
        self._check(lib().gb_ctx_check(self._h))

    def _windows(self, windows):
        key = tuple(tuple(int(x) for x in w) for w in windows)
        arr = self._win_cache.get(key)
        if arr is None:
            if len(self._win_cache) > 64:
                self._win_cache.clear()
            arr = windows_array(windows)
            self._win_cache[key] = arr
        return arr, len(windows)

    def waveform(self, theta, N, prec="fp64"):
        """A/E templates on bins q - N/2 .. q + N/2 - 1: returns hA, hE (B, N) complex128, q (B,) int64."""
        B = theta.shape[0] if theta.dim() == 2 else -1
        _need(theta, torch.float64, self.device, "theta", (B, 8))
        hA = torch.empty((B, N), dtype=torch.complex128, device=self.device)
        hE = torch.empty_like(hA)
        q = torch.empty(B, dtype=torch.int64, device=self.device)
        self._check(lib().gb_waveform(self._h, PRECISIONS[prec], _ptr(theta), B, int(N), _ptr(hA), _ptr(hE),
                                      _ptr(q), _stream(self.device)))
        return hA, hE, q

    def _data_args(self, windows, dA, dE, wA, wE, theta):
        nb = dA.shape[0]
        _need(dA, torch.complex128, self.device, "dA", (nb,))
        _need(dE, torch.complex128, self.device, "dE", (nb,))
        _need(wA, torch.float64, self.device, "wA", (nb,))
        _need(wE, torch.float64, self.device, "wE", (nb,))
        n = theta.shape[0] if theta.dim() == 2 else -1
        _need(theta, torch.float64, self.device, "theta", (n, 8))
        arr, nw = self._windows(windows)
        return arr, nw, nb, n

    def loglik(self, windows, dA, dE, wA, wE, theta, prec="fp64", out=None):
        """logL, <d|h>, <h|h> per candidate (Eq. 2 over each window)."""
        arr, nw, nb, n = self._data_args(windows, dA, dE, wA, wE, theta)
        if out is None:
            out = tuple(torch.zeros(n, dtype=torch.float64, device=self.device) for _ in range(3))
        logL, dh, hh = out
        for t, name in ((logL, "logL"), (dh, "dh"), (hh, "hh")):
            if t is not None:
                _need(t, torch.float64, self.device, name, (n,))
        self._check(lib().gb_loglik(self._h, PRECISIONS[prec], arr, nw, _ptr(dA), _ptr(dE), _ptr(wA), _ptr(wE),
                                    nb, _ptr(theta), n, _ptr(logL), _ptr(dh), _ptr(hh), _stream(self.device)))
        return logL, dh, hh

    def loglik_aet(self, windows, dA, dE, dT, wA, wE, wT, theta, prec="fp64", out=None):
        """logL, <d|h>, <h|h> with the T channel in the windows above f*/2 (see gb_loglik_aet)."""
        arr, nw, nb, n = self._data_args(windows, dA, dE, wA, wE, theta)
        _need(dT, torch.complex128, self.device, "dT", (nb,))
        _need(wT, torch.float64, self.device, "wT", (nb,))
        if out is None:
            out = tuple(torch.zeros(n, dtype=torch.float64, device=self.device) for _ in range(3))
        logL, dh, hh = out
        for t, name in ((logL, "logL"), (dh, "dh"), (hh, "hh")):
            if t is not None:
                _need(t, torch.float64, self.device, name, (n,))
        self._check(lib().gb_loglik_aet(self._h, PRECISIONS[prec], arr, nw, _ptr(dA), _ptr(dE), _ptr(dT), _ptr(wA),
                                        _ptr(wE), _ptr(wT), nb, _ptr(theta), n, _ptr(logL), _ptr(dh), _ptr(hh),
                                        _stream(self.device)))
        return logL, dh, hh

    def loglik_phase_aet(self, windows, dA, dE, dT, wA, wE, wT, theta, prec="fp64", out=None):
        """loglik_phase with the T channel above f*/2 (see gb_loglik_phase_aet)."""
        arr, nw, nb, n = self._data_args(windows, dA, dE, wA, wE, theta)
        _need(dT, torch.complex128, self.device, "dT", (nb,))
        _need(wT, torch.float64, self.device, "wT", (nb,))
        if out is None:
            out = tuple(torch.zeros(n, dtype=torch.float64, device=self.device) for _ in range(4))
        logL, dh, dh_im, hh = out
        _need(dh_im, torch.float64, self.device, "dh_im", (n,))
        for t, name in ((logL, "logL"), (dh, "dh"), (hh, "hh")):
            if t is not None:
                _need(t, torch.float64, self.device, name, (n,))
        self._check(lib().gb_loglik_phase_aet(self._h, PRECISIONS[prec], arr, nw, _ptr(dA), _ptr(dE), _ptr(dT),
                                              _ptr(wA), _ptr(wE), _ptr(wT), nb, _ptr(theta), n, _ptr(logL), _ptr(dh),
                                              _ptr(dh_im), _ptr(hh), _stream(self.device)))
        return logL, dh, dh_im, hh

    def loglik_grad_aet(self, windows, dA, dE, dT, wA, wE, wT, theta, prec="fp64", out=None):
        """logL and d logL / d theta (n, 8) with the T channel above f*/2 (see gb_loglik_grad_aet)."""
        arr, nw, nb, n = self._data_args(windows, dA, dE, wA, wE, theta)
        _need(dT, torch.complex128, self.device, "dT", (nb,))
        _need(wT, torch.float64, self.device, "wT", (nb,))
        if out is None:
            out = (torch.zeros(n, dtype=torch.float64, device=self.device),
                   torch.zeros((n, 8), dtype=torch.float64, device=self.device))
        logL, grad = out
        if logL is not None:
            _need(logL, torch.float64, self.device, "logL", (n,))
        _need(grad, torch.float64, self.device, "grad", (n, 8))
        self._check(lib().gb_loglik_grad_aet(self._h, PRECISIONS[prec], arr, nw, _ptr(dA), _ptr(dE), _ptr(dT),
                                             _ptr(wA), _ptr(wE), _ptr(wT), nb, _ptr(theta), n, _ptr(logL),
                                             _ptr(grad), _stream(self.device)))
        return logL, grad

    def waveform_aet(self, theta, N, prec="fp64"):
        """A/E/T templates: hA, hE, hT (B, N) complex128, q (B,) int64."""
        B = theta.shape[0] if theta.dim() == 2 else -1
        _need(theta, torch.float64, self.device, "theta", (B, 8))
        hA = torch.empty((B, N), dtype=torch.complex128, device=self.device)
        hE, hT = torch.empty_like(hA), torch.empty_like(hA)
        q = torch.empty(B, dtype=torch.int64, device=self.device)
        self._check(lib().gb_waveform_aet(self._h, PRECISIONS[prec], _ptr(theta), B, int(N), _ptr(hA), _ptr(hE),
                                          _ptr(hT), _ptr(q), _stream(self.device)))
        return hA, hE, hT, q

    def loglik_phase(self, windows, dA, dE, wA, wE, theta, prec="fp64", out=None):
        """logL, <d|h>, <d|h>_im, <h|h> per candidate (see gb_loglik_phase)."""
        arr, nw, nb, n = self._data_args(windows, dA, dE, wA, wE, theta)
        if out is None:
            out = tuple(torch.zeros(n, dtype=torch.float64, device=self.device) for _ in range(4))
        logL, dh, dh_im, hh = out
        _need(dh_im, torch.float64, self.device, "dh_im", (n,))
        for t, name in ((logL, "logL"), (dh, "dh"), (hh, "hh")):
            if t is not None:
                _need(t, torch.float64, self.device, name, (n,))
        self._check(lib().gb_loglik_phase(self._h, PRECISIONS[prec], arr, nw, _ptr(dA), _ptr(dE), _ptr(wA),
                                          _ptr(wE), nb, _ptr(theta), n, _ptr(logL), _ptr(dh), _ptr(dh_im),
                                          _ptr(hh), _stream(self.device)))
        return logL, dh, dh_im, hh

    def loglik_grad(self, windows, dA, dE, wA, wE, theta, prec="fp64", out=None):
        """logL and d logL / d theta (n, 8) by the adjoint kernel."""
        arr, nw, nb, n = self._data_args(windows, dA, dE, wA, wE, theta)
        if out is None:
            out = (torch.zeros(n, dtype=torch.float64, device=self.device),
                   torch.zeros((n, 8), dtype=torch.float64, device=self.device))
        logL, grad = out
        if logL is not None:
            _need(logL, torch.float64, self.device, "logL", (n,))
        _need(grad, torch.float64, self.device, "grad", (n, 8))
        self._check(lib().gb_loglik_grad(self._h, PRECISIONS[prec], arr, nw, _ptr(dA), _ptr(dE), _ptr(wA),
                                         _ptr(wE), nb, _ptr(theta), n, _ptr(logL), _ptr(grad),
                                         _stream(self.device)))
        return logL, grad

    def autotune(self, windows, dA, dE, wA, wE, theta, prec="mixed", reps=3):
        """Pick the fastest launch shape for this batch (see gb_autotune); returns a dict."""
        arr, nw, nb, n = self._data_args(windows, dA, dE, wA, wE, theta)
        logL = torch.empty(n, dtype=torch.float64, device=self.device)
        t = Tuning()
        self._check(lib().gb_autotune(self._h, PRECISIONS[prec], arr, nw, _ptr(dA), _ptr(dE), _ptr(wA), _ptr(wE),
                                      nb, _ptr(theta), n, _ptr(logL), int(reps), ctypes.byref(t),
                                      _stream(self.device)))
        return {"item": t.item, "blocks_per_sm": t.blocks_per_sm, "tile": t.tile, "ms": t.ms,
                "ms_default": t.ms_default}

    def ga_step(self, n_win, pop, theta, dh, hh, box, seed, gen_in, gen_out, params, grad=None, out=None,
                best=None, dh_im=None):
        """One generation of the genetic search (see gb_ga_step); returns (out, best).

        With dh_im (from loglik_phase) the fitness is maximised over phi0."""
        n = n_win * pop
        _need(theta, torch.float64, self.device, "theta", (n, 8))
        _need(dh, torch.float64, self.device, "dh", (n,))
        _need(hh, torch.float64, self.device, "hh", (n,))
        if dh_im is not None:
            _need(dh_im, torch.float64, self.device, "dh_im", (n,))
        _need(box, torch.float64, self.device, "box", (n_win, 16))
        _need(gen_in, torch.int64, self.device, "gen_in", (1,))
        _need(gen_out, torch.int64, self.device, "gen_out", (1,))
        if grad is not None:
            _need(grad, torch.float64, self.device, "grad", (n_win, 8))
        if out is None:
            out = torch.empty_like(theta)
        if best is None:
            best = torch.empty((n_win, 8), dtype=torch.float64, device=self.device)
        _need(out, torch.float64, self.device, "out", (n, 8))
        _need(best, torch.float64, self.device, "best", (n_win, 8))
        self._check(lib().gb_ga_step(self._h, n_win, pop, _ptr(theta), _ptr(dh), _ptr(hh), _ptr(dh_im), _ptr(box),
                                     int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(gen_in), _ptr(gen_out),
                                     ctypes.byref(params), _ptr(grad), _ptr(out), _ptr(best),
                                     _stream(self.device)))
        return out, best

    def draw_gaussian(self, mu, chol, n, seed, round_in, round_out, out=None):
        """Gaussian proposals per window (see gb_draw_gaussian): theta (n_win*n, 8), log_g, log_u (n_win, n)."""
        n_win = mu.shape[0]
        _need(mu, torch.float64, self.device, "mu", (n_win, 8))
        _need(chol, torch.float64, self.device, "chol", (n_win, 8, 8))
        _need(round_in, torch.int64, self.device, "round_in", (1,))
        _need(round_out, torch.int64, self.device, "round_out", (1,))
        if out is None:
            out = (torch.empty((n_win * n, 8), dtype=torch.float64, device=self.device),
                   torch.empty((n_win, n), dtype=torch.float64, device=self.device),
                   torch.empty((n_win, n), dtype=torch.float64, device=self.device))
        th, lg, lu = out
        _need(th, torch.float64, self.device, "theta", (n_win * n, 8))
        _need(lg, torch.float64, self.device, "log_g", (n_win, n))
        _need(lu, torch.float64, self.device, "log_u", (n_win, n))
        self._check(lib().gb_draw_gaussian(self._h, n_win, int(n), _ptr(mu), _ptr(chol),
                                           int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(round_in), _ptr(round_out),
                                           _ptr(th), _ptr(lg), _ptr(lu), _stream(self.device)))
        return th, lg, lu

    def noise_median(self, windows, dA, dE, debias=False, weights=None):
        """Median-periodogram noise of every window (see gb_noise_median): S (n_win, 2).
        weights = (wA, wE) are set to 1/S over each window's bins."""
        nb = dA.shape[0]
        _need(dA, torch.complex128, self.device, "dA", (nb,))
        _need(dE, torch.complex128, self.device, "dE", (nb,))
        arr, nw = self._windows(windows)
        S = torch.empty((nw, 2), dtype=torch.float64, device=self.device)
        wA = wE = None
        if weights is not None:
            wA, wE = weights
            _need(wA, torch.float64, self.device, "wA", (nb,))
            _need(wE, torch.float64, self.device, "wE", (nb,))
        self._check(lib().gb_noise_median(self._h, arr, nw, _ptr(dA), _ptr(dE), nb, int(bool(debias)), _ptr(S),
                                          _ptr(wA), _ptr(wE), _stream(self.device)))
        return S

    def kde_build(self, theta, chain, box, grid, floor, out):
        """Paired KDE proposal tables from each window's chain (see gb_kde_build);
        out = (cdf (n_win, 3, grid^2), ext (n_win, 3, 4))."""
        nw, n = chain.shape
        cdf, ext = out
        _need(theta, torch.float64, self.device, "theta", (nw * n, 8))
        _need(chain, torch.int32, self.device, "chain", (nw, n))
        _need(box, torch.float64, self.device, "box", (nw, 16))
        _need(cdf, torch.float64, self.device, "cdf", (nw, 3, grid * grid))
        _need(ext, torch.float64, self.device, "ext", (nw, 3, 4))
        self._check(lib().gb_kde_build(self._h, nw, n, _ptr(theta), _ptr(chain), _ptr(box), int(grid), float(floor),
                                       _ptr(cdf), _ptr(ext), _stream(self.device)))
        return cdf, ext

    def kde_draw(self, box, grid, cdf, ext, n, seed, round_in, round_out, out=None):
        """n proposals per window from the paired KDE tables (see gb_kde_draw): theta (n_win*n, 8), log_g, log_u."""
        nw = box.shape[0]
        _need(box, torch.float64, self.device, "box", (nw, 16))
        _need(cdf, torch.float64, self.device, "cdf", (nw, 3, grid * grid))
        _need(ext, torch.float64, self.device, "ext", (nw, 3, 4))
        _need(round_in, torch.int64, self.device, "round_in", (1,))
        _need(round_out, torch.int64, self.device, "round_out", (1,))
        if out is None:
            out = (torch.empty((nw * n, 8), dtype=torch.float64, device=self.device),
                   torch.empty((nw, n), dtype=torch.float64, device=self.device),
                   torch.empty((nw, n), dtype=torch.float64, device=self.device))
        th, lg, lu = out
        _need(th, torch.float64, self.device, "theta", (nw * n, 8))
        _need(lg, torch.float64, self.device, "log_g", (nw, n))
        _need(lu, torch.float64, self.device, "log_u", (nw, n))
        self._check(lib().gb_kde_draw(self._h, nw, int(n), _ptr(box), int(grid), _ptr(cdf), _ptr(ext),
                                      int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(round_in), _ptr(round_out), _ptr(th),
                                      _ptr(lg), _ptr(lu), _stream(self.device)))
        return th, lg, lu

    def gauss_refit(self, theta, chain, chol0, ratio, inflate, kappa, floor, out):
        """Gaussian refit of each window's proposal to its chain (see gb_gauss_refit).
        out = (mu, chol): chol holds the current proposal's factor on entry."""
        nw, n = chain.shape
        _need(theta, torch.float64, self.device, "theta", (nw * n, 8))
        _need(chain, torch.int32, self.device, "chain", (nw, n))
        _need(chol0, torch.float64, self.device, "chol0", (nw, 8, 8))
        mu, chol = out
        _need(mu, torch.float64, self.device, "mu", (nw, 8))
        _need(chol, torch.float64, self.device, "chol", (nw, 8, 8))
        self._check(lib().gb_gauss_refit(self._h, nw, n, _ptr(theta), _ptr(chain), _ptr(chol0), float(ratio),
                                         float(inflate), float(kappa), float(floor), _ptr(mu), _ptr(chol),
                                         _stream(self.device)))
        return mu, chol

    def philox(self, seed, n):
        """n blocks of Philox-4x32-10 with key = seed, counter (i, 0, 0, 0): (n, 4) int64 of uint32 values."""
        out = torch.empty(4 * n, dtype=torch.int32, device=self.device)
        self._check(lib().gb_philox4x32(self._h, int(seed) & 0xFFFFFFFFFFFFFFFF, int(n), _ptr(out),
                                        _stream(self.device)))
        return (out.to(torch.int64) & 0xFFFFFFFF).view(n, 4)

    def mh_independence(self, logL, log_g, log_u, temperature, literal=False, out=None):
        """Chains (n_chains, n) int32 and accept counts from (n_chains, n) float64 inputs (Alg. 4)."""
        if logL.dim() != 2:
            raise ValueError("logL must be (n_chains, n)")
        nc, n = logL.shape
        for t, name in ((logL, "logL"), (log_g, "log_g"), (log_u, "log_u")):
            _need(t, torch.float64, self.device, name, (nc, n))
        _need(temperature, torch.float64, self.device, "temperature", (nc,))
        if out is None:
            out = (torch.empty((nc, n), dtype=torch.int32, device=self.device),
                   torch.empty(nc, dtype=torch.int32, device=self.device))
        chain, acc = out
        _need(chain, torch.int32, self.device, "chain", (nc, n))
        _need(acc, torch.int32, self.device, "n_accept", (nc,))
        self._check(lib().gb_mh_independence(self._h, nc, n, _ptr(logL), _ptr(log_g), _ptr(log_u),
                                             _ptr(temperature), 1 if literal else 0, _ptr(chain), _ptr(acc),
                                             _stream(self.device)))
        return chain, acc

    def loglik_rows(self, windows, dA, dE, wA, wE, theta, rows, row_lo, row_hi, out=None):
        """FP64 logL, <d|h>, <h|h> of listed rows (see gb_loglik_rows): window w's entries are
        rows[cand_off + j], j in [row_lo[w], row_hi[w]); the other rows of the outputs are kept."""
        arr, nw, nb, n = self._data_args(windows, dA, dE, wA, wE, theta)
        _need(rows, torch.int32, self.device, "rows", (n,))
        _need(row_lo, torch.int32, self.device, "row_lo", (nw,))
        _need(row_hi, torch.int32, self.device, "row_hi", (nw,))
        if out is None:
            out = tuple(torch.zeros(n, dtype=torch.float64, device=self.device) for _ in range(3))
        logL, dh, hh = out
        for t, name in ((logL, "logL"), (dh, "dh"), (hh, "hh")):
            if t is not None:
                _need(t, torch.float64, self.device, name, (n,))
        self._check(lib().gb_loglik_rows(self._h, arr, nw, _ptr(dA), _ptr(dE), _ptr(wA), _ptr(wE), nb, _ptr(theta),
                                         n, _ptr(rows), _ptr(row_lo), _ptr(row_hi), _ptr(logL), _ptr(dh), _ptr(hh),
                                         _stream(self.device)))
        return logL, dh, hh

    def mh_certified(self, windows, dA, dE, wA, wE, theta, log_g, log_u, temperature, literal=False, eps=MIXED_EPS,
                     max_iter=2, out=None):
        """Mixed-precision logL of every proposal and the chains an all-FP64 evaluation gives
        (see gb_mh_certified).  Window w holds rows [w n, (w + 1) n).  Returns
        (chain, n_accept, logL, dh, hh, n_exact, pending); pending (1,) int32 is 0 when every
        decision is certified."""
        arr, nw, nb, nrow = self._data_args(windows, dA, dE, wA, wE, theta)
        n = nrow // max(nw, 1)
        for t, name in ((log_g, "log_g"), (log_u, "log_u")):
            _need(t, torch.float64, self.device, name, (nw, n))
        _need(temperature, torch.float64, self.device, "temperature", (nw,))
        if out is None:
            f = lambda: torch.empty(nrow, dtype=torch.float64, device=self.device)
            out = (torch.empty((nw, n), dtype=torch.int32, device=self.device),
                   torch.empty(nw, dtype=torch.int32, device=self.device), f(), f(), f(),
                   torch.empty(nw, dtype=torch.int32, device=self.device),
                   torch.empty(1, dtype=torch.int32, device=self.device))
        chain, acc, logL, dh, hh, n_exact, pending = out
        _need(chain, torch.int32, self.device, "chain", (nw, n))
        _need(acc, torch.int32, self.device, "n_accept", (nw,))
        for t, name in ((logL, "logL"), (dh, "dh"), (hh, "hh")):
            _need(t, torch.float64, self.device, name, (nrow,))
        if n_exact is not None:
            _need(n_exact, torch.int32, self.device, "n_exact", (nw,))
        _need(pending, torch.int32, self.device, "pending", (1,))
        self._check(lib().gb_mh_certified(self._h, arr, nw, _ptr(dA), _ptr(dE), _ptr(wA), _ptr(wE), nb, _ptr(theta),
                                          _ptr(log_g), _ptr(log_u), _ptr(temperature), 1 if literal else 0,
                                          float(eps), int(max_iter), _ptr(logL), _ptr(dh), _ptr(hh), _ptr(chain),
                                          _ptr(acc), _ptr(n_exact), _ptr(pending), _stream(self.device)))
        return chain, acc, logL, dh, hh, n_exact, pending

    def snr_multi(self, windows, dA, dE, wA, wE, theta, kmax=None):
        """Multi-signal SNR of each window's sources (its candidate rows; see
        gb_snr_multi): returns rho (n_win,), gram (n_win, kmax, kmax) and
        dh (n,) = <d|s_i>.  dA, dE may be None (then rho and dh are None)."""
        nb = wA.shape[0]
        _need(wA, torch.float64, self.device, "wA", (nb,))
        _need(wE, torch.float64, self.device, "wE", (nb,))
        if dA is not None:
            _need(dA, torch.complex128, self.device, "dA", (nb,))
            _need(dE, torch.complex128, self.device, "dE", (nb,))
        n = theta.shape[0] if theta.dim() == 2 else -1
        _need(theta, torch.float64, self.device, "theta", (n, 8))
        arr, nw = self._windows(windows)
        if kmax is None:
            kmax = max([1] + [int(w[5]) for w in windows])
        gram = torch.full((nw, kmax, kmax), float("nan"), dtype=torch.float64, device=self.device)
        rho = dh = None
        if dA is not None:
            rho = torch.empty(nw, dtype=torch.float64, device=self.device)
            dh = torch.zeros(n, dtype=torch.float64, device=self.device)
        self._check(lib().gb_snr_multi(self._h, arr, nw, _ptr(dA), _ptr(dE), _ptr(wA), _ptr(wE), nb, _ptr(theta), n,
                                       int(kmax), _ptr(gram), _ptr(dh), _ptr(rho), _stream(self.device)))
        return rho, gram, dh
