"""Thin ctypes binding of libp2s (include/p2s.h), same names as the C ABI.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors passed by data_ptr on the
current torch stream.  The library is loaded on first use; a missing library
raises immediately (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libp2s.so")

P2S_OK, P2S_EINVAL, P2S_ENOMEM, P2S_ECUDA, P2S_ETIMEOUT, P2S_EBUSY, P2S_EUNSUPPORTED = range(7)
PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2, "fp16": 3}
FORMS = {"scatter": 0, "gather": 1, "fft": 2}


class p2s_basis(C.Structure):
    _fields_ = [("H", C.POINTER(C.c_double)), ("K", C.c_int), ("taps_h", C.c_int), ("taps_w", C.c_int)]


class p2s_mlp(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("dims", C.POINTER(C.c_int)),
                ("W", C.POINTER(C.POINTER(C.c_double))), ("b", C.POINTER(C.POINTER(C.c_double)))]


class p2s_corr_params(C.Structure):
    _fields_ = [("anchor_spacing", C.c_int), ("n_kernels", C.c_int), ("corr_len_px", C.POINTER(C.c_double)),
                ("fft_guard", C.c_int), ("kappa", C.c_double)]


class p2s_image(C.Structure):
    _fields_ = [("data", C.c_void_p), ("H", C.c_int), ("W", C.c_int), ("C", C.c_int)]


class p2s_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int), ("total_ms", C.c_double), ("flops", C.c_double),
                ("bytes", C.c_double)]


class p2s_tune_result(C.Structure):
    _fields_ = [("option", C.c_int), ("option2", C.c_int), ("n", C.c_int), ("value", C.c_int * 8),
                ("value2", C.c_int * 8), ("ms", C.c_float * 8), ("best", C.c_int)]


class p2s_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_inflight_batches", C.c_int), ("max_batch", C.c_int)]


class p2s_server_counters(C.Structure):
    _fields_ = [("completed", C.c_longlong), ("batches", C.c_longlong), ("pending", C.c_longlong),
                ("mean_batch", C.c_double), ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t)]


class p2s_geometry(C.Structure):
    _fields_ = [("anchors_h", C.c_int), ("anchors_w", C.c_int), ("torus_h", C.c_int), ("torus_w", C.c_int),
                ("alpha_stride", C.c_int)]


# every symbol include/p2s.h declares, with its signature
_SIGS = {
    "p2s_create": (C.c_int, [C.POINTER(p2s_basis), C.POINTER(p2s_mlp), C.POINTER(p2s_corr_params), C.c_int, C.c_int,
                             C.POINTER(C.c_void_p)]),
    "p2s_destroy": (None, [C.c_void_p]),
    "p2s_status_string": (C.c_char_p, [C.c_int]),
    "p2s_last_error": (C.c_char_p, []),
    "p2s_geometry_of": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(p2s_geometry)]),
    "p2s_simulate": (C.c_int, [C.c_void_p, C.POINTER(p2s_image), C.c_int, C.POINTER(C.c_float),
                               C.POINTER(C.c_ulonglong), C.POINTER(p2s_image), C.c_void_p]),
    "p2s_simulate_host": (C.c_int, [C.c_void_p, C.POINTER(p2s_image), C.c_int, C.POINTER(C.c_float),
                                    C.POINTER(C.c_ulonglong), C.POINTER(p2s_image), C.c_void_p]),
    "p2s_stage_noise": (C.c_int, [C.c_void_p, C.c_ulonglong, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "p2s_stage_fields": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_float),
                                   C.POINTER(C.c_ulonglong), C.c_void_p, C.c_void_p]),
    "p2s_stage_warp": (C.c_int, [C.c_void_p, C.POINTER(p2s_image), C.c_void_p, C.POINTER(p2s_image), C.c_void_p]),
    "p2s_stage_mlp": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "p2s_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "p2s_selftest_stall": (C.c_int, [C.c_void_p, C.c_void_p]),
    "p2s_server_create": (C.c_int, [C.c_void_p, C.POINTER(p2s_server_config), C.POINTER(C.c_void_p)]),
    "p2s_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_float, C.c_ulonglong,
                                    C.c_void_p, C.POINTER(C.c_longlong)]),
    "p2s_server_poll": (C.c_int, [C.c_void_p, C.c_longlong, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "p2s_server_wait": (C.c_int, [C.c_void_p, C.c_longlong, C.c_double, C.POINTER(C.c_double)]),
    "p2s_server_stats": (C.c_int, [C.c_void_p, C.POINTER(p2s_server_counters)]),
    "p2s_server_destroy": (None, [C.c_void_p]),
    "p2s_autotune": (C.c_int, [C.c_void_p, C.POINTER(p2s_image), C.c_int, C.POINTER(C.c_float),
                               C.POINTER(C.c_ulonglong), C.POINTER(p2s_image), C.c_void_p, C.c_int,
                               C.POINTER(p2s_tune_result)]),
    "p2s_get_option": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "p2s_stage_mlp16": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "p2s_simulate_spectral": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(p2s_image), C.c_int, C.POINTER(C.c_float),
                                        C.POINTER(C.c_ulonglong), C.POINTER(p2s_image), C.c_void_p]),
    "p2s_contraction_scales": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_float)]),
    "p2s_stage_blur": (C.c_int, [C.c_void_p, C.POINTER(p2s_image), C.c_void_p, C.POINTER(p2s_image), C.c_void_p]),
    "p2s_stage_mlp_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "p2s_noll_covariance": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "p2s_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "p2s_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "p2s_profile_read": (C.c_int, [C.c_void_p, C.POINTER(p2s_kernel_stat), C.c_int, C.POINTER(C.c_int)]),
}

_lib = None


def lib() -> C.CDLL:
    """Load libp2s.so (built in-tree by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libp2s.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class P2SError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.p2s_status_string(status).decode()
        detail = L.p2s_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")
        self.status = status


def _check(st: int, where: str):
    if st != P2S_OK:
        raise P2SError(st, where)


def noll_covariance(j_max: int = 36) -> np.ndarray:
    """R_Z for modes 2..j_max at D/r0 = 1, computed by the library (host FP64)."""
    n = j_max - 1
    out = np.zeros(n * n, dtype=np.float64)
    _check(lib().p2s_noll_covariance(j_max, out.ctypes.data_as(C.POINTER(C.c_double))), "p2s_noll_covariance")
    return out.reshape(n, n)


def _torch():
    import torch

    return torch


def _stream_handle(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _image(t) -> p2s_image:
    if t.dtype.__str__() != "torch.float32" or not t.is_contiguous():
        raise ValueError("images must be contiguous float32 tensors [H, W, C]")
    h, w, c = t.shape
    return p2s_image(C.c_void_p(t.data_ptr()), h, w, c)


def _host_image(a: np.ndarray) -> p2s_image:
    if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host images must be contiguous float32 arrays [H, W, C]")
    h, w, c = a.shape
    return p2s_image(C.c_void_p(a.ctypes.data), h, w, c)


class Simulator:
    """p2s_create / p2s_destroy around a context, plus the per-call entry points."""

    def __init__(self, basis: np.ndarray, taps, layers, anchor_spacing: int = 8, corr_len_px=(16.0,),
                 fft_guard: int = -1, kappa: float = 0.0, precision: str = "fp32", form: str = "scatter"):
        L = lib()
        H = np.ascontiguousarray(basis, dtype=np.float64)
        self.K, self.T = H.shape
        self.taps = (int(taps[0]), int(taps[1]))
        self._keep = [H]
        b = p2s_basis(H.ctypes.data_as(C.POINTER(C.c_double)), self.K, self.taps[0], self.taps[1])
        dims = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
        dims_a = (C.c_int * len(dims))(*dims)
        Ws = [np.ascontiguousarray(W, dtype=np.float64) for W, _ in layers]
        bs = [np.ascontiguousarray(bb, dtype=np.float64) for _, bb in layers]
        self._keep += Ws + bs
        Wp = (C.POINTER(C.c_double) * len(Ws))(*[w.ctypes.data_as(C.POINTER(C.c_double)) for w in Ws])
        bp = (C.POINTER(C.c_double) * len(bs))(*[v.ctypes.data_as(C.POINTER(C.c_double)) for v in bs])
        m = p2s_mlp(len(layers), dims_a, Wp, bp)
        ell = np.ascontiguousarray(corr_len_px, dtype=np.float64)
        self._keep.append(ell)
        cp = p2s_corr_params(int(anchor_spacing), len(ell), ell.ctypes.data_as(C.POINTER(C.c_double)), int(fft_guard),
                             float(kappa))
        ctx = C.c_void_p()
        _check(L.p2s_create(C.byref(b), C.byref(m), C.byref(cp), PRECISIONS[precision], FORMS[form], C.byref(ctx)),
               "p2s_create")
        self.ctx = ctx
        self.precision, self.form = precision, form
        self.anchor_spacing = anchor_spacing

    def close(self):
        if getattr(self, "ctx", None):
            lib().p2s_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, stream=None):
        """Synchronise and raise if a device-side bounded wait gave up since the last check."""
        _check(lib().p2s_check(self.ctx, _stream_handle(stream)), "p2s_check")

    def profile(self, enable: bool):
        """Start (clearing) or stop per-kernel event timing."""
        _check(lib().p2s_profile(self.ctx, 1 if enable else 0), "p2s_profile")

    def profile_read(self) -> list:
        """[{name, launches, total_ms, flops, bytes}] aggregated per kernel name."""
        arr = (p2s_kernel_stat * 64)()
        n = C.c_int()
        _check(lib().p2s_profile_read(self.ctx, arr, 64, C.byref(n)), "p2s_profile_read")
        return [dict(name=arr[i].name.decode(), launches=arr[i].launches, total_ms=arr[i].total_ms,
                     flops=arr[i].flops, bytes=arr[i].bytes) for i in range(min(n.value, 64))]

    def geometry(self, H: int, W: int) -> dict:
        g = p2s_geometry()
        _check(lib().p2s_geometry_of(self.ctx, H, W, C.byref(g)), "p2s_geometry_of")
        return {f: getattr(g, f) for f, _ in p2s_geometry._fields_}

    @staticmethod
    def _meta(d_over_r0, seeds, n):
        dr = np.ascontiguousarray(np.broadcast_to(np.asarray(d_over_r0, dtype=np.float32), (n,)))
        sd = np.ascontiguousarray(np.broadcast_to(np.asarray(seeds, dtype=np.uint64), (n,)))
        return dr, sd

    def simulate(self, frames, d_over_r0, seeds, out=None, stream=None):
        """frames: list of CUDA tensors [H, W, C] (or a tensor [n, H, W, C]); returns the outputs."""
        torch = _torch()
        frames = list(frames)
        n = len(frames)
        if out is None:
            out = [torch.empty_like(f) for f in frames]
        dr, sd = self._meta(d_over_r0, seeds, n)
        fi = (p2s_image * max(n, 1))(*[_image(f) for f in frames])
        oi = (p2s_image * max(n, 1))(*[_image(o) for o in out])
        _check(lib().p2s_simulate(self.ctx, fi, n, dr.ctypes.data_as(C.POINTER(C.c_float)),
                                  sd.ctypes.data_as(C.POINTER(C.c_ulonglong)), oi, _stream_handle(stream)),
               "p2s_simulate")
        return out

    def autotune(self, frames, d_over_r0, seeds, out=None, reps: int = 2, stream=None):
        """Times the path's kernel and tile-shape candidates on this batch, keeps the fastest.
        Returns {"option": name or None, "option2": name or None, "candidates": {key: ms},
        "best": key}, key = the option's value, or (value, value2) when a second option is tuned
        with it (value2 0: that option left as it was)."""
        torch = _torch()
        frames = list(frames)
        n = len(frames)
        if out is None:
            out = [torch.empty_like(f) for f in frames]
        dr, sd = self._meta(d_over_r0, seeds, n)
        fi = (p2s_image * max(n, 1))(*[_image(f) for f in frames])
        oi = (p2s_image * max(n, 1))(*[_image(o) for o in out])
        r = p2s_tune_result()
        _check(lib().p2s_autotune(self.ctx, fi, n, dr.ctypes.data_as(C.POINTER(C.c_float)),
                                  sd.ctypes.data_as(C.POINTER(C.c_ulonglong)), oi, _stream_handle(stream), int(reps),
                                  C.byref(r)), "p2s_autotune")
        names = {v: k for k, v in self.OPTIONS.items()}
        key = (lambda i: (r.value[i], r.value2[i])) if r.option2 else (lambda i: r.value[i])
        cands = {key(i): float(r.ms[i]) for i in range(r.n)}
        return {"option": names.get(r.option), "option2": names.get(r.option2), "candidates": cands,
                "best": key(r.best) if r.n else None}

    def simulate_host(self, frames, d_over_r0, seeds, out=None, stream=None):
        """Host (NumPy float32) frames in and out; copies happen inside the call."""
        frames = list(frames)
        n = len(frames)
        if out is None:
            out = [np.empty_like(f) for f in frames]
        dr, sd = self._meta(d_over_r0, seeds, n)
        fi = (p2s_image * max(n, 1))(*[_host_image(f) for f in frames])
        oi = (p2s_image * max(n, 1))(*[_host_image(o) for o in out])
        _check(lib().p2s_simulate_host(self.ctx, fi, n, dr.ctypes.data_as(C.POINTER(C.c_float)),
                                       sd.ctypes.data_as(C.POINTER(C.c_ulonglong)), oi, _stream_handle(stream)),
               "p2s_simulate_host")
        return out

    def stage_noise(self, seed: int, mode: int, torus_h: int, torus_w: int, stream=None):
        torch = _torch()
        out = torch.empty(torus_h * torus_w, dtype=torch.float32, device="cuda")
        _check(lib().p2s_stage_noise(self.ctx, int(seed), int(mode), torus_h, torus_w, C.c_void_p(out.data_ptr()),
                                     _stream_handle(stream)), "p2s_stage_noise")
        return out.view(torus_h, torus_w)

    def stage_fields(self, H: int, W: int, d_over_r0, seeds, stream=None):
        torch = _torch()
        n = len(np.atleast_1d(seeds))
        g = self.geometry(H, W)
        out = torch.empty((n, g["anchors_h"], g["anchors_w"], g["alpha_stride"]), dtype=torch.float32, device="cuda")
        dr, sd = self._meta(d_over_r0, seeds, n)
        _check(lib().p2s_stage_fields(self.ctx, H, W, n, dr.ctypes.data_as(C.POINTER(C.c_float)),
                                      sd.ctypes.data_as(C.POINTER(C.c_ulonglong)), C.c_void_p(out.data_ptr()),
                                      _stream_handle(stream)), "p2s_stage_fields")
        return out

    def stage_warp(self, x, alpha, stream=None):
        torch = _torch()
        out = torch.empty_like(x)
        _check(lib().p2s_stage_warp(self.ctx, C.byref(_image(x)), C.c_void_p(alpha.data_ptr()), C.byref(_image(out)),
                                    _stream_handle(stream)), "p2s_stage_warp")
        return out

    def stage_mlp(self, H: int, W: int, alpha, stream=None):
        torch = _torch()
        out = torch.empty((H, W, self.K), dtype=torch.float32, device="cuda")
        _check(lib().p2s_stage_mlp(self.ctx, H, W, C.c_void_p(alpha.data_ptr()), C.c_void_p(out.data_ptr()),
                                   _stream_handle(stream)), "p2s_stage_mlp")
        return out

    def selftest_stall(self, stream=None):
        _check(lib().p2s_selftest_stall(self.ctx, _stream_handle(stream)), "p2s_selftest_stall")

    OPTIONS = {"scatter_segment_rows": 1, "graphs": 2, "graph_instantiations": 3, "graph_updates": 4,
               "gather_band_rows": 5, "blur_then_warp": 6, "field_method": 7,
               "gather_split": 8}

    def set_option(self, name: str, value: int):
        _check(lib().p2s_set_option(self.ctx, self.OPTIONS[name], int(value)), "p2s_set_option")

    def get_option(self, name: str) -> int:
        v = C.c_int(0)
        _check(lib().p2s_get_option(self.ctx, self.OPTIONS[name], C.byref(v)), "p2s_get_option")
        return v.value

    def stage_mlp16(self, H: int, W: int, alpha, stream=None):
        """beta in the 16-bit operand layout [H][14][W][8] (int16 tensor holding FP16/BF16 bits)."""
        torch = _torch()
        out = torch.empty((H, 14, W, 8), dtype=torch.int16, device="cuda")
        _check(lib().p2s_stage_mlp16(self.ctx, H, W, C.c_void_p(alpha.data_ptr()), C.c_void_p(out.data_ptr()),
                                     _stream_handle(stream)), "p2s_stage_mlp16")
        return out

    def contraction_scales(self):
        """FP8 contexts: (beta multipliers [K + 2] (the last two for the folded-bias columns),
        2^-c): beta_k is stored as beta_k * scale[k], basis row k as H_k * 2^c / scale[k]."""
        sc = np.zeros(self.K + 2, dtype=np.float32)
        inv = C.c_float()
        _check(lib().p2s_contraction_scales(self.ctx, sc.ctypes.data_as(C.POINTER(C.c_float)), self.K + 2,
                                            C.byref(inv)), "p2s_contraction_scales")
        return sc, float(inv.value)

    def stage_blur(self, xw, beta, stream=None):
        torch = _torch()
        out = torch.empty_like(xw)
        if not beta.is_contiguous() or beta.dtype != torch.float32:
            raise ValueError("beta must be contiguous float32 [H, W, K]")
        _check(lib().p2s_stage_blur(self.ctx, C.byref(_image(xw)), C.c_void_p(beta.data_ptr()), C.byref(_image(out)),
                                    _stream_handle(stream)), "p2s_stage_blur")
        return out


class SpectralSimulator:
    """Wavelength-dependent colour (p2s_simulate_spectral): three contexts, channel c with
    basis bases[c] and the network's first layer scaled by lambda_ref / lambda_c (alpha is in
    radians at the reference wavelength).  layers: one network for all channels or a list
    of three.  Other arguments as Simulator (shared by the three contexts)."""

    def __init__(self, bases, taps, layers, wavelengths_nm=(570.0, 540.0, 450.0), ref_nm: float = 540.0,
                 **kwargs):
        if len(bases) != 3 or len(wavelengths_nm) != 3:
            raise ValueError("three bases and three wavelengths (R, G, B)")
        per = isinstance(layers[0], list)
        self.scales = [ref_nm / lam for lam in wavelengths_nm]
        self.sims = []
        for c in range(3):
            lay = layers[c] if per else layers
            W1, b1 = lay[0]
            lay_c = [(np.asarray(W1, dtype=np.float64) * self.scales[c], b1)] + list(lay[1:])
            self.sims.append(Simulator(bases[c], taps, lay_c, **kwargs))

    def close(self):
        for sm in self.sims:
            sm.close()

    def set_option(self, name: str, value: int):
        for sm in self.sims:
            sm.set_option(name, value)

    def check(self, stream=None):
        for sm in self.sims:
            sm.check(stream)

    def simulate(self, frames, d_over_r0, seeds, out=None, stream=None):
        """frames: list of CUDA tensors [H, W, 3]; returns the outputs."""
        torch = _torch()
        frames = list(frames)
        n = len(frames)
        if out is None:
            out = [torch.empty_like(f) for f in frames]
        dr, sd = Simulator._meta(d_over_r0, seeds, n)
        fi = (p2s_image * max(n, 1))(*[_image(f) for f in frames])
        oi = (p2s_image * max(n, 1))(*[_image(o) for o in out])
        ctxs = (C.c_void_p * 3)(*[sm.ctx for sm in self.sims])
        _check(lib().p2s_simulate_spectral(ctxs, fi, n, dr.ctypes.data_as(C.POINTER(C.c_float)),
                                           sd.ctypes.data_as(C.POINTER(C.c_ulonglong)), oi, _stream_handle(stream)),
               "p2s_simulate_spectral")
        return out


class Server:
    """Request loop over a Simulator (argument marshalling for the p2s_server_* calls).

    submit() takes a host float32 [H, W, C] array and an output array of the same
    shape; both must stay alive until the request is done (this object keeps
    references until wait()/poll() reports it).  Pinned buffers copy asynchronously."""

    def __init__(self, sim: "Simulator", hbm_budget_bytes: int, max_inflight: int = 4, max_batch: int = 16):
        self.sim = sim
        cfg = p2s_server_config(int(hbm_budget_bytes), int(max_inflight), int(max_batch))
        h = C.c_void_p()
        _check(lib().p2s_server_create(sim.ctx, C.byref(cfg), C.byref(h)), "p2s_server_create")
        self.h = h
        self._keep = {}

    def submit(self, x: np.ndarray, d_over_r0: float, seed: int, out: np.ndarray) -> int:
        assert x.dtype == np.float32 and x.flags.c_contiguous and x.ndim == 3
        assert out.shape == x.shape and out.dtype == np.float32 and out.flags.c_contiguous
        t = C.c_longlong()
        _check(lib().p2s_server_submit(self.h, C.c_void_p(x.ctypes.data), x.shape[0], x.shape[1], x.shape[2],
                                       float(d_over_r0), int(seed), C.c_void_p(out.ctypes.data), C.byref(t)),
               "p2s_server_submit")
        self._keep[t.value] = (x, out)
        return t.value

    def poll(self, ticket: int):
        done, lat = C.c_int(0), C.c_double(0.0)
        _check(lib().p2s_server_poll(self.h, int(ticket), C.byref(done), C.byref(lat)), "p2s_server_poll")
        if done.value:
            self._keep.pop(ticket, None)
        return bool(done.value), lat.value

    def wait(self, ticket: int, timeout_s: float = 60.0) -> float:
        lat = C.c_double(0.0)
        _check(lib().p2s_server_wait(self.h, int(ticket), float(timeout_s), C.byref(lat)), "p2s_server_wait")
        self._keep.pop(ticket, None)
        return lat.value

    def stats(self) -> dict:
        c = p2s_server_counters()
        _check(lib().p2s_server_stats(self.h, C.byref(c)), "p2s_server_stats")
        return {f: getattr(c, f) for f, _ in p2s_server_counters._fields_}

    def close(self):
        if self.h:
            lib().p2s_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
