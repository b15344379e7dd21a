"""Thin ctypes binding of the C ABI in include/heget.h.

Argument marshalling only: every step of the hot path runs in libheget.so.
Device arrays are CUDA tensors, checked on the host (CUDA, contiguous, element
size, length) and passed as ``tensor.data_ptr()``, or raw integer addresses,
passed unchecked; streams are ``torch.cuda.Stream`` objects or their
``cuda_stream`` integers (0 = legacy default stream).
Loading fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libheget.so")

HEGET_OK, HEGET_EINVAL, HEGET_ENOMEM, HEGET_ECUDA, HEGET_ETIMEOUT, HEGET_EBUSY, HEGET_ENOTFOUND = range(7)
HEGET_FP32, HEGET_FP64 = 32, 64
HEGET_SAMPLER_FIXED, HEGET_SAMPLER_UNIFORM, HEGET_SAMPLER_TOY_PDF = 0, 1, 2
HEGET_ALG_TREE, HEGET_ALG_SUBSET = 0, 1
HEGET_OBS_PT_MAX, HEGET_OBS_PT, HEGET_OBS_ETA, HEGET_OBS_DR, HEGET_OBS_DR_MIN, HEGET_OBS_SQRT_S = range(6)
HEGET_HIST_MAX_SPECS, HEGET_HIST_MAX_BINS = 8, 1024

STATUS_NAMES = {0: "HEGET_OK", 1: "HEGET_EINVAL", 2: "HEGET_ENOMEM", 3: "HEGET_ECUDA",
                4: "HEGET_ETIMEOUT", 5: "HEGET_EBUSY", 6: "HEGET_ENOTFOUND"}


class HegetError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class heget_params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("q_charge", C.c_double), ("pt_min", C.c_double),
                ("eta_max", C.c_double), ("dr_min", C.c_double)]


class heget_sampler(C.Structure):
    _fields_ = [("kind", C.c_int), ("sqrt_s", C.c_double), ("lo", C.c_double), ("hi", C.c_double),
                ("e_beam", C.c_double), ("floor", C.c_double), ("max_tries", C.c_int)]


class heget_xsec_result(C.Structure):
    _fields_ = [("sigma_fb", C.c_double), ("err_fb", C.c_double), ("sum_w", C.c_double),
                ("sum_w2", C.c_double), ("accept", C.c_double), ("reserved", C.c_double),
                ("n_pass", C.c_int64), ("n_total", C.c_int64), ("n_tries", C.c_int64),
                ("n_escalated", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


def sampler_fixed(sqrt_s: float) -> heget_sampler:
    return heget_sampler(HEGET_SAMPLER_FIXED, sqrt_s, 0.0, 0.0, 7000.0, 100.0, 64)


def sampler_uniform(lo: float, hi: float) -> heget_sampler:
    return heget_sampler(HEGET_SAMPLER_UNIFORM, 0.0, lo, hi, 7000.0, 100.0, 64)


def sampler_toy_pdf(e_beam: float = 7000.0, floor: float = 100.0, max_tries: int = 64) -> heget_sampler:
    return heget_sampler(HEGET_SAMPLER_TOY_PDF, 0.0, 0.0, 0.0, e_beam, floor, max_tries)


class heget_xsec_request(C.Structure):
    _fields_ = [("n", C.c_int), ("precision", C.c_int), ("seed", C.c_uint64), ("i0", C.c_int64),
                ("N", C.c_int64), ("sampler", heget_sampler), ("result_dev", C.c_void_p),
                ("w_out", C.c_void_p)]


class heget_server_cfg(C.Structure):
    _fields_ = [("max_inflight", C.c_int), ("max_launch_work", C.c_double), ("hbm_reserve_frac", C.c_double),
                ("arena_bytes", C.c_uint64)]


class heget_request(C.Structure):
    _fields_ = [("n", C.c_int), ("precision", C.c_int), ("seed", C.c_uint64), ("i0", C.c_int64),
                ("N", C.c_int64), ("sampler", heget_sampler)]


class heget_result(C.Structure):
    _fields_ = [("result", heget_xsec_result), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("status", C.c_int), ("reserved", C.c_int)]


class heget_hist_spec(C.Structure):
    _fields_ = [("observable", C.c_int32), ("nbins", C.c_int32), ("lo", C.c_double), ("hi", C.c_double)]


_lib = None
P, I32, I64, U64, D = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double

# name -> (restype, argtypes); the exported symbols of include/heget.h
SIGNATURES = {
    "heget_create": (I32, [I32, C.POINTER(P)]),
    "heget_destroy": (None, [P]),
    "heget_set_params": (I32, [P, C.POINTER(heget_params)]),
    "heget_get_params": (I32, [P, C.POINTER(heget_params)]),
    "heget_last_error": (C.c_char_p, []),
    "heget_version": (C.c_char_p, []),
    "heget_phase_space": (I32, [P, U64, I64, I32, D, P, P, P]),
    "heget_phase_space_ex": (I32, [P, U64, I64, I64, I32, C.POINTER(heget_sampler), P, P, P, P, P, P, P]),
    "heget_amp2": (I32, [P, I32, I64, P, P, I32, P, P]),
    "heget_check": (I32, [P, P]),
    "heget_log_table": (I32, [P, P, I64, P]),
    "heget_sincos_2pi": (I32, [P, P, I64, P]),
    "heget_f32_round": (I32, [P, P, I64, P]),
    "heget_ward": (I32, [P, I32, I64, P, I32, I32, P, P]),
    "heget_xsec_async": (I32, [P, I32, U64, I64, I64, C.POINTER(heget_sampler), I32, P, P, P]),
    "heget_xsec": (I32, [P, I32, I64, U64, C.POINTER(heget_sampler), I32, C.POINTER(heget_xsec_result), P]),
    "heget_xsec_launch": (I32, [P, I32, U64, I64, I64, C.POINTER(heget_sampler), I32, P, P]),
    "heget_xsec_finalize": (I32, [P, P, P]),
    "heget_measure_fma_peak": (I32, [P, I32, C.POINTER(C.c_double)]),
    "heget_xsec_batch": (I32, [P, C.POINTER(heget_xsec_request), I32, P]),
    "heget_set_helicity_sampling": (I32, [P, I32]),
    "heget_get_helicity_sampling": (I32, [P]),
    "heget_hist": (I32, [P, I32, U64, I64, I64, C.POINTER(heget_sampler), P, C.POINTER(heget_hist_spec), I32, P,
                         P]),
    "heget_autotune": (I32, [P, I32, I32, I32, I64, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "heget_autotune_shape": (I32, [P, I32, I32, I64, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_double)]),
    "heget_set_shape": (I32, [P, I32, I32, I32]),
    "heget_set_graphs": (I32, [P, I32]),
    "heget_get_graphs": (I32, [P, C.POINTER(I64), C.POINTER(I64)]),
    "heget_get_shape": (I32, [P, I32, I32]),
    "heget_shape_info": (I32, [I32, I32, I32, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "heget_autotune_save": (I32, [P, C.c_char_p]),
    "heget_autotune_load": (I32, [P, C.c_char_p]),
    "heget_graph_xsec": (I32, [P, I32, I64, C.POINTER(heget_sampler), I32, P, C.POINTER(P)]),
    "heget_graph_launch": (I32, [P, U64, I64, P]),
    "heget_graph_destroy": (None, [P]),
    "heget_set_tile": (I32, [P, I32, I32, I32, I32]),
    "heget_set_algorithm": (I32, [P, I32]),
    "heget_set_escalation": (I32, [P, D]),
    "heget_get_escalation": (I32, [P, C.POINTER(C.c_double)]),
    "heget_amp2_escalated": (I32, [P, P, C.POINTER(I64)]),
    "heget_get_algorithm": (I32, [P]),
    "heget_get_tile": (I32, [P, I32, I32, I32]),
    "heget_xsec_noalloc": (I32, [I32, I32, U64, I64, I64, C.POINTER(heget_sampler), C.POINTER(heget_params),
                                 I32, P, P]),
    "heget_sum": (I32, [P, P, I64, P, P]),
    "heget_xsec_combine": (I32, [C.POINTER(heget_xsec_result), I32, I32, C.POINTER(heget_xsec_result)]),
    "heget_hist_combine": (I32, [C.POINTER(C.c_void_p), I32, I64, P]),
    "heget_server_start": (I32, [P, C.POINTER(heget_server_cfg), C.POINTER(P)]),
    "heget_submit": (I32, [P, C.POINTER(heget_request), C.POINTER(U64)]),
    "heget_poll": (I32, [P, U64, C.POINTER(heget_result)]),
    "heget_wait": (I32, [P, U64, D, C.POINTER(heget_result)]),
    "heget_server_stop": (I32, [P]),
}


def load(path: str = LIB_PATH):
    """Load libheget.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} not found: build it with paper_0908_4403_gb300.build.build() "
                              "(there is no CPU fallback)")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int):
    if status != HEGET_OK:
        raise HegetError(status, load().heget_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _dev(x, what, count, itemsize, floating=None):
    """Device address of tensor `x`, which must be a contiguous CUDA tensor
    of at least `count` elements of `itemsize` bytes (floating point or not,
    when `floating` says so).  A wrong argument raises HEGET_EINVAL here, on
    the host, instead of reaching a kernel.  None and raw integer addresses
    pass through unchecked (the library checks NULL)."""
    if x is None or isinstance(x, int):
        return x
    if not getattr(x, "is_cuda", False):
        bad = "must be a CUDA tensor"
    elif not x.is_contiguous():
        bad = "must be contiguous"
    elif x.element_size() != itemsize or (floating is not None and x.dtype.is_floating_point != floating):
        kind = "" if floating is None else (" floating-point" if floating else " integer")
        bad = f"needs {itemsize}-byte{kind} elements, got {x.dtype}"
    elif x.numel() < count:
        bad = f"holds {x.numel()} elements, needs {count}"
    else:
        return x.data_ptr()
    raise HegetError(HEGET_EINVAL, f"{what} {bad}")


def _f64s(x, what, count):
    return _dev(x, what, count, 8, True)


def _result(x, what="result_dev"):
    """A device buffer of at least sizeof(heget_xsec_result) bytes, any dtype."""
    if x is None or isinstance(x, int):
        return x
    return _dev(x, what, -(-C.sizeof(heget_xsec_result) // x.element_size()), x.element_size())


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---------------------------------------------------------------------------
# one wrapper per C entry point, same names
# ---------------------------------------------------------------------------

def heget_create(device: int = 0):
    h = P()
    _check(load().heget_create(device, C.byref(h)))
    return h


def heget_destroy(ctx):
    load().heget_destroy(ctx)


def heget_set_params(ctx, alpha=1 / 137.035999, q_charge=2 / 3, pt_min=20.0, eta_max=2.5, dr_min=0.4):
    p = heget_params(alpha, q_charge, pt_min, eta_max, dr_min)
    _check(load().heget_set_params(ctx, C.byref(p)))


def heget_get_params(ctx) -> heget_params:
    p = heget_params()
    _check(load().heget_get_params(ctx, C.byref(p)))
    return p


def heget_version() -> str:
    return load().heget_version().decode()


def heget_phase_space(ctx, seed, N, n, sqrt_s, momenta, weights=None, stream=None):
    _check(load().heget_phase_space(ctx, seed, N, n, sqrt_s, _f64s(momenta, "momenta", N * (n + 2) * 4),
                                    _f64s(weights, "weights", N), _stream(stream)))


def heget_phase_space_ex(ctx, seed, i0, N, n, sampler, momenta=None, weights=None, sqrt_s=None, y=None,
                         mask=None, tries=None, stream=None):
    _check(load().heget_phase_space_ex(ctx, seed, i0, N, n, C.byref(sampler),
                                       _f64s(momenta, "momenta", N * (n + 2) * 4), _f64s(weights, "weights", N),
                                       _f64s(sqrt_s, "sqrt_s", N), _f64s(y, "y", N), _dev(mask, "mask", N, 1),
                                       _dev(tries, "tries", N, 4, False), _stream(stream)))


def heget_amp2(ctx, n, N, momenta, amp2, hel_mask=None, precision=HEGET_FP64, stream=None):
    _check(load().heget_amp2(ctx, n, N, _f64s(momenta, "momenta", N * (n + 2) * 4),
                             _dev(hel_mask, "hel_mask", max(1, (1 << max(n + 2, 0)) // 32), 4, False), precision,
                             _f64s(amp2, "amp2", N), _stream(stream)))


def heget_ward(ctx, n, N, momenta, photon, ratio, precision=HEGET_FP64, stream=None):
    _check(load().heget_ward(ctx, n, N, _f64s(momenta, "momenta", N * (n + 2) * 4), photon, precision,
                             _f64s(ratio, "ratio", N), _stream(stream)))


def heget_log_table(x, y, N, stream=None):
    _check(load().heget_log_table(_f64s(x, "x", N), _f64s(y, "y", N), N, _stream(stream)))


def heget_sincos_2pi(words, cs, N, stream=None):
    _check(load().heget_sincos_2pi(_dev(words, "words", 2 * N, 4, False), _f64s(cs, "cs", 2 * N), N,
                                   _stream(stream)))


def heget_f32_round(x, y, N, stream=None):
    _check(load().heget_f32_round(_f64s(x, "x", N), _dev(y, "y", N, 4, True), N, _stream(stream)))


def heget_check(ctx, stream=None):
    _check(load().heget_check(ctx, _stream(stream)))


def heget_xsec_async(ctx, n, seed, i0, N, sampler, precision, result_dev, w_out=None, stream=None):
    _check(load().heget_xsec_async(ctx, n, seed, i0, N, C.byref(sampler), precision, _result(result_dev),
                                   _f64s(w_out, "w_out", N), _stream(stream)))


def heget_xsec(ctx, n, N, seed, sampler, precision=HEGET_FP32, stream=None) -> heget_xsec_result:
    out = heget_xsec_result()
    _check(load().heget_xsec(ctx, n, N, seed, C.byref(sampler), precision, C.byref(out), _stream(stream)))
    return out


def heget_xsec_launch(ctx, n, seed, i0, N, sampler, precision, w_out=None, stream=None):
    _check(load().heget_xsec_launch(ctx, n, seed, i0, N, C.byref(sampler), precision, _f64s(w_out, "w_out", N),
                                    _stream(stream)))


def heget_xsec_finalize(ctx, result_dev, stream=None):
    _check(load().heget_xsec_finalize(ctx, _result(result_dev), _stream(stream)))


def heget_measure_fma_peak(ctx, precision=HEGET_FP32) -> float:
    v = C.c_double()
    _check(load().heget_measure_fma_peak(ctx, precision, C.byref(v)))
    return v.value


def heget_set_helicity_sampling(ctx, on):
    _check(load().heget_set_helicity_sampling(ctx, int(on)))


def heget_get_helicity_sampling(ctx):
    return load().heget_get_helicity_sampling(ctx)


def hist_bins(specs):
    """Output length of heget_hist: 2 sum (nbins + 2) doubles."""
    return 2 * sum(sp[1] + 2 for sp in specs)


def heget_hist(ctx, n, seed, i0, N, sampler, w, specs, out, stream=None):
    """specs: list of (observable, nbins, lo, hi); out: device doubles of
    length hist_bins(specs), per spec (nbins + 2) rows of (sum w, sum w^2)."""
    arr = (heget_hist_spec * len(specs))(*[heget_hist_spec(*sp) for sp in specs])
    _check(load().heget_hist(ctx, n, seed, i0, N, C.byref(sampler), _f64s(w, "w", N), arr, len(specs),
                             _f64s(out, "out", hist_bins(specs)), _stream(stream)))


def heget_xsec_batch(ctx, requests, stream=None):
    """requests: list of dicts with n, precision, seed, i0, N, sampler, result_dev (tensor), w_out (tensor|None)."""
    arr = (heget_xsec_request * len(requests))()
    for a, r in zip(arr, requests):
        a.n, a.precision, a.seed, a.i0, a.N = r["n"], r["precision"], r["seed"], r.get("i0", 0), r["N"]
        a.sampler = r["sampler"]
        a.result_dev = _result(r["result_dev"])
        a.w_out = _f64s(r.get("w_out"), "w_out", r["N"])
    _check(load().heget_xsec_batch(ctx, arr, len(requests), _stream(stream)))


def heget_autotune(ctx, n, precision, kind, probe_points):
    """Returns (best_tile, best_ms); the context keeps the best tile."""
    t, ms = C.c_int(), C.c_double()
    _check(load().heget_autotune(ctx, n, precision, kind, probe_points, C.byref(t), C.byref(ms)))
    return t.value, ms.value


def heget_autotune_shape(ctx, n, precision, probe_points):
    """(best shape, best tile, ms) of the fused cross section, kept in ctx."""
    sh, t, ms = C.c_int(), C.c_int(), C.c_double()
    _check(load().heget_autotune_shape(ctx, n, precision, probe_points, C.byref(sh), C.byref(t), C.byref(ms)))
    return sh.value, t.value, ms.value


def heget_set_graphs(ctx, on):
    _check(load().heget_set_graphs(ctx, int(on)))


def heget_get_graphs(ctx):
    """(setting, captures, replays) of the batch launch graphs."""
    c, r = C.c_int64(), C.c_int64()
    v = load().heget_get_graphs(ctx, C.byref(c), C.byref(r))
    return v, c.value, r.value


def heget_set_shape(ctx, n, precision, shape):
    _check(load().heget_set_shape(ctx, n, precision, shape))


def heget_get_shape(ctx, n, precision) -> int:
    return load().heget_get_shape(ctx, n, precision)


def heget_shape_info(n, precision, shape):
    """(threads per block, helicity rows per lane, subtree groups) of a shape; zeros for shape 0."""
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(load().heget_shape_info(n, precision, shape, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def heget_autotune_save(ctx, path):
    _check(load().heget_autotune_save(ctx, str(path).encode()))


def heget_autotune_load(ctx, path):
    _check(load().heget_autotune_load(ctx, str(path).encode()))


def heget_graph_xsec(ctx, n, N, sampler, precision, result_dev):
    g = P()
    _check(load().heget_graph_xsec(ctx, n, N, C.byref(sampler), precision, _result(result_dev), C.byref(g)))
    return g


def heget_graph_launch(graph, seed, i0=0, stream=None):
    _check(load().heget_graph_launch(graph, seed, i0, _stream(stream)))


def heget_graph_destroy(graph):
    load().heget_graph_destroy(graph)


def heget_set_algorithm(ctx, alg):
    _check(load().heget_set_algorithm(ctx, alg))


def heget_get_algorithm(ctx) -> int:
    return load().heget_get_algorithm(ctx)


def heget_set_escalation(ctx, tau):
    _check(load().heget_set_escalation(ctx, tau))


def heget_get_escalation(ctx) -> float:
    v = C.c_double()
    _check(load().heget_get_escalation(ctx, C.byref(v)))
    return v.value


def heget_amp2_escalated(ctx, stream=None) -> int:
    v = I64()
    _check(load().heget_amp2_escalated(ctx, _stream(stream), C.byref(v)))
    return v.value


def heget_set_tile(ctx, n, precision, kind, tile):
    _check(load().heget_set_tile(ctx, n, precision, kind, tile))


def heget_get_tile(ctx, n, precision, kind) -> int:
    return load().heget_get_tile(ctx, n, precision, kind)


def heget_xsec_noalloc(device, n, seed, i0, N, sampler, precision, result_dev, params=None, stream=None):
    """heget_xsec_async for callers that cannot allocate device memory (no context needed)."""
    pp = C.byref(params) if params is not None else None
    _check(load().heget_xsec_noalloc(device, n, seed, i0, N, C.byref(sampler), pp, precision, _ptr(result_dev),
                                     _stream(stream)))


def heget_xsec_combine(parts, sampler_kind) -> heget_xsec_result:
    """The result of disjoint point shards (host structs, in order) merged as
    one call's (host arithmetic in the library; no GPU needed)."""
    arr = (heget_xsec_result * max(1, len(parts)))(*parts)
    out = heget_xsec_result()
    _check(load().heget_xsec_combine(arr, len(parts), sampler_kind, C.byref(out)))
    return out


def heget_hist_combine(parts):
    """Element-wise TwoSum combination of equal-length host float64 arrays
    (numpy), in order; returns a new numpy array."""
    import numpy as np
    arrs = [np.ascontiguousarray(p, dtype=np.float64).ravel() for p in parts]
    if not arrs or any(a.size != arrs[0].size for a in arrs):
        raise HegetError(HEGET_EINVAL, "histograms of different layouts (or none)")
    out = np.empty(arrs[0].size)
    ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    _check(load().heget_hist_combine(ptrs, len(arrs), out.size, out.ctypes.data_as(C.c_void_p)))
    return out


def heget_sum(ctx, x, N, out_dev, stream=None):
    _check(load().heget_sum(ctx, _f64s(x, "x", N), N, _f64s(out_dev, "out_dev", 2), _stream(stream)))


def heget_server_start(ctx, max_inflight=0, max_launch_work=0.0, hbm_reserve_frac=0.0, arena_bytes=0):
    cfg = heget_server_cfg(max_inflight, max_launch_work, hbm_reserve_frac, arena_bytes)
    s = P()
    _check(load().heget_server_start(ctx, C.byref(cfg), C.byref(s)))
    return s


def heget_submit(server, n, seed, N, sampler, precision=HEGET_FP32, i0=0) -> int:
    q = heget_request(n, precision, seed, i0, N, sampler)
    t = U64()
    _check(load().heget_submit(server, C.byref(q), C.byref(t)))
    return t.value


def heget_poll(server, ticket):
    """The finished heget_result, or None while the request runs."""
    r = heget_result()
    st = load().heget_poll(server, ticket, C.byref(r))
    if st == HEGET_EBUSY:
        return None
    _check(st)
    return r


def heget_wait(server, ticket, timeout_s=60.0) -> heget_result:
    r = heget_result()
    _check(load().heget_wait(server, ticket, timeout_s, C.byref(r)))
    return r


def heget_server_stop(server):
    _check(load().heget_server_stop(server))


def result_from_tensor(t) -> heget_xsec_result:
    """Decode a heget_xsec_result stored in a (CPU) uint8/float64 tensor of 80 bytes."""
    import numpy as np
    raw = np.ascontiguousarray(t.cpu().numpy()).view(np.uint8).tobytes()
    return heget_xsec_result.from_buffer_copy(raw[:C.sizeof(heget_xsec_result)])
