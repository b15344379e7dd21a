"""FP64 CPU oracle for u ubar -> n photons (arXiv:0908.4403).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_0908_4403_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``heget_oracle.c`` (plain C, IEEE double, built with
``-ffp-contract=off``); this module only compiles it and marshals arguments.
Functions follow the paper's Sec. 2.1 eqs. (2), (4), (6)-(8) and Sec. 2.2
eqs. (9)-(10); see the C file for the detailed citations.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "heget_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALPHA = 1.0 / 137.035999
Q_U = 2.0 / 3.0
GEV2_TO_FB = 0.3893793721e12


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Sampler(C.Structure):
    """sqrt(s-hat) sampler: kind 0 fixed, 1 uniform [lo, hi], 2 toy PDF."""
    _fields_ = [("kind", C.c_int), ("sqrt_s", C.c_double), ("lo", C.c_double),
                ("hi", C.c_double), ("e_beam", C.c_double), ("a", C.c_double),
                ("b", C.c_double), ("floor", C.c_double), ("max_tries", C.c_int)]


class Cuts(C.Structure):
    _fields_ = [("pt_min", C.c_double), ("eta_max", C.c_double), ("dr_min", C.c_double)]


def fixed(sqrt_s: float) -> Sampler:
    return Sampler(0, sqrt_s, 0.0, 0.0, 7000.0, -0.5, 3.0, 100.0, 64)


def uniform(lo: float, hi: float) -> Sampler:
    return Sampler(1, 0.0, lo, hi, 7000.0, -0.5, 3.0, 100.0, 64)


def toy_pdf(e_beam: float = 7000.0, floor: float = 100.0, max_tries: int = 64) -> Sampler:
    return Sampler(2, 0.0, 0.0, 0.0, e_beam, -0.5, 3.0, floor, max_tries)


def cuts(pt_min=20.0, eta_max=2.5, dr_min=0.4) -> Cuts:
    return Cuts(pt_min, eta_max, dr_min)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            d, i64, u64, i32, u32 = C.c_double, C.c_int64, C.c_uint64, C.c_int, C.c_uint32
            P = C.c_void_p
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_uniform.argtypes = [u64, u64, u32, u32]
            lib.oracle_uniform.restype = d
            lib.oracle_amp2_point.argtypes = [i32, P, P, d, d]
            lib.oracle_amp2_point.restype = d
            lib.oracle_amp2.argtypes = [i32, i64, P, P, d, d, i32, P]
            lib.oracle_amp_hel.argtypes = [i32, P, i32, i32, d, d, P, P, P]
            lib.oracle_amp2_metric.argtypes = [i32, P, d, d]
            lib.oracle_amp2_metric.restype = d
            lib.oracle_phase_space_volume.argtypes = [i32, d]
            lib.oracle_phase_space_volume.restype = d
            lib.oracle_rambo.argtypes = [i32, d, P, P]
            lib.oracle_rambo.restype = d
            lib.oracle_phase_space.argtypes = [i32, u64, i64, i64, P, P, P, P, P, P, P, P]
            lib.oracle_pass_cuts.argtypes = [i32, P, d, P]
            lib.oracle_pass_cuts.restype = i32
            lib.oracle_event_weight.argtypes = [i32, d, d, d, i32]
            lib.oracle_event_weight.restype = d
            lib.oracle_event_weights.argtypes = [i32, u64, i64, i64, P, P, d, d, i32, P, P, P]
            lib.oracle_hist.argtypes = [i32, i64, P, P, P, i32, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (Salmon et al., SC'11): the counter-based
    generator that stands in for the random numbers the paper's host program
    draws and copies to the GPU (Sec. 3)."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform_draw(seed: int, point: int, stream: int, draw: int) -> float:
    """Uniform number `draw` of `stream` for phase-space point `point`:
    Philox counter (point lo, point hi, draw/2, stream), key = seed, words
    2(d&1), 2(d&1)+1 -> (m + 1/2) 2^-52 with the top 52 bits m."""
    return _load().oracle_uniform(seed, point, stream, draw)


def _mask_words(n, mask):
    if mask is None:
        return None
    m = np.asarray(mask, dtype=np.uint32)
    if m.size != max(1, (1 << (n + 2)) // 32):
        raise ValueError("hel_mask needs 2^(n+2) bits")
    return np.ascontiguousarray(m)


def amp2(n: int, mom, hel_mask=None, alpha=ALPHA, Q=Q_U, threads: int | None = None):
    """sum_{h in mask} |M_h|^2 for each point (Sec. 2.1 eqs. (6)-(8), summed
    over helicities as in eq. (2), couplings included, no colour, spin
    average or 1/n!); mom shape (N, n+2, 4)."""
    lib = _load()
    m = _f64(mom).reshape(-1, n + 2, 4)
    out = np.zeros(m.shape[0])
    mw = _mask_words(n, hel_mask)
    th = threads if threads is not None else (os.cpu_count() or 1)
    lib.oracle_amp2(n, m.shape[0], _ptr(m), _ptr(mw), alpha, Q, th, _ptr(out))
    return out


def amp_hel(n: int, mom, h: int, ward: int = -1, alpha=ALPHA, Q=Q_U):
    """Complex helicity amplitude M_h (Sec. 2.1 eq. (6): the sum over the n!
    orderings) and the sum over orderings of |A_pi|; ward >= 0 replaces that
    photon's polarisation by k/k^0."""
    lib = _load()
    m = _f64(mom).reshape(n + 2, 4)
    re, im, sa = C.c_double(), C.c_double(), C.c_double()
    lib.oracle_amp_hel(n, _ptr(m), h, ward, alpha, Q, C.byref(re), C.byref(im), C.byref(sa))
    return complex(re.value, im.value), sa.value


def amp2_metric(n: int, mom, alpha=ALPHA, Q=Q_U) -> float:
    """sum_h |M_h|^2 by a second route: each photon's polarisation sum
    replaced by -g_mu,nu (valid for the gauge-invariant sum over orderings),
    so no polarisation vectors enter."""
    lib = _load()
    return lib.oracle_amp2_metric(n, _ptr(_f64(mom).reshape(n + 2, 4)), alpha, Q)


def phase_space_volume(n: int, s: float) -> float:
    """Volume of flat massless n-body phase space in the normalisation of
    Sec. 2.1 eq. (4)."""
    return _load().oracle_phase_space_volume(n, s)


def rambo(n: int, sqrt_s: float, r):
    """RAMBO (Kleiss, Stirling, Ellis 1986) for n massless momenta at sqrt_s
    from 4n uniforms r: (momenta (n, 4), the constant weight of eq. (4))."""
    lib = _load()
    rr = _f64(r).reshape(4 * n)
    out = np.zeros((n, 4))
    w = lib.oracle_rambo(n, sqrt_s, _ptr(rr), _ptr(out))
    return out, w


def phase_space(n: int, seed: int, i0: int, N: int, sampler: Sampler, cut: Cuts | None = None):
    """Regenerate points i0..i0+N-1 (the per-event phase-space step of
    Sec. 3: sqrt(s-hat) sampler, RAMBO, the cuts of Sec. 2.2): dict of momenta
    (N, n+2, 4), weight, sqrt_s, y, mask, tries."""
    lib = _load()
    mom = np.zeros((N, n + 2, 4))
    w, rs, y = np.zeros(N), np.zeros(N), np.zeros(N)
    mask = np.zeros(N, dtype=np.uint8)
    tries = np.zeros(N, dtype=np.int32)
    lib.oracle_phase_space(n, seed, i0, N, C.byref(sampler), C.byref(cut) if cut else None,
                           _ptr(mom), _ptr(w), _ptr(rs), _ptr(y), _ptr(mask), _ptr(tries))
    return dict(momenta=mom, weight=w, sqrt_s=rs, y=y, mask=mask, tries=tries)


def pass_cuts(n: int, k, y: float, cut: Cuts) -> bool:
    """Cut decision of Sec. 2.2 for photon momenta k (n, 4) at boost rapidity y."""
    kk = _f64(k).reshape(n, 4)
    return bool(_load().oracle_pass_cuts(n, _ptr(kk), y, C.byref(cut)))


def event_weight(n: int, s: float, amp2_value: float, phi_n: float, mask: int = 1) -> float:
    """dsigma-hat weight of one event in fb (Sec. 2.1 eq. (2))."""
    return _load().oracle_event_weight(n, s, amp2_value, phi_n, mask)


def event_weights(n: int, seed: int, i0: int, N: int, sampler: Sampler, cut: Cuts | None,
                  alpha=ALPHA, Q=Q_U, threads: int | None = None):
    """Per-event dsigma-hat weights (fb, Sec. 2.1 eq. (2)) for points
    i0..i0+N-1, plus mask and tries."""
    lib = _load()
    w = np.zeros(N)
    mask = np.zeros(N, dtype=np.uint8)
    tries = np.zeros(N, dtype=np.int32)
    th = threads if threads is not None else (os.cpu_count() or 1)
    lib.oracle_event_weights(n, seed, i0, N, C.byref(sampler), C.byref(cut) if cut else None,
                             alpha, Q, th, _ptr(w), _ptr(mask), _ptr(tries))
    return w, mask, tries


class HistSpec(C.Structure):
    """One histogram: observable kind (0 max pT, 1 pT, 2 eta, 3 Delta R of
    each pair, 4 smallest Delta R, 5 sqrt(s-hat)), nbins uniform bins on
    [lo, hi) plus an underflow and an overflow bin."""
    _fields_ = [("kind", C.c_int), ("nbins", C.c_int), ("lo", C.c_double), ("hi", C.c_double)]


def hist(n: int, mom, y, w, specs):
    """Weighted histograms of the Sec. 5 / Fig. 2 observables of events
    (momenta (N, n+2, 4), boost rapidities y (N,), weights w (N,)): a list
    with one (nbins + 2, 2) array per spec (rows: underflow, the bins,
    overflow; columns: sum w, sum w^2)."""
    lib = _load()
    mm = _f64(mom).reshape(-1)
    yy, ww = _f64(y), _f64(w)
    N = ww.size
    arr = (HistSpec * len(specs))(*[HistSpec(*sp) for sp in specs])
    total = sum(sp[1] + 2 for sp in specs)
    out = np.zeros(2 * total)
    lib.oracle_hist(n, N, _ptr(mm), _ptr(yy), _ptr(ww), len(specs), arr, _ptr(out))
    res, off = [], 0
    for sp in specs:
        res.append(out[2 * off:2 * (off + sp[1] + 2)].reshape(sp[1] + 2, 2))
        off += sp[1] + 2
    return res


def xsec_from_weights(w, tries=None, sampler_kind: int = 0):
    """sigma and its standard error from per-event weights (the summation
    step of Sec. 3.1; N-1 in the variance).

    Toy-PDF sampling (kind 2) multiplies by 2 P_acc (the q <-> qbar assignment
    of Sec. 2.1 eq. (1) and the sqrt(s-hat) floor acceptance from draw counts).
    """
    w = np.asarray(w, dtype=np.float64)
    N = w.size
    mean = float(np.mean(w))
    var = float(np.sum((w - mean) ** 2)) / (N - 1) if N > 1 else 0.0
    scale = 1.0
    if sampler_kind == 2:
        scale = 2.0 * N / float(np.sum(tries))
    return scale * mean, scale * np.sqrt(var / N)
