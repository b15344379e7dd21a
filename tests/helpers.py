"""Small kinematics helpers for the tests (Minkowski products, boosts, rotations).

These transform or inspect momenta; none of them computes an amplitude, a
phase-space point or a weight.
"""
import math

import numpy as np


def mdot(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return a[..., 0] * b[..., 0] - np.sum(a[..., 1:] * b[..., 1:], axis=-1)


def boost_matrix(beta):
    """Pure boost with velocity vector beta (|beta| < 1), acting on (E, px, py, pz)."""
    beta = np.asarray(beta, dtype=np.float64)
    b2 = float(beta @ beta)
    g = 1.0 / math.sqrt(1.0 - b2)
    L = np.eye(4)
    L[0, 0] = g
    L[0, 1:] = g * beta
    L[1:, 0] = g * beta
    if b2 > 0:
        L[1:, 1:] += (g - 1.0) * np.outer(beta, beta) / b2
    return L


def rotation_matrix(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    x, y, z = axis
    c, s = math.cos(angle), math.sin(angle)
    R3 = np.array([[c + x * x * (1 - c), x * y * (1 - c) - z * s, x * z * (1 - c) + y * s],
                   [y * x * (1 - c) + z * s, c + y * y * (1 - c), y * z * (1 - c) - x * s],
                   [z * x * (1 - c) - y * s, z * y * (1 - c) + x * s, c + z * z * (1 - c)]])
    R = np.eye(4)
    R[1:, 1:] = R3
    return R


def transform(mom, L):
    """Apply a 4x4 Lorentz matrix to every momentum in mom[..., 4]."""
    return np.einsum("ij,...j->...i", L, mom)


def helicity_index(s1, s2, lams):
    """Helicity index: bit0 = s1 (+1 -> 1), bit1 = s2, bit(2+i) = lambda_{i+1}."""
    h = (1 if s1 > 0 else 0) | ((1 if s2 > 0 else 0) << 1)
    for i, l in enumerate(lams):
        h |= (1 if l > 0 else 0) << (2 + i)
    return h


def propagator_condition(mom):
    """s-hat / min_T |t_T| over all proper photon subsets T, t_T = (p1 - K_T)^2.

    Input momenta conserve momentum only to FP64 rounding (~1e-16 sqrt(s));
    two exact-arithmetic-equivalent forms of a denominator, (p1 - K_T)^2 and
    (K_{T^c} - p2)^2, then differ by ~1e-16 s-hat, i.e. relatively by
    ~1e-16 s-hat/|t_T|.  This is the factor by which input rounding reaches
    |M|^2 through the propagators."""
    mom = np.asarray(mom, dtype=np.float64)
    n = mom.shape[-2] - 2
    p1, p2, ks = mom[..., 0, :], mom[..., 1, :], mom[..., 2:, :]
    s = mdot(p1 + p2, p1 + p2)
    tmin = np.full(s.shape, np.inf)
    for T in range(1, (1 << n) - 1):
        sel = [i for i in range(n) if T >> i & 1]
        q = p1 - ks[..., sel, :].sum(axis=-2)
        tmin = np.minimum(tmin, np.abs(mdot(q, q)))
    return s / tmin


def momentum_violation(mom):
    """max(u_64, |sum k - p1 - p2|_inf / sqrt(s-hat)): how well the input
    conserves momentum (RAMBO's boost amplifies rounding at small n)."""
    mom = np.asarray(mom, dtype=np.float64)
    p1, p2, ks = mom[..., 0, :], mom[..., 1, :], mom[..., 2:, :]
    rs = np.sqrt(np.abs(mdot(p1 + p2, p1 + p2)))
    d = np.max(np.abs(ks.sum(axis=-2) - p1 - p2), axis=-1) / rs
    return np.maximum(2.22e-16, d)


def fp64_tolerance(mom, floor=1e-12):
    """Per-point relative tolerance of an FP64 |M|^2 against the oracle:
    a floor for rounding-order differences over the ordering and helicity
    sums, plus 16 n times the momentum-conservation violation of the input
    times the propagator condition number (the two sides evaluate equivalent
    but differently rounded forms of each denominator)."""
    mom = np.asarray(mom, dtype=np.float64)
    n = mom.shape[-2] - 2
    return floor + 16 * n * momentum_violation(mom) * propagator_condition(mom)


def mask_words(n, hels):
    """uint32 word array with the bits of the helicities in `hels` set."""
    words = np.zeros(max(1, (1 << (n + 2)) // 32), dtype=np.uint32)
    for h in hels:
        words[h >> 5] |= np.uint32(1 << (h & 31))
    return words
