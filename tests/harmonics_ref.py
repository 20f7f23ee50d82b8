"""Test-side solid harmonics in the paper's normalisation (Sec. 2), written
with scipy's associated Legendre functions (Condon-Shortley phase), for
checking the library's host tables.  Independent of the library's own
recurrences.

    y_n^m(v) = |v|^n sqrt((n-m)!/(n+m)!) P_n^m(cos t) e^{i m phi}
    z_n^m(v) = sqrt((n-m)!/(n+m)!) P_n^m(cos t) e^{i m phi} / |v|^{n+1}
for 0 <= m <= n, stored at index n(n+1)/2 + m.
"""
import math

import numpy as np
from scipy.special import lpmv


def tri(n, m):
    return n * (n + 1) // 2 + m


def ncoef(p):
    return (p + 1) * (p + 2) // 2


def _angles(v):
    v = np.asarray(v, dtype=np.float64)
    r = np.linalg.norm(v, axis=-1)
    ct = np.where(r > 0, v[..., 2] / np.where(r > 0, r, 1), 1.0)
    ph = np.arctan2(v[..., 1], v[..., 0])
    return r, np.clip(ct, -1, 1), ph


def regular(v, p):
    """y_n^m for points v (..., 3) -> (..., ncoef(p)) complex."""
    r, ct, ph = _angles(v)
    out = np.zeros(np.shape(r) + (ncoef(p),), dtype=complex)
    for n in range(p + 1):
        for m in range(n + 1):
            c = math.sqrt(math.factorial(n - m) / math.factorial(n + m))
            out[..., tri(n, m)] = r ** n * c * lpmv(m, n, ct) * np.exp(1j * m * ph)
    return out


def irregular(v, p):
    r, ct, ph = _angles(v)
    out = np.zeros(np.shape(r) + (ncoef(p),), dtype=complex)
    for n in range(p + 1):
        for m in range(n + 1):
            c = math.sqrt(math.factorial(n - m) / math.factorial(n + m))
            out[..., tri(n, m)] = c * lpmv(m, n, ct) * np.exp(1j * m * ph) / r ** (n + 1)
    return out


def eval_real(coef, h):
    """sum_{n,m>=0} w_m Re(coef * h), w_0 = 1, w_m = 2 (real field of a conj-symmetric expansion)."""
    w = np.ones(coef.shape[-1])
    p = int((math.sqrt(8 * coef.shape[-1] + 1) - 3) / 2)
    for n in range(p + 1):
        for m in range(1, n + 1):
            w[tri(n, m)] = 2.0
    return np.real(np.sum(w * coef * h, axis=-1))


def p2m(src, q, centre, h, p):
    """M_n^m = sum_j q_j conj(y_n^m((y_j - c)/h))."""
    return np.sum(q[:, None] * np.conj(regular((src - centre) / h, p)), axis=0)


def p2l(src, q, centre, h, p):
    """L_n^m = sum_j q_j conj(z_n^m((y_j - c)/h))."""
    return np.sum(q[:, None] * np.conj(irregular((src - centre) / h, p)), axis=0)


def as_real(c):
    """complex (nc,) -> interleaved real (2 nc,)."""
    return np.stack([c.real, c.imag], axis=-1).reshape(c.shape[:-1] + (-1,))


def from_real(r):
    return r[..., 0::2] + 1j * r[..., 1::2]
