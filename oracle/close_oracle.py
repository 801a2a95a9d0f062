"""FP64 NumPy oracle of a vesicle's single layer at targets close to the vesicle (close evaluation).

TEST INFRASTRUCTURE ONLY: used by the tests, never by the product path; it imports nothing from
the CUDA package.

What it computes -- the plain definition of the quantity that close evaluation approximates
(the paper applies a cited scheme to vesicle-to-vesicle and vesicle-to-wall interactions at
close range, Sec. 1 and Sec. 3.2, and gives none itself): the stokeslet single layer of Eq. (S)
of one closed curve, with the curve and the density taken as the trigonometric interpolants of
their n equispaced samples,

    u(x) = (1 / (4 pi mu)) int_0^{2 pi} [ -log|r| f(t) + (r . f(t)) r / |r|^2 ] |y'(t)| dt,
    r = x - y(t),

at targets x off the curve.  The n-point trapezoid rule of the layer-potential sum is this
integral's discretisation; its error grows like exp(-2 pi delta / h) as a target at distance
delta from a curve of node spacing h comes close.  Here both interpolants are resampled K-fold
by FFT (exact for trigonometric polynomials of degree < n/2; the Nyquist mode is split evenly
between +-n/2 so the interpolant is real), y' is taken spectrally, and the trapezoid rule runs
on the n K fine points, whose error falls like exp(-2 pi K delta / h).
"""
from __future__ import annotations

import math

import numpy as np

PI = math.pi


def _fine_spectrum(v: np.ndarray, K: int) -> tuple[np.ndarray, np.ndarray]:
    """Fourier coefficients of the trigonometric interpolant of the n samples v (n, ...) placed
    in a length-nK spectrum, and the matching wavenumbers."""
    n = v.shape[0]
    m = n * K
    c = np.fft.fft(v, axis=0) / n
    C = np.zeros((m,) + v.shape[1:], dtype=complex)
    h = n // 2
    if n % 2 == 0:
        C[:h] = c[:h]
        C[m - h + 1:] = c[h + 1:]
        C[h] = 0.5 * c[h]          # the Nyquist mode, split between +n/2 and -n/2
        C[m - h] = 0.5 * c[h]
    else:
        C[:h + 1] = c[:h + 1]
        C[m - h:] = c[h + 1:]
    k = np.fft.fftfreq(m, d=1.0 / m)  # integer wavenumbers, index m - n/2 -> -n/2
    return C, k


def upsample(v: np.ndarray, K: int, derivative: bool = False) -> np.ndarray:
    """The interpolant of periodic samples v (n, ...) at n K equispaced parameters in [0, 2 pi),
    or its derivative with respect to the parameter."""
    C, k = _fine_spectrum(np.asarray(v, float), K)
    if derivative:
        C = C * (1j * k).reshape((-1,) + (1,) * (C.ndim - 1))
    return np.real(np.fft.ifft(C, axis=0) * C.shape[0])


def fine_curve(x_nodes: np.ndarray, K: int):
    """Fine points y(t_j), arc-length weights |y'(t_j)| 2 pi / (n K)."""
    y = upsample(x_nodes, K)
    dy = upsample(x_nodes, K, derivative=True)
    w = np.sqrt((dy * dy).sum(1)) * (2 * PI / y.shape[0])
    return y, w


def log_potential(x_nodes, sigma, targets, K=64):
    """int log|x - y| sigma ds over the interpolated curve, sigma at the nodes (n,)."""
    y, w = fine_curve(np.asarray(x_nodes, float), K)
    s = upsample(np.asarray(sigma, float), K)
    t = np.asarray(targets, float)
    r = t[:, None, :] - y[None]
    return (0.5 * np.log((r * r).sum(-1)) * (s * w)[None]).sum(1)


def close_slp(x_nodes, f, targets, mu, K=64):
    """The stokeslet single layer (1/(4 pi mu)) int [-log|r| f + (r.f) r / |r|^2] ds of one closed
    curve at targets (T, 2), the curve and the density f (n, 2) interpolated from their nodes."""
    y, w = fine_curve(np.asarray(x_nodes, float), K)
    fv = upsample(np.asarray(f, float), K) * w[:, None]
    t = np.asarray(targets, float)
    out = np.zeros((t.shape[0], 2))
    for a in range(0, t.shape[0], 256):  # bounded memory
        r = t[a:a + 256, None, :] - y[None]
        rr = (r * r).sum(-1)
        rf = (r * fv[None]).sum(-1)
        out[a:a + 256] = ((-0.5 * np.log(rr))[..., None] * fv[None]
                          + (rf / rr)[..., None] * r).sum(1)
    return out / (4 * PI * mu)
