"""Oracle incident fields, radiated fields, far field and closed-form references.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  * plane wave v(x) = exp(i k d.x) and point-source fields phi(x, s) (Sec. 2, Sec. 6);
  * the field of a density, u(x) = sum_j w_j K(x, x_j) sigma_j (Eq. (intHelm1)
    discretised with the smooth rule, valid away from the surface);
  * the far-field pattern of that field, with u(x) ~ e^{ik|x|}/|x| u_inf(x^):
        u_inf(x^) = (1/4pi) sum_j w_j e^{-ik x^.x_j} (-ik x^.n_j - i eta) sigma_j,
    the large-|x| limit of the same kernel;
  * the Mie series of a sound-soft sphere (textbook closed form) and the
    eigenvalues of the combined-field operator on a sphere, used as pins.
"""
from __future__ import annotations

import numpy as np
from scipy import special

from . import _native as nat
from .geometry import SurfaceNodes


def plane_wave(x: np.ndarray, d: np.ndarray, k: float) -> np.ndarray:
    """v(x) = exp(i k d . x) for nodes x (N,3) and directions d (R,3) -> (N, R)."""
    return np.exp(1j * k * (np.asarray(x) @ np.atleast_2d(d).T))


def point_source_field(x: np.ndarray, sources: np.ndarray, k: float) -> np.ndarray:
    """w(x) = sum_s exp(ik|x - s|) / (4 pi |x - s|)  (unit strengths)."""
    d = np.asarray(x)[:, None, :] - np.asarray(sources)[None, :, :]
    R = np.sqrt((d * d).sum(-1))
    return (np.exp(1j * k * R) / (4.0 * np.pi * R)).sum(axis=1)


def field(nodes: SurfaceNodes, sigma: np.ndarray, k: float, eta: float, pts: np.ndarray) -> np.ndarray:
    """u at off-surface points pts (T,3) for sigma (N,) or (N,R)."""
    sig = np.asarray(sigma, dtype=np.complex128)
    one = sig.ndim == 1
    sig2 = sig.reshape(nodes.w.size, -1)
    R = sig2.shape[1]
    P = nat.as_f64(pts)
    out = np.zeros(2 * P.shape[0] * R)
    nat.lib().orc_field(int(nodes.w.size), nat.dptr(nat.as_f64(nodes.x)), nat.dptr(nat.as_f64(nodes.n)),
                        nat.dptr(nat.as_f64(nodes.w)), R, nat.dptr(nat.as_c128_view(sig2)),
                        float(k), float(eta), int(P.shape[0]), nat.dptr(P), nat.dptr(out))
    u = out.view(np.complex128).reshape(P.shape[0], R)
    return u[:, 0] if one else u


def far_field(nodes: SurfaceNodes, sigma: np.ndarray, k: float, eta: float, xhat: np.ndarray) -> np.ndarray:
    """u_inf at unit directions xhat (T,3) for sigma (N,)."""
    xh = np.atleast_2d(xhat)
    ph = np.exp(-1j * k * (xh @ nodes.x.T))                     # (T, N)
    fac = -1j * k * (xh @ nodes.n.T) - 1j * eta                  # (T, N)
    return (ph * fac * nodes.w[None, :]) @ np.asarray(sigma, dtype=np.complex128) / (4.0 * np.pi)


def _h1(n, x):
    return special.spherical_jn(n, x) + 1j * special.spherical_yn(n, x)


def mie_far_field(a: float, k: float, cos_angle: np.ndarray, nmax: int = None) -> np.ndarray:
    """Sound-soft sphere of radius a hit by exp(ik d.x):
    u_inf(x^) = (i/k) sum_n (2n+1) j_n(ka)/h_n(ka) P_n(x^.d)."""
    if nmax is None:
        nmax = int(k * a + 40)
    c = np.asarray(cos_angle, dtype=np.float64)
    out = np.zeros(c.shape, dtype=np.complex128)
    for n in range(nmax + 1):
        out += (2 * n + 1) * special.spherical_jn(n, k * a) / _h1(n, k * a) * special.eval_legendre(n, c)
    return 1j / k * out


def mie_scattered(a: float, k: float, r: np.ndarray, cos_angle: np.ndarray, nmax: int = None) -> np.ndarray:
    """Scattered field u = -sum_n i^n (2n+1) j_n(ka)/h_n(ka) h_n(kr) P_n(cos angle), r >= a."""
    if nmax is None:
        nmax = int(k * a + 40)
    out = np.zeros(np.shape(r), dtype=np.complex128)
    for n in range(nmax + 1):
        out -= (1j ** n) * (2 * n + 1) * special.spherical_jn(n, k * a) / _h1(n, k * a) \
            * _h1(n, k * np.asarray(r)) * special.eval_legendre(n, np.asarray(cos_angle))
    return out


def sphere_eigenvalue(n: int, a: float, k: float, eta: float) -> complex:
    """Eigenvalue of 1/2 I + K_dl - i eta S_sl on the sphere of radius a for the
    spherical harmonics of degree n:
        lambda_n = i k a^2 h_n(ka) [k j_n'(ka) - i eta j_n(ka)]
    (addition theorem for phi: single layer i k a^2 j_n h_n; exterior trace of the
    double layer i k^2 a^2 j_n' h_n)."""
    ka = k * a
    return 1j * k * a * a * _h1(n, ka) * (k * special.spherical_jn(n, ka, derivative=True)
                                          - 1j * eta * special.spherical_jn(n, ka))
