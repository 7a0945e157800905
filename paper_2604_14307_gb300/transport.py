"""Host-side analysis of the transport protocols of Sec. III.B.

Shear viscosity.  It comes from reverse non-equilibrium simulation: the device
exchanges v_x between two slabs (mpcd_set_rnemd), which drives a bidirectional
linear shear flow, and Eq. 14 relates the rate of exchanged momentum to the
shear rate of the mass-averaged velocity profile (mpcd_velocity_profile):

    eta = p_dot / (2 A gamma_dot),

with A the area of a slab (L^2 for the paper's square cross-section) and the
factor 2 because the momentum leaves the exchange slabs through two planes.

Velocity autocorrelations.  C_T(t) = <V(0).V(t)> and C_R(t) = <omega(0).omega(t)>
(Sec. III.A) with every sample as a time origin; the device accumulates them
per body (mpcd_set_vacf); `velocity_autocorrelation` is the same average over
host samples.

Self-diffusion.  The long-time self-diffusion coefficient follows from the
mean squared displacement of the bodies (Eq. 15, Einstein relation), with every
sample as a time origin, and the finite-size correction of the periodic box,
Delta D = xi kT / (6 pi eta L), xi = 2.837297, is added.

This module only post-processes host arrays; every per-particle operation runs
on the device.
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np


def bin_centres(n_bins: int, length: float) -> np.ndarray:
    """Centres of n_bins equal bins over [0, length)."""
    w = length / n_bins
    return (np.arange(n_bins) + 0.5) * w


def shear_rate(y: np.ndarray, u: np.ndarray, length: float, y_a: float, y_b: float, width: float,
               margin: float = 1.0) -> Dict[str, float]:
    """Shear rate of a bidirectional profile u(y) driven by slabs A at
    [y_a, y_a + width) and B at [y_b, y_b + width) (y_a < y_b) in a periodic box
    of this length.  Each of the two regions between the slabs gets a least-
    squares line, leaving `margin` on either side of each slab; gamma_dot is
    the mean magnitude of the two slopes."""
    if not y_a < y_b:
        raise ValueError("expects y_a < y_b")
    y = np.asarray(y, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    lo1, hi1 = y_a + width + margin, y_b - margin              # A -> B
    m1 = (y >= lo1) & (y <= hi1)
    yy = np.where(y < y_a + width, y + length, y)              # B -> A + length
    lo2, hi2 = y_b + width + margin, y_a + length - margin
    m2 = (yy >= lo2) & (yy <= hi2)
    if m1.sum() < 2 or m2.sum() < 2:
        raise ValueError("too few bins between the slabs")
    s1 = np.polyfit(y[m1], u[m1], 1)[0]
    s2 = np.polyfit(yy[m2], u[m2], 1)[0]
    return dict(slope_ab=float(s1), slope_ba=float(s2), gamma_dot=0.5 * (abs(s1) + abs(s2)))


def viscosity_rnemd(p_exchanged: float, duration: float, area: float, gamma_dot: float) -> float:
    """Eq. 14: eta = (p_exchanged / duration) / (2 area gamma_dot)."""
    return (p_exchanged / duration) / (2.0 * area * gamma_dot)


def srd_viscosity(density: float, kT: float, m: float, dt: float, alpha_deg: float, a: float = 1.0) -> Dict[str, float]:
    """Kinetic and collisional shear viscosity of SRD with random grid shift
    (Kikuchi et al. 2003; Tuzel et al. 2003), the literature values behind the
    paper's eta_0 = 3.96 (Sec. II.A) for 5 particles per cell, kT = 1,
    m = 1, dt = 0.1 and 130 degrees."""
    n = density * a ** 3
    al = np.radians(alpha_deg)
    g = n - 1.0 + np.exp(-n)
    kin = (n * kT * dt / a ** 3) * (5.0 * n / (g * (4.0 - 2.0 * np.cos(al) - 2.0 * np.cos(2.0 * al))) - 0.5)
    col = (m / (18.0 * a * dt)) * g * (1.0 - np.cos(al))
    return dict(kinetic=float(kin), collisional=float(col), total=float(kin + col))


def mean_profile(mass: Sequence[np.ndarray], momentum: Sequence[np.ndarray]) -> np.ndarray:
    """Mass-averaged velocity per bin from sampled (mass, momentum) profiles."""
    M = np.sum(np.asarray(mass, dtype=np.float64), axis=0)
    P = np.sum(np.asarray(momentum, dtype=np.float64), axis=0)
    return np.where(M > 0, P / np.where(M > 0, M, 1.0), 0.0)


XI_CUBIC = 2.837297     # periodic-lattice constant of the finite-size corrections (Sec. III.B)


def mean_squared_displacement(D: np.ndarray, max_lag: int) -> np.ndarray:
    """MSD(k) for lags k = 0..max_lag samples from unwrapped displacements D
    [n_samples, n_bodies, 3], averaged over every time origin and body."""
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    out = np.zeros(max_lag + 1)
    for k in range(1, min(max_lag, n - 1) + 1):
        d = D[k:] - D[:-k]
        out[k] = np.mean(np.sum(d * d, axis=-1))
    return out


def diffusion_coefficient(msd: np.ndarray, dt_sample: float, lag_lo: int, lag_hi: int) -> float:
    """Eq. 15: D = (1/6) d MSD / dt, the least-squares slope over lags
    [lag_lo, lag_hi] (the long-time regime)."""
    k = np.arange(lag_lo, lag_hi + 1)
    slope = np.polyfit(k * dt_sample, msd[lag_lo: lag_hi + 1], 1)[0]
    return float(slope / 6.0)


def finite_size_correction(kT: float, eta: float, L: float) -> float:
    """Delta D = xi kT / (6 pi eta L) for a cubic periodic box of edge L."""
    return XI_CUBIC * kT / (6.0 * np.pi * eta * L)


def rotation_matrix(q: np.ndarray) -> np.ndarray:
    """Body-to-space rotation of unit quaternions (w, x, y, z), [..., 3, 3]."""
    q = np.asarray(q, dtype=np.float64)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], axis=-1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], axis=-1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], axis=-1)], axis=-2)


def angular_velocity(q: np.ndarray, L: np.ndarray, Ihat: np.ndarray) -> np.ndarray:
    """Space-frame omega = Q Ihat^-1 Q^T L of bodies with principal moments Ihat."""
    Q = rotation_matrix(q)
    Lb = np.einsum("...ji,...j->...i", Q, np.asarray(L, dtype=np.float64))
    return np.einsum("...ij,...j->...i", Q, Lb / np.asarray(Ihat, dtype=np.float64))


def velocity_autocorrelation(X: np.ndarray, n_lags: int) -> np.ndarray:
    """<X(t).X(t + k)> per body for k = 0..n_lags-1 over every time origin, from
    samples X [n_samples, n_bodies, 3]; returns [n_bodies, n_lags]."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    out = np.zeros((X.shape[1], n_lags))
    for k in range(min(n_lags, n)):
        out[:, k] = np.mean(np.sum(X[k:] * X[: n - k], axis=-1), axis=0)
    return out
