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


# --------------------------------------------------------------------------
# Hydrodynamic theory of the single-sphere autocorrelations (Sec. III.A,
# Eqs. 10-13): a neutrally buoyant no-slip sphere of radius R in a compressible
# solvent of density rho0, shear viscosity eta0, bulk viscosity eta_b and
# isothermal speed of sound c0.  Reading of Eq. 11: the variable s in the
# definition of zeta is the Laplace variable s = -i omega of the transform.
# --------------------------------------------------------------------------
def friction_translational(omega, R: float, eta0: float, rho0: float, c0: float, eta_b: float):
    """Frequency-dependent translational friction gamma_T(omega) (Eq. 11) with
    x = R sqrt(-i omega / nu0), zeta = s R / sqrt(c0^2 - i omega (4 eta0/3 +
    eta_b) / rho0), s = -i omega (principal square roots, Re >= 0).  For
    c0 -> infinity it is the incompressible 6 pi eta0 R (1 + x + x^2/9)."""
    w = np.asarray(omega, dtype=np.complex128)
    s = -1j * w
    nu = eta0 / rho0
    x = R * np.sqrt(s / nu)
    zeta = s * R / np.sqrt(c0 * c0 + s * (4.0 * eta0 / 3.0 + eta_b) / rho0)
    num = (1.0 + x) * (9.0 - 9.0j * zeta - 2.0 * zeta * zeta) + x * x * (1.0 - 1j * zeta)
    den = 2.0 * x * x * (1.0 - 1j * zeta) - (1.0 + x) * zeta * zeta - x * x * zeta * zeta
    with np.errstate(invalid="ignore", divide="ignore"):
        g = (4.0 * np.pi / 3.0) * eta0 * R * x * x * num / den
    # omega = 0: the Stokes limit (x, zeta -> 0)
    return np.where(w == 0, 6.0 * np.pi * eta0 * R + 0j, g)


def friction_rotational(s, R: float, eta0: float, rho0: float):
    """Frequency-dependent rotational friction gamma_R(s) in the Laplace variable
    s (Eq. 13): 8 pi eta0 R^3 [1 + (R^2 s / nu0) / (3 (1 + sqrt(R^2 s / nu0)))]."""
    s = np.asarray(s, dtype=np.complex128)
    y = R * R * s / (eta0 / rho0)
    return 8.0 * np.pi * eta0 * R ** 3 * (1.0 + y / (3.0 * (1.0 + np.sqrt(y))))


def vacf_translational_theory(t, kT: float, R: float, eta0: float, rho0: float, c0: float, eta_b: float,
                              M: float = None, d_omega: float = 1e-3, omega_max: float = 1e3) -> np.ndarray:
    """C_T(t) = <V(0).V(t)> of Eq. 10 for t > 0, by the trapezoid rule on
    [-omega_max, omega_max] with step d_omega (the paper's 1e-3 and 1e3).  M is
    the sphere's mass, M_S = 4 pi R^3 rho0 / 3 (neutrally buoyant) by default.
    The integrand is the transform of a real function, so the integral is
    twice the real part over omega >= 0."""
    if M is None:
        M = 4.0 * np.pi * R ** 3 * rho0 / 3.0
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    w = np.arange(0.0, omega_max + 0.5 * d_omega, d_omega)
    F = 1.0 / (friction_translational(w, R, eta0, rho0, c0, eta_b) - 1j * w * M)
    wt = np.full(w.size, d_omega)
    wt[0] = wt[-1] = 0.5 * d_omega            # trapezoid weights (the omega = 0 point counts once)
    out = np.empty(t.size)
    Fr, Fi = (F.real * wt), (F.imag * wt)
    for i0 in range(0, t.size, 16):            # e^{-i w t} F: Re = Fr cos + Fi sin
        tt = t[i0:i0 + 16, None]
        ph = w[None, :] * tt
        out[i0:i0 + 16] = (np.cos(ph) @ Fr + np.sin(ph) @ Fi)
    return 3.0 * kT / np.pi * out


def talbot_inverse(F, t, n: int = 32) -> np.ndarray:
    """Inverse Laplace transform f(t) of F(s) for t > 0 by the fixed Talbot
    contour method (Talbot 1979; Abate and Valko 2004): with r = 2n/(5t),
    theta_k = k pi / n and s(theta) = r theta (cot theta + i),
    f(t) = (r/n) [F(r) e^{r t}/2 + sum_k Re(e^{t s_k} F(s_k) (1 + i sigma_k))],
    sigma(theta) = theta + (theta cot theta - 1) cot theta.  F is called on
    complex arrays; its singularities must lie on or left of the negative real
    axis (a branch cut there is allowed)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    k = np.arange(1, n)
    th = k * np.pi / n
    cot = 1.0 / np.tan(th)
    sig = th + (th * cot - 1.0) * cot
    out = np.empty(t.size)
    for i, ti in enumerate(t):
        r = 2.0 * n / (5.0 * ti)
        sk = r * th * (cot + 1j)
        term = np.real(np.exp(ti * sk) * F(sk) * (1.0 + 1j * sig))
        out[i] = (r / n) * (0.5 * np.real(F(np.array([r + 0j]))[0]) * np.exp(r * ti) + term.sum())
    return out


def vacf_rotational_theory(t, kT: float, R: float, eta0: float, rho0: float, I: float = None,
                           n: int = 32) -> np.ndarray:
    """C_R(t) = <omega(0).omega(t)> of Eq. 12: (3 kT / I) times the inverse
    Laplace transform of 1/(s + gamma_R(s)/I) (Eq. 13), for t > 0, by the fixed
    Talbot method.  I is the sphere's moment of inertia, I_S = 2 M_S R^2 / 5 of a
    solid neutrally buoyant sphere by default."""
    if I is None:
        I = 2.0 * (4.0 * np.pi * R ** 3 * rho0 / 3.0) * R * R / 5.0
    return 3.0 * kT / I * talbot_inverse(lambda s: 1.0 / (s + friction_rotational(s, R, eta0, rho0) / I), t, n)


def vacf_translational_tail(t, kT: float, eta0: float, rho0: float):
    """Long-time tail of C_T: kT / (4 rho0 (pi nu0 t)^{3/2}), from the sqrt(s)
    term of the low-frequency friction 6 pi eta0 R (1 + R sqrt(s/nu0) + ...)."""
    nu = eta0 / rho0
    return kT / (4.0 * rho0 * (np.pi * nu * np.asarray(t, dtype=np.float64)) ** 1.5)


def vacf_rotational_tail(t, kT: float, eta0: float, rho0: float):
    """Long-time tail of C_R: 3 pi kT / (32 rho0 (pi nu0 t)^{5/2}), from the
    s^{3/2} term of gamma_R(s) at small s (Eq. 13)."""
    nu = eta0 / rho0
    return 3.0 * np.pi * kT / (32.0 * rho0 * (np.pi * nu * np.asarray(t, dtype=np.float64)) ** 2.5)
