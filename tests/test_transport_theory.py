"""Hydrodynamic theory of the single-sphere autocorrelations (Sec. III.A,
Eqs. 10-13), evaluated on the host (paper_2604_14307_gb300.transport), pinned
by closed forms and limits rather than by re-typing the formulas:

* Eq. 11 in the incompressible limit (c0 -> infinity) is the Stokes-Boussinesq
  friction 6 pi eta R (1 + x + x^2/9), and 6 pi eta R at zero frequency;
* Eq. 10 (trapezoid rule, the paper's step and bounds): C_T(0+) = 3 kT / M_S for
  the compressible solvent (the added mass needs sound to build up), and the
  long-time tail kT / (4 rho (pi nu t)^{3/2}); in the incompressible limit the
  trapezoid result equals an independent inversion (fixed Talbot contour) of
  the same transform;
* the fixed Talbot inversion reproduces known transform pairs;
* Eq. 12-13: C_R(0+) = 3 kT / I_S, the long-time tail 3 pi kT / (32 rho
  (pi nu t)^{5/2}), and, with the frequency-dependent bracket of Eq. 13 removed,
  the exponential decay of a sphere with the Stokes rotational friction.
The solvent parameters are the paper's: kT = 1, rho0 = 5, eta0 = 3.96,
c0 = 1, eta_b = 1.22 (nu0 = 0.792), d = 6.
"""
import math

import numpy as np
import pytest

from paper_2604_14307_gb300 import transport as T

KT, R, ETA, RHO, C0, ETAB = 1.0, 3.0, 3.96, 5.0, 1.0, 1.22
MS = 4.0 * math.pi * R ** 3 * RHO / 3.0
IS = 2.0 * MS * R * R / 5.0


def test_translational_friction_limits():
    w = np.array([0.01, 0.3, 2.0, 30.0])
    x = R * np.sqrt(-1j * w / (ETA / RHO))
    g = T.friction_translational(w, R, ETA, RHO, 1e9, ETAB)
    assert np.allclose(g, 6 * math.pi * ETA * R * (1 + x + x * x / 9), rtol=1e-6)
    assert T.friction_translational(np.array([0.0]), R, ETA, RHO, C0, ETAB)[0] == pytest.approx(6 * math.pi * ETA * R)
    g = T.friction_translational(np.array([1e-6]), R, ETA, RHO, C0, ETAB)[0]
    assert g.real == pytest.approx(6 * math.pi * ETA * R, rel=1e-2)


def test_translational_vacf_initial_value_and_tail():
    c0 = T.vacf_translational_theory([0.005], KT, R, ETA, RHO, C0, ETAB)[0]
    assert c0 * MS / (3 * KT) == pytest.approx(1.0, abs=0.02)
    t = np.array([200.0, 400.0])
    ratio = T.vacf_translational_theory(t, KT, R, ETA, RHO, C0, ETAB) / T.vacf_translational_tail(t, KT, ETA, RHO)
    assert np.all(np.abs(ratio - 1) < 0.03), ratio
    # monotonic decay over the window the paper shows (t <= 50 tau)
    tt = np.linspace(0.05, 50, 60)
    c = T.vacf_translational_theory(tt, KT, R, ETA, RHO, C0, ETAB)
    assert np.all(np.diff(c) < 0) and np.all(c > 0)


def test_translational_vacf_two_inversions_agree_incompressible():
    t = np.array([0.5, 2.0, 10.0, 50.0])
    c_fourier = T.vacf_translational_theory(t, KT, R, ETA, RHO, 1e5, ETAB)
    F = lambda s: 1.0 / (T.friction_translational(1j * s, R, ETA, RHO, 1e5, ETAB) + s * MS)
    c_talbot = 3 * KT * T.talbot_inverse(F, t)
    assert np.allclose(c_fourier, c_talbot, rtol=1e-2)
    # incompressible: the initial value carries the added mass M_f/2 = M_S/2
    c = T.vacf_translational_theory([0.02], KT, R, ETA, RHO, 1e5, ETAB)[0]
    assert 0.55 < c * MS / (3 * KT) < 2.0 / 3.0 + 1e-3


def test_talbot_known_pairs():
    t = np.array([0.05, 0.7, 3.0])
    assert np.allclose(T.talbot_inverse(lambda s: 1.0 / (s + 2.0), t), np.exp(-2 * t), rtol=1e-8)
    assert np.allclose(T.talbot_inverse(lambda s: 1.0 / np.sqrt(s), t), 1 / np.sqrt(math.pi * t), rtol=1e-8)
    assert np.allclose(T.talbot_inverse(lambda s: 1.0 / s ** 2, t), t, rtol=1e-8)


def test_rotational_vacf_limits():
    c = T.vacf_rotational_theory(np.array([1e-5]), KT, R, ETA, RHO)[0]
    assert c * IS / (3 * KT) == pytest.approx(1.0, abs=0.01)
    t = np.array([300.0, 600.0])
    ratio = T.vacf_rotational_theory(t, KT, R, ETA, RHO) / T.vacf_rotational_tail(t, KT, ETA, RHO)
    assert np.all(np.abs(ratio - 1) < 0.05), ratio
    # the Stokes rotational friction alone: exponential decay
    g0 = 8 * math.pi * ETA * R ** 3
    t = np.array([0.1, 1.0, 4.0])
    c = 3 * KT / IS * T.talbot_inverse(lambda s: 1.0 / (s + g0 / IS), t)
    assert np.allclose(c, 3 * KT / IS * np.exp(-g0 * t / IS), rtol=1e-8)
