"""Pins of the unwrapped body displacement (the input of Eq. 15) and of the
host-side diffusion analysis, on CPU.

* The oracle's displacement is the sum of the drifts: under a constant force
  with no collision it follows P0 t / M + F t^2 / (2 M), and through whole steps
  the wrapped position always equals R0 + D modulo the box.
* The mean squared displacement of ballistic paths is |v|^2 t^2 exactly; of
  Brownian paths with a known D it gives D back within the sampling error.
* The finite-size constant is the paper's xi = 2.837297.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I
from paper_2604_14307_gb300 import transport as T

from test_oracle_sedimentation import one_sphere


@pytest.fixture(scope="module")
def lib():
    O.build()


def test_displacement_is_the_sum_of_the_drifts(lib):
    system = one_sphere()
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    f = np.array([0.5, -0.2, 0.1])
    osys.set_body_force(f)
    ost = O.OracleState(osys, st)
    n, dt = 9, system.params.dt
    for _ in range(n):
        O.stream(osys, ost)
    t = n * dt
    M = system.shapes[0].m.sum()
    assert np.allclose(ost.D[0], st.P[0] * t / M + 0.5 * f * t * t / M, rtol=0, atol=1e-13)


@pytest.mark.parametrize("precision", [I.P64, I.P32])
def test_wrapped_position_is_start_plus_displacement(lib, precision):
    system = I.suspension(14, 5.0, 0.1, 2.0, 2, 5.0, I.SRD, 1, precision, seed=3)
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)
    O.step(osys, ost, 6)
    L = np.array(system.replicas[0].L, dtype=np.float64)
    d = np.mod(st.R + ost.D[: system.n_bodies] - ost.R, L)
    assert np.all(np.minimum(d, L - d) < 1e-12)
    assert np.any(np.abs(ost.D[: system.n_bodies]) > 1e-3)


def test_msd_of_ballistic_paths_is_exact():
    rng = np.random.default_rng(0)
    v = rng.normal(size=(50, 3))
    dt = 0.2
    t = np.arange(40)[:, None, None] * dt
    D = v[None] * t
    msd = T.mean_squared_displacement(D, 10)
    k = np.arange(11)
    assert np.allclose(msd, np.mean(np.sum(v * v, axis=1)) * (k * dt) ** 2, rtol=1e-12, atol=1e-14)


def test_msd_of_brownian_paths_gives_d_back():
    rng = np.random.default_rng(1)
    Dc, dt, n, B = 0.037, 0.5, 4000, 64
    steps = rng.normal(scale=np.sqrt(2 * Dc * dt), size=(n, B, 3))
    D = np.cumsum(steps, axis=0)
    msd = T.mean_squared_displacement(D, 40)
    est = T.diffusion_coefficient(msd, dt, 5, 40)
    assert est == pytest.approx(Dc, rel=0.05)


def test_finite_size_constant(golden):
    assert T.XI_CUBIC == golden["finite_size_xi"]["value"]
    # the correction shrinks as 1/L and grows as 1/eta
    a = T.finite_size_correction(1.0, 3.96, 60.0)
    assert T.finite_size_correction(1.0, 3.96, 120.0) == pytest.approx(a / 2)
    assert T.finite_size_correction(1.0, 7.92, 60.0) == pytest.approx(a / 2)
