"""Pins of the host-side velocity autocorrelation helpers (Sec. III.A), on CPU.

* The angular velocity omega = Q Ihat^-1 Q^T L gives the oracle's rotational
  kinetic energy omega.L / 2 for every body of a suspension, and the rigid
  site velocities V + omega x d of the oracle's Eq. 5 reset.
* The autocorrelation of a constant signal is |X|^2 at every lag, of an
  alternating one (-1)^k |X|^2, and lag 0 is the mean square.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I
from paper_2604_14307_gb300 import transport as T


@pytest.fixture(scope="module")
def lib():
    O.build()


def test_angular_velocity_matches_the_oracles_energies_and_site_velocities(lib):
    system = I.suspension(14, 5.0, 0.15, 2.0, 2, 5.0, I.SRD, 1, I.P64, seed=4)
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)
    O.step(osys, ost, 2)
    nb = system.n_bodies
    # principal moments: the templates are given in their principal-axis frame
    Ihat = np.array([np.sum(system.shapes[s].m[:, None] * (np.sum(system.shapes[s].b ** 2, axis=1)[:, None]
                                                           - system.shapes[s].b ** 2), axis=0)
                     for s in system.body_shape_array()])
    W = T.angular_velocity(ost.q[:nb], ost.Lm[:nb], Ihat)
    _, ER = O.body_energies(osys, ost)
    assert np.allclose(0.5 * np.sum(W * ost.Lm[:nb], axis=1), ER, rtol=1e-10)
    # the oracle's rigid site velocities: V + omega x d, d = Q b
    vs = O.rigid_site_velocities(osys, ost)
    sh = system.shapes[system.body_shape_array()[0]]
    Q = T.rotation_matrix(ost.q[0])
    d = sh.b @ Q.T
    M = sh.m.sum()
    assert np.allclose(vs[: sh.n_sites], ost.P[0] / M + np.cross(W[0], d), rtol=1e-10, atol=1e-12)


def test_autocorrelation_of_simple_signals():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(5, 3))
    const = np.repeat(x[None], 20, axis=0)
    c = T.velocity_autocorrelation(const, 6)
    assert np.allclose(c, np.sum(x * x, axis=1)[:, None])
    sign = (-1.0) ** np.arange(20)
    alt = sign[:, None, None] * x[None]
    c = T.velocity_autocorrelation(alt, 6)
    assert np.allclose(c, np.sum(x * x, axis=1)[:, None] * (-1.0) ** np.arange(6)[None, :])
    X = rng.normal(size=(50, 4, 3))
    assert np.allclose(T.velocity_autocorrelation(X, 3)[:, 0], np.mean(np.sum(X * X, axis=-1), axis=0))
