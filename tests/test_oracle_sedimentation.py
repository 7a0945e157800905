"""Pins of the oracle's sedimentation forcing (Sec. III.B): a constant force on
every body at its centre of mass, balanced by an equal share on every solvent
particle, on CPU.

* Streaming alone (no collision) has closed forms: under a constant force the
  kick-drift-kick step is exact, so after n steps a solvent particle sits at
  x0 + v0 t + g t^2 / 2 (wrapped) with velocity v0 + g t, g = -B f / (N_s m), and
  a lone body has P0 + f t and R0 + P0 t / M + f t^2 / (2 M).
* The box stays force free: solvent plus body momentum is conserved through
  whole steps (streaming, collision, transfer).
* A zero force reproduces the unforced step bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    O.build()


def one_sphere(precision=I.P64, seed=4, L=12):
    prm = I.Params(rule=I.SRD, thermostat=1, precision=precision, seed=seed)
    sh = I.sphere_shape(2.0, 2, 5.0)
    R_q = [(np.array([[L / 2.0, L / 2.0, L / 2.0]]), np.array([[1.0, 0.0, 0.0, 0.0]]))]
    return I.build_system(prm, [sh], [(L, L, L)], 5.0, [[0]], "one_sphere", R_q=R_q)


def test_streaming_under_a_constant_force_has_the_closed_form(lib):
    system = one_sphere()
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    f = np.array([0.5, -0.2, 0.1])
    osys.set_body_force(f)
    ost = O.OracleState(osys, st)
    n, dt = 7, system.params.dt
    t = n * dt
    for _ in range(n):
        O.stream(osys, ost)
    Ns, B, m = system.n_solvent, 1, system.params.m_solvent
    g = -B * f / (Ns * m)
    L = np.array(system.replicas[0].L, dtype=np.float64)
    assert np.allclose(ost.v, st.v + g * t, rtol=0, atol=1e-13)
    x = np.mod(st.x + st.v * t + 0.5 * g * t * t, L)
    d = np.abs(ost.x - x)
    assert np.all(np.minimum(d, L - d) < 1e-11)
    M = system.shapes[0].m.sum()
    assert np.allclose(ost.P[0], st.P[0] + f * t, rtol=0, atol=1e-12)
    R = np.mod(st.R[0] + st.P[0] * t / M + 0.5 * f * t * t / M, L)
    assert np.allclose(ost.R[0], R, rtol=0, atol=1e-12)
    # balance: the solvent gained exactly what the body did not
    dps = m * (ost.v - st.v).sum(axis=0)
    assert np.allclose(dps + (ost.P[0] - st.P[0]), 0.0, atol=1e-10)


@pytest.mark.parametrize("precision", [I.P64, I.P32])
def test_whole_steps_keep_the_box_force_free(lib, precision):
    system = one_sphere(precision)
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    osys.set_body_force([0.5, 0.0, 0.0])
    ost = O.OracleState(osys, st)
    m = system.params.m_solvent
    p0 = m * ost.v.sum(axis=0) + ost.P.sum(axis=0)
    O.step(osys, ost, 5)
    p1 = m * ost.v.sum(axis=0) + ost.P.sum(axis=0)
    tol = 1e-9 if precision == I.P64 else 2e-3
    assert np.allclose(p1, p0, atol=tol)
    assert ost.P[0, 0] > st.P[0, 0]          # the body is pushed along +x


def test_zero_force_is_the_plain_step(lib):
    system = one_sphere(I.P32)
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    a = O.OracleState(osys, st)
    O.step(osys, a, 3)
    osys.set_body_force([0.0, 0.0, 0.0])
    b = O.OracleState(osys, st)
    O.step(osys, b, 3)
    for k in ("x", "v", "R", "q", "P", "Lm"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
