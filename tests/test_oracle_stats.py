"""Statistical pins of the oracle: the distributions the paper validates.

* Sec. III.A: <E_T> = <E_R> = 3kT/2 for a rigid sphere (the paper prints
  1.4999 +- 0.0003 and 1.50015 +- 0.00009).  In a small periodic box the total
  momentum is conserved, so the translational expectation is
  (3/2) kT (1 - M/M_total); the rotational one is 3kT/2.
* Supplementary Fig. S1: without thermalisation the naive transfer drains
  energy (no thermostat) - the negative control.
* Sec. II.A: the thermostatted solvent relaxes to Maxwell-Boltzmann at T.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2604_14307_gb300 import inputs as I


def block_mean_err(x, nblocks=20):
    x = np.asarray(x)
    n = len(x) // nblocks
    b = x[: n * nblocks].reshape(nblocks, n).mean(1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nblocks)


def test_equipartition_rigid_sphere(golden):
    n_rep, L, steps, burn = 6, 10, 2500, 200
    prm = I.Params(kT=1.0, dt=0.1, alpha_deg=130.0, rule=I.SRD, thermostat=1, seed=21)
    sh = I.sphere_shape(2.0, 2, 5.0)
    rng = np.random.default_rng(8)
    R_q = [(np.array([[5.0, 5.0, 5.0]]), I.random_quaternions(rng, 1)) for _ in range(n_rep)]
    s = I.build_system(prm, [sh], [(L, L, L)] * n_rep, 5.0, [[0]] * n_rep, "eq", R_q=R_q)
    osys = O.OracleSystem(s)
    ost = O.OracleState(osys, I.initial_state(s))
    ET, ER = [], []
    for k in range(steps):
        O.step(osys, ost, 1)
        if k >= burn:
            et, er = O.body_energies(osys, ost)
            ET.append(et.mean())
            ER.append(er.mean())
    M = sh.m.sum()
    Mtot = M + 5.0 * L**3
    expect_T = golden["mean_E_T"]["expected"] * (1 - M / Mtot)
    mT, eT = block_mean_err(ET)
    mR, eR = block_mean_err(ER)
    assert abs(mT - expect_T) < 3.5 * eT + 0.02, (mT, eT, expect_T)
    assert abs(mR - golden["mean_E_R"]["expected"]) < 3.5 * eR + 0.02, (mR, eR)


def _solvent_temperature(ost):
    return (ost.v ** 2).mean()


@pytest.mark.parametrize("naive", [1, 0])
def test_naive_transfer_drains_energy_fig_s1(naive):
    prm = I.Params(kT=1.0, dt=0.1, alpha_deg=130.0, rule=I.SRD, thermostat=0, seed=31,
                   naive_transfer=naive)
    sh = I.sphere_shape(2.0, 2, 5.0)
    R = np.array([[3.0, 3.0, 3.0], [3.0, 9.0, 9.0], [9.0, 3.0, 9.0], [9.0, 9.0, 3.0]])
    q = I.random_quaternions(np.random.default_rng(3), 4)
    s = I.build_system(prm, [sh], [(12, 12, 12)], 5.0, [[0] * 4], "neg", R_q=[(R, q)])
    osys = O.OracleSystem(s)
    ost = O.OracleState(osys, I.initial_state(s))
    T0 = _solvent_temperature(ost)
    O.step(osys, ost, 300)
    T1 = _solvent_temperature(ost)
    if naive:
        assert T1 < 0.6 * T0
    else:
        assert abs(T1 / T0 - 1) < 0.06


def test_thermostat_relaxes_solvent_to_maxwell_boltzmann():
    prm = I.Params(kT=1.0, dt=0.1, alpha_deg=130.0, rule=I.SRD, thermostat=1, seed=41)
    s = I.build_system(prm, [I.sphere_shape(1.0, 0, 1.0)], [(12, 12, 12)], 5.0, [[]], "mb")
    st = I.initial_state(s)
    rng = np.random.default_rng(0)
    st.v = rng.uniform(-1.0, 1.0, st.v.shape) * 2.5   # far from MB and too hot
    st.v -= st.v.mean(0)
    osys = O.OracleSystem(s)
    ost = O.OracleState(osys, st)
    O.step(osys, ost, 40)
    v = ost.v - ost.v.mean(0)
    for a in range(3):
        assert stats.kstest(v[:, a], "norm").pvalue > 1e-3
    assert abs(v.var() - 1.0) < 0.03
