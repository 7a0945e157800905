"""Pins of the oracle's angular-momentum-conserving collision variants (SRD+a,
MPCD-AT+a), which Sec. II.A cites as a modification of the collision rule.

What fixes the variant independently of the oracle's formula:

* conservation: in every cell with two or more members the linear momentum
  and the angular momentum about the cell's centre of mass (positions on the
  2^-20 lattice of the binning rule) are unchanged by the collision, while
  the plain rules change the angular momentum (the negative control);
* least change: the +a velocities differ from the plain rule's by the
  smallest mass-weighted change that restores the angular momentum and keeps
  the momentum, found here by a generic least-squares solve of those six
  linear constraints (numpy lstsq, minimum norm) and not by the inertia
  tensor;
* MPCD-AT+a energy law: the rule keeps the cell's rigid motion (translation
  and rotation) and replaces the rest by Gaussian noise projected off the
  rigid motions, so the kinetic energy after the collision is the rigid-motion
  energy before it plus kT/2 per remaining degree of freedom, 3N - 6 for
  N >= 3 members and 1 for N = 2, whatever the velocities were (plain MPCD-AT
  redraws the rotation as well and misses the law from a hot start);
* Galilean invariance and special cases: a uniform velocity c added before
  the collision comes out as c; SRD+a with alpha = 0 and no thermostat is the
  identity; single-member cells are unchanged.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I


def solvent_box(rule, thermostat=0, angular=1, precision=I.P64, seed=3, L=(8, 8, 8), alpha=130.0):
    prm = I.Params(rule=rule, thermostat=thermostat, precision=precision, seed=seed, alpha_deg=alpha,
                   angular=angular)
    return I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [L], 5.0, [[]], "solvent_only",
                          placement_seed=seed)


def suspension_box(rule, angular=1, precision=I.P64, seed=6):
    prm = I.Params(rule=rule, thermostat=1, precision=precision, seed=seed, angular=angular)
    return I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [(12, 12, 12)], 5.0, [[0, 0]], "suspension",
                          placement_seed=seed)


def lattice_offsets(r, S):
    """position inside the shifted cell on the 2^-20 lattice of the binning rule"""
    X = np.floor(np.asarray(r, dtype=np.float64) * 2.0**20).astype(np.int64)
    t = X - np.asarray(S, dtype=np.int64)[None, :]
    return (t - np.floor_divide(t, 2**20) * 2**20) * 2.0**-20


def collide(system, angular, st=None, dv=None):
    """one collision of the oracle from the system's initial state (or st);
    returns (members' positions, masses, v before, v after, trace, state)"""
    osys = O.OracleSystem(system, angular=angular)
    st = I.initial_state(system) if st is None else st
    ost = O.OracleState(osys, st)
    if dv is not None:
        ost.v += dv
    v0 = ost.v.copy()
    tr = O.collide(osys, ost)
    Ns, Nb = osys.n_solvent, osys.n_sites

    def sites(a):
        return a[: 3 * Nb].reshape(-1, 3) if Nb else np.zeros((0, 3))
    pos = np.concatenate([ost.x, sites(tr["site_r"].ravel())])
    m_site = []
    for b in range(osys.n_bodies):
        sh = system.shapes[system.body_shape_array()[b]]
        m_site.append(sh.m)
    m = np.concatenate([np.full(Ns, osys.params["m_solvent"])] + m_site)
    vin = np.concatenate([v0, sites(tr["site_v"].ravel())])
    vout = np.concatenate([ost.v, sites(tr["site_vpost"].ravel())])
    return pos, m, vin, vout, tr, osys


def cells(tr, n_cells):
    st = tr["cell_start"]
    for c in range(n_cells):
        yield c, tr["order"][st[c]: st[c + 1]]


def cell_frame(pos, m, S, ids):
    q = lattice_offsets(pos[ids], S)
    mm = m[ids]
    com = (mm[:, None] * q).sum(0) / mm.sum()
    return q - com, mm


def ang(rc, mm, v):
    return (mm[:, None] * np.cross(rc, v)).sum(0)


CASES = [(I.SRD, 0), (I.SRD, 1), (I.AT, 0)]


@pytest.mark.parametrize("rule,thermostat", CASES)
def test_cell_momentum_and_angular_momentum_conserved(rule, thermostat):
    for angular in (1, 0):
        system = solvent_box(rule, thermostat, angular)
        pos, m, vin, vout, tr, osys = collide(system, angular)
        S = tr["shift"][0]
        worst_p, worst_l, changed = 0.0, 0.0, 0.0
        for c, ids in cells(tr, osys.n_cells):
            if len(ids) < 2:
                assert np.array_equal(vout[ids], vin[ids])
                continue
            rc, mm = cell_frame(pos, m, S, ids)
            dp = (mm[:, None] * (vout[ids] - vin[ids])).sum(0)
            dl = ang(rc, mm, vout[ids]) - ang(rc, mm, vin[ids])
            worst_p = max(worst_p, np.abs(dp).max())
            if angular:
                worst_l = max(worst_l, np.abs(dl).max())
            else:
                changed = max(changed, np.abs(dl).max())
        assert worst_p < 1e-12
        if angular:
            assert worst_l < 1e-11, worst_l
        else:
            assert changed > 0.1          # the plain rule does not conserve it


@pytest.mark.parametrize("rule", [I.SRD, I.AT])
def test_conserved_with_colloid_sites(rule):
    """sites take part like solvent; the velocities they leave with (before the
    reset to rigid motion) carry the correction"""
    system = suspension_box(rule)
    pos, m, vin, vout, tr, osys = collide(system, 1)
    assert osys.n_sites > 0
    S = tr["shift"][0]
    n_with_sites = 0
    for c, ids in cells(tr, osys.n_cells):
        if len(ids) < 2:
            continue
        n_with_sites += bool((ids >= osys.n_solvent).any())
        rc, mm = cell_frame(pos, m, S, ids)
        scale = 1.0 + np.abs(mm[:, None] * vin[ids]).sum()
        assert np.abs((mm[:, None] * (vout[ids] - vin[ids])).sum(0)).max() < 1e-12 * scale
        assert np.abs(ang(rc, mm, vout[ids]) - ang(rc, mm, vin[ids])).max() < 1e-11 * scale
    assert n_with_sites > 100


def test_float32_form_conserves_to_float_rounding():
    system = solvent_box(I.SRD, 1, 1, precision=I.P32)
    pos, m, vin, vout, tr, osys = collide(system, 1)
    S = tr["shift"][0]
    worst = 0.0
    for c, ids in cells(tr, osys.n_cells):
        if len(ids) >= 2:
            rc, mm = cell_frame(pos, m, S, ids)
            worst = max(worst, np.abs(ang(rc, mm, vout[ids]) - ang(rc, mm, vin[ids])).max())
    assert worst < 1e-5


@pytest.mark.parametrize("rule,thermostat", CASES)
def test_correction_is_the_least_change(rule, thermostat):
    """v'_+a - v'_plain is the minimum mass-weighted-norm change with zero net
    momentum that restores the cell's angular momentum"""
    system = solvent_box(rule, thermostat, seed=11)
    pos, m, vin, va, tr, osys = collide(system, 1)
    _, _, _, vp, tr0, _ = collide(system, 0)
    assert np.array_equal(tr["order"], tr0["order"])
    S = tr["shift"][0]
    checked = {2: 0, 3: 0}
    for c, ids in cells(tr, osys.n_cells):
        n = len(ids)
        if n < 2:
            continue
        rc, mm = cell_frame(pos, m, S, ids)
        # constraints on delta (3n): sum m delta = 0; sum m rc x delta = L_in - L(plain)
        A = np.zeros((6, 3 * n))
        for i in range(n):
            A[0:3, 3 * i: 3 * i + 3] = mm[i] * np.eye(3)
            x, y, z = rc[i]
            A[3:6, 3 * i: 3 * i + 3] = mm[i] * np.array([[0, -z, y], [z, 0, -x], [-y, x, 0]])
        b = np.concatenate([np.zeros(3), ang(rc, mm, vin[ids]) - ang(rc, mm, vp[ids])])
        w = np.repeat(1.0 / np.sqrt(mm), 3)          # y = sqrt(m) delta: plain minimum norm
        y = np.linalg.lstsq(A * w[None, :], b, rcond=1e-10)[0]
        delta = (y * w).reshape(n, 3)
        assert np.abs(va[ids] - vp[ids] - delta).max() < 1e-9, (c, n)
        checked[min(n, 3)] += 1
    assert checked[2] > 20 and checked[3] > 300


def rigid_energy(rc, mm, v):
    """kinetic energy of the cell's rigid motion: the translation with the
    centre-of-mass velocity and the rotation that carries the angular momentum
    about the centre of mass (least-norm for collinear members)"""
    M = mm.sum()
    u = (mm[:, None] * v).sum(0) / M
    Lc = ang(rc, mm, v - u)
    Pi = (mm[:, None, None] * ((rc * rc).sum(1)[:, None, None] * np.eye(3)[None] -
                                rc[:, :, None] * rc[:, None, :])).sum(0)
    om = np.linalg.pinv(Pi, rcond=1e-12) @ Lc
    return 0.5 * M * (u @ u) + 0.5 * (om @ Lc)


@pytest.mark.parametrize("angular", [1, 0])
def test_at_keeps_rigid_energy_and_thermalises_the_rest(angular):
    """MPCD-AT+a: E_kin after = E_rigid before + kT/2 chi^2(f), f = 3N - 6
    (N >= 3) or 1 (N = 2), from a hot start (sd 3) far from kT = 1; plain
    MPCD-AT redraws the rotation too and misses the law by far"""
    kT = 1.0
    system = solvent_box(I.AT, 0, angular, seed=17, L=(14, 14, 14))
    st = I.initial_state(system)
    st.v = np.random.default_rng(2).normal(0.0, 3.0, st.v.shape)
    pos, m, vin, vout, tr, osys = collide(system, angular, st=st)
    S = tr["shift"][0]
    E = {2: 0.0, 3: 0.0}
    dof = {2: 0, 3: 0}
    for c, ids in cells(tr, osys.n_cells):
        n = len(ids)
        if n < 2:
            continue
        rc, mm = cell_frame(pos, m, S, ids)
        k = min(n, 3)
        E[k] += 0.5 * (mm[:, None] * vout[ids] ** 2).sum() - rigid_energy(rc, mm, vin[ids])
        dof[k] += 1 if n == 2 else 3 * n - 6
    for k in (2, 3):
        mean = E[k] / dof[k]
        sd = 0.5 * kT * math.sqrt(2.0 / dof[k])
        if angular:
            assert abs(mean - 0.5 * kT) < 5 * sd, (k, mean, sd)
        else:
            assert abs(mean - 0.5 * kT) > 10 * sd, (k, mean, sd)


@pytest.mark.parametrize("rule,thermostat", CASES)
def test_galilean_invariance(rule, thermostat):
    system = solvent_box(rule, thermostat, seed=5)
    c = np.array([0.7, -1.3, 2.1])
    _, _, _, v1, _, _ = collide(system, 1)
    _, _, _, v2, _, _ = collide(system, 1, dv=c)
    assert np.abs(v2 - v1 - c).max() < 1e-11


def test_srd_a_without_rotation_is_the_identity():
    system = solvent_box(I.SRD, 0, 1, alpha=0.0, seed=9)
    _, _, vin, vout, _, _ = collide(system, 1)
    assert np.abs(vout - vin).max() < 1e-12
