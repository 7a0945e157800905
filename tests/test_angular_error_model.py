"""Error model behind the parity bar of the +a variants (angular-momentum-
conserving SRD+a / MPCD-AT+a, Sec. II.A), on the CPU.

The GPU forms the correction from exact integer cell sums (lattice offsets Q,
quantised momenta P = round(fl32(m v) 2^20) in P32), solves Pi w = dL per cell in
FP64 by the adjugate (least-norm for collinear members) and applies
v' = v* + w' x (M Q - sum mu Q) in the working precision.  This test restates
that arithmetic with numpy, feeds it the oracle's own pre- and post-rule
velocities (rounded where the P32 form stores them), and checks it against the
oracle's +a result:

the error stays below 0.1 tol (|v| + 1 + |w_c|), tol = 1e-5 (P32) and 1e-12
(P64), w_c the cell's correction, in a 30^3 solvent box (nearly collinear
cells with |w_c| in the hundreds) and beside colloid sites.  The largest
errors come from the quantised momenta of ordinary cells (P32: 3.8e-7 of the
scale); the |w_c| term covers the rounding of w x r_c in the rare cells where
w_c is large.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I

f32 = np.float32
TOL = {I.P32: 1e-5, I.P64: 1e-12}


def solve(Cm, dL):
    """G x = dL with G = tr(C) I - C by the adjugate; least-norm x for rank-one C"""
    tr = np.trace(Cm)
    if not tr > 0:
        return np.zeros(3)
    G = tr * np.eye(3) - Cm
    adj = np.array([[G[1, 1] * G[2, 2] - G[1, 2] ** 2, G[0, 2] * G[1, 2] - G[0, 1] * G[2, 2],
                     G[0, 1] * G[1, 2] - G[0, 2] * G[1, 1]],
                    [0, G[0, 0] * G[2, 2] - G[0, 2] ** 2, G[0, 1] * G[0, 2] - G[0, 0] * G[1, 2]],
                    [0, 0, G[0, 0] * G[1, 1] - G[0, 1] ** 2]])
    adj = np.triu(adj) + np.triu(adj, 1).T
    det = G[0] @ adj[:, 0]
    if det > 1e-12 * tr ** 3:
        return adj @ dL / det
    return (dL - Cm @ dL / tr) / tr


def model(system):
    prec = system.params.precision
    st = I.initial_state(system)
    o0 = O.OracleSystem(system, angular=0)
    s0 = O.OracleState(o0, st)
    O.stream(o0, s0)
    x, vpre = s0.x.copy(), s0.v.copy()
    tr = O.collide(o0, s0)
    o1 = O.OracleSystem(system, angular=1)
    s1 = O.OracleState(o1, st)
    O.stream(o1, s1)
    tr1 = O.collide(o1, s1)
    Ns, Nb = o0.n_solvent, o0.n_sites

    def sites(a):
        return a.ravel()[: 3 * Nb].reshape(-1, 3)
    pos = np.concatenate([x, sites(tr["site_r"])])
    vin = np.concatenate([vpre, sites(tr["site_v"])])
    vst = np.concatenate([s0.v, sites(tr["site_vpost"])])
    ref = np.concatenate([s1.v, sites(tr1["site_vpost"])])
    site = np.arange(Ns + Nb) >= Ns
    ms = system.params.m_solvent
    mb = float(system.shapes[0].m[0]) if Nb else 0.0
    m = np.where(site, mb, ms)
    S = tr["shift"][0].astype(np.int64)
    cell = np.concatenate([tr["cell_solvent"], tr["cell_site"].ravel()[:Nb]]).astype(np.int64)
    p32 = prec == I.P32
    if p32:
        X = np.floor(pos.astype(f32).astype(np.float64) * 2.0 ** 20).astype(np.int64)
        mf = m.astype(f32)[:, None]
        P = np.rint((mf * vin.astype(f32)).astype(np.float64) * 2.0 ** 20).astype(np.int64)
        Ps = np.rint((mf * vst.astype(f32)).astype(np.float64) * 2.0 ** 20).astype(np.int64)
        mus, mub = float(np.rint(float(f32(ms)) * 2 ** 24)), float(np.rint(float(f32(mb)) * 2 ** 24))
        unit = 2.0 ** -20 / 2.0 ** -24
    else:
        X = np.floor(pos * 2.0 ** 20).astype(np.int64)
        P, Ps = m[:, None] * vin, m[:, None] * vst
        mus, mub, unit = ms, mb, 1.0
    Q = (X - S[None, :]) & 0xFFFFF
    out = vst.copy()
    order = np.argsort(cell, kind="stable")
    bounds = np.searchsorted(cell[order], np.arange(o0.n_cells + 1))
    mu = np.where(site, mub, mus)
    for c in range(o0.n_cells):
        ids = order[bounds[c]: bounds[c + 1]]
        if len(ids) < 2:
            continue
        q, w8 = Q[ids], mu[ids]
        M = w8.sum()
        sw = (w8[:, None] * q).sum(0)
        Qc = sw / M
        Cm = (w8[:, None, None] * q[:, :, None] * q[:, None, :]).sum(0) - np.outer(sw, Qc)
        dPq = P[ids] - Ps[ids]
        dL = np.cross(q, dPq).sum(0).astype(np.float64) - np.cross(Qc, dPq.sum(0).astype(np.float64))
        wp = solve(Cm, dL) * unit / M          # w' = w / (M 2^20)
        if p32:
            rc = (np.int64(M) * q - sw.astype(np.int64)[None, :]).astype(f32)
            w, vs = wp.astype(f32), vst[ids].astype(f32)
            out[ids] = (vs + np.cross(w, rc).astype(f32)).astype(np.float64)
        else:
            out[ids] = vst[ids] + np.cross(wp, M * q - sw[None, :])
    wc = np.linalg.norm(tr1["cell_omega"], axis=1)[cell]
    ratio = np.abs(out - ref).max(1) / (np.abs(ref).max(1) + 1.0 + wc)
    return ratio, wc


def solvent(prec, L, seed, rule=I.SRD):
    prm = I.Params(rule=rule, thermostat=1, precision=prec, seed=seed)
    return I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [L], 5.0, [[]], "solvent_only",
                          placement_seed=seed)


def suspension(prec, rule):
    prm = I.Params(rule=rule, thermostat=1, precision=prec, seed=6)
    return I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [(12, 16, 12)], 5.0, [[0, 0, 0]], "suspension",
                          placement_seed=6)


@pytest.mark.parametrize("prec", [I.P32, I.P64])
def test_bar_holds_with_margin_in_a_large_box(prec):
    ratio, wc = model(solvent(prec, (30, 30, 30), 9))
    assert wc.max() > 100                      # nearly collinear cells are present
    assert ratio.max() < 0.1 * TOL[prec], ratio.max()


@pytest.mark.parametrize("prec,rule", [(I.P32, I.SRD), (I.P32, I.AT), (I.P64, I.SRD)])
def test_bar_holds_beside_colloid_sites(prec, rule):
    ratio, _ = model(suspension(prec, rule))
    assert ratio.max() < 0.1 * TOL[prec], ratio.max()

