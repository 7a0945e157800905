"""Parity at full size, in the launch configuration bench.py times.

The oracle cannot step 80-145 million particles in a test, so one GPU step
(the pipelined mpcd_step path, autotuned like bench.py) is checked by what can
be computed independently at any size:

* streaming (row a1): every particle's position equals x + v dt wrapped into
  [0, L), recomputed in float32 with the same rounding - bit-exact;
* binning and cell sums (rows a2, a5, a6): every cell's P32 words equal the
  integer sums recomputed with numpy from the streamed positions, the grid
  shift, the stored velocities and the sites' thermalised velocities -
  bit-exact (for MPCD-AT the three noise words are compared after decoding,
  since the GPU draws its noise with float32 transcendentals);
* collision parameters and velocities (row a7) of a random sample of cells:
  the SRD axis and the thermostat's E' come from the oracle's generator
  (orc_srd_axis, orc_thermostat_energy, orc_normals), u and E_rel from the
  recomputed words; the post-collision velocities of the sample's particles
  then follow from Sec. II.A and must agree within 1e-5 (|v'| + 1);
* total momentum (solvent + bodies) is conserved to float32 rounding: ten
  times the random walk of one float32 rounding (2^-23 m |v|, |v| ~ 1) per
  particle and component.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14307_gb300 import binding, build_lib
    build_lib.build()
    return binding


def q(x, scale):
    """round-half-even(float32 value x 2^scale) as int64 (exact in float64)"""
    return np.rint(x.astype(np.float64) * 2.0**scale).astype(np.int64)


def cells_of(xs, S, L, base):
    """binning rule: X = floor(x 2^20), cell = floor((X - S) / 2^20) mod L"""
    c = []
    for k in range(3):
        X = np.floor(xs[:, k].astype(np.float64) * 2.0**20).astype(np.int64)
        c.append(np.mod(np.floor_divide(X - S[:, k], 2**20), L[:, k]))
    return base + c[0] + L[:, 0] * (c[1] + L[:, 1] * c[2])


def check_full_step(B, system, n_sample=2000, seed=0):
    st = I.initial_state(system)
    sim = B.Simulation(system)
    sim.set_state(st)
    sim.autotune(steps_per_trial=10)          # the launch configuration bench.py times
    sim.set_state(st)
    sim.set_debug(True)
    p_before = sim.diagnostics()
    sim.step(1)
    d = sim.debug_cells()
    g = sim.get_state()
    p_after = sim.diagnostics()
    sim.close()
    return verify_step(system, st, g.x, g.v, d, p_before, p_after, n_sample, seed)


def verify_step(system, st, gx, gv_all, d, p_before, p_after, n_sample=2000, seed=0):
    """Checks of one collision step (see the module docstring) from the state
    before it (st), the positions and velocities after it, and the debug
    capture of the cell words, parameters, grid shift and site velocities."""
    prm = system.params
    assert prm.precision == I.P32
    x0 = st.x.astype(np.float32)
    v0 = st.v.astype(np.float32)
    n_rep = system.n_rep
    so = system.solvent_offsets()
    Lr = system.L_array().astype(np.int64)
    ncell = np.prod(Lr, axis=1)
    cbase = np.concatenate([[0], np.cumsum(ncell)[:-1]]).astype(np.int64)
    rep_of = np.repeat(np.arange(n_rep), np.diff(so))
    Lp = Lr[rep_of]

    # a1: streaming, bit-exact
    dt = np.float32(prm.dt)
    Lf = Lp.astype(np.float32)
    y = x0 + v0 * dt
    y = np.where(y >= Lf, y - Lf, y)
    yw = y + Lf
    y = np.where(y < 0, np.where(yw >= Lf, np.float32(0), yw), y)
    assert np.array_equal(np.asarray(gx, dtype=np.float32), y)
    del yw, Lf

    # a2, a5, a6: cell of every particle and every cell's words
    S = np.asarray(d["shift"], dtype=np.int64).reshape(n_rep, 3)
    cell = cells_of(y, S[rep_of], Lp, cbase[rep_of])
    C = int(ncell.sum())
    m_f = np.float32(prm.m_solvent)
    p = (m_f * v0).astype(np.float32)
    qp = [q(p[:, k], 32) for k in range(3)]
    # exact in float64: integers below 2^36 each, a few dozen per cell
    sums = [np.bincount(cell, weights=qp[k].astype(np.float64), minlength=C) for k in range(3)]
    ns = np.bincount(cell, minlength=C).astype(np.int64)
    nb = np.zeros(C, dtype=np.int64)
    if prm.rule == I.SRD:
        e = ((p[:, 0] * v0[:, 0]) + (p[:, 1] * v0[:, 1])) + (p[:, 2] * v0[:, 2])
        se = np.bincount(cell, weights=q(e, 28).astype(np.float64), minlength=C)
    # sites: their thermalised velocities enter the same words
    if system.n_sites:
        bo = system.body_offsets()
        body_rep = np.repeat(np.arange(n_rep), np.diff(bo))
        nsb = np.array([system.shapes[s].n_sites for s in system.body_shape_array()])
        site_rep = np.repeat(body_rep, nsb)
        msite = np.float32(system.shapes[system.body_shape_array()[0]].m[0])
        sc = np.asarray(d["site_cell"], dtype=np.int64) + cbase[site_rep]
        sv = np.asarray(d["site_v"]).astype(np.float32)
        ps = (msite * sv).astype(np.float32)
        for k in range(3):
            sums[k] += np.bincount(sc, weights=q(ps[:, k], 32).astype(np.float64), minlength=C)
        nb = np.bincount(sc, minlength=C).astype(np.int64)
        if prm.rule == I.SRD:
            es = ((ps[:, 0] * sv[:, 0]) + (ps[:, 1] * sv[:, 1])) + (ps[:, 2] * sv[:, 2])
            se += np.bincount(sc, weights=q(es, 28).astype(np.float64), minlength=C)
    s1 = [np.rint(sums[k]).astype(np.int64) for k in range(3)]
    w = np.asarray(d["sums"])
    assert np.array_equal(w[0], s1[0] + (ns << 48))
    assert np.array_equal(w[1], s1[1] + (nb << 48))
    assert np.array_equal(w[2], s1[2])
    if prm.rule == I.SRD:
        assert np.array_equal(w[3], np.rint(se).astype(np.int64))

    # a7 on a sample of colliding cells
    n_part = ns + nb
    Mq = ns * float(prm.m_solvent)
    if system.n_sites:
        Mq = Mq + nb * float(msite)
    rng = np.random.default_rng(seed)
    live = np.where(n_part >= 2)[0]
    sample = np.sort(rng.choice(live, size=min(n_sample, live.size), replace=False))
    osys = O.OracleSystem(system)
    par = np.asarray(d["params"], dtype=np.float64)
    rep_c = np.searchsorted(cbase, sample, side="right") - 1
    u = np.stack([s1[k][sample] * 2.0**-32 / Mq[sample] for k in range(3)], axis=1)
    assert np.all(np.abs(par[sample, 0:3] - u) <= TOL * (np.abs(u) + 1.0))
    al = math.radians(prm.alpha_deg)
    in_sample = np.zeros(C, dtype=bool)
    in_sample[sample] = True
    sel = np.where(in_sample[cell])[0]
    pos = np.searchsorted(sample, cell[sel])
    vs = v0[sel].astype(np.float64)
    uu = u[pos]
    if prm.rule == I.SRD:
        axis = np.array([O.srd_axis(osys, int(r), 0, int(c - cbase[r])) for r, c in zip(rep_c, sample)])
        assert np.all(np.abs(par[sample, 4:7] - axis) <= TOL)
        kappa = np.ones(sample.size)
        if prm.thermostat:
            S2 = w[3][sample].astype(np.float64) * 2.0**-28
            erel = 0.5 * (S2 - np.sum(u * u, axis=1) * Mq[sample])
            ep = np.array([O.thermostat_energy(osys, int(r), 0, int(c - cbase[r]), int(n))
                           for r, c, n in zip(rep_c, sample, n_part[sample])])
            kappa = np.sqrt(ep / erel)
            assert np.all(np.abs(par[sample, 3] - kappa) <= 5 * TOL * kappa)
        a = axis[pos]
        wv = vs - uu
        nd = np.sum(a * wv, axis=1, keepdims=True)
        rot = wv * math.cos(al) + np.cross(a, wv) * math.sin(al) + a * nd * (1.0 - math.cos(al))
        vnew = uu + kappa[pos][:, None] * rot
    else:
        xib = np.stack([w[3 + k][sample] for k in range(3)], axis=1) * 2.0**-32 / Mq[sample][:, None]
        assert np.all(np.abs(par[sample, 4:7] - xib) <= TOL * (np.abs(xib) + 1.0))
        tags = sel - so[rep_of[sel]]
        scale = math.sqrt(prm.kT / prm.m_solvent)
        xi = np.concatenate([O.normals(osys, int(r), 0, tags[rep_of[sel] == r], O.TAG_AT)
                             for r in np.unique(rep_of[sel])]) * scale
        order = np.argsort(rep_of[sel], kind="stable")
        xi_sel = np.empty_like(xi)
        xi_sel[order] = xi
        vnew = uu + xi_sel - xib[pos]
    gv = np.asarray(gv_all)[sel].astype(np.float64)
    assert np.all(np.abs(gv - vnew) <= TOL * (np.abs(vnew) + 1.0))

    # momentum: solvent + bodies, conserved to float32 rounding of the new velocities
    P0 = np.asarray(p_before["p_solvent"]) + np.asarray(p_before["p_bodies"])
    P1 = np.asarray(p_after["p_solvent"]) + np.asarray(p_after["p_bodies"])
    m2 = system.n_solvent * float(prm.m_solvent) ** 2
    if system.n_sites:
        m2 += system.n_sites * float(msite) ** 2
    bar = 10.0 * math.sqrt(m2) * 2.0**-23
    assert np.all(np.abs(P1 - P0) < bar), (np.abs(P1 - P0), bar)
    return sample.size, sel.size


@pytest.mark.parametrize("thermostat", [2, 1])
def test_full_size_suspension_L200(B, thermostat):
    """The benchmark workload: L=200, 80 M solvent, 8952 642-site spheres, SRD +
    thermostat (E' by Marsaglia-Tsang rejection, as bench.py times it, and as a
    sum of exponentials)."""
    ns, np_ = check_full_step(B, I.suspension_L200(I.P32, seed=1, thermostat=thermostat))
    assert ns >= 1000 and np_ >= 5000


def test_full_size_batched_single_sphere(B):
    """4096 uneven boxes L in {12, 16, 20, 24}, one 162-site sphere each, SRD."""
    check_full_step(B, I.batched_single_sphere(n_rep=4096, precision=I.P32, seed=1))


def test_batched_mixed_shapes_sampled(B):
    """MPCD-AT with spheres, dumbbells and rods; 24 of the 256 boxes (placing all
    256 by random sequential addition takes minutes on the host)."""
    check_full_step(B, I.batched_mixed_shapes(n_rep=24, precision=I.P32, seed=1))
