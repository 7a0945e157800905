"""Pins of the oracle's reverse non-equilibrium exchange (Sec. III.B) and of the
host-side viscosity analysis (Eq. 14), on CPU.

The exchange is checked against properties that characterise it, not against a
retyped copy of its sort:
* a swap of v_x between equal masses: positions, v_y, v_z and every other
  particle are untouched, the multiset of v_x values, the total x momentum and
  the kinetic energy are unchanged;
* the returned momentum equals the x momentum slab A lost;
* selection: every exchanged particle of a slab is at least as close to its
  target (ties: lower id) as every particle of that slab that was not, counted
  pair by pair;
* pairing: the k-th closest of A is exchanged with the k-th closest of B, with
  ranks counted by brute force;
* degenerate cases: no pairs, an empty slab, fewer particles than pairs.
The viscosity analysis recovers a planted shear rate exactly, and the SRD
viscosity formula gives the paper's eta_0 = 3.96 at its parameters.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I
from paper_2604_14307_gb300 import transport as T


def box(L=(6, 8, 5), precision=I.P32, seed=3, density=5.0):
    prm = I.Params(rule=I.SRD, thermostat=1, precision=precision, seed=seed)
    return I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [L], density, [[]], "solvent_only",
                          placement_seed=seed)


def ranks_brute(keys, ids):
    """rank of each particle: how many others are closer (ties: lower id)"""
    k = np.asarray(keys)
    return np.array([np.sum((k < k[j]) | ((k == k[j]) & (ids < ids[j]))) for j in range(len(k))])


@pytest.fixture(scope="module")
def lib():
    O.build()


@pytest.mark.parametrize("precision", [I.P32, I.P64])
@pytest.mark.parametrize("max_pairs", [0, 1, 7, 40, 10000])
def test_exchange_properties(lib, precision, max_pairs):
    system = box(precision=precision)
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st, compute_forces=False)
    x0, v0 = ost.x.copy(), ost.v.copy()
    y_a, y_b, w, vt = 0.5, 4.0, 1.0, 0.5
    dp, n = O.rnemd_exchange(osys, ost, y_a, y_b, w, vt, max_pairs)
    y = x0[:, 1]
    in_a = (y >= y_a) & (y < y_a + w)
    in_b = (y >= y_b) & (y < y_b + w)
    changed = np.where(ost.v[:, 0] != v0[:, 0])[0]
    assert np.array_equal(ost.x, x0) and np.array_equal(ost.v[:, 1:], v0[:, 1:])
    assert np.all(in_a[changed] | in_b[changed])
    assert n == min(max_pairs, in_a.sum(), in_b.sum())
    assert len(changed) <= 2 * n
    assert np.array_equal(np.sort(ost.v[:, 0]), np.sort(v0[:, 0]))
    assert np.sum(ost.v[:, 0]) == pytest.approx(np.sum(v0[:, 0]), abs=1e-12)
    assert np.sum(ost.v ** 2) == pytest.approx(np.sum(v0 ** 2), rel=1e-15)
    m = system.params.m_solvent
    assert dp == pytest.approx(m * (v0[in_a, 0].sum() - ost.v[in_a, 0].sum()), abs=1e-9)
    # selection and pairing, by brute-force ranks
    ids = np.arange(len(y))
    f = np.float32 if precision == I.P32 else np.float64
    ka = np.abs(v0[:, 0].astype(f) - f(vt))
    kb = np.abs(v0[:, 0].astype(f) + f(vt))
    ra = ranks_brute(ka[in_a], ids[in_a])
    rb = ranks_brute(kb[in_b], ids[in_b])
    sel_a = ids[in_a][ra < n]
    sel_b = ids[in_b][rb < n]
    # the selected particles now carry the partner's old v_x: rank k of A <-> rank k of B
    for k in range(n):
        ia = ids[in_a][ra == k][0]
        ib = ids[in_b][rb == k][0]
        assert ost.v[ia, 0] == v0[ib, 0] and ost.v[ib, 0] == v0[ia, 0]
    others = np.setdiff1d(ids, np.concatenate([sel_a, sel_b]))
    assert np.array_equal(ost.v[others], v0[others])


def test_exchange_with_an_empty_slab(lib):
    system = box()
    st = I.initial_state(system)
    st.x[:, 1] = np.where((st.x[:, 1] >= 3.0) & (st.x[:, 1] < 4.0), 2.5, st.x[:, 1])
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st, compute_forces=False)
    v0 = ost.v.copy()
    dp, n = O.rnemd_exchange(osys, ost, 0.0, 3.0, 1.0, 0.5, 100)
    assert n == 0 and dp == 0.0 and np.array_equal(ost.v, v0)


def test_equal_distances_are_ranked_by_id(lib):
    system = box()
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st, compute_forces=False)
    y = ost.x[:, 1]
    in_a = np.where((y >= 0.0) & (y < 1.0))[0]
    in_b = np.where((y >= 4.0) & (y < 5.0))[0]
    ost.v[in_a, 0] = 0.25            # every A particle at the same distance 0.25
    ost.v[in_b[::2], 0] = -0.5       # half of B exactly on target
    v0 = ost.v.copy()
    dp, n = O.rnemd_exchange(osys, ost, 0.0, 4.0, 1.0, 0.5, 5)
    assert n == 5
    chosen_a = np.where(ost.v[in_a, 0] != v0[in_a, 0])[0]
    assert np.array_equal(in_a[chosen_a], in_a[:5])           # lowest ids
    chosen_b = np.where(ost.v[in_b, 0] != v0[in_b, 0])[0]
    assert np.array_equal(in_b[chosen_b], in_b[::2][:5])
    assert dp == pytest.approx(5 * (0.25 + 0.5))


def test_step_rnemd_period(lib):
    system = box()
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    a = O.OracleState(osys, st)
    dp, n = O.step_rnemd(osys, a, 3, 0.0, 4.0, 1.0, 0.5, 3, period=2)
    assert a.step == 3 and n == 6                 # steps 0 and 2 exchange
    b = O.OracleState(osys, st)
    O.step(osys, b, 3)
    assert not np.array_equal(a.v, b.v)
    c = O.OracleState(osys, st)
    O.step_rnemd(osys, c, 3, 0.0, 4.0, 1.0, 0.5, 0)
    assert np.array_equal(c.v, b.v) and np.array_equal(c.x, b.x)   # no pairs: the plain step


def test_viscosity_analysis_recovers_a_planted_shear():
    Ly, n_bins = 40.0, 80
    y = T.bin_centres(n_bins, Ly)
    g = 0.0321
    # bidirectional profile: rises from slab A (y = 0) to slab B (y = 20), falls back
    u = np.where(y < 20.0, -0.321 + g * y, 0.321 - g * (y - 20.0))
    r = T.shear_rate(y, u, Ly, 0.0, 20.0, 1.0, margin=1.0)
    assert r["slope_ab"] == pytest.approx(g) and r["slope_ba"] == pytest.approx(-g)
    assert r["gamma_dot"] == pytest.approx(g)
    assert T.viscosity_rnemd(2 * 400.0 * 3.96 * g * 1000.0, 1000.0, 400.0, g) == pytest.approx(3.96)


def test_srd_viscosity_formula_gives_the_papers_eta0(golden):
    e = T.srd_viscosity(density=5.0, kT=1.0, m=1.0, dt=0.1, alpha_deg=130.0)
    assert e["total"] == pytest.approx(golden["eta0_solvent"]["value"], abs=0.005)
    assert e["collisional"] > e["kinetic"] > 0
