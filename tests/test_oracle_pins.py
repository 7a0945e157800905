"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself: exact
rational arithmetic, an independent rotation library (scipy), closed forms,
conservation laws the collision rules must obey (Sec. II.A), the rigid-body
identities of Eqs. 3-5 and 7, Eq. 1's WCA potential, and distributions the
method must produce (Eq. 6).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2604_14307_gb300 import inputs as I


def rot(q):
    """scipy rotation from a scalar-first quaternion."""
    q = np.asarray(q, dtype=np.float64).reshape(-1, 4)
    return Rotation.from_quat(q[:, [1, 2, 3, 0]])


def tiny_system(L=3, density=5.0, rule=I.SRD, thermostat=0, precision=I.P64, level=1,
                radius=0.9, site_mass=2.0, n_bodies=1, seed=5, naive=0):
    prm = I.Params(kT=1.0, dt=0.1, alpha_deg=130.0, rule=rule, thermostat=thermostat,
                   precision=precision, seed=seed, naive_transfer=naive)
    shapes = [I.sphere_shape(radius, level, site_mass)]
    rng = np.random.default_rng(seed)
    R = rng.random((n_bodies, 3)) * L
    q = I.random_quaternions(rng, n_bodies)
    s = I.build_system(prm, shapes, [(L, L, L)], density, [[0] * n_bodies], "tiny", R_q=[(R, q)])
    st = I.initial_state(s)
    return s, st


def run_collision(s, st):
    osys = O.OracleSystem(s)
    ost = O.OracleState(osys, st)
    O.stream(osys, ost)
    pre = dict(x=ost.x.copy(), v=ost.v.copy(), R=ost.R.copy(), q=ost.q.copy(),
               P=ost.P.copy(), Lm=ost.Lm.copy())
    tr = O.collide(osys, ost)
    return osys, ost, pre, tr


def members(osys, pre, tr, post_state):
    """Per-particle arrays over solvent then sites: cell, mass, v_pre, v_post."""
    m_sites = np.concatenate([osys.m[osys.site_off[s]:osys.site_off[s + 1]]
                              for s in osys.body_shape[:osys.n_bodies]]) if osys.n_bodies else np.zeros(0)
    cell = np.concatenate([tr["cell_solvent"][:osys.n_solvent], tr["cell_site"][:osys.n_sites]])
    m = np.concatenate([np.full(osys.n_solvent, osys.params["m_solvent"]), m_sites])
    v0 = np.concatenate([pre["v"], tr["site_v"][:osys.n_sites]])
    v1 = np.concatenate([post_state.v, tr["site_vpost"][:osys.n_sites]])
    return cell, m, v0, v1


# ---------------------------------------------------------------- binning ---
def exact_cell(x, S, L):
    """cell = floor(x - S 2^-20) mod L in exact rational arithmetic."""
    return math.floor(Fraction(x) - Fraction(int(S), 2**20)) % L


def test_binning_rule_matches_exact_rational():
    rng = np.random.default_rng(0)
    L = 7
    xs = list(rng.random(3000) * L) + list((rng.random(2000) * L).astype(np.float32).astype(float))
    xs += [0.0, L - 2**-40, 1.0, 3.5, 2.0 + 2**-21, np.nextafter(L, 0)]
    Ss = rng.integers(-(1 << 19), 1 << 19, size=len(xs))
    Ss[:8] = [-(1 << 19), (1 << 19) - 1, 0, 1, -1, 524287, -524288, 0]
    for x, S in zip(xs, Ss):
        assert O.cell_axis(x, int(S), L) == exact_cell(x, S, L), (x, S)
    # particles exactly on a shifted boundary k + s belong to cell k
    for k in range(L):
        for S in (-(1 << 19), -12345, 0, 777, (1 << 19) - 1):
            x = k + S / 2**20
            if 0 <= x < L:
                assert O.cell_axis(x, S, L) == k % L


def test_cell_sums_and_canonical_order_brute_force():
    s, st = tiny_system(L=3, density=4.0)
    osys, ost, pre, tr = run_collision(s, st)
    # site positions: R + Q b with an independent rotation, wrapped into [0, L)
    d = rot(pre["q"][0]).apply(osys.b)
    r = pre["R"][0] + d
    r = r - 3 * np.floor(r / 3)
    assert np.allclose(tr["site_r"], r, atol=1e-13)
    S = tr["shift"][0]
    pos = np.concatenate([pre["x"], tr["site_r"]])
    cell = np.array([exact_cell(p[0], S[0], 3) + 3 * (exact_cell(p[1], S[1], 3) + 3 * exact_cell(p[2], S[2], 3))
                     for p in pos])
    cc, m, v0, _ = members(osys, pre, tr, ost)
    assert np.array_equal(cc, cell)
    for c in range(27):
        sel = cell == c
        assert tr["sums"][0, c] == sel.sum()
        assert np.isclose(tr["sums"][1, c], m[sel].sum(), rtol=1e-14, atol=1e-14)
        for a in range(3):
            assert np.isclose(tr["sums"][2 + a, c], (m[sel] * v0[sel, a]).sum(), rtol=1e-12, atol=1e-13)
        assert np.isclose(tr["sums"][5, c], (m[sel] * (v0[sel] ** 2).sum(1)).sum(), rtol=1e-12, atol=1e-13)
        # canonical order: solvent before sites, ascending id inside each group
        ids = tr["order"][tr["cell_start"][c]:tr["cell_start"][c + 1]]
        assert list(ids) == list(np.flatnonzero(sel))


def rne(x):
    """round-to-nearest-even of exactly scaled float values to int64"""
    return np.rint(x).astype(np.int64)


def unpack48(w):
    """count|momentum word -> (count, signed low 48 bits)"""
    w = np.asarray(w, dtype=np.int64)
    lo = w & np.int64(2**48 - 1)
    lo = np.where(lo >= 2**47, lo - 2**48, lo)
    cnt = ((w - lo).view(np.uint64) >> np.uint64(48)).astype(np.int64)
    return cnt, lo


def record_numpy(cell, m, v, is_site, C, rule=I.SRD, xi=None):
    """The P32 cell words recomputed with numpy: float32 products, then the
    float values scaled exactly in float64 and rounded to integers:
    w0 = p_x + 2^48 [solvent], w1 = p_y + 2^48 [site], w2 = p_z with
    p = round(fl32(m v) 2^32); SRD w3 = round(e 2^28); AT w3..w5 =
    round(fl32(m xi) 2^32)."""
    mf = m.astype(np.float32)
    vf = v.astype(np.float32)
    p = mf[:, None] * vf                                   # float32 products
    e = (p[:, 0] * vf[:, 0] + p[:, 1] * vf[:, 1]) + p[:, 2] * vf[:, 2]
    s32 = 2.0**32
    w = np.zeros((6, len(m)), dtype=np.int64)
    w[0] = rne(p[:, 0].astype(np.float64) * s32) + np.where(is_site, 0, 2**48)
    w[1] = rne(p[:, 1].astype(np.float64) * s32) + np.where(is_site, 2**48, 0)
    w[2] = rne(p[:, 2].astype(np.float64) * s32)
    if rule == I.SRD:
        w[3] = rne(e.astype(np.float64) * 2.0**28)
    else:
        q = mf[:, None] * xi.astype(np.float32)
        for k in range(3):
            w[3 + k] = rne(q[:, k].astype(np.float64) * s32)
    out = np.zeros((6, C), dtype=np.int64)
    for k in range(6):
        np.add.at(out[k], cell, w[k])
    return out


def test_fixed_point_record_is_an_exact_integer_sum():
    s, st = tiny_system(L=4, density=6.0, precision=I.P32, site_mass=5.0, thermostat=1)
    osys, ost, pre, tr = run_collision(s, st)
    cell, m, v0, _ = members(osys, pre, tr, ost)
    is_site = np.arange(len(m)) >= osys.n_solvent
    ref = record_numpy(cell, m, v0, is_site, 64)
    assert np.array_equal(tr["fixed"], ref)
    # decoding recovers the counts, the masses, the momenta and the energy
    ns, px = unpack48(tr["fixed"][0])
    nb, py = unpack48(tr["fixed"][1])
    pz = tr["fixed"][2]
    assert np.array_equal(ns + nb, tr["sums"][0].astype(np.int64))
    assert nb.sum() == osys.n_sites and ns.sum() == osys.n_solvent
    M = ns * 1.0 + nb * 5.0
    assert np.allclose(M, tr["sums"][1], rtol=0, atol=1e-12)
    # the momentum words are the exact sums of the float32 momenta fl32(m v):
    # within the float32 rounding of each m v of the FP64 sums, and exactly
    # the float64 sum of the float32 products (rounded to 2^-32) for m = 1
    mf = m.astype(np.float32)
    pf = (mf[:, None] * v0.astype(np.float32)).astype(np.float64)
    for k, h in enumerate((px, py, pz)):
        exact = np.bincount(cell, weights=pf[:, k], minlength=64)
        assert np.allclose(h * 2.0**-32, exact, rtol=0, atol=2.0**-32 * 40)
        assert np.allclose(h * 2.0**-32, tr["sums"][2 + k], rtol=0, atol=1e-6)
    assert np.allclose(tr["fixed"][3] * 2.0**-28, tr["sums"][5], rtol=1e-6, atol=1e-6)


def test_fixed_point_record_of_the_at_rule():
    """AT form: no energy; noise sums m xi at 2^-32 in words 3-5."""
    s, st = tiny_system(L=4, density=6.0, precision=I.P32, site_mass=5.0, rule=I.AT)
    osys, ost, pre, tr = run_collision(s, st)
    cell, m, v0, _ = members(osys, pre, tr, ost)
    ns = osys.n_solvent
    ids = np.concatenate([np.arange(ns), ns + np.arange(osys.n_sites)])
    xi = O.normals(osys, 0, st.step, ids, O.TAG_AT) * np.sqrt(1.0 / m)[:, None]
    ref = record_numpy(cell, m, v0, ids >= ns, 64, rule=I.AT, xi=xi)
    assert np.array_equal(tr["fixed"], ref)
    _, px = unpack48(tr["fixed"][0])
    _, py = unpack48(tr["fixed"][1])
    assert np.allclose(px * 2.0**-32, tr["sums"][2], atol=1e-6)
    assert np.allclose(py * 2.0**-32, tr["sums"][3], atol=1e-6)
    for k in range(3):
        mx = np.bincount(cell, weights=m * xi[:, k], minlength=64)
        assert np.allclose(tr["fixed"][3 + k] * 2.0**-32, mx, atol=1e-6)


def test_fixed_point_words_are_exact_below_one_ulp():
    """The 2^-32 momentum quantum against float32: every float32 |m v| >= 2^-9
    is a multiple of 2^-32, so the word holds it exactly; smaller values round
    by at most 2^-33 (the per-cell momentum sums are exact sums of the stored
    float32 momenta, Sec. II.A)."""
    rng = np.random.default_rng(5)
    f = np.concatenate([rng.standard_normal(20000), rng.standard_normal(2000) * 1e-3,
                        [2.0**-9, -2.0**-9, 3.0 * 2.0**-10, 1.5 * 2.0**-32, 2.5 * 2.0**-32, 30000.0]])
    f = f.astype(np.float32).astype(np.float64)
    q = rne(f * 2.0**32)
    big = np.abs(f) >= 2.0**-9
    assert np.array_equal(q[big] * 2.0**-32, f[big])
    assert np.all(np.abs(q * 2.0**-32 - f) <= 2.0**-33)
    # ties go to even: 1.5 -> 2, 2.5 -> 2 (in units of 2^-32)
    assert list(q[-3:-1]) == [2, 2]


# --------------------------------------------------------------- collision ---
@pytest.mark.parametrize("rule,thermostat", [(I.SRD, 0), (I.SRD, 1), (I.AT, 0)])
def test_collision_conserves_cell_mass_and_momentum(rule, thermostat):
    s, st = tiny_system(L=4, density=5.0, rule=rule, thermostat=thermostat)
    osys, ost, pre, tr = run_collision(s, st)
    cell, m, v0, v1 = members(osys, pre, tr, ost)
    for c in range(64):
        sel = cell == c
        p0 = (m[sel, None] * v0[sel]).sum(0)
        p1 = (m[sel, None] * v1[sel]).sum(0)
        assert np.allclose(p0, p1, atol=1e-12)
        if rule == I.SRD and not thermostat:
            e0 = 0.5 * (m[sel] * (v0[sel] ** 2).sum(1)).sum()
            e1 = 0.5 * (m[sel] * (v1[sel] ** 2).sum(1)).sum()
            assert abs(e0 - e1) < 1e-12 * max(1.0, e0)


def test_srd_rotates_relative_velocity_by_alpha():
    s, st = tiny_system(L=4, density=5.0)
    osys, ost, pre, tr = run_collision(s, st)
    cell, m, v0, v1 = members(osys, pre, tr, ost)
    alpha = math.radians(130.0)
    n_checked = 0
    for i in range(len(m)):
        c = cell[i]
        if tr["sums"][0, c] < 2:
            assert np.array_equal(v0[i], v1[i])
            continue
        u, n = tr["cell_u"][c], tr["cell_axis"][c]
        assert abs(np.linalg.norm(n) - 1) < 1e-14
        w0, w1 = v0[i] - u, v1[i] - u
        assert abs(n @ w0 - n @ w1) < 1e-12
        p0, p1 = w0 - (n @ w0) * n, w1 - (n @ w1) * n
        if np.linalg.norm(p0) < 1e-6:
            continue
        ang = math.atan2(n @ np.cross(p0, p1), p0 @ p1)
        assert abs(ang - alpha) < 1e-9
        assert abs(np.linalg.norm(p0) - np.linalg.norm(p1)) < 1e-12
        n_checked += 1
    assert n_checked > 100


def test_p32_thermostat_energy_is_the_relative_energy_of_the_stored_state():
    """In the P32 form kappa^2 = E'/E_rel with E_rel from the cell's words.
    Pinned against the plain definition E_rel = 1/2 sum m |v - u|^2 of the
    stored float32 velocities (FP64): the difference can only come from the
    float32 products fl32(fl32(m v_a) v_a) summed in float32 per particle
    (at most 4 roundings of 2^-24 e_i each), the 2^-29 rounding of each energy
    term and the float32 rounding of m v in the momentum sums."""
    s, st = tiny_system(L=4, density=6.0, precision=I.P32, site_mass=5.0, thermostat=1)
    osys, ost, pre, tr = run_collision(s, st)
    cell, m, v0, v1 = members(osys, pre, tr, ost)
    vf = v0.astype(np.float32).astype(np.float64)
    mf = m.astype(np.float32).astype(np.float64)
    e = (mf[:, None] * vf * vf).sum(1)
    n_checked = 0
    for c in range(64):
        sel = cell == c
        if sel.sum() < 2:
            continue
        M = mf[sel].sum()
        u = (mf[sel, None] * vf[sel]).sum(0) / M
        E = 0.5 * (mf[sel, None] * (vf[sel] - u) ** 2).sum()
        S1 = np.abs(mf[sel, None] * vf[sel]).sum(0)
        bound = 0.5 * ((4 * 2.0**-24 * e[sel] + 2.0**-29).sum() + 2 * 2.0**-24 * (S1 @ S1) / M)
        Ep = O.thermostat_energy(osys, 0, 0, c, int(sel.sum()))
        E32 = Ep / tr["cell_kappa"][c] ** 2
        assert abs(E32 - E) <= bound * (1 + 1e-9) + 1e-15 * Ep, (c, E32, E, bound)
        # and the collision realises it: post-collision relative energy = kappa^2 E_rel,
        # up to the float32 rounding of the stored new velocities
        Epost = 0.5 * (m[sel, None] * (v1[sel] - tr["cell_u"][c]) ** 2).sum()
        assert abs(Epost - Ep) < 2.0**-20 * max(Ep, 1e-3)
        n_checked += 1
    assert n_checked > 40


@pytest.mark.parametrize("sampler", [1, 2])
def test_thermostat_energy_follows_eq6_gamma(sampler):
    """Huang cell thermostat: the post-collision relative KE of a cell with Nc
    particles is Gamma(3(Nc-1)/2, kT) distributed (Eq. 6, n = 3(Nc-1)), with E'
    drawn as a sum of exponentials (1) or by Marsaglia-Tsang rejection (2)."""
    prm = I.Params(rule=I.SRD, thermostat=sampler, seed=11)
    s = I.build_system(prm, [I.sphere_shape(1.0, 0, 1.0)], [(14, 14, 14)], 4.0, [[]], "bulk")
    st = I.initial_state(s)
    osys, ost, pre, tr = run_collision(s, st)
    cell = tr["cell_solvent"]
    u = tr["cell_u"]
    w = ost.v - u[cell]
    E = np.zeros(osys.n_cells)
    np.add.at(E, cell, 0.5 * (w ** 2).sum(1))
    n = tr["sums"][0].astype(int)
    sel = n >= 2
    pit = stats.gamma.cdf(E[sel], a=1.5 * (n[sel] - 1), scale=1.0)
    assert stats.kstest(pit, "uniform").pvalue > 1e-3
    # velocities are rotated and scaled about the preserved cell velocity
    kap = tr["cell_kappa"][sel]
    assert np.all(kap > 0) and abs(np.median(kap) - 1) < 0.2


@pytest.mark.parametrize("nc", [2, 3, 6, 11, 30])
def test_marsaglia_tsang_draws_follow_eq6(nc):
    """orc_thermostat_energy with the rejection sampler: 4000 cells of Nc
    particles, E'/kT against Gamma(3(Nc-1)/2) (Eq. 6) by KS, mean and variance
    against n kT/2 and n (kT)^2/2; kT = 1.7 scales the draw."""
    prm = I.Params(rule=I.SRD, thermostat=2, seed=21, kT=1.7)
    s = I.build_system(prm, [I.sphere_shape(1.0, 0, 1.0)], [(20, 20, 10)], 1.0, [[]], "bulk")
    osys = O.OracleSystem(s)
    E = np.array([O.thermostat_energy(osys, 0, 3, c, nc) for c in range(4000)]) / 1.7
    a = 1.5 * (nc - 1)
    assert stats.kstest(E, stats.gamma(a).cdf).pvalue > 1e-3
    assert abs(E.mean() - a) < 4 * math.sqrt(a / len(E))
    assert abs(E.var() / a - 1) < 0.15
    # not the exponential-sum draws (independent streams): the samplers differ
    o1 = O.OracleSystem(s, thermostat=1)
    E1 = np.array([O.thermostat_energy(o1, 0, 3, c, nc) for c in range(50)]) / 1.7
    assert not np.allclose(E1, E[:50])


def test_at_rule_momentum_and_relative_variance():
    prm = I.Params(rule=I.AT, seed=13)
    s = I.build_system(prm, [I.sphere_shape(1.0, 0, 1.0)], [(14, 14, 14)], 5.0, [[]], "bulk")
    st = I.initial_state(s)
    osys, ost, pre, tr = run_collision(s, st)
    cell = tr["cell_solvent"]
    n = tr["sums"][0]
    w = ost.v - tr["cell_u"][cell]
    # E[sum_i m |xi_i - xibar|^2] = 3 kT (Nc - 1) in every cell
    tot = (w ** 2).sum()
    expect = 3.0 * (n[n >= 1] - 1).sum()
    assert abs(tot / expect - 1) < 4 * math.sqrt(2.0 / (3 * (n - 1).clip(0).sum()))
    p0 = np.zeros((osys.n_cells, 3))
    p1 = np.zeros((osys.n_cells, 3))
    np.add.at(p0, cell, pre["v"])
    np.add.at(p1, cell, ost.v)
    assert np.allclose(p0, p1, atol=1e-11)


# ------------------------------------------------------- rigid-body coupling ---
def inertia_space(b, m, q):
    d = rot(q).apply(b)
    r2 = (d * d).sum(1)
    return (m[:, None, None] * (r2[:, None, None] * np.eye(3) - d[:, :, None] * d[:, None, :])).sum(0), d


@pytest.mark.parametrize("naive", [0, 1])
def test_thermalisation_keeps_P_and_L(naive):
    """Eq. 7 changes the site velocities but not P (Eq. 3) or L (Eq. 4); the
    naive scheme feeds the rigid velocities of Eq. 5 into the collision."""
    s, st = tiny_system(L=8, density=2.0, level=2, radius=2.0, site_mass=5.0, naive=naive)
    osys, ost, pre, tr = run_collision(s, st)
    m = osys.m
    I_s, d = inertia_space(osys.b, m, pre["q"][0])
    v = tr["site_v"]
    assert np.allclose((m[:, None] * v).sum(0), pre["P"][0], rtol=0, atol=1e-11)
    assert np.allclose(np.cross(d, m[:, None] * v).sum(0), pre["Lm"][0], rtol=0, atol=1e-10)
    V = pre["P"][0] / m.sum()
    om = np.linalg.solve(I_s, pre["Lm"][0])
    rigid = V + np.cross(om, d)
    if naive:
        assert np.allclose(v, rigid, atol=1e-13)
    else:
        assert not np.allclose(v, rigid, atol=1e-3)


def test_thermalised_internal_energy_is_gamma_3N_minus_6():
    """The non-rigid part of the thermalised site velocities carries the 3N-6
    internal modes at temperature T: its kinetic energy is Gamma((3N-6)/2, kT)."""
    s, st = tiny_system(L=8, density=0.5, level=1, radius=2.0, site_mass=5.0)
    osys = O.OracleSystem(s)
    ost = O.OracleState(osys, st)
    m = osys.m
    N = len(m)
    E = []
    for _ in range(300):
        O.stream(osys, ost)
        q, P, Lm = ost.q[0].copy(), ost.P[0].copy(), ost.Lm[0].copy()
        tr = O.collide(osys, ost)
        I_s, d = inertia_space(osys.b, m, q)
        rigid = P / m.sum() + np.cross(np.linalg.solve(I_s, Lm), d)
        E.append(0.5 * (m[:, None] * (tr["site_v"] - rigid) ** 2).sum())
        ost.step += 1
    E = np.array(E)
    assert stats.kstest(E, stats.gamma(a=(3 * N - 6) / 2.0, scale=1.0).cdf).pvalue > 1e-3


def test_transfer_conserves_total_momentum():
    s, st = tiny_system(L=8, density=5.0, level=2, radius=2.0, site_mass=5.0, n_bodies=2)
    osys, ost, pre, tr = run_collision(s, st)
    p0 = pre["v"].sum(0) + pre["P"].sum(0)
    p1 = ost.v.sum(0) + ost.P.sum(0)
    assert np.allclose(p0, p1, atol=1e-10)
    # the body receives exactly what its sites lost
    m = osys.m
    for b in range(2):
        g = slice(osys.site_base[b], osys.site_base[b + 1])
        dp = (m[:, None] * (tr["site_vpost"][g] - tr["site_v"][g])).sum(0)
        assert np.allclose(dp, ost.P[b] - pre["P"][b], atol=1e-11)


def test_sites_reset_to_rigid_motion_eq5():
    s, st = tiny_system(L=8, density=5.0, level=2, radius=2.0, site_mass=5.0)
    osys = O.OracleSystem(s)
    ost = O.OracleState(osys, st)
    O.step(osys, ost, 3)
    v = O.rigid_site_velocities(osys, ost)
    m = osys.m
    I_s, d = inertia_space(osys.b, m, ost.q[0])
    om = np.linalg.solve(I_s, ost.Lm[0])
    assert np.allclose(v, ost.P[0] / m.sum() + np.cross(om, d), atol=1e-13)
    assert np.allclose((m[:, None] * v).sum(0), ost.P[0], atol=1e-11)
    assert np.allclose(np.cross(d, m[:, None] * v).sum(0), ost.Lm[0], atol=1e-10)


# ---------------------------------------------------------------- WCA (Eq. 1) ---
def test_wca_eq1_cutoff_continuity_and_force():
    d = 6.0
    delta = d - 1.0
    rc = delta + 2 ** (1 / 6)
    u, f = O.wca(rc, d)
    assert abs(u) < 1e-12 and abs(f) < 1e-12
    u, f = O.wca(rc - 1e-7, d)
    assert abs(u) < 1e-9 and abs(f) < 1e-5
    assert O.wca(rc + 1e-9, d) == (0.0, 0.0)
    for r in np.linspace(delta + 0.9, rc - 1e-3, 25):
        u, f = O.wca(r, d)
        h = 1e-6
        dudr = (O.wca(r + h, d)[0] - O.wca(r - h, d)[0]) / (2 * h)
        assert abs(f + dudr) < 1e-5 * max(1, abs(f))
        s6 = (1 / (r - delta)) ** 6
        assert abs(u - (4 * (s6 * s6 - s6) + 1)) < 1e-12 * max(1, u)


def test_body_forces_newton3_torques_and_gradient():
    prm = I.Params(seed=3)
    sh = I.dumbbell_shape(3.0, 3.0, 1, 5.0)
    rng = np.random.default_rng(4)
    # search a configuration inside the repulsive shell (5.2 < r < 6.12) of at
    # least two centre pairs, with no pair inside the core (r <= Delta = 5)
    while True:
        R = 20.0 + rng.random((3, 3)) * 9.0
        q = I.random_quaternions(rng, 3)
        c = np.concatenate([R[i] + rot(q[i]).apply(sh.centres) for i in range(3)])
        owner = np.repeat(np.arange(3), len(sh.centres))
        dd = np.linalg.norm(c[:, None] - c[None], axis=-1)
        other = owner[:, None] != owner[None, :]
        if dd[other].min() > 5.2 and (dd[other] < 6.1).sum() >= 4:
            break
    s = I.build_system(prm, [sh], [(48, 48, 48)], 0.0, [[0, 0, 0]], "dumb", R_q=[(R, q)])
    st = I.initial_state(s)
    osys = O.OracleSystem(s)
    ost = O.OracleState(osys, st)
    E0 = O.forces(osys, ost)
    assert E0 > 0
    F, T = ost.F.copy(), ost.T.copy()
    assert np.allclose(F.sum(0), 0, atol=1e-9)
    assert np.allclose((np.cross(ost.R, F) + T).sum(0), 0, atol=1e-8)
    h = 1e-6
    for i in range(3):
        for a in range(3):
            ost.R[i, a] += h
            ep = O.forces(osys, ost)
            ost.R[i, a] -= 2 * h
            em = O.forces(osys, ost)
            ost.R[i, a] += h
            assert abs(-(ep - em) / (2 * h) - F[i, a]) < 1e-4 * max(1, abs(F[i, a]))
        # torque = -dE/dtheta for a small space-frame rotation about each axis
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            q0 = ost.q[i].copy()
            for sgn in (1, -1):
                r = Rotation.from_rotvec(sgn * e) * rot(q0)
                qq = r.as_quat()[0] if r.as_quat().ndim == 2 else r.as_quat()
                ost.q[i] = [qq[3], qq[0], qq[1], qq[2]]
                if sgn == 1:
                    ep = O.forces(osys, ost)
                else:
                    em = O.forces(osys, ost)
            ost.q[i] = q0
            assert abs(-(ep - em) / (2 * h) - T[i, a]) < 1e-4 * max(1, abs(T[i, a]))


# ------------------------------------------------------- rigid integrator ---
def free_body_system(shape, q0, Lm, dt=0.1):
    prm = I.Params(dt=dt, seed=2)
    s = I.build_system(prm, [shape], [(40, 40, 40)], 0.0, [[0]], "free",
                       R_q=[(np.array([[20.0, 20.0, 20.0]]), np.array([q0]))])
    st = I.initial_state(s)
    st.P[:] = 0.0
    st.Lm[0] = Lm
    osys = O.OracleSystem(s)
    return osys, O.OracleState(osys, st)


def test_free_sphere_rotates_uniformly():
    """Isotropic inertia: L and omega = L/I stay constant and the orientation
    follows the exact rotation exp(omega t); the splitting error of the
    3-2-1-2-3 rotor is second order in dt."""
    sh = I.sphere_shape(2.0, 2, 5.0)
    I0 = I.shape_inertia_diag(sh)[0]
    q0 = I.random_quaternions(np.random.default_rng(1), 1)[0]
    Lm = np.array([30.0, -110.0, 70.0])
    errs = []
    for dt in (0.1, 0.05):
        osys, ost = free_body_system(sh, q0, Lm, dt=dt)
        n = int(round(20.0 / dt))
        for _ in range(n):
            O.stream(osys, ost)
        expect = Rotation.from_rotvec(Lm / I0 * 20.0) * rot(q0)
        errs.append((expect.inv() * rot(ost.q[0])).magnitude()[0])
        assert np.allclose(ost.Lm[0], Lm, rtol=1e-12, atol=1e-10)
    assert errs[0] < 1e-4
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_symmetric_top_precesses_about_L():
    """Free symmetric top (I1 = I2): the symmetry axis precesses about L at the
    rate |L|/I1 (Euler); NO_SQUISH reproduces it to O(dt^2)."""
    ph = 2 * np.pi * np.arange(8) / 8
    ring = np.stack([3 * np.cos(ph), 3 * np.sin(ph), np.zeros(8)], 1)
    b = np.concatenate([ring + [0, 0, z] for z in (-4.0, 0.0, 4.0)])
    sh = I.Shape(b=b, m=np.full(len(b), 5.0), centres=np.zeros((1, 3)), wca_d=6.0)
    Id = I.shape_inertia_diag(sh)
    assert abs(Id[0] - Id[1]) < 1e-9 * Id[0] and abs(Id[2] - Id[0]) > 0.1 * Id[0]
    q0 = I.random_quaternions(np.random.default_rng(2), 1)[0]
    Lm = np.array([40.0, 10.0, -25.0])
    dt = 0.01
    osys, ost = free_body_system(sh, q0, Lm, dt=dt)
    n = 2000
    E0 = O.body_energies(osys, ost)[1][0]
    for _ in range(n):
        O.stream(osys, ost)
    Lh = Lm / np.linalg.norm(Lm)
    e3_0 = rot(q0).apply([0, 0, 1])[0]
    rate = np.linalg.norm(Lm) / Id[0]
    e3_expect = Rotation.from_rotvec(Lh * rate * dt * n).apply(e3_0)
    e3_got = rot(ost.q[0]).apply([0, 0, 1])[0]
    assert np.linalg.norm(e3_got - e3_expect) < 2e-3
    assert np.allclose(ost.Lm[0], Lm, atol=1e-10)
    E1 = O.body_energies(osys, ost)[1][0]
    assert abs(E1 - E0) < 1e-3 * E0


def test_asymmetric_rotor_conserves_L_and_energy():
    sh = I.spherocylinder_shape(6.0, 24.0, 1.0, 5.0, cap_level=1)
    sh2 = I.Shape(b=sh.b * np.array([1.0, 1.3, 1.0]), m=sh.m, centres=sh.centres, wca_d=6.0)
    q0 = I.random_quaternions(np.random.default_rng(5), 1)[0]
    Lm = np.array([300.0, -120.0, 80.0])
    osys, ost = free_body_system(sh2, q0, Lm)
    E0 = O.body_energies(osys, ost)[1][0]
    Es = []
    for _ in range(500):
        O.stream(osys, ost)
        Es.append(O.body_energies(osys, ost)[1][0])
    assert np.allclose(ost.Lm[0], Lm, rtol=1e-12, atol=1e-10)
    Es = np.array(Es)
    assert np.max(np.abs(Es - E0)) < 5e-3 * E0          # bounded, symplectic
    assert abs(Es[-100:].mean() - Es[:100].mean()) < 2e-3 * E0   # no drift


# --------------------------------------------------------------- templates ---
def test_icosphere_counts_radius_density_and_isotropy(golden):
    for k, n in enumerate([12, 42, 162, 642]):
        v = I.icosphere_vertices(k)
        assert len(v) == n == 10 * 4**k + 2
        assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-14)
        assert len(np.unique(np.round(v, 12), axis=0)) == n
    sh = I.sphere_shape(3.0, 2, 5.0)
    assert sh.n_sites == golden["n_sites_two_subdivisions"]["value"]
    dens = sh.n_sites / (4 * math.pi * 3.0**2)
    assert abs(dens - golden["surface_density_162_sites_d6"]["value"]) < 0.005
    Ib = (sh.m[:, None, None] * ((sh.b**2).sum(1)[:, None, None] * np.eye(3)
                                 - sh.b[:, :, None] * sh.b[:, None, :])).sum(0)
    iso = 2.0 / 3.0 * (sh.m * (sh.b**2).sum(1)).sum()
    assert np.allclose(Ib, iso * np.eye(3), rtol=0, atol=1e-10 * iso)


@pytest.mark.parametrize("maker", [
    lambda: I.dumbbell_shape(3.0, 3.0, 3, 5.0),
    lambda: I.spherocylinder_shape(6.0, 24.0, 0.5, 5.0),
    lambda: I.sphere_shape(4.0, 3, 10.0)])
def test_templates_are_principal_and_centred(maker):
    sh = maker()
    assert np.allclose((sh.m[:, None] * sh.b).sum(0), 0, atol=1e-10)
    Ib = (sh.m[:, None, None] * ((sh.b**2).sum(1)[:, None, None] * np.eye(3)
                                 - sh.b[:, :, None] * sh.b[:, None, :])).sum(0)
    off = Ib - np.diag(np.diag(Ib))
    assert np.abs(off).max() < 1e-9 * np.abs(Ib).max()


def test_exported_axis_and_thermostat_match_the_collision():
    """orc_srd_axis / orc_thermostat_energy are the pieces orc_collide uses:
    the axis it traces, and the kappa = sqrt(E'/E_rel) it traces with E_rel from
    the P32 fixed-point words (Sec. II.A, Eq. 6)."""
    s = I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, I.SRD, 1, I.P32, seed=3, name="small")
    osys = O.OracleSystem(s)
    ost = O.OracleState(osys, I.initial_state(s))
    O.stream(osys, ost)
    tr = O.collide(osys, ost)
    n = tr["sums"][0]
    M = tr["sums"][1]
    sel = np.where(n >= 2)[0][:300]
    for c in sel:
        assert np.array_equal(O.srd_axis(osys, 0, 0, int(c)), tr["cell_axis"][c])
        fx = tr["fixed"][:, c]
        S1 = np.array([unpack48(fx[0])[1], unpack48(fx[1])[1], fx[2]], dtype=np.float64) * 2.0**-32
        erel = 0.5 * (float(fx[3]) * 2.0**-28 - float(S1 @ S1) / M[c])
        kappa = np.sqrt(O.thermostat_energy(osys, 0, 0, int(c), int(n[c])) / erel)
        assert abs(kappa - tr["cell_kappa"][c]) <= 1e-12 * kappa
