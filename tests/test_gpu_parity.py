"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (stated once, used everywhere):
  * integer work - cell indices, counts, masses in the fixed-point count|mass
    word, streamed positions - must be bit-exact;
  * floating point: |gpu - oracle| <= tol * (|oracle| + scale) with
    tol = 1e-12 for the FP64 form and 1e-5 for the FP32 form, scale the
    thermal value of the quantity (sqrt(kT/m) for velocities, sqrt(M kT) for
    body momenta, sqrt(I kT) for angular momenta).
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {I.P64: 1e-12, I.P32: 1e-5}


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14307_gb300 import binding, build_lib
    build_lib.build()
    return binding


def close(a, b, tol, scale):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    err = np.abs(a - b) / (np.abs(b) + scale)
    return err.max() if err.size else 0.0


def body_scales(system):
    Ms = np.array([system.shapes[s].m.sum() for s in system.body_shape_array()])
    Is = np.array([I.shape_inertia_diag(system.shapes[s]).max() for s in system.body_shape_array()])
    return np.sqrt(Ms)[:, None], np.sqrt(Is)[:, None]


def site_mask_cells(osys, tr):
    """cells that contain at least one site"""
    m = np.zeros(osys.n_cells, dtype=bool)
    if osys.n_sites:
        for r in range(len(osys.L)):
            b0, b1 = osys.body_off[r], osys.body_off[r + 1]
            g0, g1 = osys.site_base[b0], osys.site_base[b1]
            m[osys.cell_base[r] + tr["cell_site"][g0:g1]] = True
    return m


def unpack48(w):
    """count|momentum word -> (count, signed low 48 bits)"""
    w = np.asarray(w, dtype=np.int64)
    lo = w & np.int64(2**48 - 1)
    lo = np.where(lo >= 2**47, lo - 2**48, lo)
    return ((w - lo).view(np.uint64) >> np.uint64(48)).astype(np.int64), lo


def decode_record(w, rule):
    """P32 cell words -> physical sums (see include/mpcd.h)"""
    out = {}
    out["p0"] = unpack48(w[0])[1] * 2.0**-32
    out["p1"] = unpack48(w[1])[1] * 2.0**-32
    out["p2"] = w[2] * 2.0**-32
    if rule == I.SRD:
        out["e"] = w[3] * 2.0**-28
    else:
        for k in range(3):
            out[f"q{k}"] = w[3 + k] * 2.0**-32
    return out


def one_step(B, system, check_sums=True):
    prec = system.params.precision
    tol = TOL[prec]
    st = I.initial_state(system)
    sim = B.Simulation(system)
    sim.set_debug(True)
    sim.set_state(st)
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)

    # a1 + a9: streaming is bit-exact; bodies agree to rounding
    sim.stream()
    O.stream(osys, ost)
    g = sim.get_state()
    assert np.array_equal(g.x, ost.x)
    sM, sI = body_scales(system)
    if osys.n_bodies:
        assert close(g.R, ost.R, tol, 1.0) < 1e-14
        assert close(g.q, ost.q, tol, 1.0) < 1e-13
        assert close(g.P, ost.P, tol, sM) < tol
        assert close(g.Lm, ost.Lm, tol, sI) < tol

    # a2-a8
    sim.couple(B.MPCD_PRE)
    sim.collide()
    d = sim.debug_cells()
    sim.couple(B.MPCD_POST)
    tr = O.collide(osys, ost)
    ost.step += 1

    assert np.array_equal(d["shift"], tr["shift"])
    if osys.n_sites:
        assert np.array_equal(d["site_cell"], tr["cell_site"])
        ms = np.concatenate([osys.m[osys.site_off[s]:osys.site_off[s + 1]]
                             for s in osys.body_shape[:osys.n_bodies]])
        assert close(d["site_v"], tr["site_v"], tol, np.sqrt(1.0 / ms)[:, None]) < tol
    n = tr["sums"][0]
    if check_sums:
        if prec == I.P32:
            w, fx = d["sums"], tr["fixed"]
            sm = site_mask_cells(osys, tr)
            # counts (high 16 bits of w0, w1): integer, bit-exact everywhere
            assert np.array_equal(unpack48(w[0])[0], unpack48(fx[0])[0])
            assert np.array_equal(unpack48(w[1])[0], unpack48(fx[1])[0])
            if system.params.rule == I.SRD:
                # only solvent (identical float inputs): every word bit-exact
                assert np.array_equal(w[:, ~sm], fx[:4, ~sm])
            else:
                assert np.array_equal(w[:3, ~sm], fx[:3, ~sm])
            # with sites: decoded values within the tolerance
            gd, od = decode_record(w, system.params.rule), decode_record(fx, system.params.rule)
            M = tr["sums"][1]
            for k in gd:
                assert np.all(np.abs(gd[k] - od[k]) <= tol * (4.0 * M + 1.0)), k
        else:
            w = d["sums"]
            assert np.array_equal(w[0], n)
            assert close(w[1], tr["sums"][1], tol, 1.0) < tol
            for k in range(2, 5):
                assert close(w[k], tr["sums"][k], tol, np.sqrt(np.maximum(tr["sums"][1], 1.0))) < tol
    # cell parameters of every cell that collides
    sel = n >= 2
    p = d["params"].astype(np.float64)
    assert np.all(p[~sel, 3] < 0)
    assert close(p[sel, 0:3], tr["cell_u"][sel], tol, 1.0) < tol
    if system.params.rule == I.SRD:
        assert close(p[sel, 3], tr["cell_kappa"][sel], tol, 1.0) < 5 * tol
        assert close(p[sel, 4:7], tr["cell_axis"][sel], tol, 1.0) < tol
    else:
        assert close(p[sel, 4:7], tr["cell_xibar"][sel], tol, 1.0) < tol

    g = sim.get_state()
    assert np.array_equal(g.x, ost.x)
    assert close(g.v, ost.v, tol, 1.0) < tol
    if osys.n_bodies:
        assert close(g.P, ost.P, tol, sM) < tol
        assert close(g.Lm, ost.Lm, tol, sI) < tol
    assert g.step == 1
    sim.close()
    return g, ost


@pytest.mark.parametrize("prec", [I.P64, I.P32])
def test_one_step_single_sphere_L10(B, prec):
    one_step(B, I.single_sphere_L10(prec))


@pytest.mark.parametrize("prec", [I.P64, I.P32])
@pytest.mark.parametrize("rule,thermo", [(I.SRD, 1), (I.SRD, 2), (I.AT, 0)])
def test_one_step_small_suspension(B, prec, rule, thermo):
    system = I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, rule, thermo, prec, seed=3, name="small")
    assert system.n_bodies >= 3
    one_step(B, system)


@pytest.mark.parametrize("prec", [I.P64, I.P32])
def test_one_step_suspension_L50(B, prec):
    """L=50, density 5, 221 radius-3 642-site spheres, MPCD-AT."""
    one_step(B, I.suspension_L50(prec))


def test_one_step_ragged_replicas(B):
    """Several uneven replicas, one with no colloid and one tiny box."""
    prm = I.Params(rule=I.SRD, thermostat=1, precision=I.P32, seed=9)
    shapes = [I.sphere_shape(2.0, 2, 5.0), I.dumbbell_shape(2.0, 2.0, 2, 5.0)]
    rng = np.random.default_rng(0)
    Ls = [(16, 16, 16), (3, 3, 3), (9, 14, 11), (20, 20, 20)]
    ids = [[0, 1], [], [0], [1, 0, 1]]
    system = I.build_system(prm, shapes, Ls, 3.3, ids, "ragged", placement_seed=5)
    system.replicas[1].n_solvent = 7          # ragged tail, not a multiple of 4
    system._placements[1] = (np.zeros((0, 3)), np.zeros((0, 4)))
    one_step(B, system)


def test_pipelined_steps_equal_unfused_bitwise(B):
    """mpcd_step(n) (fused solvent pass, CUDA graph, re-sorts) reproduces the
    unfused stream/couple/collide/couple sequence bit for bit (FP32 form)."""
    for rule in (I.SRD, I.AT):
        system = I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, rule, 1, I.P32, seed=4, name="pipe")
        st = I.initial_state(system)
        a = B.Simulation(system, sort_period=3)
        a.set_state(st)
        a.step(7)
        a.step(1)
        ga = a.get_state()
        b = B.Simulation(system, sort_period=-1)
        b.set_state(st)
        for _ in range(8):
            b.stream()
            b.couple(B.MPCD_PRE)
            b.collide()
            b.couple(B.MPCD_POST)
        gb = b.get_state()
        for k in ("x", "v", "R", "q", "P", "Lm"):
            assert np.array_equal(getattr(ga, k), getattr(gb, k)), (rule, k)
        assert ga.step == gb.step == 8
        a.close()
        b.close()


def test_restart_and_input_order_are_bitwise_reproducible(B):
    system = I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, I.SRD, 1, I.P32, seed=6, name="restart")
    st = I.initial_state(system)
    s1 = B.Simulation(system)
    s1.set_state(st)
    s1.step(12)
    ref = s1.get_state()
    s1.set_state(st)
    s1.step(5)
    mid = s1.get_state()
    s2 = B.Simulation(system)
    s2.set_state(mid)
    s2.step(7)
    out = s2.get_state()
    for k in ("x", "v", "R", "q", "P", "Lm"):
        assert np.array_equal(getattr(out, k), getattr(ref, k)), k
    # permuted solvent input order: SRD draws are per cell, so the physics is
    # unchanged and the (permuted-back) result is bit-identical
    perm = np.random.default_rng(1).permutation(system.n_solvent)
    stp = st.copy()
    stp.x, stp.v = st.x[perm], st.v[perm]
    s3 = B.Simulation(system)
    s3.set_state(stp)
    s3.step(12)
    o3 = s3.get_state()
    inv = np.argsort(perm)
    assert np.array_equal(o3.x[inv], ref.x) and np.array_equal(o3.v[inv], ref.v)
    for s in (s1, s2, s3):
        s.close()


def test_multi_step_fp64_tracks_oracle(B):
    system = I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, I.SRD, 1, I.P64, seed=8, name="track")
    st = I.initial_state(system)
    sim = B.Simulation(system)
    sim.set_state(st)
    sim.step(10)
    g = sim.get_state()
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)
    O.step(osys, ost, 10)
    assert np.array_equal(np.floor(g.x * 2**20), np.floor(ost.x * 2**20))
    assert close(g.v, ost.v, 0, 1.0) < 1e-10
    sM, sI = body_scales(system)
    assert close(g.P, ost.P, 0, sM) < 1e-10
    assert close(g.Lm, ost.Lm, 0, sI) < 1e-10
    sim.close()


def test_conservation_and_canonical_sort(B):
    system = I.suspension(20, 5.0, 0.2, 2.0, 2, 5.0, I.SRD, 1, I.P32, seed=10, name="cons")
    st = I.initial_state(system)
    sim = B.Simulation(system)
    sim.set_state(st)
    d0 = sim.diagnostics()
    sim.step(20)
    d1 = sim.diagnostics()
    p0 = d0["p_solvent"] + d0["p_bodies"]
    p1 = d1["p_solvent"] + d1["p_bodies"]
    # Only the FP32 rounding of each written velocity changes the total: a
    # random walk of N steps x N_s roundings of about one ulp(1) = 2^-23 each
    # (|v| ~ sqrt(kT/m) = 1).  Ten times its size: the loss of one site's
    # momentum (m |v| ~ 1) or of one cell's would be 100x above the bar.
    m2 = system.n_solvent * system.params.m_solvent ** 2 + system.n_sites * system.shapes[0].m[0] ** 2
    bar = 10.0 * np.sqrt(20 * m2) * 2.0**-23
    print("total momentum change", np.abs(p1 - p0), "bar", bar)
    assert np.all(np.abs(p1 - p0) < bar), (np.abs(p1 - p0), bar)
    before = sim.get_state()
    sim.sort(canonical=True)
    after = sim.get_state()
    for k in ("x", "v", "R", "q", "P", "Lm"):
        assert np.array_equal(getattr(before, k), getattr(after, k))
    sim.close()


def test_invalid_arguments_are_rejected(B):
    system = I.single_sphere_L10(I.P32)
    st = I.initial_state(system)
    sim = B.Simulation(system)
    bad = st.copy()
    bad.x[5, 1] = 10.0        # == L: outside [0, L)
    with pytest.raises(B.MPCDError) as e:
        sim.set_state(bad)
    assert e.value.status == B.MPCD_ERR_ARG
    sim.set_state(st)         # the context is still usable
    sim.step(2)
    with pytest.raises(B.MPCDError):
        sim.step(-1)
    sim.close()


@pytest.mark.parametrize("rule", [I.SRD, I.AT])
def test_staged_and_direct_solvent_passes_agree_bitwise(B, rule):
    """The direct pass, the shared-memory staged pass (bulk async copies), the
    warp-specialised pass and the per-warp ring compute the same thing; every
    launch shape gives bit-identical P32 states."""
    system = I.suspension(18, 5.0, 0.15, 2.0, 2, 5.0, rule, 1, I.P32, seed=12, name="ab")
    system.replicas[0].n_solvent -= 3          # a ragged tail
    st = I.initial_state(system)
    ref = None
    for staged, block, tile, ctas in [(0, 256, 8192, 4), (1, 128, 1024, 1), (1, 256, 2048, 2),
                                      (1, 512, 4096, 1), (1, 96, 1000, 3), (2, 256, 1024, 2),
                                      (2, 512, 2048, 1), (2, 96, 1000, 3), (3, 512, 128, 1),
                                      (3, 256, 256, 2), (3, 96, 200, 3)]:
        sim = B.Simulation(system)
        sim.set_tuning(block=block, tile=tile, ctas_per_sm=ctas, staged=staged)
        sim.set_state(st)
        sim.step(6)
        g = sim.get_state()
        sim.close()
        if ref is None:
            ref = g
            continue
        for k in ("x", "v", "R", "q", "P", "Lm"):
            assert np.array_equal(getattr(g, k), getattr(ref, k)), (staged, block, tile, k)


def test_pipelined_resorts_over_many_replicas_equal_unfused_bitwise(B):
    """The pipelined step's re-sort orders each replica by the cells of the next
    collision (its own grid shift), with the counts the cell words hold: over
    boxes of different edges, with ragged tails, a re-sort every other step gives
    the state of the unfused sequence bit for bit."""
    system = I.batched_single_sphere(24, I.P32, seed=6, Ls=(6, 7, 9, 12))
    system.params.thermostat = 1
    st = I.initial_state(system)
    a = B.Simulation(system, sort_period=2)
    a.set_tuning(block=128, tile=512, ctas_per_sm=2, staged=1)
    a.set_state(st)
    a.step(7)
    ga = a.get_state()
    b = B.Simulation(system, sort_period=-1)
    b.set_state(st)
    for _ in range(7):
        b.stream()
        b.couple(B.MPCD_PRE)
        b.collide()
        b.couple(B.MPCD_POST)
    gb = b.get_state()
    for k in ("x", "v", "R", "q", "P", "Lm"):
        assert np.array_equal(getattr(ga, k), getattr(gb, k)), k
    a.close()
    b.close()


@pytest.mark.parametrize("rule", [I.SRD, I.AT])
def test_launch_forms_agree_bitwise_over_many_replicas(B, rule):
    """Boxes of different edges in one context: a CTA's tiles cross replica
    boundaries, so the launch forms' per-replica set-up (grid shifts, box,
    cell base, keys - cached across tiles of one replica) changes between
    tiles; every form gives bit-identical P32 states."""
    system = I.batched_single_sphere(24, I.P32, seed=4, Ls=(6, 7, 9, 12))
    system.params.rule = rule
    system.params.thermostat = 1 if rule == I.SRD else 0
    st = I.initial_state(system)
    ref = None
    for staged, block, tile, ctas in [(0, 256, 1024, 1), (1, 128, 256, 1), (1, 256, 512, 2), (2, 128, 256, 1),
                                      (3, 256, 128, 1), (3, 96, 64, 2)]:
        sim = B.Simulation(system)
        sim.set_tuning(block=block, tile=tile, ctas_per_sm=ctas, staged=staged)
        sim.set_state(st)
        sim.step(5)
        g = sim.get_state()
        sim.close()
        if ref is None:
            ref = g
            continue
        for k in ("x", "v", "R", "q", "P", "Lm"):
            assert np.array_equal(getattr(g, k), getattr(ref, k)), (staged, block, tile, k)


@pytest.mark.parametrize("prec", [I.P32, I.P64])
def test_state_round_trip_is_exact(B, prec):
    """mpcd_set_state stores the solvent cell-sorted (radix sort of (cell, row)
    pairs, then a gather) and mpcd_get_state brings it back to row order (radix
    sort of (row, slot) pairs): with no step in between the round trip is the
    identity, for uneven replicas with ragged tails, a box large enough for
    three digit passes and one large enough for the chunked egress (rows gathered
    and copied to the host in eight chunks)."""
    for system in (I.batched_single_sphere(n_rep=5, precision=prec, seed=6, Ls=(6, 8, 12)),
                   I.suspension(60, 10.0, 0.1, 4.0, 3, 10.0, I.SRD, 1, prec, seed=2, name="rt"),
                   # 4.4 M solvent particles: the egress gathers and copies in row chunks
                   I.suspension(76, 10.0, 0.05, 4.0, 3, 10.0, I.SRD, 1, prec, seed=3, name="rt_big")):
        system.replicas[0].n_solvent -= 5
        st = I.initial_state(system)
        sim = B.Simulation(system)
        sim.set_state(st)
        g = sim.get_state()
        sim.close()
        real = np.float32 if prec == I.P32 else np.float64
        assert np.array_equal(g.x, st.x.astype(real)) and np.array_equal(g.v, st.v.astype(real))
        assert np.array_equal(g.R, st.R) and np.array_equal(g.P, st.P)


def test_resorts_per_call_follow_the_fused_pass_count(B):
    """A call of n steps runs n - 1 fused passes, each of which counts towards
    the next re-sort, so from `since` passes after a re-sort it re-sorts
    (since + n - 1) // period times and ends at (since + n - 1) % period;
    bench.py places its timed call in the replay cycle by this rule."""
    system = I.suspension(24, 5.0, 0.1, 2.0, 2, 5.0, I.SRD, 1, I.P32, seed=3, name="phase")
    st = I.initial_state(system)
    sim = B.Simulation(system)
    sim.set_state(st)
    period = 4
    sim.set_tuning(sort_period=period)
    sim.sort()
    since = 0
    for n in (3, 5, 2, 7, 4, 9, 1, 6):
        sim.set_profiling(True)
        sim.reset_profile()
        sim.step(n)
        prof = sim.profile()
        sim.set_profiling(False)
        got = prof["sort"]["launches"] if "sort" in prof else 0
        assert got == (since + n - 1) // period, (since, n, got)
        since = (since + n - 1) % period
    sim.close()
