"""Spatial domain decomposition on the GPU: two and three slab contexts of one
box (mpcd_create_slab and the slab calls, driven by domain.SlabDomain with
in-process message routing) against one context holding the whole box, both
through the C ABI on the same device.

* Pure solvent, FP32 form, SRD with the cell thermostat: after every one of
  five steps the gathered positions and velocities equal the single context's
  bit for bit (the completed face-layer words are the whole box's words), and
  particles did migrate.
* With colloids (their sites split between slabs by z): after one step the
  solvent is bit-identical; each body's momentum and angular momentum, summed
  over the slabs, agree with the single context to FP32 rounding (the sums of
  the sites' momentum changes are taken in another order).
* Argument checks of the slab calls.
"""
import numpy as np
import pytest

from paper_2604_14307_gb300 import domain as D
from paper_2604_14307_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14307_gb300 import binding, build_lib
    build_lib.build()
    return binding


def single(B, system, st, steps):
    sim = B.Simulation(system, sort_period=-1)
    sim.set_state(st)
    out = []
    for _ in range(steps):
        sim.stream()
        sim.couple(B.MPCD_PRE)
        sim.collide()
        sim.couple(B.MPCD_POST)
        out.append(sim.get_state())
    sim.close()
    return out


def slabs(B, system, st, world, steps):
    part = D.Partition(system.replicas[0].L[2], world)
    rows = D.split_state(part, st.x)
    cap = int(1.3 * max(len(r) for r in rows)) + 256
    real = np.float32 if system.params.precision == I.P32 else np.float64
    sl = {}
    for r in range(world):
        s = B.Slab(system, int(part.bounds[r]), int(part.bounds[r + 1]), min(cap, system.n_solvent))
        s.set_slab_state(rows[r].astype(np.uint32), st.x[rows[r]].astype(real), st.v[rows[r]].astype(real),
                         st.R, st.q, st.P, st.Lm, st.step)
        sl[r] = s
    dom = D.SlabDomain(part, D.LoopbackComm(world), {r: D.GpuSlab(s) for r, s in sl.items()}, sort_period=0)
    out = []
    for _ in range(steps):
        dom.step(1)
        parts = [sl[r].get_slab_state() for r in range(world)]
        x, v = D.gather([(p[0], p[1], p[2]) for p in parts], system.n_solvent)
        out.append((x, v, parts))
    for s in sl.values():
        s.close()
    return out, dom.migrated


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_reproduce_one_context_bitwise_solvent(B, world):
    prm = I.Params(rule=I.SRD, thermostat=1, precision=I.P32, seed=17)
    system = I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [(16, 12, 24)], 5.0, [[]], "slabs", placement_seed=3)
    st = I.initial_state(system)
    ref = single(B, system, st, 5)
    got, mig = slabs(B, system, st, world, 5)
    assert mig > 0
    for k in range(5):
        assert np.array_equal(got[k][0], ref[k].x), k
        assert np.array_equal(got[k][1], ref[k].v), k


@pytest.mark.parametrize("rule", [I.SRD, I.AT])
def test_slabs_with_colloids(B, rule):
    system = I.suspension(24, 5.0, 0.12, 2.0, 2, 5.0, rule, 1, I.P32, seed=5, name="slab_colloids")
    assert system.n_bodies >= 4
    st = I.initial_state(system)
    ref = single(B, system, st, 1)[0]
    got, _ = slabs(B, system, st, 2, 1)
    x, v, parts = got[0]
    assert np.array_equal(x, ref.x)
    assert np.array_equal(v, ref.v)
    M = system.shapes[0].m.sum()
    Ib = I.shape_inertia_diag(system.shapes[0]).max()
    for p in parts:   # every slab holds the same bodies
        R, q, P, Lm = p[3], p[4], p[5], p[6]
        assert np.array_equal(R, parts[0][3]) and np.array_equal(P, parts[0][5])
        assert np.max(np.abs(P - ref.P) / (np.abs(ref.P) + np.sqrt(M))) < 1e-5
        assert np.max(np.abs(Lm - ref.Lm) / (np.abs(ref.Lm) + np.sqrt(Ib))) < 1e-5


def test_slab_arguments(B):
    prm = I.Params(rule=I.SRD, thermostat=1, precision=I.P32, seed=1)
    system = I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [(8, 8, 8)], 5.0, [[]], "slab_args", placement_seed=1)
    with pytest.raises(B.MPCDError):
        B.Slab(system, 3, 4, 100)                       # one cell layer: too thin
    with pytest.raises(B.MPCDError):
        B.Slab(system, 0, 9, 100)                       # beyond the box
    s = B.Slab(system, 0, 4, 64)
    st = I.initial_state(system)
    sel = np.flatnonzero(st.x[:, 2] < 4)[:100]
    with pytest.raises(B.MPCDError):                    # more than the capacity
        s.set_slab_state(sel.astype(np.uint32), st.x[sel].astype(np.float32), st.v[sel].astype(np.float32),
                         st.R, st.q, st.P, st.Lm, 0)
    s.close()
    sim = B.Simulation(system)
    with pytest.raises(B.MPCDError):                    # only a slab takes slab calls
        sim.lib and sim._check(sim.lib.mpcd_slab_insert(sim.ctx, 0, None, None, None, None))
    sim.close()
