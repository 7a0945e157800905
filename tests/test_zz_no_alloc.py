"""mpcd_collide_solvent_static (static device scratch, no allocation) against
mpcd_collide of a context that holds the same solvent-only box, and against
the oracle.

Two collisions in a row (steps 0 and 1) on both paths.  The two paths run the
same binning, parameter and collision kernels on the same particles (only the
storage order and the scratch pointers differ), and the cell sums are exact
integer sums, so the velocities must agree bit for bit after each call;
positions must be untouched.  The first collision must also agree with the
oracle's collision of the same state within the FP32 parity bar of the other
GPU tests (|a - b| <= 1e-5 (|b| + 1), 1 = sqrt(kT/m)).  The file is named to be
collected last, so the static scratch is exercised after every other test has
used the library on the same device, and it also passes on its own.
"""
import numpy as np
import pytest

from paper_2604_14307_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14307_gb300 import binding, build_lib
    build_lib.build()
    return binding, torch


def solvent_box(rule, thermostat, L, seed):
    prm = I.Params(rule=rule, thermostat=thermostat, precision=I.P32, seed=seed)
    system = I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [L], 5.0, [[]], "solvent_only",
                            placement_seed=seed)
    system.replicas[0].n_solvent -= system.replicas[0].n_solvent % 4
    return system


def soa(torch, a):
    return [torch.tensor(np.ascontiguousarray(a[:, k], dtype=np.float32), device="cuda") for k in range(3)]


@pytest.mark.parametrize("rule,thermostat,L", [(I.SRD, 1, (20, 24, 16)), (I.SRD, 0, (40, 40, 40)),
                                               (I.AT, 0, (17, 19, 23))])
def test_static_collide_matches_context_collide(env, rule, thermostat, L):
    import oracle as O
    B, torch = env
    system = solvent_box(rule, thermostat, L, seed=21)
    st = I.initial_state(system)
    st.x, st.v = st.x.astype(np.float32), st.v.astype(np.float32)

    sim = B.Simulation(system, sort_period=-1)
    sim.set_state(st)
    sim.collide()                 # step 0
    ref0 = sim.get_state()
    sim.couple(B.MPCD_POST)       # no colloids: only advances the step
    sim.collide()                 # step 1
    ref1 = sim.get_state()
    sim.close()

    n = system.n_solvent
    x, y, z = soa(torch, st.x)
    vx, vy, vz = soa(torch, st.v)
    tag = torch.arange(n, dtype=torch.int32, device="cuda")

    def velocities():
        torch.cuda.synchronize()
        return np.stack([t.cpu().numpy() for t in (vx, vy, vz)], axis=1)

    B.collide_solvent_static(system.params, L, x, y, z, vx, vy, vz, tag, step=0)
    v0 = velocities()
    B.collide_solvent_static(system.params, L, x, y, z, vx, vy, vz, tag, step=1)
    v1 = velocities()
    pos = np.stack([t.cpu().numpy() for t in (x, y, z)], axis=1)

    assert np.array_equal(pos, st.x) and np.array_equal(ref1.x, st.x)
    assert not np.array_equal(v0, st.v)
    assert np.array_equal(v0, ref0.v), np.abs(v0 - ref0.v).max()
    assert np.array_equal(v1, ref1.v), np.abs(v1 - ref1.v).max()

    # the first collision against the oracle's collision of the same state
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)
    O.collide(osys, ost, trace=False)
    err = np.abs(v0.astype(np.float64) - ost.v) / (np.abs(ost.v) + 1.0)
    assert err.max() <= TOL, err.max()


def test_static_collide_rejects_what_does_not_fit(env):
    B, torch = env
    system = solvent_box(I.SRD, 1, (8, 8, 8), seed=3)
    st = I.initial_state(system)
    x, y, z = soa(torch, st.x)
    vx, vy, vz = soa(torch, st.v)
    p = system.params

    with pytest.raises(B.MPCDError) as e:              # more cells than the static scratch holds
        B.collide_solvent_static(p, (41, 41, 41), x, y, z, vx, vy, vz)
    assert e.value.status == B.MPCD_ERR_ARG and "exceeds" in str(e.value)

    with pytest.raises(B.MPCDError) as e:              # an edge the 32-bit binning rule cannot hold
        B.collide_solvent_static(p, (3, 3, 2048), x, y, z, vx, vy, vz)
    assert e.value.status == B.MPCD_ERR_ARG and "2047" in str(e.value)

    odd = [t[:-1] for t in (x, y, z, vx, vy, vz)]       # n not a multiple of 4
    with pytest.raises(B.MPCDError) as e:
        B.collide_solvent_static(p, (8, 8, 8), *odd)
    assert e.value.status == B.MPCD_ERR_ARG and "multiple of 4" in str(e.value)

    mis = [t[1:-3] for t in (x, y, z, vx, vy, vz)]      # 4-byte offset: not 16-byte aligned
    with pytest.raises(B.MPCDError) as e:
        B.collide_solvent_static(p, (8, 8, 8), *mis)
    assert e.value.status == B.MPCD_ERR_ARG and "aligned" in str(e.value)

    p64 = I.Params(rule=I.SRD, thermostat=1, precision=I.P64, seed=3)
    with pytest.raises(B.MPCDError) as e:
        B.collide_solvent_static(p64, (8, 8, 8), x, y, z, vx, vy, vz)
    assert e.value.status == B.MPCD_ERR_ARG

    at = I.Params(rule=I.AT, thermostat=0, precision=I.P32, seed=3)
    with pytest.raises(B.MPCDError) as e:              # MPCD_AT without particle ids
        B.collide_solvent_static(at, (8, 8, 8), x, y, z, vx, vy, vz)
    assert e.value.status == B.MPCD_ERR_ARG

    # nothing was changed by the rejected calls
    assert np.array_equal(vx.cpu().numpy(), st.v[:, 0].astype(np.float32))
