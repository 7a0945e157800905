"""GPU tests of the sedimentation forcing (Sec. III.B): a constant force on
every body, balanced on the solvent.

* One step with the force from the same state as the oracle, through mpcd_step
  (the solvent pass kicks, drifts and kicks inside the fused pass) and through
  stream, couple, collide: solvent positions bit-exact, solvent velocities,
  body momenta and positions within the parity bars.
* Many steps keep the box force free: solvent plus body momentum stays at its
  initial value to float rounding, while the bodies gain momentum along f.
* A force on a context with several replicas, or without solvent, is refused.
* The unwrapped body displacements (mpcd_body_displacements, the input of the
  diffusion coefficient of Eq. 15) match the oracle and the wrapped positions.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {I.P64: 1e-12, I.P32: 1e-5}
F = np.array([0.5, 0.0, 0.0])


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14307_gb300 import binding, build_lib
    build_lib.build()
    return binding


def box(precision, rule=I.SRD, n_bodies=3, seed=8):
    prm = I.Params(rule=rule, thermostat=1, precision=precision, seed=seed)
    return I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [(14, 14, 14)], 5.0, [[0] * n_bodies],
                          "sediment", placement_seed=seed)


@pytest.mark.parametrize("pipelined", [True, False])
@pytest.mark.parametrize("precision,rule", [(I.P32, I.SRD), (I.P64, I.SRD), (I.P32, I.AT)])
def test_one_forced_step_matches_oracle(B, pipelined, precision, rule):
    system = box(precision, rule)
    tol = TOL[precision]
    st = I.initial_state(system)
    sim = B.Simulation(system)
    sim.set_state(st)
    sim.set_body_force(F)
    if pipelined:
        sim.step(1)
    else:
        sim.stream()
        sim.couple(B.MPCD_PRE)
        sim.collide()
        sim.couple(B.MPCD_POST)
    g = sim.get_state()
    sim.close()
    osys = O.OracleSystem(system)
    osys.set_body_force(F)
    ost = O.OracleState(osys, st)
    O.step(osys, ost, 1)
    assert np.array_equal(g.x, ost.x)
    assert np.max(np.abs(g.v - ost.v) / (np.abs(ost.v) + 1.0)) <= tol
    M = system.shapes[0].m.sum()
    assert np.max(np.abs(g.P - ost.P)) <= tol * np.sqrt(M) * 10
    assert np.max(np.abs(g.R - ost.R)) <= 1e-12
    assert np.all(g.P[:, 0] != st.P[:, 0])


def test_forced_box_stays_force_free(B):
    """Total momentum stays constant under the balanced force, while the bodies'
    momentum along f, averaged over the second half of the run, is positive.
    The thermal momentum of the four bodies fluctuates by about sqrt(4 M kT) ~ 57
    around a mean of ~100 at this force (oracle runs, four seeds: time averages
    101-162), so the average over 20 samples, not one instant, is tested."""
    system = box(I.P32, n_bodies=4, seed=9)
    st = I.initial_state(system)
    sim = B.Simulation(system)
    sim.set_state(st)
    sim.set_body_force(40 * F)      # strong enough to beat the bodies' thermal momentum
    d0 = sim.diagnostics()
    p0 = np.asarray(d0["p_solvent"]) + np.asarray(d0["p_bodies"])
    sim.step(200)
    pb = []
    for _ in range(20):
        sim.step(10)
        pb.append(sim.diagnostics()["p_bodies"][0])
    d1 = sim.diagnostics()
    p1 = np.asarray(d1["p_solvent"]) + np.asarray(d1["p_bodies"])
    sim.close()
    assert np.all(np.abs(p1 - p0) < 1e-2 * np.sqrt(system.n_solvent + system.n_sites))
    print("time-averaged body momentum along f:", np.mean(pb), "+-", np.std(pb))
    assert np.mean(pb) > 0.0


def test_force_needs_one_replica_with_solvent(B):
    two = I.batched_single_sphere(n_rep=2, precision=I.P32, seed=1, Ls=(12,))
    sim = B.Simulation(two)
    with pytest.raises(B.MPCDError) as e:
        sim.set_body_force(F)
    assert e.value.status == B.MPCD_ERR_ARG
    sim.set_body_force([0.0, 0.0, 0.0])       # turning it off is always allowed
    sim.close()


@pytest.mark.parametrize("precision", [I.P32, I.P64])
def test_body_displacements_match_oracle(B, precision):
    """Unwrapped displacement (the input of Eq. 15): the oracle's value, and the
    wrapped position equals start + displacement modulo the box."""
    system = I.suspension(14, 5.0, 0.1, 2.0, 2, 5.0, I.SRD, 1, precision, seed=3)
    st = I.initial_state(system)
    sim = B.Simulation(system)
    sim.set_state(st)
    sim.step(6)
    D = sim.body_displacements()
    g = sim.get_state()
    sim.close()
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)
    O.step(osys, ost, 6)
    assert np.allclose(D, ost.D[: system.n_bodies], rtol=1e-4, atol=1e-9)
    L = np.array(system.replicas[0].L, dtype=np.float64)
    d = np.mod(st.R + D - g.R, L)
    assert np.all(np.minimum(d, L - d) < 1e-9)
