"""GPU tests of replica ensembles (many uneven boxes in one context).

* one step of the batched single-colloid and mixed-shape workloads against the
  oracle (parity bars of test_gpu_parity);
* an ensemble split over several contexts (as over several GPUs) evolves
  bit for bit as the ensemble in one context: each replica's random streams
  are keyed by its stream id, not by its position;
* equipartition on the GPU (Sec. III.A): over a large ensemble of single
  spheres the mean translational and rotational kinetic energies per body are
  (3/2) kT (1 - M/M_total) and (3/2) kT within 3 standard errors (50 block
  averages of a long run), with no other slack.
"""
import math

import numpy as np
import pytest

from paper_2604_14307_gb300 import inputs as I
from paper_2604_14307_gb300 import replicas as RP

from test_gpu_parity import one_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14307_gb300 import binding, build_lib
    build_lib.build()
    return binding


@pytest.mark.parametrize("prec", [I.P64, I.P32])
def test_one_step_batched_single_sphere(B, prec):
    """Uneven boxes L in {12, 16, 20, 24}, one 162-site sphere each."""
    one_step(B, I.batched_single_sphere(n_rep=48, precision=prec, seed=2))


def test_one_step_batched_mixed_shapes(B):
    """Spheres, dumbbells and spherocylinders in boxes L in [20, 40], MPCD-AT."""
    system = I.batched_mixed_shapes(n_rep=3, precision=I.P32, seed=4)
    assert len(set(system.body_shape_array())) >= 2
    one_step(B, system)


def test_split_ensemble_equals_one_context_bitwise(B):
    full = I.batched_single_sphere(n_rep=7, precision=I.P32, seed=5, Ls=(12, 16, 20))
    st = I.initial_state(full)
    a = B.Simulation(full)
    a.set_state(st)
    a.step(5)
    ga = a.get_state()
    a.close()
    so, bo = full.solvent_offsets(), full.body_offsets()
    parts = RP.shard(RP.replica_cost(full), 3)
    assert sum(len(p) for p in parts) == full.n_rep
    for ids in parts:
        sub = full.subset(ids)
        b = B.Simulation(sub)
        b.set_state(I.initial_state(sub))
        b.step(5)
        gb = b.get_state()
        b.close()
        so2, bo2 = sub.solvent_offsets(), sub.body_offsets()
        for k, r in enumerate(ids):
            for name, off, off2 in (("x", so, so2), ("v", so, so2), ("R", bo, bo2), ("q", bo, bo2),
                                    ("P", bo, bo2), ("Lm", bo, bo2)):
                u = getattr(ga, name)[off[r]:off[r + 1]]
                w = getattr(gb, name)[off2[k]:off2[k + 1]]
                assert np.array_equal(u, w), (r, name)


def block_mean_err(x, nblocks=20):
    x = np.asarray(x)
    n = len(x) // nblocks
    b = x[: n * nblocks].reshape(nblocks, n).mean(1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nblocks)


def test_equipartition_of_the_rigid_sphere_ensemble(B, golden):
    n_rep, L, burn, steps, every = 512, 12, 300, 10000, 5
    system = I.batched_single_sphere(n_rep=n_rep, precision=I.P32, seed=11, Ls=(L,))
    sim = B.Simulation(system)
    sim.set_state(I.initial_state(system))
    sim.step(burn)
    ET, ER = [], []
    for _ in range(steps // every):
        sim.step(every)
        d = sim.diagnostics()
        ET.append(d["ke_trans"] / n_rep)
        ER.append(d["ke_rot"] / n_rep)
    sim.close()
    M = system.shapes[0].m.sum()
    Mtot = M + 5.0 * L**3
    expect_T = golden["mean_E_T"]["expected"] * (1 - M / Mtot)
    expect_R = golden["mean_E_R"]["expected"]
    mT, eT = block_mean_err(ET, nblocks=50)
    mR, eR = block_mean_err(ER, nblocks=50)
    print("E_T", mT, "+-", eT, "expected", expect_T, "; E_R", mR, "+-", eR, "expected", expect_R)
    assert abs(mT - expect_T) < 3 * eT, (mT, eT, expect_T)
    assert abs(mR - expect_R) < 3 * eR, (mR, eR, expect_R)
    assert eT < 0.01 and eR < 0.01        # the ensemble is large enough to mean something
