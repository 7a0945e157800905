"""GPU parity of the binning step as a counting sort (Sec. II.A, the cell
assignment under the random grid shift).

mpcd_cell_order builds, on the GPU, the canonical member order of the
collision at the current step: histogram of the cell occupancies, exclusive
scan, scatter, and within each cell solvent before sites, each by ascending
id.  It is integer work, so it must equal the oracle's `order` and
`cell_start` of the same collision bit for bit: for the FP32 and FP64 forms,
SRD and MPCD-AT, with colloid sites, on uneven replicas with a ragged
7-particle tail, an empty box and a 3^3 box, and on the L=50 suspension at full
size.  The order must also not depend on the storage order of the solvent
(a re-sort before the call changes nothing).
"""
import numpy as np
import pytest

import oracle as O
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


def ragged(rule, prec):
    prm = I.Params(rule=rule, thermostat=1, precision=prec, seed=9)
    shapes = [I.sphere_shape(2.0, 2, 5.0), I.dumbbell_shape(2.0, 2.0, 2, 5.0)]
    Ls = [(16, 16, 16), (3, 3, 3), (9, 14, 11), (5, 4, 6), (20, 20, 20)]
    ids = [[0, 1], [], [0], [], [1, 0, 1]]
    system = I.build_system(prm, shapes, Ls, 3.3, ids, "ragged_order", placement_seed=5)
    system.replicas[1].n_solvent = 7          # ragged tail, not a multiple of 4
    system._placements[1] = (np.zeros((0, 3)), np.zeros((0, 4)))
    system.replicas[3].n_solvent = 0          # an empty box
    system._placements[3] = (np.zeros((0, 3)), np.zeros((0, 4)))
    return system


def check_order(B, system, resort=False, steps_before=0):
    st = I.initial_state(system)
    sim = B.Simulation(system, sort_period=-1)
    sim.set_state(st)
    if steps_before:
        sim.step(steps_before)
        st = sim.get_state()
    if resort:
        sim.sort(canonical=False)
    sim.stream()
    sim.couple(B.MPCD_PRE)
    order, start = sim.cell_order()
    sim.close()
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)
    O.stream(osys, ost)
    tr = O.collide(osys, ost)
    n = osys.n_solvent + osys.n_sites
    assert np.array_equal(start, tr["cell_start"])
    assert np.array_equal(order, tr["order"][:n])
    # the order is a permutation of all members
    assert np.array_equal(np.sort(order), np.arange(n))
    return order, start


@pytest.mark.parametrize("prec", [I.P32, I.P64])
@pytest.mark.parametrize("rule", [I.SRD, I.AT])
def test_cell_order_ragged_replicas(B, prec, rule):
    order, start = check_order(B, ragged(rule, prec))
    counts = np.diff(start)
    assert counts.max() > 1 and (counts == 0).any()


def test_cell_order_after_steps_and_resort(B):
    """After pipelined steps (the storage is cell-sorted and re-sorted) the
    order of the next collision still equals the oracle's from the same state."""
    system = I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, I.SRD, 1, I.P32, seed=3, name="order_steps")
    check_order(B, system, resort=True, steps_before=5)


def test_cell_order_suspension_L50(B):
    """Full size: 625,000 solvent particles and 141,882 sites in 125,000 cells."""
    check_order(B, I.suspension_L50(I.P32))
