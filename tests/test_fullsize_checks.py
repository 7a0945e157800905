"""The full-size checks of test_gpu_fullsize.py, run on the oracle's own step
(small boxes, CPU): they must accept the oracle's result, and reject it when a
velocity, a position or a cell word is perturbed - so a GPU step that passes
them agrees with the method, not merely with the checker."""
import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I

from test_gpu_fullsize import verify_step


def oracle_step(system):
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)

    def momenta():
        return {"p_solvent": system.params.m_solvent * ost.v.sum(0), "p_bodies": ost.P.sum(0)}

    p0 = momenta()
    O.stream(osys, ost)
    tr = O.collide(osys, ost)
    nw = 4 if system.params.rule == I.SRD else 6
    C = osys.n_cells
    par = np.zeros((C, 8))
    par[:, 0:3] = tr["cell_u"]
    par[:, 3] = np.where(tr["sums"][0] >= 2, tr["cell_kappa"], -1.0)
    par[:, 4:7] = tr["cell_axis"] if system.params.rule == I.SRD else tr["cell_xibar"]
    d = {"shift": tr["shift"], "sums": tr["fixed"][:nw].astype(np.int64), "params": par,
         "site_cell": tr["cell_site"], "site_v": tr["site_v"]}
    return st, ost.x.copy(), ost.v.copy(), d, p0, momenta()


@pytest.mark.parametrize("make", [
    lambda: I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, I.SRD, 1, I.P32, seed=3, name="srd"),
    lambda: I.batched_single_sphere(n_rep=6, precision=I.P32, seed=2, Ls=(12, 16)),
    lambda: I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, I.AT, 0, I.P32, seed=4, name="at"),
])
def test_checks_accept_the_oracle_and_reject_perturbations(make):
    system = make()
    st, gx, gv, d, p0, p1 = oracle_step(system)
    ns, npart = verify_step(system, st, gx, gv, d, p0, p1, n_sample=300)
    assert ns > 50 and npart > 200
    # a perturbed velocity of a particle in a checked cell is caught
    bad = gv.copy()
    bad[:] += 1e-3
    with pytest.raises(AssertionError):
        verify_step(system, st, gx, bad, d, p0, p1, n_sample=300)
    # a position one ulp off is caught
    badx = gx.astype(np.float32).copy()
    badx[7, 1] = np.nextafter(badx[7, 1], np.float32(0))
    with pytest.raises(AssertionError):
        verify_step(system, st, badx, gv, d, p0, p1, n_sample=300)
    # a cell word off by one unit is caught
    dd = dict(d)
    dd["sums"] = d["sums"].copy()
    live = np.where(d["sums"][0] != 0)[0]
    dd["sums"][0, live[3]] += 1
    with pytest.raises(AssertionError):
        verify_step(system, st, gx, gv, dd, p0, p1, n_sample=300)
