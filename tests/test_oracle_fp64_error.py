"""The comparison of the FP32 form with the plain FP64 method (oracle.parity),
checked on the CPU with the oracle's own FP32 mode standing in for the GPU.

* The oracle in its FP32 mode (float32 storage and float32 decisions, the
  fixed-point cell words) against the same oracle in its plain FP64 mode, one
  step from the same float32-representable state: velocities, body momenta
  and positions within the FP32 bar (1e-5 of the thermal scale, one float32
  rounding of the box edge).
* The comparison itself: a planted velocity error is reported at its size; a
  particle moved into another cell is counted as a split cell and its cell is
  left out of the velocity comparison; a planted body error is reported.
"""
import numpy as np
import pytest

import oracle as O
from oracle import parity as OP
from paper_2604_14307_gb300 import inputs as I


def fp32_oracle_step(system, st):
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)
    O.stream(osys, ost)
    tr = O.collide(osys, ost)
    ost.step += 1
    return ost, tr["cell_site"][:osys.n_sites].copy(), tr["shift"].copy()


@pytest.mark.parametrize("rule,thermo", [(I.SRD, 1), (I.AT, 0), (I.SRD, 0)])
def test_fp32_mode_is_within_the_bar_of_fp64(rule, thermo):
    system = I.suspension(12, 5.0, 0.15, 2.0, 2, 5.0, rule, thermo, I.P32, seed=3, name="e")
    st = I.initial_state(system)
    g, sc, sh = fp32_oracle_step(system, st)
    r = OP.compare(system, st, g, sc, sh)
    assert r["v"] <= 1e-5 and r["P"] <= 1e-5 and r["L"] <= 1e-5, r
    assert r["x"] <= 2.0**-23, r
    assert r["split_cells"] == 0
    # the two modes really differ (float32 storage): not a comparison of equals
    assert r["v"] > 0.0 and r["x"] > 0.0


def test_comparison_reports_planted_errors():
    system = I.suspension(12, 5.0, 0.15, 2.0, 2, 5.0, I.SRD, 1, I.P32, seed=4, name="e")
    st = I.initial_state(system)
    g, sc, sh = fp32_oracle_step(system, st)
    ref = OP.fp64_reference(system, st)
    base = OP.compare(system, st, g, sc, sh, ref=ref)
    # a velocity error of 3e-4 on one particle of an unsplit cell
    g2 = type(g).__new__(type(g))
    g2.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in g.__dict__.items()})
    g2.v[10, 1] += 3e-4 * (abs(ref[1].v[10, 1]) + 1.0)
    r = OP.compare(system, st, g2, sc, sh, ref=ref)
    assert r["v"] == pytest.approx(3e-4, rel=1e-3)
    # move particle 20 by one cell along x: its old and new cells are split
    g3 = type(g).__new__(type(g))
    g3.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in g.__dict__.items()})
    g3.x[20, 0] = (g3.x[20, 0] + 1.0) % system.L_array()[0][0]
    g3.v[20, 0] += 1.0                                   # and give it a wrong velocity
    r = OP.compare(system, st, g3, sc, sh, ref=ref)
    assert r["split_cells"] == 2 and r["split_particles"] == 1
    assert r["v"] == pytest.approx(base["v"])            # its cell is not compared
    assert r["v_split_cells"] > 0.1
    # a body momentum error
    g4 = type(g).__new__(type(g))
    g4.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in g.__dict__.items()})
    g4.P[0, 2] += 1e-3 * (abs(ref[1].P[0, 2]) + np.sqrt(system.shapes[0].m.sum()))
    r = OP.compare(system, st, g4, sc, sh, ref=ref)
    assert r["P"] == pytest.approx(1e-3, rel=1e-3)
