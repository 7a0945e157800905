"""The oracle's all-core form: its per-particle and per-cell loops run on
several host threads (OpenMP) with every output computed by the same
arithmetic in the same order, so a run on four threads equals the run on one
thread bit for bit (FP32 and FP64 forms, SRD with either thermostat sampler and
MPCD-AT, with colloids, several steps)."""
import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I


@pytest.mark.parametrize("prec,rule,thermo", [(I.P32, I.SRD, 1), (I.P64, I.SRD, 2), (I.P32, I.AT, 0),
                                              (I.P64, I.AT, 0)])
def test_threads_do_not_change_the_result(prec, rule, thermo):
    system = I.suspension(14, 5.0, 0.15, 2.0, 2, 5.0, rule, thermo, prec, seed=5, name="omp")
    st = I.initial_state(system)
    out = []
    for n in (1, 4):
        used = O.set_threads(n)
        assert used in (1, n)
        osys = O.OracleSystem(system)
        ost = O.OracleState(osys, st)
        O.step(osys, ost, 3)
        out.append(ost)
    O.set_threads(1)
    for k in ("x", "v", "R", "q", "P", "Lm"):
        assert np.array_equal(getattr(out[0], k), getattr(out[1], k)), k


def test_threads_with_the_collision_trace():
    system = I.suspension(12, 5.0, 0.15, 2.0, 2, 5.0, I.SRD, 1, I.P32, seed=6, name="omp_tr")
    st = I.initial_state(system)
    trs = []
    for n in (1, 3):
        O.set_threads(n)
        osys = O.OracleSystem(system)
        ost = O.OracleState(osys, st)
        O.stream(osys, ost)
        trs.append((O.collide(osys, ost), ost.v.copy()))
    O.set_threads(1)
    for k in ("fixed", "sums", "cell_kappa", "order", "cell_start", "dP", "dL"):
        assert np.array_equal(trs[0][0][k], trs[1][0][k]), k
    assert np.array_equal(trs[0][1], trs[1][1])
