"""Error of the FP32 form (FP32 state, integer fixed-point cell sums, FP64
bodies) against the plain FP64 method, and its per-cell momentum.

1. One GPU step of the FP32 form from float32-representable inputs against one
   step of the oracle in its plain FP64 mode (no float32 decision, no
   fixed-point word; oracle.parity): velocities within 1e-5 (|v| + sqrt(kT/m)),
   body momenta within 1e-5 of their thermal scale, positions within one
   float32 rounding of the box edge.  Cells split by a binning difference
   (a particle within one float32 rounding of a shifted cell face lands in
   another cell in the two runs) are counted, not compared; there may be only
   a handful of them.
2. Per-cell momentum of the plain rules on the GPU's own data (Sec. II.A: the
   collision conserves each cell's momentum; with the exact fixed-point sums
   the FP32 form adds only the float32 evaluation of the rule).  In every cell
   that holds no colloid site, |sum m (v' - v)| is measured in units of
   N_c m ulp(max |v|, |v'|): each new velocity comes from about ten float32
   operations on values no larger than that maximum, which bounds the ratio by
   a few units; the test asserts a mean below 1/2 and a maximum of 4
   (measured 0.23-0.29 and 1.6-2.4; with the former 2^-20 momentum words,
   1.4-1.5 and 10-19).
"""
import numpy as np
import pytest

import oracle as O
from oracle import parity as OP
from paper_2604_14307_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14307_gb300 import binding, build_lib
    build_lib.build()
    return binding


def gpu_step(B, system, st):
    """one unpipelined step; returns (state after, site cells, shifts, v before, v after, x)"""
    sim = B.Simulation(system, sort_period=-1)
    sim.set_debug(True)
    sim.set_state(st)
    sim.stream()
    sim.couple(B.MPCD_PRE)
    before = sim.get_state()
    sim.collide()
    d = sim.debug_cells()
    sim.couple(B.MPCD_POST)
    g = sim.get_state()
    sim.close()
    return g, d, before


CASES = {
    "sphere_L10_srd": lambda: I.single_sphere_L10(I.P32),
    "suspension_L16_srd_thermostat": lambda: I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, I.SRD, 1, I.P32, seed=3,
                                                          name="err_srd"),
    "suspension_L16_srd_thermostat_mt": lambda: I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, I.SRD, 2, I.P32, seed=3,
                                                             name="err_srd_mt"),
    "suspension_L16_at": lambda: I.suspension(16, 5.0, 0.15, 2.0, 2, 5.0, I.AT, 0, I.P32, seed=3, name="err_at"),
    "suspension_L50_at": lambda: I.suspension_L50(I.P32),
}


@pytest.mark.parametrize("case", list(CASES))
def test_fp32_form_against_fp64_method(B, case):
    system = CASES[case]()
    st = I.initial_state(system)
    g, d, _ = gpu_step(B, system, st)
    r = OP.compare(system, st, g, d["site_cell"], d["shift"], params=d["params"])
    print(case, r)
    assert r["v"] <= TOL, r
    assert r["x"] <= 2.0**-23, r
    if system.n_bodies:
        assert r["P"] <= TOL and r["L"] <= TOL, r
        assert r["split_bodies"] <= max(2, system.n_bodies // 50), r
    # binning differences are rare: one float32 rounding of a coordinate
    assert r["split_cells"] <= max(4, r["n_cells"] // 10000), r
    # so are different accept/reject decisions of the rejection sampler
    assert r["thermostat_flips"] <= max(1, r["n_cells"] // 100000), r


def cell_momentum_change(system, before, after, d):
    """per solvent-only cell: (sum m (v' - v) [3], N_c, max |component| of v and v')"""
    Ls = system.L_array()
    so = system.solvent_offsets()
    C = int(np.prod(Ls, axis=1).sum())
    cb = np.concatenate([[0], np.cumsum(np.prod(Ls, axis=1))])
    cell = np.zeros(system.n_solvent, dtype=np.int64)
    for r in range(len(Ls)):
        i0, i1 = so[r], so[r + 1]
        cell[i0:i1] = OP.cells_from_positions(before.x[i0:i1], d["shift"][r], Ls[r]) + cb[r]
    has_site = np.zeros(C, dtype=bool)
    if system.n_sites:
        bo = system.body_offsets()
        sizes = [system.shapes[s].n_sites for s in system.body_shape_array()]
        site_rep = np.repeat(np.repeat(np.arange(len(Ls)), np.diff(bo)), sizes)
        has_site[d["site_cell"].astype(np.int64) + cb[site_rep]] = True
    m = float(np.float32(system.params.m_solvent))
    dp = np.zeros((C, 3))
    for k in range(3):
        # exact: float32 values summed in float64 (<= 2^10 terms of 24-bit mantissas)
        dp[:, k] = np.bincount(cell, weights=m * after.v[:, k], minlength=C) - \
            np.bincount(cell, weights=m * before.v[:, k], minlength=C)
    n = np.bincount(cell, minlength=C)
    vmax = np.zeros(C)
    np.maximum.at(vmax, cell, np.maximum(np.abs(before.v).max(1), np.abs(after.v).max(1)))
    return dp, n, vmax, ~has_site


@pytest.mark.parametrize("rule,thermo", [(I.SRD, 0), (I.SRD, 1), (I.AT, 0)])
def test_per_cell_momentum_is_conserved_to_float_rounding(B, rule, thermo):
    system = I.suspension(20, 5.0, 0.15, 2.0, 2, 5.0, rule, thermo, I.P32, seed=7, name="cellp")
    st = I.initial_state(system)
    g, d, before = gpu_step(B, system, st)
    dp, n, vmax, solvent_only = cell_momentum_change(system, before, g, d)
    m = float(np.float32(system.params.m_solvent))
    ulp = np.spacing(vmax.astype(np.float32)).astype(np.float64)
    bound = n * m * ulp
    sel = solvent_only & (n >= 2)
    ratio = np.abs(dp[sel]).max(1) / bound[sel]
    print(rule, thermo, "cells", int(sel.sum()), "max |dP| / (N m ulp)", float(ratio.max()),
          "mean", float(ratio.mean()))
    assert ratio.mean() <= 0.5 and ratio.max() <= 4.0, (float(ratio.mean()), float(ratio.max()))
