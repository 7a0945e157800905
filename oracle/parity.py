"""Error of the FP32 form against the plain FP64 method, one step.

TEST INFRASTRUCTURE ONLY (the test-suite and the benchmark's CPU-baseline leg).
The oracle runs the step in its plain FP64 mode (no float32 decision, no
fixed-point word) from the same float32-representable state that the FP32 run
starts from; the FP32 result is then compared element by element.

Positions of the two runs differ by the float32 rounding of x + v dt, so a
particle within that distance of a shifted cell face can land in another cell
in the two runs.  Every cell that holds such a particle in either run is
"split": its members' velocities and the bodies with a site in it are left out
of the element-wise comparison and counted instead.  Everything else is
compared with the relative measures the FP32 parity bar uses:
  velocities   |v32 - v64| / (|v64| + sqrt(kT/m))
  body P       |P32 - P64| / (|P64| + sqrt(M kT))
  body L       |L32 - L64| / (|L64| + sqrt(I kT))
  positions    |x32 - x64| / L   (L the box edge)
"""
from __future__ import annotations

import numpy as np

from . import OracleState, OracleSystem, P64, collide, stream


def cells_from_positions(x: np.ndarray, S: np.ndarray, L) -> np.ndarray:
    """Replica-local cells of positions x [n][3] under the integer shift S:
    floor((floor(x 2^20) - S) / 2^20) mod L per axis (the binning reading)."""
    X = np.floor(np.asarray(x, dtype=np.float64) * 2.0**20).astype(np.int64)
    c = ((X - np.asarray(S, dtype=np.int64)[None, :]) >> 20) % np.asarray(L, dtype=np.int64)[None, :]
    return c[:, 0] + L[0] * (c[:, 1] + L[1] * c[:, 2])


def fp64_reference(system, st):
    """One whole step (stream, then collision) of the plain FP64 oracle from st.
    Returns (oracle system, state after the step, collision trace)."""
    osys = OracleSystem(system, precision=P64)
    ost = OracleState(osys, st)
    stream(osys, ost)
    tr = collide(osys, ost)
    ost.step += 1
    return osys, ost, tr


def compare(system, st, g, site_cell, shift, ref=None, params=None) -> dict:
    """Compare an FP32-form step (g: state after one step from st; site_cell,
    shift: the GPU's site cells and grid shifts of that collision; params: its
    per-cell collision records, if given) with the FP64 oracle.  Returns the
    largest relative errors and the split counts.  With the rejection sampler
    of the thermostat (thermostat = 2) the two forms may take a different
    accept/reject decision in a rare cell; such cells (kappa differing by more
    than 1e-3 relative) are counted as `thermostat_flips` and, like split
    cells, left out of the velocity comparison."""
    osys, ost, tr = ref if ref is not None else fp64_reference(system, st)
    p = system.params
    Ls = system.L_array()
    so, bo = system.solvent_offsets(), system.body_offsets()
    # per replica: members whose cell differs between the runs -> split cells
    split = np.zeros(osys.n_cells, dtype=bool)
    gcell_s = np.zeros(osys.n_solvent, dtype=np.int64)
    for r in range(len(Ls)):
        i0, i1 = so[r], so[r + 1]
        if i1 > i0:
            gcell_s[i0:i1] = cells_from_positions(g.x[i0:i1], shift[r], Ls[r]) + osys.cell_base[r]
    ocell_s = tr["cell_solvent"][:osys.n_solvent].astype(np.int64)
    for r in range(len(Ls)):
        ocell_s[so[r]:so[r + 1]] += osys.cell_base[r]
    bad = gcell_s != ocell_s
    split[gcell_s[bad]] = True
    split[ocell_s[bad]] = True
    n_split_particles = int(bad.sum())
    site_rep = np.repeat(np.arange(len(Ls)), np.diff(osys.site_base[bo]))
    if osys.n_sites:
        gsite = np.asarray(site_cell, dtype=np.int64)[:osys.n_sites] + osys.cell_base[site_rep]
        osite = tr["cell_site"][:osys.n_sites].astype(np.int64) + osys.cell_base[site_rep]
        sbad = gsite != osite
        split[gsite[sbad]] = True
        split[osite[sbad]] = True
        n_split_particles += int(sbad.sum())
    else:
        gsite = np.zeros(0, dtype=np.int64)
    flips = np.zeros(osys.n_cells, dtype=bool)
    if params is not None and p.rule == 0 and p.thermostat:
        kg = np.asarray(params, dtype=np.float64)[:, 3]
        ko = tr["cell_kappa"][:osys.n_cells]
        live = (tr["sums"][0] >= 2) & ~split
        flips = live & (np.abs(kg - ko) > 1e-3 * np.abs(ko))
    keep = ~(split | flips)[ocell_s]
    sv = np.sqrt(p.kT / p.m_solvent)
    ev = np.abs(g.v - ost.v) / (np.abs(ost.v) + sv)
    out = dict(n_solvent=int(osys.n_solvent), n_bodies=int(osys.n_bodies), n_cells=int(osys.n_cells),
               split_cells=int(split.sum()), split_particles=n_split_particles,
               thermostat_flips=int(flips.sum()),
               v=float(ev[keep].max()) if keep.any() else 0.0,
               v_split_cells=float(ev[~keep].max()) if (~keep).any() else 0.0)
    xe = np.zeros(0)
    for r in range(len(Ls)):
        i0, i1 = so[r], so[r + 1]
        if i1 > i0:
            xe = np.concatenate([xe, (np.abs(g.x[i0:i1] - ost.x[i0:i1]) / np.asarray(Ls[r])[None, :]).ravel()])
    # a coordinate near 0 may wrap to near L in one run only
    xe = np.minimum(xe, np.abs(1.0 - xe))
    out["x"] = float(xe.max()) if xe.size else 0.0
    if osys.n_bodies:
        body_split = np.zeros(osys.n_bodies, dtype=bool)
        site_body = np.repeat(np.arange(osys.n_bodies), np.diff(osys.site_base))
        body_split[site_body[(split | flips)[gsite]]] = True
        Ms = np.array([system.shapes[s].m.sum() for s in system.body_shape_array()])
        from_inertia = [np.asarray(_inertia_diag(system.shapes[s])).max() for s in system.body_shape_array()]
        Is = np.array(from_inertia)
        eP = np.abs(g.P - ost.P) / (np.abs(ost.P) + np.sqrt(Ms * p.kT)[:, None])
        eL = np.abs(g.Lm - ost.Lm) / (np.abs(ost.Lm) + np.sqrt(Is * p.kT)[:, None])
        ok = ~body_split
        out.update(P=float(eP[ok].max()) if ok.any() else 0.0, L=float(eL[ok].max()) if ok.any() else 0.0,
                   split_bodies=int(body_split.sum()))
    return out


def _inertia_diag(shape):
    b, m = np.asarray(shape.b, dtype=np.float64), np.asarray(shape.m, dtype=np.float64)
    r2 = (b * b).sum(1)
    return np.array([(m * (r2 - b[:, k] ** 2)).sum() for k in range(3)])
