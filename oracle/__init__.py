"""FP64 CPU oracle for the MPCD + rigid-body step (arXiv 2604.14307).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
the benchmark's CPU-baseline leg may import this module.  It shares no code
with the CUDA path: it compiles its own C source (``mpcd_oracle.c``) with gcc
and calls it through ctypes.  System descriptions are read duck-typed from the
objects built by the seeded input generator (``paper_2604_14307_gb300.inputs``),
which it does not import.

Parity status of each function is recorded in the C source header and in the
design notes; every function here is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpcd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

P64, P32 = 0, 1
SRD, AT = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle (FP64, no fused multiply-add) into oracle/_build."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        # with OpenMP where the compiler has it (orc_set_threads; one thread by default)
        if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
            subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Sys(C.Structure):
    _fields_ = [("kT", C.c_double), ("dt", C.c_double), ("alpha_deg", C.c_double),
                ("m_solvent", C.c_double), ("rule", C.c_int32), ("thermostat", C.c_int32),
                ("precision", C.c_int32), ("naive_transfer", C.c_int32), ("seed", C.c_uint64),
                ("n_rep", C.c_int32), ("L", C.c_void_p), ("solv_off", C.c_void_p),
                ("body_off", C.c_void_p), ("n_shapes", C.c_int32), ("site_off", C.c_void_p),
                ("b", C.c_void_p), ("m", C.c_void_p), ("cent_off", C.c_void_p),
                ("cent", C.c_void_p), ("wca_d", C.c_void_p), ("body_shape", C.c_void_p),
                ("stream_id", C.c_void_p), ("f_ext", C.c_void_p), ("angular", C.c_int32)]


class _State(C.Structure):
    _fields_ = [("x", C.c_void_p), ("v", C.c_void_p), ("R", C.c_void_p), ("q", C.c_void_p),
                ("P", C.c_void_p), ("Lm", C.c_void_p), ("F", C.c_void_p), ("T", C.c_void_p),
                ("step", C.c_int64), ("D", C.c_void_p)]


_TRACE_FIELDS = ["shift", "cell_solvent", "cell_site", "site_r", "site_v", "site_vpost",
                 "fixed", "sums", "cell_u", "cell_axis", "cell_kappa", "cell_xibar",
                 "order", "cell_start", "dP", "dL", "cell_omega"]


class _Trace(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in _TRACE_FIELDS]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            _lib.orc_cell_axis.argtypes = [C.c_double, C.c_int32, C.c_int32]
            _lib.orc_cell_axis.restype = C.c_int32
            _lib.orc_grid_shift.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_void_p]
            _lib.orc_srd_axis.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_uint32, C.c_void_p]
            _lib.orc_thermostat_energy.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_uint32, C.c_int64]
            _lib.orc_thermostat_energy.restype = C.c_double
            for fn in ("orc_forces",):
                getattr(_lib, fn).argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            for fn in ("orc_stream",):
                getattr(_lib, fn).argtypes = [C.c_void_p, C.c_void_p]
            _lib.orc_collide.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            _lib.orc_step.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
            _lib.orc_rigid_site_velocities.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            _lib.orc_body_energies.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            _lib.orc_wca.argtypes = [C.c_double, C.c_double, C.c_void_p, C.c_void_p]
            _lib.orc_rotation_matrix.argtypes = [C.c_void_p, C.c_void_p]
            _lib.orc_normals.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_uint32,
                                         C.c_uint32, C.c_void_p]
            _lib.orc_set_threads.argtypes = [C.c_int]
            _lib.orc_set_threads.restype = C.c_int
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleSystem:
    """ctypes view of a system description (keeps the arrays alive)."""

    def __init__(self, system, **overrides):
        p = system.params
        self.system = system
        self.L = np.ascontiguousarray(system.L_array(), dtype=np.int32)
        self.solv_off = np.ascontiguousarray(system.solvent_offsets(), dtype=np.int64)
        self.body_off = np.ascontiguousarray(system.body_offsets(), dtype=np.int64)
        so, b, m, co, cen, d = system.shape_tables()
        self.site_off, self.b, self.m = so, b, m
        self.cent_off, self.cent, self.wca_d = co, cen, d
        self.stream_id = np.ascontiguousarray(system.stream_ids(), dtype=np.int32)
        self.body_shape = np.ascontiguousarray(system.body_shape_array(), dtype=np.int32)
        if self.body_shape.size == 0:
            self.body_shape = np.zeros(1, dtype=np.int32)
        vals = dict(kT=p.kT, dt=p.dt, alpha_deg=p.alpha_deg, m_solvent=p.m_solvent,
                    rule=p.rule, thermostat=p.thermostat, precision=p.precision,
                    naive_transfer=p.naive_transfer, seed=p.seed, angular=getattr(p, "angular", 0))
        vals.update(overrides)
        self.params = vals
        self.c = _Sys(vals["kT"], vals["dt"], vals["alpha_deg"], vals["m_solvent"],
                      vals["rule"], vals["thermostat"], vals["precision"],
                      vals["naive_transfer"], vals["seed"], len(self.L), _ptr(self.L),
                      _ptr(self.solv_off), _ptr(self.body_off), len(system.shapes),
                      _ptr(self.site_off), _ptr(self.b), _ptr(self.m), _ptr(self.cent_off),
                      _ptr(self.cent), _ptr(self.wca_d), _ptr(self.body_shape),
                      _ptr(self.stream_id), None, vals["angular"])
        self.f_ext = None
        self.n_solvent = int(self.solv_off[-1])
        self.n_bodies = int(self.body_off[-1])
        sizes = [int(so[s + 1] - so[s]) for s in self.body_shape[: self.n_bodies]]
        self.site_base = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.n_sites = int(self.site_base[-1])
        self.cell_base = np.concatenate([[0], np.cumsum(np.prod(self.L, axis=1))]).astype(np.int64)
        self.n_cells = int(self.cell_base[-1])

    def set_body_force(self, f):
        """Constant force on every body at its centre of mass, balanced on the
        solvent (Sec. III.B sedimentation); None or zeros: none."""
        if f is None or not np.any(np.asarray(f, dtype=np.float64)):
            self.f_ext = None
            self.c.f_ext = None
        else:
            self.f_ext = np.ascontiguousarray(f, dtype=np.float64).reshape(3).copy()
            self.c.f_ext = _ptr(self.f_ext)


class OracleState:
    """Oracle state arrays: solvent (x, v), bodies (R, q, P, Lm, F, T)."""

    def __init__(self, osys: OracleSystem, st, compute_forces: bool = True):
        self.x = np.ascontiguousarray(st.x, dtype=np.float64).copy()
        self.v = np.ascontiguousarray(st.v, dtype=np.float64).copy()
        self.R = np.ascontiguousarray(st.R, dtype=np.float64).copy().reshape(-1, 3)
        self.q = np.ascontiguousarray(st.q, dtype=np.float64).copy().reshape(-1, 4)
        self.P = np.ascontiguousarray(st.P, dtype=np.float64).copy().reshape(-1, 3)
        self.Lm = np.ascontiguousarray(st.Lm, dtype=np.float64).copy().reshape(-1, 3)
        nb = max(1, self.R.shape[0])
        self.F = np.zeros((nb, 3))
        self.T = np.zeros((nb, 3))
        self.D = np.zeros((nb, 3))      # unwrapped body displacement since construction
        self.step = int(st.step)
        self.osys = osys
        if compute_forces:
            forces(osys, self)

    def c(self) -> _State:
        self._keep = []

        def pp(a):
            if a.size:
                return _ptr(a)
            z = np.zeros(4)
            self._keep.append(z)
            return _ptr(z)
        self._c = _State(pp(self.x), pp(self.v), pp(self.R), pp(self.q), pp(self.P),
                         pp(self.Lm), pp(self.F), pp(self.T), self.step, pp(self.D))
        return self._c

    def sync(self):
        self.step = int(self._c.step)


def forces(osys: OracleSystem, st: OracleState) -> float:
    e = np.zeros(1)
    cs = st.c()
    lib().orc_forces(C.byref(osys.c), C.byref(cs), _ptr(e))
    return float(e[0])


def stream(osys: OracleSystem, st: OracleState) -> None:
    cs = st.c()
    rc = lib().orc_stream(C.byref(osys.c), C.byref(cs))
    if rc:
        raise RuntimeError(f"oracle stream failed ({rc})")


def collide(osys: OracleSystem, st: OracleState, trace: bool = True) -> dict:
    """One collision keyed on st.step (a2-a8); returns the per-collision trace."""
    out = {}
    tr = _Trace()
    if trace:
        Ns, Nsite, Ct, B, R = osys.n_solvent, osys.n_sites, osys.n_cells, osys.n_bodies, len(osys.L)
        nw = 6
        shapes = dict(shift=((R, 3), np.int32), cell_solvent=((Ns,), np.int32),
                      cell_site=((Nsite,), np.int32), site_r=((Nsite, 3), np.float64),
                      site_v=((Nsite, 3), np.float64), site_vpost=((Nsite, 3), np.float64),
                      fixed=((nw, Ct), np.int64), sums=((6, Ct), np.float64),
                      cell_u=((Ct, 3), np.float64), cell_axis=((Ct, 3), np.float64),
                      cell_kappa=((Ct,), np.float64), cell_xibar=((Ct, 3), np.float64),
                      order=((Ns + Nsite,), np.int64), cell_start=((Ct + 1,), np.int64),
                      dP=((max(B, 1), 3), np.float64), dL=((max(B, 1), 3), np.float64),
                      cell_omega=((Ct, 3), np.float64))
        for k, (shp, dt) in shapes.items():
            a = np.zeros(shp, dtype=dt)
            if a.size == 0:
                a = np.zeros(max(1, a.size), dtype=dt)
            out[k] = a
            setattr(tr, k, _ptr(a))
    cs = st.c()
    rc = lib().orc_collide(C.byref(osys.c), C.byref(cs), C.byref(tr) if trace else None)
    if rc:
        raise RuntimeError(f"oracle collide failed ({rc})")
    return out


def step(osys: OracleSystem, st: OracleState, n: int = 1) -> None:
    cs = st.c()
    rc = lib().orc_step(C.byref(osys.c), C.byref(cs), n)
    st.sync()
    if rc:
        raise RuntimeError(f"oracle step failed ({rc})")


def rigid_site_velocities(osys: OracleSystem, st: OracleState) -> np.ndarray:
    out = np.zeros((max(osys.n_sites, 1), 3))
    cs = st.c()
    rc = lib().orc_rigid_site_velocities(C.byref(osys.c), C.byref(cs), _ptr(out))
    if rc:
        raise RuntimeError("singular inertia tensor")
    return out[: osys.n_sites]


def body_energies(osys: OracleSystem, st: OracleState):
    ET = np.zeros(max(osys.n_bodies, 1))
    ER = np.zeros(max(osys.n_bodies, 1))
    cs = st.c()
    lib().orc_body_energies(C.byref(osys.c), C.byref(cs), _ptr(ET), _ptr(ER))
    return ET[: osys.n_bodies], ER[: osys.n_bodies]


def set_threads(n: int) -> int:
    """Threads of the oracle's independent per-particle and per-cell loops
    (OpenMP; the results do not depend on it).  Returns the count in use: 1 if
    the oracle was built without OpenMP."""
    return int(lib().orc_set_threads(int(n)))


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def srd_axis(osys: OracleSystem, rep: int, step_: int, cell: int) -> np.ndarray:
    """SRD rotation axis of replica-local cell `cell` at collision `step_`."""
    out = np.zeros(3)
    lib().orc_srd_axis(C.byref(osys.c), int(rep), int(step_), int(cell), _ptr(out))
    return out


def thermostat_energy(osys: OracleSystem, rep: int, step_: int, cell: int, n: int) -> float:
    """E' of the cell-level thermostat for a cell of n particles (Eq. 6)."""
    return float(lib().orc_thermostat_energy(C.byref(osys.c), int(rep), int(step_), int(cell), int(n)))


def grid_shift(osys: OracleSystem, rep: int, step_: int) -> np.ndarray:
    S = np.zeros(3, dtype=np.int32)
    lib().orc_grid_shift(C.byref(osys.c), rep, step_, _ptr(S))
    return S


def cell_axis(x: float, S: int, L: int) -> int:
    return int(lib().orc_cell_axis(float(x), int(S), int(L)))


def wca(r: float, d: float):
    u, f = np.zeros(1), np.zeros(1)
    lib().orc_wca(r, d, _ptr(u), _ptr(f))
    return float(u[0]), float(f[0])


def rotation_matrix(q) -> np.ndarray:
    qq = np.ascontiguousarray(q, dtype=np.float64)
    Q = np.zeros((3, 3))
    lib().orc_rotation_matrix(_ptr(qq), _ptr(Q))
    return Q


def normals(osys: OracleSystem, rep: int, step_: int, ids, tag: int) -> np.ndarray:
    """The three Box-Muller normals of each id (one Philox block per id)."""
    ids = np.asarray(ids, dtype=np.int64)
    out = np.zeros((len(ids), 3))
    one = np.zeros(3)
    for k, i in enumerate(ids):
        lib().orc_normals(C.byref(osys.c), rep, step_, int(i), tag, _ptr(one))
        out[k] = one
    return out


TAG_SHIFT, TAG_AXIS, TAG_THERMO, TAG_THERMO_ODD, TAG_SITE, TAG_AT = 1, 2, 3, 4, 5, 6


# --------------------------------------------------------------------------
# Transport protocols of Sec. III.B (shear viscosity, Eq. 14)
# --------------------------------------------------------------------------
def rnemd_exchange(osys: OracleSystem, st: OracleState, y_a: float, y_b: float, width: float,
                   v_target: float, max_pairs: int, rep: int = 0):
    """Reverse non-equilibrium (Mueller-Plathe) momentum exchange, Sec. III.B.

    The solvent particles of slab A, y in [y_a, y_a + width), are ranked by how
    close their v_x is to +v_target, those of slab B, y in [y_b, y_b + width), by
    how close it is to -v_target (ascending |v_x -+ v_target|, equal distances by
    particle id); the first min(max_pairs, n_A, n_B) of each ranking are paired in
    rank order and every pair exchanges v_x.  In the P32 form the slab test and
    the distances are evaluated on the stored float32 values in float32, the
    precision in which that form takes these decisions.  Returns (x momentum
    moved from A to B = sum of m (v_A - v_B), number of pairs).  Modifies st.v.
    """
    so = osys.solv_off
    i0, i1 = int(so[rep]), int(so[rep + 1])
    y = st.x[i0:i1, 1]
    vx = st.v[i0:i1, 0]
    if osys.params["precision"] == P32:
        f = np.float32
        y, vxk = y.astype(f), vx.astype(f)
        a0, a1, b0, b1 = f(y_a), f(y_a + width), f(y_b), f(y_b + width)
        key_a, key_b = np.abs(vxk - f(v_target)), np.abs(vxk + f(v_target))
    else:
        a0, a1, b0, b1 = y_a, y_a + width, y_b, y_b + width
        key_a, key_b = np.abs(vx - v_target), np.abs(vx + v_target)
    ids = np.arange(i1 - i0)
    in_a = (y >= a0) & (y < a1)
    in_b = (y >= b0) & (y < b1)
    rank_a = ids[in_a][np.lexsort((ids[in_a], key_a[in_a]))]
    rank_b = ids[in_b][np.lexsort((ids[in_b], key_b[in_b]))]
    n = min(int(max_pairs), len(rank_a), len(rank_b))
    pa, pb = rank_a[:n], rank_b[:n]
    va, vb = vx[pa].copy(), vx[pb].copy()
    st.v[i0 + pa, 0] = vb
    st.v[i0 + pb, 0] = va
    m = osys.params["m_solvent"]
    if osys.params["precision"] == P32:
        m = float(np.float32(m))
    return float(np.sum(m * (va - vb))), n


def step_rnemd(osys: OracleSystem, st: OracleState, n: int, y_a: float, y_b: float, width: float,
               v_target: float, max_pairs: int, period: int = 1):
    """n whole steps with the exchange before the collision of every step whose
    index is a multiple of `period` (after streaming, the order of the stream,
    collide sequence of Sec. II).  Returns the summed (momentum, pairs)."""
    dp, npairs = 0.0, 0
    for _ in range(n):
        stream(osys, st)
        if st.step % period == 0:
            d, k = rnemd_exchange(osys, st, y_a, y_b, width, v_target, max_pairs)
            dp += d
            npairs += k
        collide(osys, st, trace=False)
        st.step += 1
    return dp, npairs
