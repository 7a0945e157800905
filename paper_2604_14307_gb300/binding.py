"""Thin ctypes binding of the C ABI in include/mpcd.h (libmpcd.so).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device memory comes from PyTorch's caching allocator (through
the ABI's allocator callbacks) and work is enqueued on PyTorch's current CUDA
stream when PyTorch is available; otherwise the library allocates with
cudaMalloc and uses the legacy default stream.  If the library cannot be
loaded, every entry point raises - there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import inputs as I

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmpcd.so")

MPCD_OK, MPCD_ERR_ARG, MPCD_ERR_CUDA, MPCD_ERR_OOM, MPCD_ERR_TIMEOUT, MPCD_ERR_STATE = 0, -1, -2, -3, -4, -5
MPCD_PRE, MPCD_POST = 0, 1
_STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "out of device memory",
           -4: "device wait timed out", -5: "invalid device state"}

# every function the header declares (the CPU test checks they are exported)
EXPORTS = ["mpcd_create", "mpcd_destroy", "mpcd_set_state", "mpcd_get_state", "mpcd_stream",
           "mpcd_couple", "mpcd_collide", "mpcd_step", "mpcd_sort", "mpcd_diagnostics",
           "mpcd_sizes", "mpcd_last_error", "mpcd_set_debug", "mpcd_debug_cells",
           "mpcd_set_profiling", "mpcd_get_profile", "mpcd_reset_profile", "mpcd_get_tuning",
           "mpcd_set_tuning", "mpcd_autotune", "mpcd_collide_solvent_static", "mpcd_set_rnemd",
           "mpcd_rnemd_totals", "mpcd_velocity_profile", "mpcd_set_body_force",
           "mpcd_body_displacements", "mpcd_set_vacf", "mpcd_get_vacf", "mpcd_cell_order",
           "mpcd_create_slab", "mpcd_slab_set_state", "mpcd_slab_get_state", "mpcd_slab_extract",
           "mpcd_slab_export", "mpcd_slab_insert", "mpcd_collide_begin", "mpcd_collide_end",
           "mpcd_layer_words", "mpcd_couple_post_partial", "mpcd_apply_impulse"]


class MPCDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)} ({status}): {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("kT", C.c_double), ("dt", C.c_double), ("alpha_deg", C.c_double),
                ("m_solvent", C.c_double), ("rule", C.c_int32), ("thermostat", C.c_int32),
                ("precision", C.c_int32), ("naive_transfer", C.c_int32), ("seed", C.c_uint64),
                ("sort_period", C.c_int32), ("angular", C.c_int32)]


class ShapeDesc(C.Structure):
    _fields_ = [("n_sites", C.c_int32), ("b", C.c_void_p), ("m", C.c_void_p),
                ("n_centres", C.c_int32), ("centres", C.c_void_p), ("wca_d", C.c_double)]


class ReplicaDesc(C.Structure):
    _fields_ = [("L", C.c_int32 * 3), ("n_solvent", C.c_int64), ("n_bodies", C.c_int32),
                ("stream_id", C.c_int32), ("body_shape", C.c_void_p)]


AllocFn = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FreeFn = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", AllocFn), ("free", FreeFn), ("user", C.c_void_p)]


class HostState(C.Structure):
    _fields_ = [("x", C.c_void_p), ("v", C.c_void_p), ("R", C.c_void_p), ("q", C.c_void_p),
                ("P", C.c_void_p), ("Lm", C.c_void_p), ("step", C.c_int64)]


class Sizes(C.Structure):
    _fields_ = [("n_solvent", C.c_int64), ("n_bodies", C.c_int64), ("n_sites", C.c_int64),
                ("n_cells", C.c_int64), ("n_replicas", C.c_int32), ("n_shapes", C.c_int32),
                ("device_bytes", C.c_int64), ("sum_words", C.c_int32), ("param_bytes", C.c_int32)]


class Diag(C.Structure):
    _fields_ = [("p_solvent", C.c_double * 3), ("p_bodies", C.c_double * 3),
                ("ke_solvent", C.c_double), ("ke_trans", C.c_double), ("ke_rot", C.c_double),
                ("step", C.c_int64)]


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("bytes_per_launch", C.c_double)]


class Rnemd(C.Structure):
    _fields_ = [("enabled", C.c_int32), ("max_pairs", C.c_int32), ("period", C.c_int32),
                ("reserved", C.c_int32), ("y_a", C.c_double), ("y_b", C.c_double), ("width", C.c_double),
                ("v_target", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("block", C.c_int32), ("tile", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("sort_period", C.c_int32), ("staged", C.c_int32)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libmpcd.so; raises if it is missing (build it with build_lib.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run paper_2604_14307_gb300.build_lib.build())")
        lib = C.CDLL(path)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "mpcd_create": [C.POINTER(Params), i32, vp, i32, vp, vp, i32, C.POINTER(vp)],
            "mpcd_destroy": [vp],
            "mpcd_set_state": [vp, C.POINTER(HostState), vp],
            "mpcd_get_state": [vp, C.POINTER(HostState), vp],
            "mpcd_stream": [vp, vp],
            "mpcd_couple": [vp, i32, vp],
            "mpcd_collide": [vp, vp],
            "mpcd_step": [vp, i64, vp],
            "mpcd_sort": [vp, i32, vp],
            "mpcd_diagnostics": [vp, C.POINTER(Diag), vp],
            "mpcd_sizes": [vp, C.POINTER(Sizes)],
            "mpcd_set_debug": [vp, i32],
            "mpcd_debug_cells": [vp, vp, vp, vp, vp, vp, vp],
            "mpcd_set_profiling": [vp, i32],
            "mpcd_get_profile": [vp, vp, i32],
            "mpcd_reset_profile": [vp],
            "mpcd_get_tuning": [vp, C.POINTER(Tuning)],
            "mpcd_set_tuning": [vp, C.POINTER(Tuning)],
            "mpcd_autotune": [vp, i32, vp],
            "mpcd_set_rnemd": [vp, C.POINTER(Rnemd)],
            "mpcd_set_body_force": [vp, C.POINTER(C.c_double * 3), vp],
            "mpcd_body_displacements": [vp, vp, vp],
            "mpcd_set_vacf": [vp, i32, i32],
            "mpcd_get_vacf": [vp, vp, vp, vp, vp],
            "mpcd_rnemd_totals": [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), vp],
            "mpcd_velocity_profile": [vp, i32, i32, i32, vp, vp, vp],
            "mpcd_cell_order": [vp, vp, vp, vp],
            "mpcd_create_slab": [C.POINTER(Params), i32, vp, C.POINTER(C.c_int32 * 3), i64, i64, i32, vp, i32, i32,
                                 vp, i32, C.POINTER(vp)],
            "mpcd_slab_set_state": [vp, i64, vp, vp, vp, vp, vp, vp, vp, i64, vp],
            "mpcd_slab_get_state": [vp, C.POINTER(C.c_int64), vp, vp, vp, vp, vp, vp, vp, vp],
            "mpcd_slab_extract": [vp, C.POINTER(C.c_int64), vp],
            "mpcd_slab_export": [vp, vp, vp, vp, vp],
            "mpcd_slab_insert": [vp, i64, vp, vp, vp, vp],
            "mpcd_collide_begin": [vp, vp],
            "mpcd_collide_end": [vp, vp],
            "mpcd_layer_words": [vp, i32, i32, vp, i32, vp],
            "mpcd_couple_post_partial": [vp, vp, vp],
            "mpcd_apply_impulse": [vp, vp, vp],
            "mpcd_collide_solvent_static": [C.POINTER(Params), C.POINTER(C.c_int32 * 3), i64, vp, vp, vp,
                                            vp, vp, vp, vp, i64, vp, C.c_char_p, C.c_size_t],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        lib.mpcd_last_error.argtypes = [vp]
        lib.mpcd_last_error.restype = C.c_char_p
        _lib = lib
        return lib


def _torch_cuda():
    try:
        import torch
        if torch.cuda.is_available():
            return torch
    except Exception:
        pass
    return None


def current_stream() -> int:
    t = _torch_cuda()
    return int(t.cuda.current_stream().cuda_stream) if t is not None else 0


class _TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(n, _user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(n), self.device))
            except Exception:
                return None

        def _free(p, _user):
            try:
                torch.cuda.caching_allocator_delete(int(p))
            except Exception:
                pass

        self._a = AllocFn(_alloc)
        self._f = FreeFn(_free)
        self.c = Allocator(self._a, self._f, None)


class Simulation:
    """One MPCD context: all replicas of `system` simulated together on one GPU."""

    def __init__(self, system: I.System, device: int = 0, sort_period: int = 0,
                 use_torch_allocator: bool = True):
        self.lib = load()
        self.system = system
        p = system.params
        self.precision = p.precision
        self.prm = Params(p.kT, p.dt, p.alpha_deg, p.m_solvent, p.rule, p.thermostat,
                          p.precision, p.naive_transfer, p.seed, sort_period, getattr(p, "angular", 0))
        self._keep = []
        shapes = self._shape_descs(system)
        reps = (ReplicaDesc * system.n_rep)()
        sids = system.stream_ids()
        for r, rep in enumerate(system.replicas):
            ids = np.ascontiguousarray(rep.body_shapes, dtype=np.int32)
            self._keep.append(ids)
            reps[r] = ReplicaDesc((C.c_int32 * 3)(*rep.L), rep.n_solvent, len(ids), int(sids[r]),
                                  ids.ctypes.data if len(ids) else None)
        self._alloc = None
        t = _torch_cuda()
        if use_torch_allocator and t is not None:
            self._alloc = _TorchAllocator(device)
        ctx = C.c_void_p()
        rc = self.lib.mpcd_create(C.byref(self.prm), len(system.shapes), C.cast(shapes, C.c_void_p),
                                  system.n_rep, C.cast(reps, C.c_void_p),
                                  C.byref(self._alloc.c) if self._alloc else None, device,
                                  C.byref(ctx))
        if rc != MPCD_OK:
            raise MPCDError(rc, "mpcd_create failed")
        self.ctx = ctx
        self.sizes = Sizes()
        self._check(self.lib.mpcd_sizes(self.ctx, C.byref(self.sizes)))
        self.real = np.float32 if self.precision == I.P32 else np.float64

    def _shape_descs(self, system):
        shapes = (ShapeDesc * max(1, len(system.shapes)))()
        for k, sh in enumerate(system.shapes):
            b = np.ascontiguousarray(sh.b, dtype=np.float64)
            m = np.ascontiguousarray(sh.m, dtype=np.float64)
            cen = np.ascontiguousarray(sh.centres, dtype=np.float64).reshape(-1, 3)
            self._keep += [b, m, cen]
            shapes[k] = ShapeDesc(len(m), b.ctypes.data, m.ctypes.data, len(cen),
                                  cen.ctypes.data if len(cen) else None, sh.wca_d)
        return shapes

    # ------------------------------------------------------------------
    def _check(self, rc: int):
        if rc < 0:
            msg = self.lib.mpcd_last_error(self.ctx).decode() if getattr(self, "ctx", None) else ""
            raise MPCDError(rc, msg)
        return rc

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mpcd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @staticmethod
    def _s(stream):
        return current_stream() if stream is None else int(stream)

    # ------------------------------------------------------------------
    def host_buffers(self, pinned: bool = False):
        """Host state buffers of the right shapes (optionally page-locked via torch)."""
        ns, nb = self.sizes.n_solvent, self.sizes.n_bodies
        if pinned and _torch_cuda() is not None:
            import torch
            dt = torch.float32 if self.real == np.float32 else torch.float64
            mk = lambda shp, d=dt: torch.empty(shp, dtype=d).pin_memory()  # noqa: E731
            t = dict(x=mk((ns, 3)), v=mk((ns, 3)), R=mk((nb, 3), torch.float64),
                     q=mk((nb, 4), torch.float64), P=mk((nb, 3), torch.float64),
                     Lm=mk((nb, 3), torch.float64))
            self._pinned = t
            return {k: v.numpy() for k, v in t.items()}
        return dict(x=np.zeros((ns, 3), self.real), v=np.zeros((ns, 3), self.real),
                    R=np.zeros((nb, 3)), q=np.zeros((nb, 4)), P=np.zeros((nb, 3)),
                    Lm=np.zeros((nb, 3)))

    def _hs(self, b: dict, step: int) -> HostState:
        ptr = lambda a: a.ctypes.data if a.size else None  # noqa: E731
        return HostState(ptr(b["x"]), ptr(b["v"]), ptr(b["R"]), ptr(b["q"]), ptr(b["P"]),
                         ptr(b["Lm"]), step)

    def set_state_buffers(self, b: dict, step: int = 0, stream=None):
        hs = self._hs(b, step)
        self._check(self.lib.mpcd_set_state(self.ctx, C.byref(hs), self._s(stream)))

    def get_state_buffers(self, b: dict, stream=None) -> int:
        hs = self._hs(b, 0)
        self._check(self.lib.mpcd_get_state(self.ctx, C.byref(hs), self._s(stream)))
        return int(hs.step)

    def set_state(self, st: I.State, stream=None):
        b = dict(x=np.ascontiguousarray(st.x, dtype=self.real), v=np.ascontiguousarray(st.v, dtype=self.real),
                 R=np.ascontiguousarray(st.R, dtype=np.float64).reshape(-1, 3),
                 q=np.ascontiguousarray(st.q, dtype=np.float64).reshape(-1, 4),
                 P=np.ascontiguousarray(st.P, dtype=np.float64).reshape(-1, 3),
                 Lm=np.ascontiguousarray(st.Lm, dtype=np.float64).reshape(-1, 3))
        self.set_state_buffers(b, st.step, stream)

    def get_state(self, stream=None) -> I.State:
        b = self.host_buffers()
        step = self.get_state_buffers(b, stream)
        return I.State(x=b["x"].astype(np.float64), v=b["v"].astype(np.float64), R=b["R"], q=b["q"],
                       P=b["P"], Lm=b["Lm"], step=step)

    # ------------------------------------------------------------------ steps
    def stream(self, stream=None):
        self._check(self.lib.mpcd_stream(self.ctx, self._s(stream)))

    def couple(self, phase: int, stream=None):
        self._check(self.lib.mpcd_couple(self.ctx, phase, self._s(stream)))

    def collide(self, stream=None):
        self._check(self.lib.mpcd_collide(self.ctx, self._s(stream)))

    def step(self, n: int = 1, stream=None):
        self._check(self.lib.mpcd_step(self.ctx, int(n), self._s(stream)))

    def sort(self, canonical: bool = False, stream=None):
        self._check(self.lib.mpcd_sort(self.ctx, int(canonical), self._s(stream)))

    def cell_order(self, stream=None):
        """Canonical member order of the collision at the current step (call it
        after couple(PRE)): (order int64[N_s + N_sites], cell_start int64[C + 1])."""
        n = self.sizes.n_solvent + self.sizes.n_sites
        order = np.zeros(max(n, 1), dtype=np.int64)
        start = np.zeros(self.sizes.n_cells + 1, dtype=np.int64)
        self._check(self.lib.mpcd_cell_order(self.ctx, order.ctypes.data, start.ctypes.data, self._s(stream)))
        return order[:n], start

    def diagnostics(self, stream=None) -> dict:
        d = Diag()
        self._check(self.lib.mpcd_diagnostics(self.ctx, C.byref(d), self._s(stream)))
        return dict(p_solvent=np.array(d.p_solvent[:]), p_bodies=np.array(d.p_bodies[:]),
                    ke_solvent=d.ke_solvent, ke_trans=d.ke_trans, ke_rot=d.ke_rot, step=d.step)

    # ------------------------------------------------- transport protocols
    def set_rnemd(self, y_a: float, y_b: float, width: float = 1.0, v_target: float = 0.5,
                  max_pairs: int = 100, period: int = 1, enabled: bool = True):
        """Reverse non-equilibrium exchange of v_x between slabs [y_a, y_a + width)
        and [y_b, y_b + width) (Sec. III.B); see mpcd_set_rnemd."""
        cfg = Rnemd(int(enabled), int(max_pairs), int(period), 0, float(y_a), float(y_b), float(width),
                    float(v_target))
        self._check(self.lib.mpcd_set_rnemd(self.ctx, C.byref(cfg)))

    def set_body_force(self, f, stream=None):
        """Constant force on every body, balanced on the solvent (Sec. III.B
        sedimentation); see mpcd_set_body_force."""
        arr = (C.c_double * 3)(*[float(v) for v in f])
        self._check(self.lib.mpcd_set_body_force(self.ctx, C.byref(arr), self._s(stream)))

    def body_displacements(self, stream=None) -> np.ndarray:
        """Unwrapped displacement of every body since set_state, [n_bodies, 3]."""
        D = np.zeros((max(1, self.sizes.n_bodies), 3))
        self._check(self.lib.mpcd_body_displacements(self.ctx, D.ctypes.data, self._s(stream)))
        return D[: self.sizes.n_bodies]

    def set_vacf(self, n_lags: int, every: int = 1):
        """Start (or with n_lags = 0 stop) the per-body velocity autocorrelations
        of Sec. III.A; see mpcd_set_vacf."""
        self._vacf_lags = int(n_lags)
        self._check(self.lib.mpcd_set_vacf(self.ctx, int(n_lags), int(every)))

    def vacf(self, stream=None):
        """(C_T, C_R) per body and lag, averaged over the origins: [n_bodies, n_lags]."""
        nl, nb = getattr(self, "_vacf_lags", 0), self.sizes.n_bodies
        ct = np.zeros((max(1, nb), nl))
        cr = np.zeros((max(1, nb), nl))
        cnt = np.zeros(nl, dtype=np.int64)
        self._check(self.lib.mpcd_get_vacf(self.ctx, ct.ctypes.data, cr.ctypes.data, cnt.ctypes.data,
                                           self._s(stream)))
        den = np.maximum(cnt, 1)[None, :]
        return ct[:nb] / den, cr[:nb] / den, cnt

    def rnemd_totals(self, stream=None):
        """(x momentum moved from slab A to slab B, number of exchanged pairs)."""
        p, n = C.c_double(), C.c_int64()
        self._check(self.lib.mpcd_rnemd_totals(self.ctx, C.byref(p), C.byref(n), self._s(stream)))
        return p.value, n.value

    def velocity_profile(self, n_bins: int, bin_axis: int = 1, vel_axis: int = 0, stream=None):
        """(mass, momentum) per bin of coordinate `bin_axis` (solvent and bodies)."""
        mass = np.zeros(n_bins)
        mom = np.zeros(n_bins)
        self._check(self.lib.mpcd_velocity_profile(self.ctx, int(bin_axis), int(vel_axis), int(n_bins),
                                                   mass.ctypes.data, mom.ctypes.data, self._s(stream)))
        return mass, mom

    # ------------------------------------------------------------------ debug
    def set_debug(self, on: bool = True):
        self._check(self.lib.mpcd_set_debug(self.ctx, int(on)))

    def debug_cells(self, stream=None) -> dict:
        s = self.sizes
        sums = np.zeros((s.sum_words, s.n_cells), dtype=np.int64 if self.precision == I.P32 else np.float64)
        pw = s.param_bytes // (4 if self.precision == I.P32 else 8)
        params = np.zeros((s.n_cells, pw), dtype=self.real)
        site_cell = np.zeros(max(1, s.n_sites), dtype=np.int32)
        site_v = np.zeros((3, max(1, s.n_sites)), dtype=self.real)
        shift = np.zeros((s.n_replicas, 3), dtype=np.int32)
        self._check(self.lib.mpcd_debug_cells(self.ctx, sums.ctypes.data, params.ctypes.data,
                                              site_cell.ctypes.data, site_v.ctypes.data,
                                              shift.ctypes.data, self._s(stream)))
        return dict(sums=sums, params=params, site_cell=site_cell[: s.n_sites],
                    site_v=site_v[:, : s.n_sites].T.astype(np.float64), shift=shift)

    # ----------------------------------------------------------- profiling
    def set_profiling(self, on: bool = True):
        self._check(self.lib.mpcd_set_profiling(self.ctx, int(on)))

    def reset_profile(self):
        self._check(self.lib.mpcd_reset_profile(self.ctx))

    def profile(self) -> dict:
        arr = (KernelTime * 64)()
        n = self._check(self.lib.mpcd_get_profile(self.ctx, C.cast(arr, C.c_void_p), 64))
        return {arr[i].name.decode(): dict(launches=arr[i].launches, total_ms=arr[i].total_ms,
                                           bytes_per_launch=arr[i].bytes_per_launch)
                for i in range(min(n, 64))}

    def tuning(self) -> dict:
        t = Tuning()
        self._check(self.lib.mpcd_get_tuning(self.ctx, C.byref(t)))
        return dict(block=t.block, tile=t.tile, ctas_per_sm=t.ctas_per_sm, sort_period=t.sort_period,
                    staged=t.staged)

    def set_tuning(self, block=0, tile=0, ctas_per_sm=0, sort_period=0, staged=-1):
        t = Tuning(block, tile, ctas_per_sm, sort_period, staged)
        self._check(self.lib.mpcd_set_tuning(self.ctx, C.byref(t)))

    def autotune(self, steps_per_trial: int = 3, stream=None) -> dict:
        self._check(self.lib.mpcd_autotune(self.ctx, steps_per_trial, self._s(stream)))
        return self.tuning()


class Slab(Simulation):
    """One slab [z_lo, z_hi) of a single-box system (spatial domain
    decomposition along z; see mpcd_create_slab): a subset of the solvent with
    box-wide ids, every body, the sites of its z range."""

    def __init__(self, system: I.System, z_lo: int, z_hi: int, capacity: int, device: int = 0,
                 sort_period: int = 0, use_torch_allocator: bool = True):
        if system.n_rep != 1:
            raise ValueError("a slab is a part of a single box")
        self.lib = load()
        self.system = system
        p = system.params
        self.precision = p.precision
        self.prm = Params(p.kT, p.dt, p.alpha_deg, p.m_solvent, p.rule, p.thermostat,
                          p.precision, p.naive_transfer, p.seed, sort_period, getattr(p, "angular", 0))
        self._keep = []
        shapes = self._shape_descs(system)
        rep = system.replicas[0]
        ids = np.ascontiguousarray(rep.body_shapes, dtype=np.int32)
        self._keep.append(ids)
        self._alloc = None
        if use_torch_allocator and _torch_cuda() is not None:
            self._alloc = _TorchAllocator(device)
        ctx = C.c_void_p()
        rc = self.lib.mpcd_create_slab(C.byref(self.prm), len(system.shapes), C.cast(shapes, C.c_void_p),
                                       C.byref((C.c_int32 * 3)(*rep.L)), int(rep.n_solvent), int(capacity),
                                       len(ids), ids.ctypes.data if len(ids) else None, int(z_lo), int(z_hi),
                                       C.byref(self._alloc.c) if self._alloc else None, device, C.byref(ctx))
        if rc != MPCD_OK:
            raise MPCDError(rc, "mpcd_create_slab failed")
        self.ctx = ctx
        self.z_lo, self.z_hi = int(z_lo), int(z_hi)
        self.sizes = Sizes()
        self._check(self.lib.mpcd_sizes(self.ctx, C.byref(self.sizes)))
        self.real = np.float32 if self.precision == I.P32 else np.float64

    def _rows(self, x):
        return np.ascontiguousarray(np.asarray(x, dtype=self.real).reshape(-1, 3))

    def set_slab_state(self, tags, x, v, R, q, P, Lm, step: int = 0, stream=None):
        tags = np.ascontiguousarray(tags, dtype=np.uint32)
        x, v = self._rows(x), self._rows(v)
        bodies = [np.ascontiguousarray(a, dtype=np.float64) for a in (R, q, P, Lm)]
        self._check(self.lib.mpcd_slab_set_state(self.ctx, len(tags), tags.ctypes.data, x.ctypes.data,
                                                 v.ctypes.data, *[b.ctypes.data for b in bodies], int(step),
                                                 self._s(stream)))

    def get_slab_state(self, stream=None):
        """(ids, x, v, R, q, P, Lm, step) with the solvent in storage order."""
        n = C.c_int64()
        self._check(self.lib.mpcd_slab_get_state(self.ctx, C.byref(n), None, None, None, None, None, None,
                                                 None, self._s(stream)))
        nb = self.sizes.n_bodies
        tags = np.zeros(max(1, n.value), dtype=np.uint32)
        x = np.zeros((max(1, n.value), 3), dtype=self.real)
        v = np.zeros_like(x)
        R, P, Lm = (np.zeros((max(1, nb), 3)) for _ in range(3))
        q = np.zeros((max(1, nb), 4))
        self._check(self.lib.mpcd_slab_get_state(self.ctx, C.byref(n), tags.ctypes.data, x.ctypes.data,
                                                 v.ctypes.data, R.ctypes.data, q.ctypes.data, P.ctypes.data,
                                                 Lm.ctypes.data, self._s(stream)))
        k = n.value
        return tags[:k], x[:k], v[:k], R[:nb], q[:nb], P[:nb], Lm[:nb]

    def extract(self, stream=None):
        """Remove the particles outside [z_lo, z_hi); returns (ids, x, v) of the leavers."""
        n = C.c_int64()
        self._check(self.lib.mpcd_slab_extract(self.ctx, C.byref(n), self._s(stream)))
        k = n.value
        tags = np.zeros(max(1, k), dtype=np.uint32)
        x = np.zeros((max(1, k), 3), dtype=self.real)
        v = np.zeros_like(x)
        self._check(self.lib.mpcd_slab_export(self.ctx, tags.ctypes.data, x.ctypes.data, v.ctypes.data,
                                              self._s(stream)))
        return tags[:k], x[:k], v[:k]

    def insert(self, tags, x, v, stream=None):
        tags = np.ascontiguousarray(tags, dtype=np.uint32)
        x, v = self._rows(x), self._rows(v)
        self._check(self.lib.mpcd_slab_insert(self.ctx, len(tags), tags.ctypes.data, x.ctypes.data,
                                              v.ctypes.data, self._s(stream)))

    def collide_begin(self, stream=None):
        self._check(self.lib.mpcd_collide_begin(self.ctx, self._s(stream)))

    def collide_end(self, stream=None):
        self._check(self.lib.mpcd_collide_end(self.ctx, self._s(stream)))

    def layer_words(self, layer0: int, n_layers: int, stream=None) -> np.ndarray:
        Lx, Ly = self.system.replicas[0].L[:2]
        dt = np.int64 if self.precision == I.P32 else np.float64
        w = np.zeros((self.sizes.sum_words, n_layers * Lx * Ly), dtype=dt)
        self._check(self.lib.mpcd_layer_words(self.ctx, int(layer0), int(n_layers), w.ctypes.data, 0,
                                              self._s(stream)))
        return w

    def add_layer_words(self, layer0: int, words: np.ndarray, stream=None):
        Lx, Ly = self.system.replicas[0].L[:2]
        dt = np.int64 if self.precision == I.P32 else np.float64
        w = np.ascontiguousarray(words, dtype=dt)
        n_layers = w.shape[1] // (Lx * Ly)
        self._check(self.lib.mpcd_layer_words(self.ctx, int(layer0), int(n_layers), w.ctypes.data, 1,
                                              self._s(stream)))

    def post_partial(self, stream=None) -> np.ndarray:
        nb = self.sizes.n_bodies
        d = np.zeros((max(1, nb), 6))
        self._check(self.lib.mpcd_couple_post_partial(self.ctx, d.ctypes.data, self._s(stream)))
        return d[:nb]

    def apply_impulse(self, dPL, stream=None):
        d = np.ascontiguousarray(dPL, dtype=np.float64).reshape(-1, 6)
        self._check(self.lib.mpcd_apply_impulse(self.ctx, d.ctypes.data if d.size else None, self._s(stream)))


def collide_solvent_static(params: I.Params, L, x, y, z, vx, vy, vz, tag=None, step: int = 0,
                           stream=None) -> None:
    """mpcd_collide_solvent_static: one collision of a single solvent-only box
    on caller-owned CUDA float32 tensors (vx, vy, vz updated in place), with
    the library's static scratch instead of any device allocation.  `tag`
    (int32/uint32 particle ids) is needed for MPCD_AT.  Calls on one device
    must not overlap in time: they share the scratch."""
    lib = load()
    prm = Params(params.kT, params.dt, params.alpha_deg, params.m_solvent, params.rule,
                 params.thermostat, params.precision, params.naive_transfer, params.seed, 0,
                 getattr(params, "angular", 0))
    arrs = [x, y, z, vx, vy, vz]
    n = int(x.numel())
    for t in arrs + ([tag] if tag is not None else []):
        if not t.is_cuda or not t.is_contiguous() or t.numel() != n:
            raise ValueError("solvent arrays must be contiguous CUDA tensors of one length")
    for t in arrs:
        if t.element_size() != 4 or not t.is_floating_point():
            raise ValueError("solvent arrays must be float32")
    Ls = (C.c_int32 * 3)(*[int(a) for a in L])
    msg = C.create_string_buffer(256)
    rc = lib.mpcd_collide_solvent_static(C.byref(prm), C.byref(Ls), n, *[t.data_ptr() for t in arrs],
                                         tag.data_ptr() if tag is not None else None, int(step),
                                         current_stream() if stream is None else int(stream), msg, 256)
    if rc != MPCD_OK:
        raise MPCDError(rc, msg.value.decode())
