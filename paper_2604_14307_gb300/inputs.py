"""Seeded synthetic inputs for MPCD suspensions with rigid discrete-particle colloids.

This module only *generates inputs*: site templates (the surface discretisations
of Sec. II.B), colloid placements, orientations and Maxwell-Boltzmann initial
velocities. It performs none of the time-stepping arithmetic (streaming, grid
shift, binning, collision, thermalisation, transfer, rigid-body integration);
both the CUDA path and the FP64 oracle consume what it returns.

Conventions shared by every consumer:
  * lengths in units of the cell size a = 1, boxes are periodic with integer
    edge lengths L (cells per edge), positions are stored in [0, L);
  * quaternions are scalar-first (w, x, y, z), unit norm, body -> space;
  * body angular momentum is given in the space frame (Eq. 4);
  * a site template is expressed in its principal-axis frame with its
    centre of mass at the origin, so R of Eq. 3-5 is the site centre of mass.

The paper's equilibrated suspension configurations are not available, so the
suspension workloads are built by random sequential addition (RSA) at the
target volume fraction, with uniform random orientations.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Names of the two arithmetic forms and the two collision rules.
P64 = 0          # FP64 state on the GPU
P32 = 1          # FP32 state, int64 fixed-point cell sums, FP64 bodies
SRD = 0          # stochastic rotation dynamics (Sec. II.A)
AT = 1           # Andersen-thermostat collision (MPCD-AT)

WCA_SIGMA = 1.0
WCA_RCUT_EXTRA = 2.0 ** (1.0 / 6.0) * WCA_SIGMA   # Eq. 1 cutoff beyond Delta


# --------------------------------------------------------------------------
# Site templates (Sec. II.B: icosphere discretisation; other shapes are
# builder choices for the mixed-shape batch, the paper says only that the
# method accepts arbitrary discretisations).
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Shape:
    """A rigid discrete-particle colloid template.

    b:       (n, 3) site offsets in the body (principal-axis) frame
    m:       (n,) site masses
    centres: (k, 3) excluded-volume (WCA) centres in the body frame; these
             are massless and take no part in collisions (Sec. II.B)
    wca_d:   diameter d of each centre, Delta = d - sigma in Eq. 1
    name:    label
    """
    b: np.ndarray
    m: np.ndarray
    centres: np.ndarray
    wca_d: float
    name: str = "shape"

    @property
    def n_sites(self) -> int:
        return int(self.b.shape[0])

    @property
    def bound_radius(self) -> float:
        """Largest distance of a WCA centre from the origin."""
        return float(np.max(np.linalg.norm(self.centres, axis=1)))


def _icosahedron() -> tuple[np.ndarray, np.ndarray]:
    """Regular icosahedron: vertices (0, +-1, +-phi) and cyclic permutations."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v.append((0.0, s1, s2 * phi))
            v.append((s1, s2 * phi, 0.0))
            v.append((s2 * phi, 0.0, s1))
    v = np.array(v)
    # faces: triples of mutually adjacent vertices (edge length 2)
    n = len(v)
    d2 = ((v[:, None, :] - v[None, :, :]) ** 2).sum(-1)
    adj = np.abs(d2 - 4.0) < 1e-9
    faces = []
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    faces.append((i, j, k))
    return v, np.array(faces, dtype=np.int64)


def icosphere_vertices(level: int) -> np.ndarray:
    """Unit-sphere vertices of an icosahedron subdivided `level` times.

    Each subdivision splits every triangular face into four by its edge
    midpoints; vertices are projected back to the sphere after every
    subdivision.  Vertex count is 10 * 4**level + 2 (12, 42, 162, 642, ...).
    """
    v, faces = _icosahedron()
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    verts = [tuple(x) for x in v]
    for _ in range(level):
        mid = {}
        new_faces = []

        def midpoint(i: int, j: int) -> int:
            key = (min(i, j), max(i, j))
            if key not in mid:
                p = (np.array(verts[i]) + np.array(verts[j])) / 2.0
                p = p / np.linalg.norm(p)
                verts.append(tuple(p))
                mid[key] = len(verts) - 1
            return mid[key]

        for (a, b, c) in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = np.array(new_faces, dtype=np.int64)
    return np.array(verts, dtype=np.float64)


def _centre(b: np.ndarray, m: np.ndarray) -> np.ndarray:
    com = (m[:, None] * b).sum(0) / m.sum()
    return b - com


def sphere_shape(radius: float, level: int, site_mass: float,
                 wca_d: Optional[float] = None) -> Shape:
    """Icosphere shell of `radius` with one WCA centre at the origin."""
    b = icosphere_vertices(level) * radius
    m = np.full(b.shape[0], float(site_mass))
    b = _centre(b, m)
    d = 2.0 * radius if wca_d is None else wca_d
    return Shape(b=b, m=m, centres=np.zeros((1, 3)), wca_d=float(d),
                 name=f"sphere_r{radius:g}_n{b.shape[0]}")


def dumbbell_shape(radius: float, separation: float, level: int,
                   site_mass: float) -> Shape:
    """Two fused icosphere shells with centres `separation` apart along z.

    Sites of one shell lying strictly inside the other sphere are removed.
    """
    s = icosphere_vertices(level) * radius
    top = s + np.array([0.0, 0.0, separation / 2])
    bot = s - np.array([0.0, 0.0, separation / 2])
    keep_top = np.linalg.norm(top + np.array([0, 0, separation / 2]), axis=1) >= radius - 1e-9
    keep_bot = np.linalg.norm(bot - np.array([0, 0, separation / 2]), axis=1) >= radius - 1e-9
    b = np.concatenate([top[keep_top], bot[keep_bot]])
    m = np.full(b.shape[0], float(site_mass))
    b = _centre(b, m)
    cen = np.array([[0, 0, separation / 2], [0, 0, -separation / 2]], dtype=np.float64)
    return Shape(b=b, m=m, centres=cen, wca_d=2.0 * radius,
                 name=f"dumbbell_r{radius:g}_s{separation:g}_n{b.shape[0]}")


def spherocylinder_shape(diameter: float, length: float, spacing: float,
                         site_mass: float, cap_level: int = 3) -> Shape:
    """Spherocylinder of total `length` along z, surface sampled at ~`spacing`.

    The cylinder carries rings of sites (even count per ring, so the x and y
    mirror planes are symmetry planes); each cap is the z >= 0 half of an
    icosphere shell.  WCA centres are spaced <= sigma along the axis.
    """
    r = diameter / 2.0
    h = length / 2.0 - r                      # half-length of the cylinder part
    nphi = int(round(2.0 * math.pi * r / spacing))
    nphi += nphi % 2
    nz = max(1, int(round(2.0 * h / spacing)))
    rings = []
    for k in range(1, nz):
        z = -h + 2.0 * h * k / nz
        for i in range(nphi):
            ph = 2.0 * math.pi * i / nphi
            rings.append((r * math.cos(ph), r * math.sin(ph), z))
    cap = icosphere_vertices(cap_level) * r
    cap = cap[cap[:, 2] >= -1e-12]
    top = cap + np.array([0.0, 0.0, h])
    bot = cap * np.array([1.0, 1.0, -1.0]) - np.array([0.0, 0.0, h])
    b = np.concatenate([np.array(rings).reshape(-1, 3), top, bot])
    m = np.full(b.shape[0], float(site_mass))
    b = _centre(b, m)
    ncen = int(math.ceil(2.0 * h / WCA_SIGMA)) + 1
    zc = np.linspace(-h, h, ncen)
    cen = np.stack([np.zeros(ncen), np.zeros(ncen), zc], axis=1)
    return Shape(b=b, m=m, centres=cen, wca_d=diameter,
                 name=f"rod_d{diameter:g}_l{length:g}_n{b.shape[0]}")


def shape_inertia_diag(shape: Shape) -> np.ndarray:
    """Diagonal of the body-frame inertia tensor of the sites (input scale only)."""
    b, m = shape.b, shape.m
    r2 = (b * b).sum(1)
    return np.array([(m * (r2 - b[:, k] ** 2)).sum() for k in range(3)])


# --------------------------------------------------------------------------
# System description
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    kT: float = 1.0
    dt: float = 0.1
    alpha_deg: float = 130.0
    m_solvent: float = 1.0
    rule: int = SRD
    thermostat: int = 0
    precision: int = P64
    naive_transfer: int = 0
    seed: int = 1
    angular: int = 0              # 1: angular-momentum-conserving variant of the rule (SRD+a, MPCD-AT+a)


@dataclasses.dataclass
class Replica:
    L: tuple                      # (Lx, Ly, Lz) cells per edge
    n_solvent: int
    body_shapes: List[int]        # shape index of each body
    id: int = -1                  # index in the whole ensemble (-1: its position);
                                  # keys the replica's random streams


@dataclasses.dataclass
class System:
    params: Params
    shapes: List[Shape]
    replicas: List[Replica]
    name: str = "system"

    # flattened views -------------------------------------------------------
    @property
    def n_rep(self) -> int:
        return len(self.replicas)

    def solvent_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([r.n_solvent for r in self.replicas])]).astype(np.int64)

    def body_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([len(r.body_shapes) for r in self.replicas])]).astype(np.int64)

    def body_shape_array(self) -> np.ndarray:
        out = []
        for r in self.replicas:
            out += list(r.body_shapes)
        return np.array(out, dtype=np.int32)

    def stream_ids(self) -> np.ndarray:
        """Per-replica stream id: the replica's index in the whole ensemble, so
        that its random streams do not depend on how the ensemble is split."""
        return np.array([r.id if r.id >= 0 else i for i, r in enumerate(self.replicas)], dtype=np.int32)

    def subset(self, ids: Sequence[int]) -> "System":
        """The replicas `ids` (indices into this system) as a system of their own;
        each keeps its stream id, so it evolves exactly as it does here."""
        sid = self.stream_ids()
        reps = [dataclasses.replace(self.replicas[i], body_shapes=list(self.replicas[i].body_shapes),
                                    id=int(sid[i])) for i in ids]
        sub = System(params=dataclasses.replace(self.params), shapes=self.shapes, replicas=reps,
                     name=f"{self.name}[{len(reps)}]")
        pl = getattr(self, "_placements", None)
        if pl is not None:
            sub._placements = [pl[i] for i in ids]
        return sub

    def L_array(self) -> np.ndarray:
        return np.array([r.L for r in self.replicas], dtype=np.int32).reshape(-1, 3)

    @property
    def n_solvent(self) -> int:
        return int(sum(r.n_solvent for r in self.replicas))

    @property
    def n_bodies(self) -> int:
        return int(sum(len(r.body_shapes) for r in self.replicas))

    @property
    def n_sites(self) -> int:
        return int(sum(self.shapes[s].n_sites for r in self.replicas for s in r.body_shapes))

    @property
    def n_cells(self) -> int:
        return int(sum(int(np.prod(r.L)) for r in self.replicas))

    def shape_tables(self):
        """Concatenated template tables: site offsets/masses and WCA centres."""
        site_off = np.concatenate([[0], np.cumsum([s.n_sites for s in self.shapes])]).astype(np.int64)
        cent_off = np.concatenate([[0], np.cumsum([len(s.centres) for s in self.shapes])]).astype(np.int64)
        b = np.ascontiguousarray(np.concatenate([s.b for s in self.shapes]).astype(np.float64))
        m = np.ascontiguousarray(np.concatenate([s.m for s in self.shapes]).astype(np.float64))
        cen = np.ascontiguousarray(np.concatenate([s.centres for s in self.shapes]).astype(np.float64))
        d = np.array([s.wca_d for s in self.shapes], dtype=np.float64)
        return site_off, b, m, cent_off, cen, d


@dataclasses.dataclass
class State:
    """Host state. Solvent and bodies of all replicas are concatenated."""
    x: np.ndarray        # (Ns, 3) solvent positions in [0, L)
    v: np.ndarray        # (Ns, 3) solvent velocities
    R: np.ndarray        # (B, 3) body centres of mass in [0, L)
    q: np.ndarray        # (B, 4) orientation quaternions (w, x, y, z)
    P: np.ndarray        # (B, 3) linear momenta (Eq. 3)
    Lm: np.ndarray       # (B, 3) space-frame angular momenta (Eq. 4)
    step: int = 0

    def copy(self) -> "State":
        return State(self.x.copy(), self.v.copy(), self.R.copy(), self.q.copy(),
                     self.P.copy(), self.Lm.copy(), self.step)


# --------------------------------------------------------------------------
# Random placement
# --------------------------------------------------------------------------
def _rotate(q: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Rotate vectors v (k,3) by unit quaternion q (w,x,y,z)."""
    w, u = q[0], q[1:]
    t = 2.0 * np.cross(u, v)
    return v + w * t + np.cross(u, t)


def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed unit quaternions (Shoemake's method)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], axis=1)
    # reorder to (w, x, y, z) with w the last component of Shoemake's tuple
    return np.ascontiguousarray(q[:, [3, 0, 1, 2]])


def rsa_place(rng: np.random.Generator, L: Sequence[int], shapes: List[Shape],
              shape_ids: Sequence[int], gap: float = 0.2,
              max_attempts: int = 2000) -> tuple[np.ndarray, np.ndarray, List[int]]:
    """Random sequential addition of bodies without overlap.

    Two bodies are accepted when every pair of their WCA centres is farther
    apart than d + gap (d the mean centre diameter), i.e. beyond the cutoff of
    Eq. 1 when gap > 2^(1/6) - 1.  Bodies that cannot be placed within
    `max_attempts` tries are dropped; returns (R, q, placed shape ids).
    """
    L = np.asarray(L, dtype=np.float64)
    R_out, q_out, ids_out = [], [], []
    cen_pos: List[np.ndarray] = []      # placed centres (space frame)
    cen_d: List[float] = []
    reach = max(s.bound_radius for s in shapes) * 2 + max(s.wca_d for s in shapes) + gap
    cell = max(reach, 1.0)
    ncell = np.maximum((L // cell).astype(int), 1)
    grid: dict = {}

    def key(p):
        return tuple((np.floor(p / L * ncell).astype(int)) % ncell)

    for sid in shape_ids:
        sh = shapes[sid]
        for _ in range(max_attempts):
            R = rng.random(3) * L
            q = random_quaternions(rng, 1)[0]
            c = (R + _rotate(q, sh.centres)) % L
            k0 = np.array(key(R))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        kk = tuple((k0 + (dx, dy, dz)) % ncell)
                        for j in grid.get(kk, ()):
                            dd = c[:, None, :] - cen_pos[j][None, :, :]
                            dd -= L * np.round(dd / L)
                            r2 = (dd * dd).sum(-1)
                            lim = 0.5 * (sh.wca_d + cen_d[j]) + gap
                            if np.any(r2 < lim * lim):
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                j = len(R_out)
                R_out.append(R)
                q_out.append(q)
                ids_out.append(sid)
                cen_pos.append(c)
                cen_d.append(sh.wca_d)
                grid.setdefault(key(R), []).append(j)
                break
    R = np.array(R_out, dtype=np.float64).reshape(-1, 3)
    q = np.array(q_out, dtype=np.float64).reshape(-1, 4)
    return R, q, ids_out


# --------------------------------------------------------------------------
# Initial state
# --------------------------------------------------------------------------
def _as_f32_positions(x: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Round positions to float32 values that still lie in [0, L)."""
    xf = x.astype(np.float32)
    Lf = L.astype(np.float32)
    xf = np.where(xf >= Lf, np.float32(0.0), xf)
    return xf.astype(np.float64)


def initial_state(system: System, seed: Optional[int] = None) -> State:
    """Seeded initial state: uniform solvent with Maxwell-Boltzmann velocities
    at kT (zero net momentum per replica), bodies from the given placements
    with MB linear momentum and isotropic angular momentum of matching scale.
    Each replica draws from its own generator, seeded by (seed, stream id), so
    a subset of an ensemble starts from the same state as in the whole.

    For the P32 form every solvent value is rounded to float32 so that both
    implementations start from the same stored numbers.
    """
    p = system.params
    base = p.seed if seed is None else seed
    sids = system.stream_ids()
    Ns, B = system.n_solvent, system.n_bodies
    soff, boff = system.solvent_offsets(), system.body_offsets()
    x = np.empty((Ns, 3))
    v = np.empty((Ns, 3))
    R = np.empty((B, 3))
    q = np.empty((B, 4))
    P = np.empty((B, 3))
    Lm = np.empty((B, 3))
    placements = getattr(system, "_placements", None)
    for r, rep in enumerate(system.replicas):
        rng = np.random.default_rng([int(base), int(sids[r])])   # per replica: independent of the split
        L = np.array(rep.L, dtype=np.float64)
        s0, s1 = soff[r], soff[r + 1]
        b0, b1 = boff[r], boff[r + 1]
        n = s1 - s0
        xr = rng.random((n, 3)) * L
        vr = rng.standard_normal((n, 3)) * math.sqrt(p.kT / p.m_solvent)
        Pb = np.zeros((b1 - b0, 3))
        for i, sid in enumerate(rep.body_shapes):
            sh = system.shapes[sid]
            M = sh.m.sum()
            Pb[i] = rng.standard_normal(3) * math.sqrt(M * p.kT)
            Ibar = shape_inertia_diag(sh).mean()
            Lm[b0 + i] = rng.standard_normal(3) * math.sqrt(Ibar * p.kT)
        if placements is not None:
            R[b0:b1], q[b0:b1] = placements[r]
        P[b0:b1] = Pb
        # zero net momentum of the replica (solvent absorbs the bodies' momentum)
        tot = p.m_solvent * vr.sum(0) + Pb.sum(0)
        if n > 0:
            vr -= tot / (p.m_solvent * n)
        if p.precision == P32:
            xr = _as_f32_positions(xr, L)
            vr = vr.astype(np.float32).astype(np.float64)
        x[s0:s1] = xr
        v[s0:s1] = vr
    return State(x=x, v=v, R=R, q=q, P=P, Lm=Lm, step=0)


def rsa_spheres(rng: np.random.Generator, L: Sequence[int], n: int, d: float,
                gap: float = 0.2, batch: int = 65536, max_proposals: int = 50_000_000):
    """Random sequential addition of up to n equal spheres (centre distance
    >= d + gap), vectorised: proposals are screened in batches against a grid
    of the spheres already placed, and the survivors are then added one at a
    time with a check against the ones added before them in the same batch.
    Every accepted sphere has been tested against all earlier ones, as in
    sequential RSA.  Returns centres (k, 3), k <= n."""
    L = np.asarray(L, dtype=np.float64)
    dmin = d + gap
    cs = dmin / math.sqrt(3.0) * 0.999              # at most one centre per grid cell
    ng = np.maximum((L // cs).astype(int), 1)
    csz = L / ng
    reach = int(math.ceil(dmin / csz.min()))
    grid = -np.ones(tuple(ng), dtype=np.int64)
    R = np.zeros((n, 3))
    k, proposals = 0, 0
    offs = np.array([(a, b, c) for a in range(-reach, reach + 1) for b in range(-reach, reach + 1)
                     for c in range(-reach, reach + 1)])
    while k < n and proposals < max_proposals:
        P = rng.random((batch, 3)) * L
        proposals += batch
        cell = np.minimum((P / csz).astype(int), ng - 1)
        ok = np.ones(batch, dtype=bool)
        for o in np.array_split(offs, 5):
            nb = (cell[:, None, :] + o[None, :, :]) % ng
            idx = grid[nb[..., 0], nb[..., 1], nb[..., 2]]
            has = idx >= 0
            dv = P[:, None, :] - R[np.maximum(idx, 0)]
            dv -= L * np.round(dv / L)
            close_ = has & ((dv * dv).sum(-1) < dmin * dmin)
            ok &= ~close_.any(1)
        for i in np.flatnonzero(ok):
            if k >= n:
                break
            nb = (cell[i] + offs) % ng
            idx = grid[nb[:, 0], nb[:, 1], nb[:, 2]]
            idx = idx[idx >= 0]
            if idx.size:
                dv = P[i] - R[idx]
                dv -= L * np.round(dv / L)
                if ((dv * dv).sum(-1) < dmin * dmin).any():
                    continue
            if grid[tuple(cell[i])] >= 0:
                continue
            R[k] = P[i]
            grid[tuple(cell[i])] = k
            k += 1
    return R[:k]


def build_system(params: Params, shapes: List[Shape], Ls: Sequence[Sequence[int]],
                 density: float, bodies_per_rep: Sequence[Sequence[int]],
                 name: str, placement_seed: int = 12345,
                 R_q: Optional[list] = None) -> System:
    """Assemble a System; bodies are placed by RSA unless R_q is given."""
    rng = np.random.default_rng(placement_seed)
    reps, placements = [], []
    for i, (L, ids) in enumerate(zip(Ls, bodies_per_rep)):
        L = tuple(int(a) for a in L)
        n_s = int(round(density * L[0] * L[1] * L[2]))
        if R_q is not None:
            R, q = R_q[i]
            placed = list(ids)
        elif ids and len(set(ids)) == 1 and len(shapes[ids[0]].centres) == 1 \
                and np.allclose(shapes[ids[0]].centres, 0.0):
            R = rsa_spheres(rng, L, len(ids), shapes[ids[0]].wca_d)
            q = random_quaternions(rng, len(R))
            placed = [ids[0]] * len(R)
        else:
            R, q, placed = rsa_place(rng, L, shapes, ids)
        reps.append(Replica(L=L, n_solvent=n_s, body_shapes=list(placed)))
        placements.append((np.asarray(R, dtype=np.float64).reshape(-1, 3),
                           np.asarray(q, dtype=np.float64).reshape(-1, 4)))
    sysm = System(params=params, shapes=shapes, replicas=reps, name=name)
    sysm._placements = placements
    return sysm


def n_bodies_for_phi(L: Sequence[int], phi: float, radius: float) -> int:
    vol = float(np.prod(L))
    return int(round(phi * vol / (4.0 / 3.0 * math.pi * radius ** 3)))


# --------------------------------------------------------------------------
# The workloads
# --------------------------------------------------------------------------
def single_sphere_L10(precision: int = P64, seed: int = 1) -> System:
    """L=10, density 5, one radius-2 sphere of 162 unit-mass sites, SRD 130 deg,
    no thermostat, dt=0.1 (the small validation case)."""
    prm = Params(kT=1.0, dt=0.1, alpha_deg=130.0, rule=SRD, thermostat=0,
                 precision=precision, seed=seed)
    sh = sphere_shape(2.0, 2, 1.0)
    return build_system(prm, [sh], [(10, 10, 10)], 5.0, [[0]],
                        name="single_sphere_L10",
                        R_q=[(np.array([[5.0, 5.0, 5.0]]), np.array([[1.0, 0.0, 0.0, 0.0]]))])


def suspension(L: int, density: float, phi: float, radius: float, level: int,
               site_mass: float, rule: int, thermostat: int, precision: int,
               seed: int = 1, name: Optional[str] = None) -> System:
    prm = Params(kT=1.0, dt=0.1, alpha_deg=130.0, rule=rule, thermostat=thermostat,
                 precision=precision, seed=seed)
    sh = sphere_shape(radius, level, site_mass)
    nb = n_bodies_for_phi((L, L, L), phi, radius)
    return build_system(prm, [sh], [(L, L, L)], density, [[0] * nb],
                        name=name or f"suspension_L{L}_phi{phi:g}", placement_seed=seed + 1000)


def suspension_L50(precision: int = P32, seed: int = 1) -> System:
    """L=50, density 5, 221 radius-3 spheres of 642 sites (phi~0.2), MPCD-AT."""
    return suspension(50, 5.0, 0.2, 3.0, 3, 5.0, AT, 1, precision, seed, "suspension_L50_phi0.2")


def suspension_L200(precision: int = P32, seed: int = 1, thermostat: int = 2) -> System:
    """L=200, density 10, ~8950 radius-4 spheres of 642 sites (phi~0.3),
    SRD with the cell-level thermostat (E' drawn by Marsaglia-Tsang rejection
    by default, 1: as a sum of exponentials)."""
    return suspension(200, 10.0, 0.3, 4.0, 3, 10.0, SRD, thermostat, precision, seed, "suspension_L200_phi0.3")


def batched_single_sphere(n_rep: int = 4096, precision: int = P32, seed: int = 1,
                          Ls: Sequence[int] = (12, 16, 20, 24)) -> System:
    """n_rep independent boxes, L drawn uniformly from Ls, density 5, one
    162-site radius-2 sphere (site mass 5) per box, SRD 130 deg."""
    rng = np.random.default_rng(seed + 77)
    Lr = rng.choice(np.array(Ls), size=n_rep)
    prm = Params(kT=1.0, dt=0.1, alpha_deg=130.0, rule=SRD, thermostat=0,
                 precision=precision, seed=seed)
    sh = sphere_shape(2.0, 2, 5.0)
    R_q = [(np.array([[L / 2.0, L / 2.0, L / 2.0]]), random_quaternions(rng, 1)) for L in Lr]
    return build_system(prm, [sh], [(L, L, L) for L in Lr], 5.0, [[0]] * n_rep,
                        name=f"batched_single_sphere_{n_rep}", R_q=R_q)


def batched_mixed_shapes(n_rep: int = 256, precision: int = P32, seed: int = 1,
                         Lmin: int = 20, Lmax: int = 40, phimin: float = 0.05,
                         phimax: float = 0.35) -> System:
    """n_rep boxes with L uniform in [Lmin, Lmax] and phi uniform in
    [phimin, phimax]; colloids are a mix of radius-3 642-site spheres, rigid
    dumbbells (two fused radius-3 spheres 3 apart) and 1:4 spherocylinders
    (diameter 6, sites spaced ~0.5); MPCD-AT, density 5, site mass 5.
    Rods are only used in boxes with L >= 30 so that minimum images stay valid."""
    rng = np.random.default_rng(seed + 99)
    prm = Params(kT=1.0, dt=0.1, alpha_deg=130.0, rule=AT, thermostat=1,
                 precision=precision, seed=seed)
    shapes = [sphere_shape(3.0, 3, 5.0), dumbbell_shape(3.0, 3.0, 3, 5.0),
              spherocylinder_shape(6.0, 24.0, 0.5, 5.0)]
    vol = [4.0 / 3.0 * math.pi * 27.0,
           2 * 4.0 / 3.0 * math.pi * 27.0 - math.pi * (4 * 3.0 + 3.0) * (2 * 3.0 - 3.0) ** 2 / 12.0,
           math.pi * 9.0 * 18.0 + 4.0 / 3.0 * math.pi * 27.0]
    Ls, ids = [], []
    for _ in range(n_rep):
        L = int(rng.integers(Lmin, Lmax + 1))
        phi = float(rng.uniform(phimin, phimax))
        allowed = [0, 1, 2] if L >= 30 else [0, 1]
        target = phi * L ** 3
        lst, acc = [], 0.0
        while acc < target:
            s = int(rng.choice(allowed))
            lst.append(s)
            acc += vol[s]
        if lst and acc - target > vol[lst[-1]] / 2:
            lst.pop()
        Ls.append((L, L, L))
        ids.append(lst)
    return build_system(prm, shapes, Ls, 5.0, ids, name=f"batched_mixed_shapes_{n_rep}",
                        placement_seed=seed + 2000)
