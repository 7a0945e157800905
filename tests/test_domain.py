"""Spatial domain decomposition of one box into slabs (domain.py), on CPU.

The decomposition logic - slab bounds, migration of the particles that left
a slab, completion of the cell words of the shifted layers next to each slab
face by integer addition of the neighbour's partial words, the all-reduce of
the bodies' momentum change - runs over two and three gloo ranks with a numpy
slab backend that restates the oracle's FP32-form collision arithmetic
(float32 streaming, the exact integer cell words, the cell velocity and E_rel
from the completed words in FP64, the oracle's axis and thermostat draws).  Against the single-box oracle, after every step: the
positions, velocities and ids are bit-identical, and each slab's completed
words equal the oracle's words of every cell the slab's particles occupy.
"""
import math
import multiprocessing
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import domain as D
from paper_2604_14307_gb300 import inputs as I

STEPS = 3


def box(seed=5):
    prm = I.Params(rule=I.SRD, thermostat=1, precision=I.P32, seed=seed)
    return I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [(8, 7, 12)], 5.0, [[]], "slabbox", placement_seed=seed)


class NumpySlab:
    """Solvent-only P32 SRD slab on the host (test backend)."""

    def __init__(self, system, osys, rows, st, zlo, zhi):
        self.s, self.osys = system, osys
        self.L = np.array(system.replicas[0].L, dtype=np.int64)
        self.C = int(np.prod(self.L))
        self.ids = rows.astype(np.int64)
        self.x = st.x[rows].astype(np.float32)
        self.v = st.v[rows].astype(np.float32)
        self.zlo, self.zhi = zlo, zhi
        self.step_ = int(st.step)
        self.m = float(np.float32(system.params.m_solvent))
        self.words = np.zeros((4, self.C), dtype=np.int64)
        self.words_log = []

    def stream(self):
        dt = np.float32(self.s.params.dt)
        for a in range(3):
            La = np.float32(self.L[a])
            y = self.x[:, a] + self.v[:, a] * dt
            y = np.where(y >= La, y - La, y)
            yw = (y + La).astype(np.float32)
            y = np.where(y < 0, np.where(yw >= La, np.float32(0), yw), y)
            self.x[:, a] = y.astype(np.float32)

    def extract(self):
        z = self.x[:, 2]
        out = ~((z >= self.zlo) & (z < self.zhi))
        res = (self.ids[out].astype(np.uint32), self.x[out].copy(), self.v[out].copy())
        keep = ~out
        self.ids, self.x, self.v = self.ids[keep], self.x[keep], self.v[keep]
        return res

    def insert(self, ids, x, v):
        self.ids = np.concatenate([self.ids, ids.astype(np.int64)])
        self.x = np.concatenate([self.x, x.astype(np.float32)])
        self.v = np.concatenate([self.v, v.astype(np.float32)])

    def couple_pre(self):
        pass

    def _cells(self):
        S = O.grid_shift(self.osys, 0, self.step_).astype(np.int64)
        X = np.floor(self.x.astype(np.float64) * 2.0**20).astype(np.int64)
        c = ((X - S[None, :]) >> 20) % self.L[None, :]
        return c[:, 0] + self.L[0] * (c[:, 1] + self.L[1] * c[:, 2])

    def collide_begin(self):
        self.cell = self._cells()
        p = np.float32(self.m) * self.v
        e = (p[:, 0] * self.v[:, 0] + p[:, 1] * self.v[:, 1]) + p[:, 2] * self.v[:, 2]
        terms = [np.rint(p[:, 0].astype(np.float64) * 2.0**32).astype(np.int64) + 2**48,
                 np.rint(p[:, 1].astype(np.float64) * 2.0**32).astype(np.int64),
                 np.rint(p[:, 2].astype(np.float64) * 2.0**32).astype(np.int64),
                 np.rint(e.astype(np.float64) * 2.0**28).astype(np.int64)]
        self.words[:] = 0
        for k in range(4):
            np.add.at(self.words[k], self.cell, terms[k])

    def layer_words(self, layer, n):
        plane = int(self.L[0] * self.L[1])
        return self.words[:, layer * plane:(layer + n) * plane].copy()

    def add_layer_words(self, layer, w):
        plane = int(self.L[0] * self.L[1])
        n = w.shape[1] // plane
        self.words[:, layer * plane:(layer + n) * plane] += w

    def collide_end(self):
        al = self.s.params.alpha_deg * 3.14159265358979323846264338327950288 / 180.0
        ca, sa = math.cos(al), math.sin(al)
        order = np.lexsort((self.ids, self.cell))
        cells, starts = np.unique(self.cell[order], return_index=True)
        ends = np.append(starts[1:], len(order))
        vnew = self.v.astype(np.float64).copy()
        self.words_log.append({int(c): self.words[:, c].copy() for c in cells})
        for c, b, e in zip(cells, starts, ends):
            mem = order[b:e]
            # the cell's totals come from its completed words: members of a face
            # cell live on two slabs
            w = self.words[:, c]
            lo0 = int(w[0]) & (2**48 - 1)
            lo0 = lo0 - 2**48 if lo0 >= 2**47 else lo0
            n = (int(w[0]) - lo0) >> 48
            if n < 2:
                continue
            M = n * self.m
            S1 = [lo0 * 2.0**-32, int(w[1]) * 2.0**-32, int(w[2]) * 2.0**-32]
            u = [S1[a] / M for a in range(3)]
            pp = 0.0
            for a in range(3):
                pp += S1[a] * S1[a]
            Erel = 0.5 * (float(w[3]) * 2.0**-28 - pp / M)
            Ep = O.thermostat_energy(self.osys, 0, self.step_, int(c), n)
            kappa = math.sqrt(Ep / Erel) if Erel > 0.0 else 1.0
            ax = O.srd_axis(self.osys, 0, self.step_, int(c))
            for i in mem:
                wv = [float(self.v[i, a]) - u[a] for a in range(3)]
                nx = [ax[1] * wv[2] - ax[2] * wv[1], ax[2] * wv[0] - ax[0] * wv[2], ax[0] * wv[1] - ax[1] * wv[0]]
                nd = ax[0] * wv[0] + ax[1] * wv[1] + ax[2] * wv[2]
                for a in range(3):
                    vnew[i, a] = u[a] + kappa * (wv[a] * ca + nx[a] * sa + ax[a] * nd * (1.0 - ca))
        self.v = vnew.astype(np.float32)

    def post_partial(self):
        return np.zeros((0, 6))

    def apply_impulse(self, dPL):
        self.step_ += 1

    def sort(self):
        pass


def oracle_steps(system, st, n):
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)
    out = []
    for _ in range(n):
        O.stream(osys, ost)
        tr = O.collide(osys, ost)
        ost.step += 1
        out.append((ost.x.copy(), ost.v.copy(), tr["fixed"][:4].copy()))
    return out


def run_slabs(system, comm, ranks, world):
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    part = D.Partition(system.replicas[0].L[2], world)
    rows = D.split_state(part, st.x)
    slabs = {r: NumpySlab(system, osys, rows[r], st, int(part.bounds[r]), int(part.bounds[r + 1])) for r in ranks}
    dom = D.SlabDomain(part, comm, slabs, sort_period=0)
    snaps = []
    for _ in range(STEPS):
        dom.step(1)
        snaps.append({r: (s.ids.copy(), s.x.copy(), s.v.copy(), s.words_log[-1]) for r, s in slabs.items()})
    return snaps, dom.migrated


def check(system, snaps_all, world):
    ref = oracle_steps(system, I.initial_state(system), STEPS)
    n = system.n_solvent
    for k in range(STEPS):
        parts = [snaps_all[r][k] for r in range(world)]
        x, v = D.gather([(p[0], p[1], p[2]) for p in parts], n)
        assert np.array_equal(x.astype(np.float64), ref[k][0]), k
        assert np.array_equal(v.astype(np.float64), ref[k][1]), k
        for p in parts:
            for c, w in p[3].items():
                assert np.array_equal(w, ref[k][2][:, c]), (k, c)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        snaps, mig = run_slabs(box(), D.TorchComm(), [rank], world)
        per_step = [s[rank] for s in snaps]
        allp = [None] * world
        dist.all_gather_object(allp, (per_step, mig))
        if rank == 0:
            q.put(allp)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_and_faces():
    p = D.Partition(12, 3)
    assert list(p.bounds) == [0, 4, 8, 12]
    assert list(p.owner(np.array([0.0, 3.99, 4.0, 11.9]))) == [0, 0, 1, 2]
    assert p.faces(0) == [(0, 2, 0), (4, 1, 1)] and p.faces(2) == [(8, 1, 2), (0, 0, 0)]
    assert p.face_layers(0) == [11, 0]
    with pytest.raises(ValueError):
        D.Partition(5, 3)
    assert D.Partition(7, 1).faces(0) == []


@pytest.mark.parametrize("world", [2, 3])
def test_loopback_slabs_reproduce_the_single_box_oracle(world):
    snaps, mig = run_slabs(box(), D.LoopbackComm(world), list(range(world)), world)
    assert mig > 0                                   # particles did cross slab faces
    check(box(), {r: [s[r] for s in snaps] for r in range(world)}, world)


def test_two_gloo_ranks_reproduce_the_single_box_oracle():
    O.build()
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allp = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sum(m for _, m in allp) > 0
    check(box(), {r: allp[r][0] for r in range(2)}, 2)
