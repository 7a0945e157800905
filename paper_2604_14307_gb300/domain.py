"""Spatial domain decomposition of one periodic box into slabs along z.

The paper runs every simulation on one GPU; a box too large for one device is
split here into slabs [z_r, z_{r+1}) of whole cells, one rank (process, GPU) per
slab.  What each rank holds and does per step (Sec. II.A collision, Sec. II.B
rigid bodies):

* its solvent particles (box-wide ids), the cell grid of the whole box, and
  every body (replicated: the bodies' forces and integration need no
  communication, every rank computes them alike);
* streaming; then the particles that left the slab are sent to the rank that
  owns their new z (a neighbour: no particle moves a cell in a step);
* the surface sites of every body are placed and thermalised on every rank
  (Eq. 7 needs each body's sums over all of its sites), but a rank bins and
  collides only the sites whose z lies in its slab;
* binning into exact integer cell words.  Under the random grid shift
  s in [-1/2, 1/2) the shifted cell layer next to a slab face - layer
  z_face - 1 or z_face - holds particles of both neighbours.  Each rank sends
  its partial words of the two layers z_face - 1 and z_face to the neighbour
  across the face and adds the neighbour's: integer addition makes every
  completed word equal to the single-box word bit for bit;
* collision parameters and the collision of its own particles and sites;
* each body's momentum change is summed over the ranks (all-reduce, in rank
  order, so that every rank applies the same FP64 sum) and applied.

Communication goes through a `comm` object: `TorchComm` (one slab per process,
torch.distributed point-to-point and all-reduce on host buffers; gloo or NCCL)
or `LoopbackComm` (every slab in this process, e.g. several contexts on one
GPU, exchanged in host memory).  `SlabDomain.step()` advances every local slab
by one step, phase by phase, so that the slabs of one process never wait on
one another inside a kernel.
"""
from __future__ import annotations

import io
from typing import Dict, List, Sequence

import numpy as np


# ------------------------------------------------------------------ layout
class Partition:
    """Slab bounds z_0 = 0 < z_1 < ... < z_N = L_z (cells), each slab at least
    two cells thick (so that the face layers of one slab are distinct)."""

    def __init__(self, Lz: int, n: int):
        if n < 1 or (n > 1 and Lz < 2 * n):
            raise ValueError("each slab needs at least two cell layers")
        self.Lz, self.n = int(Lz), int(n)
        self.bounds = np.array([(r * Lz) // n for r in range(n + 1)], dtype=np.int64)

    def owner(self, z: np.ndarray) -> np.ndarray:
        """The slab of each z in [0, L_z)."""
        z = np.asarray(z, dtype=np.float64)
        return np.searchsorted(self.bounds, z, side="right") - 1

    def faces(self, r: int):
        """The faces of slab r as (z of the face, neighbour across it, face id);
        the face between slab k-1 and slab k (cyclically) has id k."""
        if self.n == 1:
            return []
        lo, hi = int(self.bounds[r]), int(self.bounds[r + 1])
        return [(lo, (r - 1) % self.n, r), (hi % self.Lz, (r + 1) % self.n, (r + 1) % self.n)]

    def face_layers(self, z_face: int):
        """The two shifted-grid layers that may straddle a face at z_face."""
        return [(z_face - 1) % self.Lz, z_face % self.Lz]


# --------------------------------------------------------------- messaging
def pack(*arrays: np.ndarray) -> bytes:
    buf = io.BytesIO()
    np.savez(buf, *[np.ascontiguousarray(a) for a in arrays])
    return buf.getvalue()


def unpack(b: bytes) -> List[np.ndarray]:
    with np.load(io.BytesIO(b)) as z:
        return [z[f"arr_{k}"] for k in range(len(z.files))]


class LoopbackComm:
    """All slabs in this process: messages are routed in host memory."""

    def __init__(self, n: int):
        self.size = n
        self.local = list(range(n))

    def exchange(self, sends: Dict[int, Dict[int, List[bytes]]]) -> Dict[int, Dict[int, List[bytes]]]:
        """sends[src][dst] = list of messages -> recvs[dst][src] = the same list."""
        out: Dict[int, Dict[int, List[bytes]]] = {r: {} for r in self.local}
        for src, d in sends.items():
            for dst, msgs in d.items():
                out[dst].setdefault(src, []).extend(msgs)
        return out

    def allreduce_sum(self, arrays: Dict[int, np.ndarray]) -> np.ndarray:
        tot = None
        for r in sorted(arrays):
            tot = arrays[r].copy() if tot is None else tot + arrays[r]
        return tot


class TorchComm:
    """One slab per process over torch.distributed (host buffers; gloo, or NCCL
    with device staging).  Messages to a neighbour travel as one length and
    one byte tensor; every rank posts its sends and receives together."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.size = dist.get_world_size()
        self.rank = dist.get_rank()
        self.local = [self.rank]
        self.device = device if device is not None else (
            torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu"))

    def _p2p(self, peers_send: Dict[int, bytes], peers_recv: Sequence[int]) -> Dict[int, bytes]:
        torch, dist = self.torch, self.dist
        ops, lens_in = [], {}
        for dst, b in peers_send.items():
            ops.append(dist.P2POp(dist.isend, torch.tensor([len(b)], dtype=torch.int64, device=self.device), dst))
        for src in peers_recv:
            lens_in[src] = torch.zeros(1, dtype=torch.int64, device=self.device)
            ops.append(dist.P2POp(dist.irecv, lens_in[src], src))
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        ops, bufs = [], {}
        for dst, b in peers_send.items():
            t = torch.frombuffer(bytearray(b), dtype=torch.uint8).to(self.device)
            ops.append(dist.P2POp(dist.isend, t, dst))
        for src in peers_recv:
            bufs[src] = torch.zeros(int(lens_in[src].item()), dtype=torch.uint8, device=self.device)
            ops.append(dist.P2POp(dist.irecv, bufs[src], src))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        return {src: bytes(bufs[src].cpu().numpy().tobytes()) for src in peers_recv}

    def exchange(self, sends: Dict[int, Dict[int, List[bytes]]]) -> Dict[int, Dict[int, List[bytes]]]:
        me = self.rank
        peers = sorted({(me - 1) % self.size, (me + 1) % self.size} - {me})
        outgoing = {dst: pack(*[np.frombuffer(m, dtype=np.uint8) for m in sends.get(me, {}).get(dst, [])])
                    for dst in peers}
        got = self._p2p(outgoing, peers)
        return {me: {src: [a.tobytes() for a in unpack(b)] for src, b in got.items()}}

    def allreduce_sum(self, arrays: Dict[int, np.ndarray]) -> np.ndarray:
        torch, dist = self.torch, self.dist
        a = arrays[self.rank]
        # all-gather then a sum in rank order: every rank applies the same value
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(self.device)
        parts = [torch.zeros_like(t) for _ in range(self.size)]
        dist.all_gather(parts, t)
        tot = parts[0].clone()
        for p in parts[1:]:
            tot += p
        return tot.cpu().numpy()


# ------------------------------------------------------------------- driver
class SlabDomain:
    """The slabs of one box held by this process (`slabs[r]` for the ranks in
    comm.local) and the step that couples them.  A slab backend provides:
    stream(), extract() -> (ids, x, v), insert(ids, x, v), couple_pre(),
    collide_begin(), layer_words(layer, 1) / add_layer_words(layer, words),
    collide_end(), post_partial() -> dPL, apply_impulse(dPL), sort()."""

    def __init__(self, partition: Partition, comm, slabs: Dict[int, object], sort_period: int = 20):
        self.part, self.comm, self.slabs = partition, comm, slabs
        self.sort_period = sort_period
        self.steps = 0
        self.migrated = 0

    def _migrate(self):
        sends: Dict[int, Dict[int, List[bytes]]] = {}
        for r, s in self.slabs.items():
            ids, x, v = s.extract()
            self.migrated += len(ids)
            dst = self.part.owner(np.floor(np.asarray(x, dtype=np.float64)[:, 2])) if len(ids) else np.zeros(0, int)
            nbrs = {(r - 1) % self.part.n, (r + 1) % self.part.n}
            if len(ids) and not set(np.unique(dst).tolist()) <= nbrs:
                raise RuntimeError("a particle crossed more than one slab in one step")
            sends[r] = {d: [pack(ids[dst == d], x[dst == d], v[dst == d])] for d in nbrs if d != r}
        recvs = self.comm.exchange(sends)
        for r, s in self.slabs.items():
            for src in sorted(recvs.get(r, {})):
                for m in recvs[r][src]:
                    ids, x, v = unpack(m)
                    if len(ids):
                        s.insert(ids, x, v)

    def _complete_face_words(self):
        sends: Dict[int, Dict[int, List[bytes]]] = {}
        for r, s in self.slabs.items():
            sends[r] = {}
            for z, nb, fid in self.part.faces(r):
                for layer in self.part.face_layers(z):
                    w = s.layer_words(layer, 1)
                    sends[r].setdefault(nb, []).append(pack(np.array([fid, layer], dtype=np.int64), w))
        recvs = self.comm.exchange(sends)
        for r, s in self.slabs.items():
            mine = {fid for _, _, fid in self.part.faces(r)}
            for src in sorted(recvs.get(r, {})):
                for m in recvs[r][src]:
                    head, w = unpack(m)
                    if int(head[0]) in mine:
                        s.add_layer_words(int(head[1]), w)

    def step(self, n: int = 1):
        for _ in range(n):
            for s in self.slabs.values():
                s.stream()
            if self.part.n > 1:
                self._migrate()
            for s in self.slabs.values():
                s.couple_pre()
                s.collide_begin()
            if self.part.n > 1:
                self._complete_face_words()
            parts = {}
            for r, s in self.slabs.items():
                s.collide_end()
                parts[r] = s.post_partial()
            tot = self.comm.allreduce_sum(parts) if self.part.n > 1 else next(iter(parts.values()))
            for s in self.slabs.values():
                s.apply_impulse(tot)
            self.steps += 1
            if self.sort_period > 0 and self.steps % self.sort_period == 0:
                for s in self.slabs.values():
                    s.sort()


def split_state(partition: Partition, x: np.ndarray):
    """Row indices of each slab's solvent from host positions x[N][3]."""
    own = partition.owner(np.floor(np.asarray(x, dtype=np.float64)[:, 2]))
    return [np.flatnonzero(own == r) for r in range(partition.n)]


def gather(parts: Sequence[tuple], n_total: int):
    """(x, v) in box-wide id order from per-slab (ids, x, v)."""
    ids = np.concatenate([p[0] for p in parts]).astype(np.int64)
    if len(ids) != n_total or np.any(np.bincount(ids, minlength=n_total) != 1):
        raise RuntimeError("the slabs do not hold every particle exactly once")
    x = np.empty((n_total, 3), dtype=parts[0][1].dtype)
    v = np.empty((n_total, 3), dtype=parts[0][2].dtype)
    x[ids] = np.concatenate([p[1] for p in parts])
    v[ids] = np.concatenate([p[2] for p in parts])
    return x, v


class GpuSlab:
    """The CUDA backend of a slab: a `binding.Slab` context."""

    def __init__(self, sim):
        self.sim = sim

    def stream(self):
        self.sim.stream()

    def extract(self):
        return self.sim.extract()

    def insert(self, ids, x, v):
        self.sim.insert(ids, x, v)

    def couple_pre(self):
        from .binding import MPCD_PRE
        self.sim.couple(MPCD_PRE)

    def collide_begin(self):
        self.sim.collide_begin()

    def layer_words(self, layer, n):
        return self.sim.layer_words(layer, n)

    def add_layer_words(self, layer, w):
        self.sim.add_layer_words(layer, w)

    def collide_end(self):
        self.sim.collide_end()

    def post_partial(self):
        return self.sim.post_partial()

    def apply_impulse(self, dPL):
        self.sim.apply_impulse(dPL)

    def sort(self):
        self.sim.sort()
