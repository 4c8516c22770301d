"""The workload's natural shards split over ranks (one process per GPU).

The method's work splits three ways (Sec. "Particle-In-Cell Scheme" and
"Test Particle Method" of arXiv:1607.04069):

* the superparticles of one discharge: every step is per particle except the
  field solve, which needs the total charge.  Each rank holds a contiguous
  range of the initial loading's ids (``pic_params.id_offset``) and after
  every step the ranks sum the exact int64 deposits (``pic_exchange_slot``)
  with one all-reduce; random words are keyed by particle id and step, so the
  split run equals the one-rank run of the same discharge;
* the atoms of one test-particle source: ranks launch disjoint id ranges
  (``tp_source.first_id``) and never talk until their histograms are summed;
* independent discharges (a batch or a stream of requests): each rank runs
  its own members.

Counts and histograms are sums over ranks; the time-averaged charge,
potential and fluxes of a split discharge are already global on every rank.
Argument marshalling and collectives only: the stepping is the library's.
"""
from __future__ import annotations

import numpy as np

from . import Discharge, params_from_workload

#: diagnostics whose value on a rank is that rank's own part (summed over ranks)
PER_RANK_DIAG = ("eedf", "iedf_l", "iedf_r", "ieadf_l", "ieadf_r", "sputter_e_l", "sputter_e_r", "sputter_ang_l",
                 "sputter_ang_r", "tp_dens", "tpf_time")
#: counters that add up over ranks (the rest are per-rank slot counts and step indices)
SUMMED_COUNTERS = ("imp_e_l", "imp_e_r", "imp_i_l", "imp_i_r", "ionizations", "sputtered_l", "sputtered_r",
                   "tp_dep_l", "tp_dep_r", "numerics", "elastic", "excitation", "cx", "iso", "tp_coll", "capacity")


def part(n: int, rank: int, world: int) -> tuple[int, int]:
    """The contiguous block of rank ``rank`` among ``world`` in 0 .. n-1:
    (first index, count).  The blocks cover 0 .. n-1 exactly once."""
    if not (0 <= rank < world):
        raise ValueError("rank must lie in [0, world)")
    a = n * rank // world
    b = n * (rank + 1) // world
    return a, b - a


def members(n: int, rank: int, world: int) -> range:
    """Independent discharges 0 .. n-1 of rank ``rank``: a contiguous block."""
    a, c = part(n, rank, world)
    return range(a, a + c)


def shard_workload(cfg: dict, rank: int, world: int) -> dict:
    """One rank's share of a discharge: the particles id_offset .. of both
    charged species (n_e0 = n_i0 required) and slot capacities scaled to the
    share; the weight is the whole discharge's."""
    if cfg["n_e0"] != cfg["n_i0"]:
        raise ValueError("a split discharge loads as many electrons as ions")
    if cfg.get("circuit", 0):
        raise ValueError("a split discharge needs the ideal source (circuit 0)")
    first, count = part(cfg["n_e0"], rank, world)
    c = dict(cfg, n_e0=count, n_i0=count, id_offset=first)
    for k in ("cap_e", "cap_i"):
        if c.get(k):
            c[k] = -(-c[k] * count // max(cfg["n_e0"], 1)) + 65536
    return c


def allreduce_(t, group=None):
    """Sum a tensor over the ranks in place (int64 sums are exact and do not
    depend on the order).  On one rank, nothing."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def sum_host(a: np.ndarray, group=None, device=None) -> np.ndarray:
    """Sum a host array over the ranks (through the device for NCCL)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1):
        return a
    dev = device if device is not None else ("cuda" if dist.get_backend(group) == "nccl" else "cpu")
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


class SplitDischarge:
    """One rank's share of a discharge whose superparticles are split over
    ``world`` ranks (one context per rank on its own GPU).  ``step`` runs the
    library's step and then sums the deposit block over the ranks before the
    next step; with world = 1 it is the plain discharge."""

    def __init__(self, cfg: dict, rank: int, world: int, group=None, stream=None, **over):
        self.rank, self.world, self.group = rank, world, group
        self.cfg = shard_workload(cfg, rank, world)
        self.d = Discharge(params_from_workload(self.cfg, **over), stream=stream)
        self._exchange()

    def _exchange(self):
        if self.world > 1:
            allreduce_(self.d.exchange_slot(), self.group)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.d.step(1)
            self._exchange()

    def sync(self):
        self.d.sync()

    def diag(self, kind) -> np.ndarray:
        """The whole discharge's diagnostic: charge, potential and flux
        averages as the rank holds them, per-rank histograms summed.  Ratios
        of per-rank sums (tp_v, tpf_vx) do not add up and are refused."""
        if kind in ("tp_v", "tpf_vx"):
            raise ValueError(f"{kind} is a ratio of per-rank sums; combine tp_dens and the moments instead")
        v = self.d.diag(kind)
        return sum_host(v, self.group) if kind in PER_RANK_DIAG else v

    def counters(self) -> dict:
        """Event counts summed over the ranks (slot counts stay per rank)."""
        c = self.d.counters()
        tot = sum_host(np.array([c[k] for k in SUMMED_COUNTERS], dtype=np.int64), self.group)
        return dict(c, **dict(zip(SUMMED_COUNTERS, tot.tolist())))

    def alive(self) -> int:
        """Charged superparticles of the whole discharge."""
        n = sum(len(self.d.get_species(s)["id"]) for s in (0, 1))
        return int(sum_host(np.array([n], dtype=np.int64), self.group)[0])

    def close(self):
        self.d.close()
