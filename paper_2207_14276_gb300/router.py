"""Request router over independent replicas, one per GPU.

Energy+force requests (gas-phase molecules, or new solute coordinates for a
solvated box kept resident on one replica) are independent, so a multi-GPU
deployment runs one replica of the potential per GPU and routes requests
between them; there is no data-path collective.  This module holds the
host-side policy and the sharded evaluation loop over a process group:

- ``Router``: online assignment.  A request for a resident box goes to the
  replica that holds the box; any other request to the replica with the least
  outstanding work, counted in ML-region atoms (the unit the evaluation cost
  scales with).  Ties go to the lowest replica index, so assignment is
  deterministic for a given arrival order.
- ``shard``: the same policy applied to a known list of requests (in order).
- ``serve_sharded``: every rank evaluates the requests assigned to it with a
  caller-supplied function and rank 0 gathers the results in request order.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence


class Router:
    def __init__(self, n_replicas: int):
        if n_replicas < 1:
            raise ValueError("at least one replica")
        self.n = n_replicas
        self.load = [0] * n_replicas          # outstanding ML-region atoms per replica
        self.resident_at = {}                 # resident box id -> replica
        self.resident_atoms = [0] * n_replicas

    def place_resident(self, box_id: int, n_atoms: int) -> int:
        """Choose the replica that keeps box `box_id` (n_atoms atoms) resident: the
        one with the fewest resident atoms."""
        if box_id in self.resident_at:
            return self.resident_at[box_id]
        r = min(range(self.n), key=lambda k: (self.resident_atoms[k], k))
        self.resident_at[box_id] = r
        self.resident_atoms[r] += n_atoms
        return r

    def assign(self, n_ml: int, box_id: Optional[int] = None) -> int:
        """Replica for a request with n_ml atoms in its ML region."""
        if box_id is not None:
            if box_id not in self.resident_at:
                raise KeyError(f"resident box {box_id} was not placed")
            r = self.resident_at[box_id]
        else:
            r = min(range(self.n), key=lambda k: (self.load[k], k))
        self.load[r] += n_ml
        return r

    def complete(self, replica: int, n_ml: int) -> None:
        """A request of n_ml atoms finished on `replica`."""
        self.load[replica] -= n_ml
        if self.load[replica] < 0:
            raise ValueError("more work completed than assigned")


def shard(sizes: Sequence[int], n_replicas: int,
          box_ids: Optional[Sequence[Optional[int]]] = None,
          box_atoms: Optional[dict] = None) -> List[int]:
    """Replica of each request of a known list (sizes = ML atoms per request),
    assigned in order with nothing completing in between."""
    router = Router(n_replicas)
    box_ids = box_ids or [None] * len(sizes)
    for b in sorted({b for b in box_ids if b is not None}):
        router.place_resident(b, (box_atoms or {}).get(b, 0))
    return [router.assign(n, b) for n, b in zip(sizes, box_ids)]


def serve_sharded(requests: Sequence, sizes: Sequence[int], evaluate: Callable,
                  dist=None, box_ids=None, box_atoms=None):
    """Evaluate `requests` across the ranks of a process group: each rank runs
    `evaluate(request)` on the requests `shard` assigns to it, and rank 0 returns
    every result in request order (other ranks return None).  Without a process
    group (or with one rank) everything runs locally."""
    world = dist.get_world_size() if (dist is not None and dist.is_initialized()) else 1
    rank = dist.get_rank() if world > 1 else 0
    owner = shard(sizes, world, box_ids, box_atoms)
    mine = [(i, evaluate(requests[i])) for i in range(len(requests)) if owner[i] == rank]
    if world == 1:
        return [r for _, r in sorted(mine, key=lambda t: t[0])]
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(mine, gathered, dst=0)
    if rank != 0:
        return None
    out = [None] * len(requests)
    for part in gathered:
        for i, r in part:
            out[i] = r
    return out
