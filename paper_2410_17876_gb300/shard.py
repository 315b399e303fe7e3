"""A state partitioned over G processes by its most significant wires, with
the wire-swap exchange step (the paper names distributed execution as
future work, section "Conclusion").

Layout.  The logical wires are mapped to physical digit positions; the
lowest ``n_local`` positions are *local* (each rank stores the
``D / G`` amplitudes that share its *global* digits) and the positions above
them are *global*: rank ``r``'s global digits are the mixed-radix digits of
``r`` over the global positions' dimensions (the first global position least
significant), so ``prod(global dims) = G``.  The initial global wires are
taken from the most significant logical wire down, each one whose dimension
still divides what is left of ``G``.

Gates (section "Superposition gates": a gate only mixes the amplitudes of
a class, which differ only in the gate's own digits):
  * every target on a local position: each rank applies the gate to its
    shard on the mapped positions.  A control on a global position has one
    digit per rank (section "Controlled and Multi-Controlled Gates"): a rank
    whose digit differs skips the gate, the others drop that control;
  * a target on a global position g: first *swap* g with a local position l
    of the same dimension d that the gate does not target.  An amplitude
    with digit x at g and y at l moves from the rank whose digit at g is x
    (local digit y) to the rank whose digit at g is y (local digit x): each
    rank keeps the block y = x and exchanges the other d - 1 blocks of
    ``D / (G d)`` amplitudes with the d - 1 ranks that differ from it only
    in the digit at g -- ``D / G (1 - 1/d)`` amplitudes sent per rank, in one
    ``all_to_all_single``.  Position l is moved to the top of the local
    order first (``Backend.to_top``) so that each block is contiguous, and
    moved back after the exchange (``Backend.from_top``).

The local steps run in a ``Backend``: :class:`CudaBackend` drives the C ABI
(gates through ``qd_apply_*``, the moves through ``qd_state_wire_to_top`` /
``qd_state_wire_from_top``), and the exchange goes through
``torch.distributed`` (NCCL between GPUs).  A backend is injectable so that
the rank logic and the exchange can be exercised on CPU processes (gloo).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = ["ShardLayout", "ShardedState", "CudaBackend"]


class ShardLayout:
    """Logical wire <-> physical position map of a state over ``world`` ranks."""

    def __init__(self, dims: Sequence[int], world: int):
        self.dims = tuple(int(d) for d in dims)
        self.world = int(world)
        n = len(self.dims)
        glob: List[int] = []
        prod = 1
        for w in range(n - 1, -1, -1):  # most significant first; |0...0> is the same in any wire order
            if prod == self.world:
                break
            if self.world % (prod * self.dims[w]) == 0:
                glob.append(w)
                prod *= self.dims[w]
        if prod != self.world:
            raise ValueError(f"no set of the wires {self.dims} has dimensions multiplying to {self.world} ranks")
        glob = sorted(glob)
        local = [w for w in range(n) if w not in glob]
        if not local:
            raise ValueError("every wire would be global")
        self.n_local = len(local)
        self.pos2wire = local + glob  # physical position -> logical wire
        self._sync()

    def _sync(self):
        self.wire2pos = {w: p for p, w in enumerate(self.pos2wire)}

    def pos_dims(self) -> Tuple[int, ...]:
        return tuple(self.dims[w] for w in self.pos2wire)

    def local_dims(self) -> Tuple[int, ...]:
        return self.pos_dims()[:self.n_local]

    def global_dims(self) -> Tuple[int, ...]:
        return self.pos_dims()[self.n_local:]

    def rank_digits(self, rank: int) -> Tuple[int, ...]:
        """Digits of the global positions on ``rank`` (first global position least significant)."""
        out = []
        r = int(rank)
        for d in self.global_dims():
            out.append(r % d)
            r //= d
        return tuple(out)

    def rank_of(self, digits: Sequence[int]) -> int:
        r, m = 0, 1
        for x, d in zip(digits, self.global_dims()):
            r += int(x) * m
            m *= d
        return r

    def is_global(self, wire: int) -> bool:
        return self.wire2pos[wire] >= self.n_local

    def swap_partner(self, gwire: int, busy: Sequence[int]) -> int:
        """Local wire to swap with global ``gwire``: the same dimension, not in
        ``busy`` (the gate's targets), the highest local position first."""
        d = self.dims[gwire]
        for p in range(self.n_local - 1, -1, -1):
            w = self.pos2wire[p]
            if self.dims[w] == d and w not in busy:
                return w
        raise ValueError(f"no local wire of dimension {d} to swap with wire {gwire}")

    def swap(self, gwire: int, lwire: int) -> None:
        pg, pl = self.wire2pos[gwire], self.wire2pos[lwire]
        self.pos2wire[pg], self.pos2wire[pl] = lwire, gwire
        self._sync()


def exchange_splits(layout: ShardLayout, rank: int, gpos: int, block: int) -> List[int]:
    """Split sizes (amplitudes per destination rank, rank order) of the swap
    at global position ``gpos``: ``block`` for each rank that differs from
    ``rank`` only in that position's digit (itself included), 0 otherwise."""
    digits = list(layout.rank_digits(rank))
    gi = gpos - layout.n_local
    d = layout.global_dims()[gi]
    splits = [0] * layout.world
    for y in range(d):
        dd = list(digits)
        dd[gi] = y
        splits[layout.rank_of(dd)] = block
    return splits


class ShardedState:
    """One rank's shard of a partitioned state (see the module docstring).

    ``backend`` holds the local amplitudes and runs the local steps;
    ``group`` is a ``torch.distributed`` process group (None: the default)."""

    def __init__(self, dims: Sequence[int], backend, rank: int, world: int, group=None):
        self.layout = ShardLayout(dims, world)
        self.rank = int(rank)
        self.world = int(world)
        self.group = group
        self.backend = backend
        self.swaps = 0
        self.sent_amplitudes = 0
        backend.init_zero(self.layout.local_dims(), self.rank == 0)

    # --- gates -----------------------------------------------------------------------------
    def apply(self, gate) -> None:
        """Apply an ``inputs.Gate`` (logical wires)."""
        L = self.layout
        for w in gate.wires:
            if L.is_global(w):
                self._swap(w, L.swap_partner(w, gate.wires))
        digits = L.rank_digits(self.rank)
        cw, cv = [], []
        for c, v in zip(gate.controls, gate.values):
            p = L.wire2pos[c]
            if p >= L.n_local:
                if digits[p - L.n_local] != v:
                    return  # this rank's classes all fail the control
            else:
                cw.append(p)
                cv.append(int(v))
        self.backend.apply([L.wire2pos[w] for w in gate.wires], gate.U, cw, cv)

    def run(self, circuit) -> None:
        for g in circuit.gates:
            self.apply(g)

    # --- exchange --------------------------------------------------------------------------
    def _swap(self, gwire: int, lwire: int) -> None:
        import torch.distributed as dist

        L = self.layout
        gpos, lpos = L.wire2pos[gwire], L.wire2pos[lwire]
        local_D = int(np.prod(L.local_dims(), dtype=np.int64))
        d = L.dims[gwire]
        block = local_D // d
        send = self.backend.to_top(lpos)          # blocks by local digit y, contiguous (2 reals per amplitude)
        recv = self.backend.empty_like(send)
        splits = [2 * s for s in exchange_splits(L, self.rank, gpos, block)]
        dist.all_to_all_single(recv, send, splits, splits, group=self.group)
        self.backend.from_top(lpos, recv)         # block from the rank with digit y goes to local digit y
        L.swap(gwire, lwire)
        self.swaps += 1
        self.sent_amplitudes += block * (d - 1)

    # --- readouts --------------------------------------------------------------------------
    def norm(self) -> float:
        import torch
        import torch.distributed as dist

        t = torch.tensor([self.backend.norm()], dtype=torch.float64, device=self.backend.reduce_device())
        dist.all_reduce(t, group=self.group)
        return float(t.item())

    def gather(self) -> Optional[np.ndarray]:
        """The whole state in logical order on rank 0 (None elsewhere): for tests and small states."""
        import torch
        import torch.distributed as dist

        mine = torch.from_numpy(self.backend.host_amplitudes().view(np.float64).copy())
        mine = mine.to(self.backend.reduce_device())
        parts = [torch.empty_like(mine) for _ in range(self.world)] if self.rank == 0 else None
        dist.gather(mine, parts, dst=0, group=self.group)
        if self.rank != 0:
            return None
        L = self.layout
        shards = [p.cpu().numpy().view(np.complex128) for p in parts]
        pdims = L.pos_dims()
        # physical index = local index + D_local * rank; shape (global..., local...) reversed for C order
        phys = np.concatenate(shards).reshape(tuple(reversed(pdims)))
        # axis k of phys (C order) is physical position n-1-k; reorder to logical positions
        n = len(pdims)
        axes_for_logical = [n - 1 - L.wire2pos[w] for w in range(n)]  # logical wire -> phys axis
        logical = np.transpose(phys, [axes_for_logical[w] for w in reversed(range(n))])
        return np.ascontiguousarray(logical).reshape(-1)


class CudaBackend:
    """Local steps on one GPU through the C ABI: the shard is a torch tensor
    wrapped as a qd_state; the moved order lives in a second buffer of the
    same size (the receive buffer of the exchange is a third)."""

    def __init__(self, prec: int = None, device: int = 0):
        from . import binding as qb

        self.qb = qb
        self.prec = qb.QD_C128 if prec is None else prec
        self.device = device
        self.state = None

    def init_zero(self, local_dims, is_rank0: bool) -> None:
        qb = self.qb
        self.local_dims = tuple(local_dims)
        self.state = qb.State(self.local_dims, prec=self.prec, device=self.device)
        if not is_rank0:  # |0...0> lives on rank 0 only
            self.state.buf.zero_()

    def apply(self, wires, U, cw, cv) -> None:
        qb = self.qb
        h = self.state.handle
        if len(wires) == 1 and not cw:
            qb.qd_apply_gate(h, wires[0], U)
        elif len(wires) == 1:
            qb.qd_apply_controlled(h, wires[0], U, cw, cv)
        else:
            qb.qd_apply_multi(h, wires, U, cw or None, cv or None)

    def empty_like(self, t):
        import torch

        return torch.empty_like(t)

    def to_top(self, pos: int):
        import torch

        out = torch.empty_like(self.state.buf)
        self.qb.qd_state_wire_to_top(self.state.handle, pos, out.data_ptr())
        self.state.synchronize()
        return out

    def from_top(self, pos: int, buf) -> None:
        self.qb.qd_state_wire_from_top(self.state.handle, pos, buf.data_ptr())
        self.state.synchronize()

    def norm(self) -> float:
        return self.state.norm()

    def reduce_device(self):
        return f"cuda:{self.device}"

    def host_amplitudes(self) -> np.ndarray:
        return self.state.amplitudes()
