"""A state partitioned over several processes by its most significant wires
(paper_2410_17876_gb300.shard): the layout bookkeeping, and whole circuits
that target and control the partitioned wires, run as 2, 3 and 4 gloo ranks
on CPU with the wire-swap exchange, against the oracle.  On these CPU ranks
the local steps (gates, wire moves) run in a numpy/oracle backend; on GPUs
they run through the C ABI (CudaBackend), which needs several GPUs and is
not measured here."""
import os
import socket
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_2410_17876_gb300 import inputs as gen
from paper_2410_17876_gb300.shard import ShardLayout, exchange_splits

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_layout_partitions_the_top_wires():
    L = ShardLayout((2, 3, 2, 3, 2), 2)
    assert L.global_dims() == (2,) and L.pos2wire == [0, 1, 2, 3, 4]
    L = ShardLayout((3, 2, 2, 3, 2, 2), 4)
    assert L.pos2wire[-2:] == [4, 5] and L.global_dims() == (2, 2)
    assert [L.rank_digits(r) for r in range(4)] == [(0, 0), (1, 0), (0, 1), (1, 1)]
    assert all(L.rank_of(L.rank_digits(r)) == r for r in range(4))
    L = ShardLayout((2, 3, 2, 2), 3)  # the qutrit is the only wire dividing 3
    assert L.pos2wire == [0, 2, 3, 1] and L.local_dims() == (2, 2, 2)
    with pytest.raises(ValueError):
        ShardLayout((2, 2, 2), 3)


def test_swap_bookkeeping_and_splits():
    L = ShardLayout((3, 2, 2, 3, 2, 2), 4)
    w = L.swap_partner(5, busy=(5,))
    assert L.dims[w] == 2 and not L.is_global(w) and w == 2  # highest local qubit position
    gpos = L.wire2pos[5]
    # rank 3 = digits (1, 1): partners differ in the digit at wire 5's position
    assert exchange_splits(L, 3, gpos, 7) == [0, 7, 0, 7]
    L.swap(5, w)
    assert L.is_global(2) and not L.is_global(5) and L.pos2wire[gpos] == 2


class _NumpyBackend:
    """CPU backend of the tests: the oracle applies the gates to the shard,
    numpy moves a wire to the top and back."""

    def init_zero(self, local_dims, is_rank0):
        self.dims = tuple(local_dims)
        self.psi = np.zeros(int(np.prod(self.dims)), dtype=np.complex128)
        if is_rank0:
            self.psi[0] = 1.0

    def apply(self, wires, U, cw, cv):
        import oracle

        self.psi = oracle.apply_gate(self.dims, self.psi, gen.Gate(tuple(wires), U, tuple(cw), tuple(cv)))

    def _shape(self, pos):
        lo = int(np.prod(self.dims[:pos], dtype=np.int64))
        d = self.dims[pos]
        return self.psi.size // (lo * d), d, lo

    def to_top(self, pos):
        import torch

        hi, d, lo = self._shape(pos)
        moved = np.ascontiguousarray(self.psi.reshape(hi, d, lo).transpose(1, 0, 2)).reshape(-1)
        return torch.from_numpy(moved.view(np.float64).copy())

    def empty_like(self, t):
        import torch

        return torch.empty_like(t)

    def from_top(self, pos, buf):
        hi, d, lo = self._shape(pos)
        moved = buf.numpy().view(np.complex128).reshape(d, hi, lo)
        self.psi = np.ascontiguousarray(moved.transpose(1, 0, 2)).reshape(-1)

    def norm(self):
        return float(np.vdot(self.psi, self.psi).real)

    def reduce_device(self):
        return "cpu"

    def host_amplitudes(self):
        return self.psi


def _circuit(dims, seed):
    """Random mixed circuit plus gates aimed at the top wires: targets, controls
    and a two-wire gate across the partition."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = gen.random_mixed_circuit(dims, 60, rng)
    n = len(dims)
    extra = [gen.Gate((n - 1,), gen.haar(dims[n - 1], rng)),
             gen.Gate((0,), gen.haar(dims[0], rng), (n - 1,), (1,)),
             gen.Gate((n - 2, n - 1), gen.haar(dims[n - 2] * dims[n - 1], rng)),
             gen.Gate((n - 1,), gen.x_plus(dims[n - 1]), (n - 2, 0), (1, 0))]
    return gen.Circuit(dims, extra + c.gates + extra)


RANK_SCRIPT = textwrap.dedent("""
    import os, sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch.distributed as dist
    from paper_2410_17876_gb300 import inputs as gen
    from paper_2410_17876_gb300.shard import ShardedState
    from tests.test_shard_host import _NumpyBackend, _circuit
    import oracle
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    dims = {dims!r}
    circ = _circuit(dims, {seed})
    st = ShardedState(dims, _NumpyBackend(), rank, world)
    st.run(circ)
    nrm = st.norm()
    full = st.gather()
    if rank == 0:
        ref = oracle.run_circuit(circ)
        err = float(np.max(np.abs(full - ref)))
        print(f"err={{err:.3e}} norm={{nrm:.15f}} swaps={{st.swaps}} sent={{st.sent_amplitudes}}")
        assert err < 1e-12 and abs(nrm - 1) < 1e-12 and st.swaps > 0
    dist.barrier()
    dist.destroy_process_group()
""")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("dims,world,seed", [((2, 3, 2, 3, 2), 2, 1), ((2, 2, 3, 2, 3), 3, 2),
                                             ((3, 2, 2, 3, 2, 2), 4, 3)])
def test_sharded_circuit_over_gloo_ranks(tmp_path, dims, world, seed):
    script = tmp_path / "rank.py"
    script.write_text(RANK_SCRIPT.format(root=ROOT, dims=dims, seed=seed))
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=300)[0] for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    assert "err=" in outs[0], outs[0]
