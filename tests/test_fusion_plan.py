"""Fusion planner (host logic, no GPU): every gate runs exactly once, tiles fit,
and the planner's reordering only swaps gates that commute -- checked by
running the oracle on the executed order and on the original order."""
import numpy as np
import pytest

import __graft_entry__
import oracle

__graft_entry__.build()
from paper_2410_17876_gb300 import binding as qb  # noqa: E402
from paper_2410_17876_gb300 import inputs as gen  # noqa: E402


def _reordered(circ, order):
    return gen.Circuit(circ.dims, [circ.gates[i] for i in order])


def _check_plan(circ, prec, **opts):
    order, pass_of, tiles = qb.qd_plan_circuit(circ.dims, prec, circ, **opts)
    n = len(circ.gates)
    assert sorted(order.tolist()) == list(range(n))
    assert np.all(np.diff(pass_of) >= 0)
    assert len(tiles) == pass_of[-1] + 1 if n else True
    maxt = opts.get("max_tile_amps") or (8192 if prec == qb.QD_C64 else 4096)
    assert np.all(tiles <= maxt)
    # a tile pass holds >= 2 gates; a per-gate pass exactly one
    counts = np.bincount(pass_of, minlength=len(tiles))
    for p, c in enumerate(counts):
        assert (tiles[p] > 0 and c >= 2) or (tiles[p] == 0 and c == 1)
    return order, pass_of, tiles


@pytest.mark.parametrize("prec", [0, 1])
def test_fusion_off_keeps_order(prec):
    c = gen.config0_circuit(depth=60)
    order, pass_of, tiles = qb.qd_plan_circuit(c.dims, prec, c, mode=qb.QD_FUSE_OFF)
    assert order.tolist() == list(range(60))
    assert pass_of.tolist() == list(range(60))
    assert np.all(tiles == 0)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("max_tile", [64, 512, 4096])
def test_reordering_preserves_the_result(seed, max_tile):
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = tuple(int(x) for x in rng.choice([2, 3, 4, 5], size=int(rng.integers(5, 9))))
    circ = gen.random_mixed_circuit(dims, 150, rng)
    # add diagonal gates, commuting controls and a few non-fusable gates
    extra = []
    for _ in range(30):
        t = int(rng.integers(len(dims)))
        extra.append(gen.Gate((t,), gen.z_gen(dims[t])))
    extra.append(gen.Gate((0, 1), gen.haar(dims[0] * dims[1], rng)))
    gates = circ.gates[:50] + extra + circ.gates[50:]
    circ = gen.Circuit(dims, gates)
    order, _, _ = _check_plan(circ, qb.QD_C64, mode=qb.QD_FUSE_TILE, max_tile_amps=max_tile)
    psi0 = gen.random_state(circ.D, rng)
    a = oracle.run_circuit(circ, psi0)
    b = oracle.run_circuit(_reordered(circ, order), psi0)
    assert np.max(np.abs(a - b)) < 1e-12


def test_config1_is_grouped_into_few_passes():
    c = gen.config1_circuit()
    order, pass_of, tiles = _check_plan(c, qb.QD_C64, mode=qb.QD_FUSE_TILE)
    n_pass = len(tiles)
    fused_gates = int(np.sum(np.bincount(pass_of)[tiles > 0]))
    assert n_pass < 100, n_pass
    assert fused_gates > 450
    # the wire set of each pass is chosen to take the most gates: 12 passes
    # (choosing wires in the order the gates need them gave 15)
    assert n_pass <= 12, n_pass
    # the executed order still gives the same state (checked on the 20-wire state
    # with a 12-wire-prefix variant to keep the oracle fast)
    small = gen.prefix_circuit(c, 12)
    o2, _, _ = _check_plan(small, qb.QD_C64, mode=qb.QD_FUSE_TILE, max_tile_amps=256)
    a = oracle.run_circuit(small)
    b = oracle.run_circuit(_reordered(small, o2))
    assert np.max(np.abs(a - b)) < 1e-12


def test_non_fusable_gates_run_alone():
    dims = (2, 3, 7, 2, 2)
    rng = np.random.Generator(np.random.PCG64(3))
    gates = [gen.Gate((0,), gen.haar(2, rng)), gen.Gate((2,), gen.haar(7, rng)),
             gen.Gate((1, 3), gen.haar(6, rng)), gen.Gate((4,), gen.haar(2, rng)),
             gen.Gate((3,), gen.haar(2, rng))]
    c = gen.Circuit(dims, gates)
    order, pass_of, tiles = _check_plan(c, qb.QD_C64, mode=qb.QD_FUSE_TILE, max_tile_amps=8192)
    pos = {g: i for i, g in enumerate(order)}
    for g in (1, 2):
        p = pass_of[pos[g]]
        assert tiles[p] == 0


def test_sparse_qubit_blocks_become_register_runs():
    """Four qubits with one dense gate each and controlled shifts: the cost model
    picks a run of gates applied in registers over the composed 16 x 16 block for
    complex64 (each gate's own arithmetic: 96 flop per amplitude), while complex128,
    which has no runs, composes it (128 flop per amplitude); the executed order is
    still a valid reordering."""
    rng = np.random.Generator(np.random.PCG64(950))
    dims = (2, 2, 2, 2, 3, 2, 3)
    gates = [gen.Gate((w,), gen.haar(2, rng)) for w in range(4)]
    gates += [gen.Gate(((w + 1) % 4,), gen.x_plus(2, 1), (w,), (1,)) for w in range(4)]
    circ = gen.Circuit(dims, gates)
    f64 = qb.qd_plan_circuit(dims, qb.QD_C64, circ, mode=qb.QD_FUSE_TILE, max_tile_amps=1024, with_flops=True)[3]
    f128 = qb.qd_plan_circuit(dims, qb.QD_C128, circ, mode=qb.QD_FUSE_TILE, max_tile_amps=1024, with_flops=True)[3]
    assert sum(f64) / circ.D == pytest.approx(96.0)
    assert sum(f128) / circ.D == pytest.approx(128.0)
    order, _, _ = _check_plan(circ, qb.QD_C64, mode=qb.QD_FUSE_TILE, max_tile_amps=1024)
    psi0 = gen.random_state(circ.D, rng)
    assert np.max(np.abs(oracle.run_circuit(circ, psi0) - oracle.run_circuit(_reordered(circ, order), psi0))) < 1e-12


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("block_dim", [16, 64])
def test_whole_state_blocks_preserve_the_result(seed, block_dim):
    """QD_FUSE_BLOCK plans: every gate once, every block within block_dim
    dimensions, and the executed order gives the same state."""
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    dims = tuple(int(x) for x in rng.choice([2, 3, 4, 5], size=int(rng.integers(5, 9))))
    circ = gen.random_mixed_circuit(dims, 150, rng)
    extra = [gen.Gate((int(t),), gen.z_gen(dims[int(t)])) for t in rng.integers(len(dims), size=20)]
    extra.append(gen.Gate((0, 1), gen.haar(dims[0] * dims[1], rng)))
    circ = gen.Circuit(dims, circ.gates[:60] + extra + circ.gates[60:])
    order, pass_of, _ = qb.qd_plan_circuit(dims, qb.QD_C64, circ, mode=qb.QD_FUSE_BLOCK, block_dim=block_dim)
    n = len(circ.gates)
    assert sorted(order.tolist()) == list(range(n))
    assert np.all(np.diff(pass_of) >= 0)
    for p in range(pass_of[-1] + 1):
        gates = [circ.gates[order[i]] for i in np.nonzero(pass_of == p)[0]]
        if len(gates) > 1:
            wires = set()
            for g in gates:
                assert len(g.wires) == 1
                wires |= set(g.wires) | set(g.controls)
            assert np.prod([dims[w] for w in wires]) <= block_dim
    psi0 = gen.random_state(circ.D, rng)
    a = oracle.run_circuit(circ, psi0)
    b = oracle.run_circuit(_reordered(circ, order), psi0)
    assert np.max(np.abs(a - b)) < 1e-12


def test_whole_state_block_pass_counts_of_the_workloads():
    """Blocks of up to 64 dimensions grown by the wires that take the most
    gates: 20 passes for the 200 gates of the 18-qubit + 8-qutrit workload
    (adding wires in gate order: 25) and 39 for the 500 gates of the
    12-qubit + 8-qutrit circuit."""
    for circ, most in ((gen.config2_circuit(), 20), (gen.config1_circuit(), 39)):
        _, pass_of, _ = qb.qd_plan_circuit(circ.dims, qb.QD_C64, circ, mode=qb.QD_FUSE_BLOCK, block_dim=64)
        assert pass_of[-1] + 1 <= most, pass_of[-1] + 1
