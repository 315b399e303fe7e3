"""GPU parity of fused circuits (shared-memory tile passes) against the oracle,
across tile sizes, odd and even row lengths, in-tile and outside controls,
and non-fusable gates interleaved."""
import numpy as np
import pytest

import __graft_entry__
import oracle
from tests.gpu_util import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qb():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    __graft_entry__.build()
    from paper_2410_17876_gb300 import binding

    return binding


@pytest.fixture(scope="module")
def gen():
    from paper_2410_17876_gb300 import inputs

    return inputs


def _run(qb, circ, prec, psi0=None, **opts):
    st = qb.State(circ.dims, prec=prec)
    if psi0 is not None:
        st.set_amplitudes(psi0)
    st.run(circ, fuse=True, **opts)
    out = st.amplitudes()
    st.close()
    return out


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_config0_fused_single_tile(qb, gen, prec):
    p = qb.QD_C128 if prec == "c128" else qb.QD_C64
    circ = gen.config0_circuit(seed=0, depth=200)
    order, pass_of, tiles = qb.qd_plan_circuit(circ.dims, p, circ)
    # every pass is a tile pass over (at most) the whole 216-amplitude state,
    # at most 64 gates per pass
    assert np.all(tiles > 0) and np.all(tiles <= circ.D) and len(tiles) == 4
    assert_close(_run(qb, circ, p), oracle.run_circuit(circ), p, "config0 fused")


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("max_tile,block_dim", [(64, 16), (256, 4), (2048, 8), (8192, 16), (8192, 1), (2048, 9)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_mixed_circuits_fused(qb, gen, prec, max_tile, block_dim, seed):
    p = qb.QD_C128 if prec == "c128" else qb.QD_C64
    if p == qb.QD_C128 and max_tile > 4096:
        max_tile = 4096
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    dims = tuple(int(x) for x in rng.choice([2, 3, 4, 5], size=int(rng.integers(7, 11))))
    if seed == 2:
        dims = (3, 3, 5, 3) + dims[4:]  # odd row lengths (no 16-byte path)
    circ = gen.random_mixed_circuit(dims, 160, rng)
    # interleave multi-controlled, diagonal and non-fusable gates
    extra = []
    n = len(dims)
    for _ in range(25):
        t = int(rng.integers(n))
        cw = tuple(int(x) for x in rng.permutation([w for w in range(n) if w != t])[:3])
        extra.append(gen.Gate((t,), gen.haar(dims[t], rng), cw, tuple(int(rng.integers(dims[c])) for c in cw)))
        extra.append(gen.Gate((t,), gen.z_gen(dims[t])))
    extra.append(gen.Gate((1, 0), gen.haar(dims[0] * dims[1], rng)))
    gates = circ.gates[:80] + extra + circ.gates[80:]
    circ = gen.Circuit(dims, gates)
    psi0 = gen.random_state(circ.D, rng)
    got = _run(qb, circ, p, psi0, max_tile_amps=max_tile, block_dim=block_dim)
    ref = oracle.run_circuit(circ, psi0)
    assert_close(got, ref, p, f"fused dims={dims} tile={max_tile} block={block_dim}")


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_fused_equals_unfused_on_wide_state(qb, gen, prec):
    """A 2^22-amplitude state: many tiles per pass; fused within tolerance of per-gate."""
    p = qb.QD_C128 if prec == "c128" else qb.QD_C64
    rng = np.random.Generator(np.random.PCG64(7))
    dims = (2,) * 10 + (3, 2, 2, 3) + (2,) * 6
    circ = gen.random_mixed_circuit(dims, 300, rng)
    st = qb.State(dims, prec=p)
    st.run(circ, fuse=True)
    a = st.amplitudes()
    st.reset()
    st.run(circ, fuse=False)
    b = st.amplitudes()
    st.close()
    tol = 1e-12 if p == qb.QD_C128 else 1e-5
    assert np.max(np.abs(a - b)) < tol
    assert abs(np.vdot(a, a).real - 1.0) < tol


def test_tile_too_large_is_rejected(qb, gen):
    circ = gen.config0_circuit(depth=5)
    st = qb.State(circ.dims, prec=qb.QD_C128)
    with pytest.raises(qb.QuditError) as ei:
        st.run(circ, fuse=True, max_tile_amps=1 << 20)
    assert ei.value.status == qb.QD_ERR_UNSUPPORTED
    st.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_light_passes(qb, gen, prec):
    """Passes light on arithmetic (phase and permutation gates, a few
    controlled; monomial gates run through the dense class update): 2.98M
    amplitudes in tiles of at most 4096, with controls outside the tile
    evaluated per tile."""
    p = qb.QD_C64 if prec == "c64" else qb.QD_C128
    rng = np.random.Generator(np.random.PCG64(77))
    dims = (2,) * 12 + (3,) * 6
    gates = []
    for i in range(60):
        w = int(rng.integers(0, len(dims)))
        d = dims[w]
        k = i % 3
        if k == 0:
            U = np.diag(np.exp(2j * np.pi * rng.random(d)))
        elif k == 1:
            U = gen.x_plus(d, 1)
        else:
            U = np.diag(np.exp(2j * np.pi * np.arange(d) / d))
        if i % 7 == 3:
            c = int(rng.integers(0, len(dims)))
            if c != w:
                gates.append(gen.Gate((w,), U, (c,), (int(rng.integers(0, dims[c])),)))
                continue
        gates.append(gen.Gate((w,), U))
    circ = gen.Circuit(dims, gates)
    psi0 = gen.random_state(circ.D, rng)
    plan = qb.qd_plan_circuit(dims, p, circ, mode=qb.QD_FUSE_TILE, max_tile_amps=4096, with_flops=True)
    assert any(t > 0 for t in plan[2]) and max(plan[3]) / circ.D < 150  # tile passes, all light
    got = _run(qb, circ, p, psi0, max_tile_amps=4096)
    assert_close(got, oracle.run_circuit(circ, psi0, nthreads=max(1, oracle.max_threads())), p,
                 f"light passes {prec}")


@pytest.mark.parametrize("max_tile,block_dim", [(4096, 32), (8192, 24), (2048, 32)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tensor_core_blocks_in_tiles(qb, gen, max_tile, block_dim, seed):
    """complex64 tile passes whose composed blocks of 17..32 dimensions run on
    the tensor cores (TF32x3, TMEM-staged classes, per-class norm restoration)."""
    rng = np.random.Generator(np.random.PCG64(600 + seed))
    dims = tuple(int(x) for x in rng.choice([2, 3], size=int(rng.integers(12, 16))))
    circ = gen.random_mixed_circuit(dims, 200, rng)
    psi0 = gen.random_state(circ.D, rng)
    got = _run(qb, circ, qb.QD_C64, psi0, max_tile_amps=max_tile, block_dim=block_dim)
    ref = oracle.run_circuit(circ, psi0, nthreads=max(1, oracle.max_threads()))
    assert_close(got, ref, qb.QD_C64, f"tc tiles {max_tile}/{block_dim} dims={dims}")


def test_tensor_core_tiles_on_benchmark_circuit(qb, gen):
    """The 500-gate 12-qubit + 8-qutrit circuit in tile mode with blocks up to 32
    dimensions, against the oracle; the norm stays 1 (no accumulation drift)."""
    circ = gen.config1_circuit()
    st = qb.State(circ.dims, prec=qb.QD_C64)
    st.run(circ, fuse="tile", max_tile_amps=8192, block_dim=32)
    nrm = st.norm()
    got = st.amplitudes()
    st.close()
    ref = oracle.run_circuit(circ, nthreads=max(1, oracle.max_threads()))
    assert_close(got, ref, qb.QD_C64, "benchmark circuit, tensor-core tiles")
    assert abs(nrm - 1.0) < 1e-5


def test_repeated_circuit_is_built_once_and_stays_exact(qb, gen):
    """A gate list repeated on the same state is planned, composed and
    uploaded once (the second call) and only launched afterwards: every call
    gives the same bits as the first, and changing one matrix entry, the
    fusion settings or the gate order is seen as a different circuit.  The
    library's count of uploaded gate bytes shows the uploads: every call
    uploads except a repeat of an already built circuit."""
    import oracle

    rng = np.random.Generator(np.random.PCG64(515))
    dims = (2, 3, 2, 2, 3, 2, 2, 2, 3, 2, 2, 2)
    c1 = gen.random_mixed_circuit(dims, 120, rng)
    c2 = gen.Circuit(dims, list(c1.gates))
    g = c2.gates[7]
    U = g.U.copy()
    U[0, 0] *= -1.0  # no longer unitary, still a valid gate
    c2.gates[7] = gen.Gate(g.wires, U, g.controls, g.values)
    st = qb.State(dims, prec=qb.QD_C64)
    outs, uploaded = [], []
    for c in (c1, c1, c1, c1, c2, c1, c2, c2, c2):
        st.reset()
        u0 = qb.qd_bytes_uploaded()
        st.run(c, fuse="tile")
        uploaded.append(qb.qd_bytes_uploaded() - u0)
        outs.append(st.raw().copy())
    assert [i for i, u in enumerate(uploaded) if u == 0] == [2, 3, 8], uploaded
    st.reset()
    st.run(c1, fuse="tile", block_dim=4)
    other_opts = st.raw().copy()
    st.close()
    for i in (1, 2, 3, 5):
        assert np.array_equal(outs[i], outs[0])
    for i in (6, 7, 8):
        assert np.array_equal(outs[i], outs[4])
    assert not np.array_equal(outs[4], outs[0])
    assert_close(outs[0], oracle.run_circuit(c1), qb.QD_C64, "repeated circuit")
    assert_close(outs[8], oracle.run_circuit(c2), qb.QD_C64, "changed matrix")
    assert_close(other_opts, oracle.run_circuit(c1), qb.QD_C64, "other fusion settings")
