"""GPU parity of batched independent circuits against the oracle: one-CTA
small circuits, fused programs on auxiliary streams, CUDA-graph capture and
relaunch, and the 8192-circuit batched workload (sampled against the oracle,
norms checked for every circuit)."""
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


def _mixed_batch(gen, seed, n=40):
    rng = np.random.Generator(np.random.PCG64(seed))
    circs = []
    for i in range(n):
        w = int(rng.integers(2, 9)) if i % 4 else int(rng.integers(9, 12))
        dims = tuple(int(x) for x in rng.choice([2, 3, 4, 5], size=w))
        c = gen.random_mixed_circuit(dims, int(rng.integers(5, 120)), rng)
        if i % 7 == 3 and len(dims) >= 2:  # a multi-wire gate: not eligible for the one-CTA path
            P = dims[0] * dims[1]
            if P <= 64:
                c.gates.insert(len(c.gates) // 2, gen.Gate((1, 0), gen.haar(P, rng)))
        circs.append(c)
    return circs


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("use_graph", [False, True])
def test_mixed_batch_against_oracle(qb, gen, prec, use_graph):
    p = qb.QD_C128 if prec == "c128" else qb.QD_C64
    circs = _mixed_batch(gen, 11)
    b = qb.qd_batch_create(p)
    qb.qd_batch_run(b, circs, use_graph=use_graph)
    norms = qb.qd_batch_norms(b, len(circs))
    for i, c in enumerate(circs):
        got = qb.qd_batch_get_amplitudes(b, i)
        ref = oracle.run_circuit(c)
        assert_close(got, ref, p, f"batch circuit {i} dims={c.dims}")
        tol = 1e-12 if p == qb.QD_C128 else 1e-5
        assert abs(norms[i] - oracle.norm(ref)) < tol
    qb.qd_batch_destroy(b)


def test_batch_modes_agree_bitwise(qb, gen):
    """Each circuit's kernels depend only on its own shape: streams, graph
    capture and relaunch give bit-identical states."""
    circs = _mixed_batch(gen, 12, n=24)
    outs = []
    for kw in (dict(n_streams=1), dict(n_streams=8), dict(n_streams=4, use_graph=True)):
        b = qb.qd_batch_create(qb.QD_C64)
        qb.qd_batch_run(b, circs, **kw)
        outs.append([qb.qd_batch_get_amplitudes(b, i) for i in range(len(circs))])
        if kw.get("use_graph"):
            qb.qd_batch_relaunch(b)
            outs.append([qb.qd_batch_get_amplitudes(b, i) for i in range(len(circs))])
        qb.qd_batch_destroy(b)
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert np.array_equal(a, c)


def test_batch_alone_equals_in_batch(qb, gen):
    """A circuit gives the same state alone and among others."""
    circs = _mixed_batch(gen, 13, n=16)
    b = qb.qd_batch_create(qb.QD_C64)
    qb.qd_batch_run(b, circs)
    together = [qb.qd_batch_get_amplitudes(b, i) for i in range(len(circs))]
    for i in (0, 5, 9):
        qb.qd_batch_run(b, [circs[i]])
        assert np.array_equal(qb.qd_batch_get_amplitudes(b, 0), together[i])
    qb.qd_batch_destroy(b)


def test_invalid_circuit_rejects_the_batch(qb, gen):
    circs = _mixed_batch(gen, 14, n=4)
    bad = gen.Circuit((2, 3), [gen.Gate((0,), gen.x_plus(2), (1,), (5,))])  # control value 5 >= 3
    b = qb.qd_batch_create(qb.QD_C64)
    with pytest.raises(qb.QuditError) as ei:
        qb.qd_batch_run(b, circs + [bad])
    assert ei.value.status == qb.QD_ERR_ARG and "circuit 4" in str(ei.value)
    qb.qd_batch_destroy(b)


# Sample rule for the workload's larger circuits (every circuit up to 2^16
# amplitudes is compared): a seeded draw of 24 circuits with D in
# (2^16, 2^18], 24 in (2^18, 2^20] and 16 in (2^20, 2^22].
LARGE_STRATA = ((1 << 16, 1 << 18, 24), (1 << 18, 1 << 20, 24), (1 << 20, 1 << 22, 16))


def test_batched_workload_8192_circuits(qb, gen):
    """8192 circuits (widths 4-12, dims from {2,3,4,5}, depths 20-300), complex64,
    run as one batch under a CUDA graph: every norm within 1e-5 of 1; every
    circuit with D <= 2^16 against the oracle (the one-CTA path up to 8192
    amplitudes and the tile-pass programs on auxiliary streams above it), and
    a stratified seeded sample of 64 circuits with 2^16 < D <= 2^22."""
    circs = gen.config3_batch()
    b = qb.qd_batch_create(qb.QD_C64)
    qb.qd_batch_run(b, circs, use_graph=True)
    norms = qb.qd_batch_norms(b, len(circs))
    assert np.all(np.abs(norms - 1.0) < 1e-5), np.max(np.abs(norms - 1.0))
    rng = np.random.Generator(np.random.PCG64(5))
    chosen = [i for i, c in enumerate(circs) if c.D <= (1 << 16)]
    n_small = len(chosen)
    for lo, hi, k in LARGE_STRATA:
        pool = [i for i, c in enumerate(circs) if lo < c.D <= hi]
        assert len(pool) >= k
        chosen += sorted(int(i) for i in rng.permutation(pool)[:k])
    got = [qb.qd_batch_get_amplitudes(b, i) for i in chosen]
    qb.qd_batch_destroy(b)
    refs = oracle.run_circuits([circs[i] for i in chosen])
    assert n_small > 5000 and sum(1 for i in chosen if circs[i].D > 8192) > 1500
    for i, g, r in zip(chosen, got, refs):
        assert_close(g, r, qb.QD_C64, f"workload circuit {i} (D = {circs[i].D})")


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_layer_queue_and_stream_paths_agree(qb, gen, prec):
    """Larger circuits of a batch through the device-side layer queue (one
    launch per pass position for all of them) and as programs on auxiliary
    streams: both against the oracle, each circuit's norm exactly its
    qd_norm, and the layer path's norms and states the same bits under a
    CUDA graph relaunch."""
    p = qb.QD_C128 if prec == "c128" else qb.QD_C64
    rng = np.random.Generator(np.random.PCG64(31))
    circs = []
    for i in range(30):
        w = int(rng.integers(6, 12))
        dims = tuple(int(x) for x in rng.choice([2, 3, 4, 5], size=w))
        circs.append(gen.random_mixed_circuit(dims, int(rng.integers(20, 200)), rng))
    circs.append(gen.Circuit((2, 3, 2, 3, 2, 3, 2, 3), [gen.Gate((1, 0), gen.haar(6, rng))]))  # not tile-only
    outs = {}
    for path in (qb.QD_BATCH_LAYERS, qb.QD_BATCH_STREAMS):
        b = qb.qd_batch_create(p)
        qb.qd_batch_run(b, circs, small_max_amps=1024, use_graph=True, path=path)
        st = [qb.qd_batch_get_amplitudes(b, i) for i in range(len(circs))]
        nr = qb.qd_batch_norms(b, len(circs))
        qb.qd_batch_relaunch(b)
        assert all(np.array_equal(qb.qd_batch_get_amplitudes(b, i), st[i]) for i in range(len(circs)))
        assert np.array_equal(qb.qd_batch_norms(b, len(circs)), nr)
        qb.qd_batch_destroy(b)
        outs[path] = (st, nr)
    tol = 1e-12 if p == qb.QD_C128 else 1e-5
    for i, c in enumerate(circs):
        ref = oracle.run_circuit(c)
        for path in outs:
            st, nr = outs[path]
            assert_close(st[i], ref, p, f"batch path {path} circuit {i} dims={c.dims}")
            assert abs(nr[i] - oracle.norm(ref)) < tol
        if c.D > 1024:  # outside the one-CTA path: each norm is the bits qd_norm gives the same amplitudes
            s = qb.State(c.dims, prec=p)
            s.set_amplitudes(outs[qb.QD_BATCH_LAYERS][0][i])
            assert s.norm() == outs[qb.QD_BATCH_LAYERS][1][i]
            s.close()
