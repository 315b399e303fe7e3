"""Asynchronous read-back of a state (qd_state_get_raw_async): the same bits
as the synchronous copy in both precisions, with a queued deferred gate
applied first; two states on two streams running circuits in turn, each
read-back overlapping the other state's work and each buffer holding its own
circuit's result against the oracle; a buffer smaller than the state is
rejected."""
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


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_async_read_back_matches_the_synchronous_copy(qb, prec):
    import torch
    from paper_2410_17876_gb300 import inputs as gen

    p = qb.QD_C64 if prec == "c64" else qb.QD_C128
    rng = np.random.Generator(np.random.PCG64(41))
    dims = (2,) * 16 + (3, 3, 2)  # 1,179,648 amplitudes
    circ = gen.random_mixed_circuit(dims, 50, rng)
    st = qb.State(dims, prec=p)
    st.run(circ, fuse="tile")
    st.set_fusion(4)  # a deferred gate still queued when the copy is enqueued
    st.apply(circ.gates[0])
    tdt = torch.complex64 if p == qb.QD_C64 else torch.complex128
    pinned = torch.full((st.D,), float("nan"), dtype=tdt).pin_memory()
    out = pinned.numpy()
    qb.qd_state_get_raw_async(st.handle, out)
    st.synchronize()
    want = st.raw()  # the queued gate was applied before the asynchronous copy
    assert np.array_equal(out, want)
    with pytest.raises(qb.QuditError):
        qb.qd_state_get_raw_async(st.handle, out[:-1])
    st.close()


def test_two_states_on_two_streams_in_turn(qb):
    import torch
    from paper_2410_17876_gb300 import inputs as gen

    rng = np.random.Generator(np.random.PCG64(42))
    dims = (2,) * 12 + (3,) * 4  # 331,776 amplitudes
    circs = [gen.random_mixed_circuit(dims, 60, rng) for _ in range(5)]
    refs = [oracle.run_circuit(c) for c in circs]
    states = [qb.State(dims, prec=qb.QD_C64, stream=torch.cuda.Stream()) for _ in range(2)]
    outs = [torch.zeros(states[0].D, dtype=torch.complex64).pin_memory().numpy() for _ in range(2)]
    got = {}
    for i, c in enumerate(circs):
        s, o = states[i % 2], outs[i % 2]
        s.synchronize()  # the read-back issued two steps ago has landed
        if i >= 2:
            got[i - 2] = o.copy()
        s.reset()
        s.run(c, fuse="tile")
        qb.qd_state_get_raw_async(s.handle, o)
    for i in (len(circs) - 2, len(circs) - 1):
        states[i % 2].synchronize()
        got[i] = outs[i % 2].copy()
    for i, ref in enumerate(refs):
        assert_close(got[i], ref, qb.QD_C64, f"circuit {i}")
    for s in states:
        s.close()
