"""qd_norm_noalloc: the norm for callers that cannot allocate device memory.

Code running under CUDA-graph capture, inside a framework whose caching
allocator owns all device memory, or in a loop that must not stall on an
allocation cannot create a qd_state (that allocates a reduction workspace).
qd_norm_noalloc reads caller-owned amplitudes and writes one caller-owned
device double, keeping its partial sums in a fixed array inside the library.
This test calls it through the C ABI twice in a row on each of two states of
different sizes and checks every result against qd_norm on the same
amplitudes, within the norm tolerance of the other tests (relative 1e-13).
It sits in a file of its own, collected last.
"""
import numpy as np
import pytest

import __graft_entry__

pytestmark = pytest.mark.gpu

NORM_RTOL = 1e-13


def test_norm_noalloc_matches_qd_norm_on_two_calls_in_a_row():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    __graft_entry__.build()
    from paper_2410_17876_gb300 import binding as qb
    from paper_2410_17876_gb300 import inputs as gen

    rng = np.random.Generator(np.random.PCG64(2024))
    stream = torch.cuda.current_stream()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    cases = [((3, 2, 5, 2, 4, 3, 2, 2, 3, 2, 3), 1.3), ((2, 3), 0.7)]  # 51,840 amplitudes, then 6
    for prec in (qb.QD_C128, qb.QD_C64):
        for dims, scale in cases:
            st = qb.State(dims, prec=prec, stream=stream)
            st.set_amplitudes(gen.random_state(st.D, rng) * scale)
            ref = st.norm()  # existing entry point, through its qd_state
            for call in range(2):
                out.fill_(float("nan"))
                qb.qd_norm_noalloc(st.buf.data_ptr(), st.D, prec, stream.cuda_stream, out.data_ptr())
                stream.synchronize()
                got = float(out.item())
                assert abs(got - ref) <= NORM_RTOL * ref, (prec, dims, call, got, ref)
            st.close()


def test_norm_noalloc_rejects_bad_sizes():
    import torch

    __graft_entry__.build()
    from paper_2410_17876_gb300 import binding as qb

    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for bad in (0, -5, (1 << 44) + 1):
        with pytest.raises(qb.QuditError) as ei:
            qb.qd_norm_noalloc(buf.data_ptr(), bad, qb.QD_C128, 0, out.data_ptr())
        assert ei.value.status == qb.QD_ERR_ARG
        assert "amplitudes" in qb.qd_last_error()
