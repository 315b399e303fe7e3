"""qd_norm_noalloc: the norm for callers that cannot allocate device memory.

A framework whose caching allocator owns all device memory, or a loop that
must not stall on an allocation, cannot create a qd_state (that allocates a
reduction workspace).  qd_norm_noalloc reads caller-owned amplitudes and
writes one caller-owned device double, keeping its partial sums in a fixed
array inside the library.  These tests call it through the C ABI twice in a
row on states of different sizes and check every result against qd_norm on
the same amplitudes, bit for bit as its declaration promises -- also for a
complex64 pointer that is 8- but not 16-byte aligned (one amplitude into a
buffer), whose amplitudes are compared with a state holding the same values
and with the oracle's norm.  The file is collected last.
"""
import numpy as np
import pytest

import __graft_entry__
import oracle

pytestmark = pytest.mark.gpu

NORM_RTOL = 1e-13  # the readout tolerance of the other tests, for the oracle comparison


def _setup():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    __graft_entry__.build()
    from paper_2410_17876_gb300 import binding as qb
    from paper_2410_17876_gb300 import inputs as gen

    return torch, qb, gen


def test_norm_noalloc_matches_qd_norm_on_two_calls_in_a_row():
    torch, qb, gen = _setup()
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
                assert got == ref, (prec, dims, call, got, ref)
            st.close()


@pytest.mark.parametrize("dims", [(3, 3, 3, 5, 5, 7, 11), (7,)])  # 51,975 and 7 amplitudes
def test_norm_noalloc_on_8_byte_aligned_complex64(dims):
    """Amplitudes 1..D of a complex64 buffer (the pointer is 8 mod 16): the
    same bits as qd_norm of a state holding the same values, and the oracle's
    norm of those values within the readout tolerance."""
    torch, qb, gen = _setup()
    rng = np.random.Generator(np.random.PCG64(77))
    stream = torch.cuda.current_stream()
    D = int(np.prod(dims))
    vals = (gen.random_state(D, rng) * 1.7).astype(np.complex64)
    buf = torch.zeros(2 * (D + 1), dtype=torch.float32, device="cuda")
    buf[2:] = torch.from_numpy(vals.view(np.float32).copy()).cuda()
    ptr = buf.data_ptr() + 8
    assert ptr % 16 == 8
    st = qb.State(dims, prec=qb.QD_C64, stream=stream)
    st.buf.copy_(buf[2:])
    ref = st.norm()
    st.close()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        qb.qd_norm_noalloc(ptr, D, qb.QD_C64, stream.cuda_stream, out.data_ptr())
        stream.synchronize()
        got = float(out.item())
        assert got == ref, (got, ref)
    want = oracle.norm(vals.astype(np.complex128))
    assert abs(got - want) <= NORM_RTOL * want, (got, want)


def test_norm_noalloc_rejects_bad_sizes():
    torch, qb, _ = _setup()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for bad in (0, -5, (1 << 44) + 1):
        with pytest.raises(qb.QuditError) as ei:
            qb.qd_norm_noalloc(buf.data_ptr(), bad, qb.QD_C128, 0, out.data_ptr())
        assert ei.value.status == qb.QD_ERR_ARG
        assert "amplitudes" in qb.qd_last_error()
