"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Sizes span several thread blocks with a ragged tail; every wire is used as
target and as control; every matrix kind (dense, diagonal with unit
entries, pure and phased permutation) and multi-wire gates up to P = 64 run
in both precisions.  Tolerances: complex128 max |d amp| <= 1e-12; complex64
max |d amp| <= 1e-5 and infidelity <= 1e-6.
"""
import math

import numpy as np
import pytest

import __graft_entry__
import oracle
from tests.gpu_util import assert_close, infidelity

pytestmark = pytest.mark.gpu

PRECS = ["c128", "c64"]


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


def _prec(qb, name):
    return qb.QD_C128 if name == "c128" else qb.QD_C64


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _run_both(qb, dims, gates, psi0, prec):
    st = qb.State(dims, prec=prec)
    st.set_amplitudes(psi0)
    for g in gates:
        st.apply(g)
    got = st.amplitudes()
    st.close()
    ref = psi0
    for g in gates:
        ref = oracle.apply_gate(dims, ref, g)
    return got, ref


@pytest.mark.parametrize("prec", PRECS)
def test_config0_full_circuit(qb, gen, prec):
    circ = gen.config0_circuit(seed=0, depth=200)
    st = qb.State(circ.dims, prec=_prec(qb, prec))
    st.run(circ)
    got = st.amplitudes()
    st.close()
    ref = oracle.run_circuit(circ)
    assert_close(got, ref, _prec(qb, prec), "config0")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(3, 2, 5, 2, 3, 4, 2, 3, 5, 2), (2, 2, 3, 2, 2, 2, 3, 2, 2, 2, 2, 2, 3),
                                  (3, 3, 5, 3, 3, 3, 5, 3, 3)])
def test_every_wire_every_kind(qb, gen, prec, dims):
    """Each wire as target with each matrix kind, plain and controlled by every other wire."""
    rng = _rng(sum(dims))
    p = _prec(qb, prec)
    D = int(np.prod(dims))
    n = len(dims)
    psi0 = gen.random_state(D, rng)
    gates = []
    for t in range(n):
        d = dims[t]
        phased = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, d))) @ gen.x_plus(d, 2 % d or 1)
        tdiag = np.eye(d, dtype=np.complex128)
        tdiag[d - 1, d - 1] = np.exp(1j * np.pi / 4)  # one non-unit row (T-like)
        mats = [gen.haar(d, rng), gen.z_gen(d), tdiag, gen.x_plus(d, 1), phased, gen.fourier(d)]
        for M in mats:
            gates.append(gen.Gate((t,), M))
        for c in range(n):
            if c != t:
                v = int(rng.integers(dims[c]))
                gates.append(gen.Gate((t,), mats[int(rng.integers(len(mats)))], (c,), (v,)))
    got, ref = _run_both(qb, dims, gates, psi0, p)
    assert_close(got, ref, p, f"dims={dims}")


@pytest.mark.parametrize("prec", PRECS)
def test_multi_controlled(qb, gen, prec):
    rng = _rng(5)
    p = _prec(qb, prec)
    dims = (2, 3, 2, 4, 2, 3, 2, 2, 5, 2)
    D = int(np.prod(dims))
    n = len(dims)
    psi0 = gen.random_state(D, rng)
    gates = []
    for _ in range(60):
        t = int(rng.integers(n))
        others = [w for w in range(n) if w != t]
        m = int(rng.integers(1, 6))
        cw = tuple(int(x) for x in rng.permutation(others)[:m])
        cv = tuple(int(rng.integers(dims[c])) for c in cw)
        gates.append(gen.Gate((t,), gen.haar(dims[t], rng), cw, cv))
    # all other wires as controls (a single class is touched)
    cw = tuple(w for w in range(n) if w != 3)
    gates.append(gen.Gate((3,), gen.haar(4, rng), cw, tuple(dims[c] - 1 for c in cw)))
    got, ref = _run_both(qb, dims, gates, psi0, p)
    assert_close(got, ref, p, "multi-controlled")


@pytest.mark.parametrize("prec", PRECS)
def test_multi_wire_gates(qb, gen, prec):
    rng = _rng(7)
    p = _prec(qb, prec)
    dims = (2, 4, 3, 2, 4, 2, 3, 2, 4, 2)
    D = int(np.prod(dims))
    n = len(dims)
    psi0 = gen.random_state(D, rng)
    gates = []
    for _ in range(30):
        k = int(rng.integers(2, 4))
        while True:
            wires = tuple(int(x) for x in rng.permutation(n)[:k])
            P = int(np.prod([dims[w] for w in wires]))
            if P <= 64:
                break
        rest = [w for w in range(n) if w not in wires]
        if rng.random() < 0.4:
            cw = (int(rest[int(rng.integers(len(rest)))]),)
            cv = (int(rng.integers(dims[cw[0]])),)
        else:
            cw, cv = (), ()
        gates.append(gen.Gate(wires, gen.haar(P, rng), cw, cv))
    # maximum gate dimension: 4 x 4 x 4 = 64 and 2^6 = 64
    gates.append(gen.Gate((1, 4, 8), gen.haar(64, rng)))
    gates.append(gen.Gate((0, 3, 5, 7, 9), gen.haar(32, rng)))
    got, ref = _run_both(qb, dims, gates, psi0, p)
    assert_close(got, ref, p, "multi-wire")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d", [6, 7, 8, 16, 64])
def test_wide_single_wire(qb, gen, prec, d):
    rng = _rng(d)
    p = _prec(qb, prec)
    dims = (3, d, 2, 5) if d <= 16 else (2, d, 3)
    D = int(np.prod(dims))
    psi0 = gen.random_state(D, rng)
    gates = [gen.Gate((1,), gen.haar(d, rng)), gen.Gate((1,), gen.x_plus(d, 3)), gen.Gate((1,), gen.z_gen(d)),
             gen.Gate((0,), gen.haar(dims[0], rng), (1,), (d - 1,)),
             gen.Gate((1,), gen.fourier(d), (0,), (1,))]
    got, ref = _run_both(qb, dims, gates, psi0, p)
    assert_close(got, ref, p, f"d={d}")


@pytest.mark.parametrize("prec", PRECS)
def test_readouts(qb, gen, prec):
    rng = _rng(13)
    p = _prec(qb, prec)
    dims = (3, 2, 5, 2, 4, 3, 2, 2, 3)
    D = int(np.prod(dims))
    psi = gen.random_state(D, rng) * 1.3
    st = qb.State(dims, prec=p)
    st.set_amplitudes(psi)
    if p == qb.QD_C64:
        psi = psi.astype(np.complex64).astype(np.complex128)  # what the state holds
    assert abs(st.norm() - oracle.norm(psi)) <= 1e-13 * oracle.norm(psi)
    assert np.max(np.abs(st.probabilities() - oracle.probabilities(psi))) <= 1e-15
    for w in range(len(dims)):
        assert np.max(np.abs(st.marginal(w) - oracle.marginal(dims, psi, w))) <= 1e-13
    st.close()


@pytest.mark.parametrize("prec", PRECS)
def test_identity_and_unmet_controls_leave_state_unchanged(qb, gen, prec):
    rng = _rng(17)
    p = _prec(qb, prec)
    dims = (2, 3, 2, 3, 2)
    D = int(np.prod(dims))
    psi = gen.random_state(D, rng)
    st = qb.State(dims, prec=p)
    st.set_amplitudes(psi)
    before = st.raw().copy()
    st.apply(gen.Gate((1,), np.eye(3)))
    assert np.array_equal(st.raw(), before)
    # basis state with control digit 0; controlled on value 1 -> untouched
    e = np.zeros(D, dtype=np.complex128)
    e[2] = 1.0  # digits: q0=0, q1=1, rest 0
    st.set_amplitudes(e)
    st.apply(gen.Gate((1,), gen.haar(3, rng), (3,), (1,)))
    assert np.array_equal(st.amplitudes(), e)
    st.close()


@pytest.mark.parametrize("prec", PRECS)
def test_worked_example_of_the_paper(qb, gen, prec):
    """Section "Example Circuit": dims (2, 3), F_3 on q_1, CX target q_0 control q_1 = 2."""
    st = qb.State((2, 3), prec=_prec(qb, prec))
    st.apply(gen.Gate((1,), gen.fourier(3)))
    st.apply(gen.Gate((0,), gen.x_plus(2, 1), (1,), (2,)))
    got = st.amplitudes()
    st.close()
    expect = np.zeros(6, dtype=np.complex128)
    expect[[0, 2, 5]] = 1 / math.sqrt(3)
    assert_close(got, expect, _prec(qb, prec), "worked example")


def test_state_create_and_wrap_agree(qb, gen):
    circ = gen.config0_circuit(seed=3, depth=120)
    h = qb.qd_state_create(circ.dims, qb.QD_C128)
    for g in circ.gates:
        if len(g.controls):
            qb.qd_apply_controlled(h, g.wires[0], g.U, g.controls, g.values)
        else:
            qb.qd_apply_gate(h, g.wires[0], g.U)
    a = qb.qd_state_get_amplitudes(h)
    qb.qd_state_destroy(h)
    st = qb.State(circ.dims, prec=qb.QD_C128)
    st.run(circ)
    b = st.amplitudes()
    st.close()
    assert np.array_equal(a, b)  # same kernels, same order: bitwise equal


def test_results_are_deterministic(qb, gen):
    circ = gen.config0_circuit(seed=4, depth=200)
    outs = []
    for _ in range(2):
        st = qb.State(circ.dims, prec=qb.QD_C64)
        st.run(circ)
        outs.append((st.raw().copy(), st.norm()))
        st.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


@pytest.mark.parametrize("dims,root", [((2,) * 24, 0), ((3,) * 15, 7), ((2, 3, 4, 3, 2, 3, 4, 2, 2, 3, 3, 2), 0)])
def test_ghz_closed_form_at_size(qb, gen, dims, root):
    """Property at any size: exactly d_root non-zeros of 1/sqrt(d_root) at |k...k>."""
    c = gen.ghz_circuit(dims, root)
    for p in (qb.QD_C128, qb.QD_C64):
        st = qb.State(dims, prec=p)
        st.run(c)
        a = st.raw()
        st.close()
        d = dims[root]
        b = np.cumprod((1,) + tuple(dims[:-1]))
        idx = np.array([k * int(b.sum()) for k in range(d)])
        tol = 1e-15 if p == qb.QD_C128 else 1e-7
        nz = np.flatnonzero(np.abs(a) > tol)
        assert np.array_equal(nz, idx)
        assert np.max(np.abs(a[idx] - 1 / math.sqrt(d))) < (1e-15 if p == qb.QD_C128 else 1e-7)


def test_invalid_arguments_report_errors(qb, gen):
    st = qb.State((2, 3, 2), prec=qb.QD_C64)
    with pytest.raises(qb.QuditError) as ei:
        qb.qd_apply_controlled(st.handle, 0, gen.x_plus(2), [0], [1])
    assert ei.value.status == qb.QD_ERR_ARG
    with pytest.raises(qb.QuditError):
        qb.qd_apply_gate(st.handle, 3, gen.x_plus(2))
    # the state is still usable afterwards
    st.apply(gen.Gate((1,), gen.fourier(3)))
    assert abs(st.norm() - 1.0) < 1e-6
    st.close()
