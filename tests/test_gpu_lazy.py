"""Lazy permutations and phases (qd_set_lazy): single-wire phase / permutation
gates fold into a per-wire frame without a launch; every other gate runs in
that frame; readouts in between (norm, marginal, probabilities) and the final
amplitudes match the oracle."""
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


def _mixed_gates(gen, dims, n, rng):
    gates = []
    for _ in range(n):
        t = int(rng.integers(0, len(dims)))
        d = dims[t]
        k = rng.random()
        if k < 0.45:  # foldable: phases and cyclic shifts
            U = gen.x_plus(d, int(rng.integers(1, d))) if rng.random() < 0.5 else gen.z_gen(d)
            if d == 2 and rng.random() < 0.5:
                U = gen.qubit_t() if rng.random() < 0.5 else gen.qubit_s()
            gates.append(gen.Gate((t,), U))
        elif k < 0.65:
            gates.append(gen.Gate((t,), gen.haar(d, rng) if rng.random() < 0.5 else gen.fourier(d)))
        elif k < 0.9:  # controlled permutation or Haar
            c = int(rng.integers(0, len(dims)))
            if c == t:
                continue
            U = gen.x_plus(d, 1) if rng.random() < 0.5 else gen.haar(d, rng)
            gates.append(gen.Gate((t,), U, (c,), (int(rng.integers(0, dims[c])),)))
        else:  # two-wire Haar
            u = int(rng.integers(0, len(dims)))
            if u == t:
                continue
            gates.append(gen.Gate((t, u), gen.haar(d * dims[u], rng)))
    return gates


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("seed", range(3))
def test_lazy_frame_matches_oracle(qb, gen, prec, seed):
    p = qb.QD_C64 if prec == "c64" else qb.QD_C128
    rng = np.random.Generator(np.random.PCG64(700 + seed))
    dims = tuple(int(x) for x in rng.choice([2, 3, 4], size=9))
    gates = _mixed_gates(gen, dims, 160, rng)
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    st = qb.State(dims, prec=p)
    st.set_amplitudes(psi0)
    st.set_lazy(True)
    ref = psi0
    tol = 1e-12 if p == qb.QD_C128 else 1e-5
    for i, g in enumerate(gates):
        st.apply(g)
        ref = oracle.apply_gate(dims, ref, g)
        if i % 40 == 39:  # readouts that need no materialisation ...
            assert abs(st.norm() - 1.0) < 10 * tol
            w = int(rng.integers(0, len(dims)))
            m_ref = oracle.marginal(dims, ref, w)
            assert np.max(np.abs(st.marginal(w) - m_ref)) < 10 * tol
        if i == 100:  # ... and one that does
            assert np.max(np.abs(st.probabilities() - np.abs(ref) ** 2)) < 10 * tol
    assert_close(st.amplitudes(), ref, p, f"lazy frame {prec}")
    st.close()


def test_foldable_gates_launch_nothing(qb, gen):
    dims = (2, 3, 4, 2, 5)
    rng = np.random.Generator(np.random.PCG64(77))
    gates = [gen.Gate((0,), gen.qubit_t()), gen.Gate((1,), gen.x_plus(3, 2)), gen.Gate((2,), gen.z_gen(4)),
             gen.Gate((4,), gen.x_plus(5, 1)), gen.Gate((1,), gen.z_gen(3)), gen.Gate((3,), gen.x_plus(2, 1))]
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    st = qb.State(dims, prec=qb.QD_C128)
    st.set_amplitudes(psi0)
    st.set_lazy(True)
    n0 = qb.qd_launch_count()
    for g in gates:
        st.apply(g)
    assert qb.qd_launch_count() == n0
    ref = psi0
    for g in gates:
        ref = oracle.apply_gate(dims, ref, g)
    assert_close(st.amplitudes(), ref, qb.QD_C128, "folded gates")
    assert qb.qd_launch_count() - n0 <= len(dims)  # one monomial pass per touched wire
    st.set_lazy(False)
    st.apply(gen.Gate((2,), gen.fourier(4)))
    assert_close(st.amplitudes(), oracle.apply_gate(dims, ref, gen.Gate((2,), gen.fourier(4))), qb.QD_C128,
                 "after set_lazy(False)")
    st.close()


def test_lazy_then_circuit_and_deferred_fusion(qb, gen):
    rng = np.random.Generator(np.random.PCG64(78))
    dims = (3, 2, 2, 4, 3, 2)
    gates = _mixed_gates(gen, dims, 80, rng)
    st = qb.State(dims, prec=qb.QD_C64)
    st.set_lazy(True)
    for g in gates[:40]:
        st.apply(g)
    st.run(gen.Circuit(dims, gates[40:60]), fuse="tile")  # the frame is applied first
    st.set_fusion(64)
    for g in gates[60:]:
        st.apply(g)
    ref = oracle.run_circuit(gen.Circuit(dims, gates))
    assert_close(st.amplitudes(), ref, qb.QD_C64, "lazy + circuit + deferred fusion")
    st.close()
