"""Pins for the FP64 oracle against things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle fails it:
  * transposed ``U`` or a conjugated entry     -> Kronecker / tensor brute force
    (Haar matrices are neither symmetric nor real);
  * wire order reversed (q_0 most significant) -> worked example of section
    "Example Circuit" and brute force on asymmetric dims;
  * wrong control digit or value               -> controlled brute force,
    unmet-control invariance, GHZ closed form;
  * multi-wire local index order               -> tensor contraction brute force;
  * dropped term in a sum                      -> norm preservation, identities.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2410_17876_gb300 import inputs as gen
from tests.brute import kron_unitary, tensor_apply, tensor_marginal, tensor_unitary

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

TINY_DIMS = [(2, 3), (3, 2), (2, 3, 2), (3, 2, 4), (5, 2), (2, 2, 3, 3), (4, 3, 2), (3, 5, 2),
             (2, 2, 2, 2, 2, 2, 2, 2, 2)]


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.split()
    return out


def test_worked_example_of_the_paper():
    g = _read_golden("worked_example_2x3.txt")
    dims = tuple(int(x) for x in g["dims"])
    amp = float(g["amplitude"][0])
    psi = oracle.zero_state(dims)
    psi = oracle.apply_gate(dims, psi, gen.Gate((1,), gen.fourier(3)))
    nz1 = sorted(int(x) for x in g["after_step1_nonzero"])
    assert sorted(np.flatnonzero(np.abs(psi) > 1e-12).tolist()) == nz1
    assert np.allclose(np.abs(psi[nz1]), amp, atol=1e-15)
    psi = oracle.apply_gate(dims, psi, gen.Gate((0,), gen.x_plus(2, 1), (1,), (2,)))
    nz = sorted(int(x) for x in g["final_nonzero"])
    assert sorted(np.flatnonzero(np.abs(psi) > 1e-12).tolist()) == nz
    assert np.allclose(psi[nz], amp, atol=1e-15)  # F[k, 0] = 1/sqrt(3) is real


@pytest.mark.parametrize("dims", TINY_DIMS)
def test_single_gate_matches_kronecker(dims):
    rng = _rng(11 + len(dims))
    D = int(np.prod(dims))
    for t in range(len(dims)):
        U = gen.haar(dims[t], rng)
        psi = gen.random_state(D, rng)
        ref = kron_unitary(dims, t, U) @ psi
        got = oracle.apply_gate(dims, psi, gen.Gate((t,), U))
        assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("dims", TINY_DIMS)
def test_controlled_gate_matches_kronecker(dims):
    rng = _rng(23 + len(dims))
    n = len(dims)
    D = int(np.prod(dims))
    for t in range(n):
        for c in range(n):
            if c == t:
                continue
            for v in range(dims[c]):
                U = gen.haar(dims[t], rng)
                psi = gen.random_state(D, rng)
                ref = kron_unitary(dims, t, U, (c,), (v,)) @ psi
                got = oracle.apply_gate(dims, psi, gen.Gate((t,), U, (c,), (v,)))
                assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("dims", [(2, 3, 2, 3), (3, 2, 4, 2), (2, 2, 2, 2, 2)])
def test_multi_controlled_gate_matches_kronecker(dims):
    rng = _rng(37)
    n = len(dims)
    D = int(np.prod(dims))
    for trial in range(20):
        t = int(rng.integers(n))
        others = [w for w in range(n) if w != t]
        m = int(rng.integers(2, min(3, n - 1) + 1))
        cw = tuple(int(x) for x in rng.permutation(others)[:m])
        cv = tuple(int(rng.integers(dims[c])) for c in cw)
        U = gen.haar(dims[t], rng)
        psi = gen.random_state(D, rng)
        ref = kron_unitary(dims, t, U, cw, cv) @ psi
        got = oracle.apply_gate(dims, psi, gen.Gate((t,), U, cw, cv))
        assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("dims", [(2, 3, 2), (3, 2, 4), (2, 2, 3, 2), (4, 2, 3, 2)])
def test_multi_wire_gate_matches_tensor_contraction(dims):
    rng = _rng(41)
    n = len(dims)
    D = int(np.prod(dims))
    for trial in range(25):
        k = int(rng.integers(2, min(3, n) + 1))
        wires = tuple(int(x) for x in rng.permutation(n)[:k])
        P = int(np.prod([dims[w] for w in wires]))
        rest = [w for w in range(n) if w not in wires]
        if rest and rng.random() < 0.5:
            cw = (int(rest[int(rng.integers(len(rest)))]),)
            cv = (int(rng.integers(dims[cw[0]])),)
        else:
            cw, cv = (), ()
        U = gen.haar(P, rng)
        psi = gen.random_state(D, rng)
        ref = tensor_apply(dims, psi, wires, U, cw, cv)
        got = oracle.apply_gate(dims, psi, gen.Gate(wires, U, cw, cv))
        assert np.max(np.abs(got - ref)) < 1e-14


def test_two_brute_forces_agree_on_single_target():
    """The Kronecker and tensor constructions agree with each other."""
    rng = _rng(43)
    dims = (3, 2, 2)
    for t in range(3):
        U = gen.haar(dims[t], rng)
        for c in [w for w in range(3) if w != t]:
            A = kron_unitary(dims, t, U, (c,), (1,))
            B = tensor_unitary(dims, (t,), U, (c,), (1,))
            assert np.max(np.abs(A - B)) < 1e-15


def test_pins_detect_planted_mistakes():
    """Feeding the oracle the inputs a plausible bug would produce (a transposed
    matrix, reversed wire order, an off-by-one control value) fails the pins."""
    rng = _rng(47)
    dims = (2, 3, 2)
    D = 12
    U = gen.haar(3, rng)
    psi = gen.random_state(D, rng)
    ref = kron_unitary(dims, 1, U, (2,), (1,)) @ psi
    good = oracle.apply_gate(dims, psi, gen.Gate((1,), U, (2,), (1,)))
    assert np.max(np.abs(good - ref)) < 1e-14
    transposed = oracle.apply_gate(dims, psi, gen.Gate((1,), U.T, (2,), (1,)))
    assert np.max(np.abs(transposed - ref)) > 1e-3
    reversed_dims = dims[::-1]
    rev = oracle.apply_gate(reversed_dims, psi, gen.Gate((1,), U, (0,), (1,)))
    assert np.max(np.abs(rev - ref)) > 1e-3
    off = oracle.apply_gate(dims, psi, gen.Gate((1,), U, (2,), (0,)))
    assert np.max(np.abs(off - ref)) > 1e-3


@pytest.mark.parametrize("d", [2, 3, 4, 5, 7])
def test_identities(d):
    rng = _rng(53 + d)
    dims = (2, d, 3)
    D = int(np.prod(dims))
    psi = gen.random_state(D, rng)
    X, Z, F = gen.x_plus(d, 1), gen.z_gen(d), gen.fourier(d)
    ap = lambda s, M: oracle.apply_gate(dims, s, gen.Gate((1,), M))
    # X_d^d = I
    s = psi
    for _ in range(d):
        s = ap(s, X)
    assert np.max(np.abs(s - psi)) < 1e-14
    # F_d^4 = I and F_d^2 = parity permutation |j> -> |-j mod d>
    s2 = ap(ap(psi, F), F)
    par = np.zeros((d, d))
    for j in range(d):
        par[(-j) % d, j] = 1.0
    assert np.max(np.abs(s2 - ap(psi, par))) < 1e-13
    s4 = ap(ap(s2, F), F)
    assert np.max(np.abs(s4 - psi)) < 1e-13
    # Z X = omega X Z
    w = np.exp(2j * np.pi / d)
    zx = ap(ap(psi, X), Z)
    xz = ap(ap(psi, Z), X)
    assert np.max(np.abs(zx - w * xz)) < 1e-14
    # U then U^dagger
    U = gen.haar(d, rng)
    back = ap(ap(psi, U), U.conj().T)
    assert np.max(np.abs(back - psi)) < 1e-14


def test_unmet_control_leaves_state_unchanged():
    rng = _rng(59)
    dims = (3, 2, 3, 2)
    D = int(np.prod(dims))
    # every basis state whose control digit differs from the value is untouched
    b = np.cumprod((1,) + dims[:-1])
    for j in range(D):
        e = np.zeros(D, dtype=np.complex128)
        e[j] = 1.0
        xc = (j // b[2]) % dims[2]
        v = (xc + 1) % dims[2]
        out = oracle.apply_gate(dims, e, gen.Gate((0,), gen.haar(3, rng), (2,), (v,)))
        assert np.array_equal(out, e)


def test_norm_preserved_on_random_circuits():
    for seed in range(3):
        c = gen.config0_circuit(seed=100 + seed, depth=200)
        psi = oracle.run_circuit(c)
        assert abs(oracle.norm(psi) - 1.0) < 1e-13


@pytest.mark.parametrize("dims,root", [((2,) * 10, 0), ((3,) * 6, 2), ((4, 4, 4, 4), 3),
                                       ((5, 5, 5), 1), ((2, 3, 4, 5, 3), 0), ((3, 3, 4, 5), 1)])
def test_ghz_closed_form(dims, root):
    """F on the root then controlled X_{+v}: sum_k |k...k> / sqrt(d_root); exactly
    d_root non-zero amplitudes (the count the paper states for GHZ circuits)."""
    c = gen.ghz_circuit(dims, root)
    psi = oracle.run_circuit(c)
    d = dims[root]
    b = np.cumprod((1,) + tuple(dims[:-1]))
    idx = [int(k * b.sum()) for k in range(d)]
    expect = np.zeros(int(np.prod(dims)), dtype=np.complex128)
    expect[idx] = 1.0 / math.sqrt(d)
    assert np.max(np.abs(psi - expect)) < 1e-14
    assert int(np.count_nonzero(np.abs(psi) > 1e-12)) == d


def test_readouts_against_independent_sums():
    rng = _rng(61)
    dims = (3, 2, 5, 2)
    psi = gen.random_state(int(np.prod(dims)), rng) * 1.7
    p = np.abs(psi) ** 2
    assert abs(oracle.norm(psi) - math.fsum(p.tolist())) < 1e-15 * max(1.0, math.fsum(p.tolist()))
    assert np.max(np.abs(oracle.probabilities(psi) - p)) < 1e-15
    for w in range(len(dims)):
        assert np.max(np.abs(oracle.marginal(dims, psi, w) - tensor_marginal(dims, psi, w))) < 1e-14


def test_oracle_rejects_invalid_gates():
    dims = (2, 3)
    psi = oracle.zero_state(dims)
    with pytest.raises(ValueError):
        oracle.apply_gate(dims, psi, gen.Gate((0,), gen.x_plus(2), (0,), (1,)))  # control == target
    with pytest.raises(ValueError):
        oracle.apply_gate(dims, psi, gen.Gate((0,), gen.x_plus(2), (1,), (3,)))  # value >= d_c
    with pytest.raises(ValueError):
        oracle.apply_gate(dims, psi, gen.Gate((2,), gen.x_plus(2)))  # wire out of range
