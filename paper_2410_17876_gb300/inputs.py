"""Seeded synthetic inputs: gate matrices and circuits.

This module is shared by the CUDA path, the CPU oracle, the tests and the
benchmark.  It builds *inputs only*: explicit complex128 gate matrices and
ordered gate lists.  It contains none of the block-simulation arithmetic
(no state vector is ever touched here), so that neither side of a parity
comparison can inherit a mistake from the other through it.

Conventions (paper, section "Proposed Methodology"):
  * wire ``q_0`` is the least significant digit of a basis index, so the
    stride of wire ``i`` is ``prod(dims[:i])``;
  * a gate acting on several wires lists them first-least-significant:
    the local row index of a multi-wire gate is
    ``sum_m digit(w_m) * prod(dims[w_0..w_{m-1}])``.

Gate definitions the paper names but does not spell out:
  * generalized Fourier (the paper's "generalized Hadamard"):
    ``F_d[j, k] = omega^(j k) / sqrt(d)`` with ``omega = exp(2 pi i / d)``;
  * generalized Z: ``Z_d = diag(omega^j)``;
  * generalized NOT ``X_{+a}`` (section "Permutation Gates"):
    ``|j> -> |(j + a) mod d>``, i.e. ``X[(j + a) mod d, j] = 1``;
  * qubit ``S = diag(1, i)``, ``T = diag(1, exp(i pi / 4))``;
  * Haar-random unitaries: QR of an i.i.d. complex Gaussian matrix with the
    phases of ``diag(R)`` divided out (Mezzadri, "How to generate random
    matrices from the classical compact groups", Notices AMS 2007).

Random draws use ``numpy.random.Generator(PCG64(seed))`` in a fixed order.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

__all__ = [
    "Gate", "Circuit", "haar", "haar_batch", "x_plus", "z_gen", "fourier", "qubit_s",
    "qubit_t", "random_state", "config0_circuit", "config1_circuit",
    "config2_circuit", "prefix_circuit", "config3_batch", "config4_trace",
    "random_mixed_circuit", "ghz_circuit", "product_circuit", "amp_gate_updates",
    "circuit_from_arrays",
]


# ----------------------------------------------------------------------------
# Gate and circuit containers
# ----------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Gate:
    """One gate: a ``P x P`` complex matrix on ``wires`` with optional controls.

    ``wires`` lists the target wires, first-listed least significant in the
    local index (``P = prod(dims[w] for w in wires)``).  ``controls`` and
    ``values`` are the two lists of the section "Controlled and
    Multi-Controlled Gates": the gate acts only on basis states whose digit
    on ``controls[m]`` equals ``values[m]`` for every ``m``.
    """

    wires: Tuple[int, ...]
    U: np.ndarray
    controls: Tuple[int, ...] = ()
    values: Tuple[int, ...] = ()
    name: str = "U"

    def __post_init__(self):
        object.__setattr__(self, "wires", tuple(int(w) for w in self.wires))
        object.__setattr__(self, "controls", tuple(int(c) for c in self.controls))
        object.__setattr__(self, "values", tuple(int(v) for v in self.values))
        U = np.ascontiguousarray(np.asarray(self.U, dtype=np.complex128))
        object.__setattr__(self, "U", U)

    @classmethod
    def _trusted(cls, wires: Tuple[int, ...], U: np.ndarray, controls: Tuple[int, ...] = (),
                 values: Tuple[int, ...] = (), name: str = "U") -> "Gate":
        """The same gate as ``Gate(...)`` from arguments that already have the
        normalised types (tuples of ints, a C-contiguous complex128 matrix):
        the generators build millions of gates, and the conversions dominate."""
        g = object.__new__(cls)
        g.__dict__.update(wires=wires, U=U, controls=controls, values=values, name=name)
        return g


@dataclasses.dataclass
class Circuit:
    """Wire dimensions (``q_0`` first) and an ordered gate list."""

    dims: Tuple[int, ...]
    gates: List[Gate]

    @property
    def D(self) -> int:
        return int(np.prod(np.asarray(self.dims, dtype=np.int64)))

    @property
    def n(self) -> int:
        return len(self.dims)


def amp_gate_updates(circ: Circuit) -> int:
    """Logical amplitude-gate updates: sum over gates of ``D / prod(d_controls)``."""
    D = circ.D
    total = 0
    for g in circ.gates:
        div = 1
        for c in g.controls:
            div *= circ.dims[c]
        total += D // div
    return total


# ----------------------------------------------------------------------------
# Gate matrices
# ----------------------------------------------------------------------------
def haar(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random ``d x d`` unitary (Mezzadri 2007: QR plus phase fix)."""
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    diag = np.diagonal(r)
    ph = diag / np.abs(diag)
    return np.ascontiguousarray(q * ph[np.newaxis, :])


def x_plus(d: int, a: int = 1) -> np.ndarray:
    """Generalized NOT: ``|j> -> |(j + a) mod d>``."""
    m = np.zeros((d, d), dtype=np.complex128)
    for j in range(d):
        m[(j + a) % d, j] = 1.0
    return m


def z_gen(d: int) -> np.ndarray:
    """Generalized Z: ``diag(omega^j)``, ``omega = exp(2 pi i / d)``."""
    return np.diag(np.exp(2j * np.pi * np.arange(d) / d)).astype(np.complex128)


def fourier(d: int) -> np.ndarray:
    """Generalized Fourier (Hadamard for ``d = 2``): ``omega^(jk) / sqrt(d)``."""
    j = np.arange(d)
    return (np.exp(2j * np.pi * np.outer(j, j) / d) / math.sqrt(d)).astype(np.complex128)


def qubit_s() -> np.ndarray:
    return np.diag([1.0, 1.0j]).astype(np.complex128)


def qubit_t() -> np.ndarray:
    return np.diag([1.0, np.exp(1j * np.pi / 4)]).astype(np.complex128)


def random_state(D: int, rng: np.random.Generator) -> np.ndarray:
    """Normalised complex Gaussian state of length ``D``."""
    v = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    return v / np.linalg.norm(v)


# ----------------------------------------------------------------------------
# Circuit generators (one per workload shape)
# ----------------------------------------------------------------------------
def haar_batch(d: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """``m`` Haar-random ``d x d`` unitaries (the same construction as :func:`haar`, batched)."""
    if m == 0:
        return np.zeros((0, d, d), dtype=np.complex128)
    z = (rng.standard_normal((m, d, d)) + 1j * rng.standard_normal((m, d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    diag = np.diagonal(r, axis1=1, axis2=2)
    ph = diag / np.abs(diag)
    return np.ascontiguousarray(q * ph[:, np.newaxis, :])


def random_mixed_circuit(dims: Sequence[int], depth: int, rng: np.random.Generator) -> Circuit:
    """``depth`` gates of the 50/20/30 mix: Haar single-wire / one of
    {X_{+1}, Z_d, F_d} / controlled (a control wire different from the
    target, a control value uniform in ``[0, d_c)``, and a target matrix
    that is X_{+1} or Haar with equal probability).  Wires are uniform.

    The gate skeleton is drawn first (fixed order of vectorised draws), then
    the Haar matrices, batched per dimension in gate order.
    """
    dims = tuple(int(x) for x in dims)
    n = len(dims)
    u = rng.random(depth)
    t = rng.integers(n, size=depth)
    k3 = rng.integers(3, size=depth)
    craw = rng.integers(max(n - 1, 1), size=depth)
    vu = rng.random(depth)
    xhalf = rng.random(depth) < 0.5
    kind = np.where((u < 0.5) | (n == 1), 0, np.where(u < 0.7, 1, 2))
    need_haar = (kind == 0) | ((kind == 2) & ~xhalf)
    tdims = np.asarray(dims)[t]
    mats = {}
    for d in sorted(set(int(x) for x in tdims[need_haar])):
        idx = np.flatnonzero(need_haar & (tdims == d))
        mats.update(zip(idx.tolist(), haar_batch(d, len(idx), rng)))
    gates: List[Gate] = []
    fixed = {}
    mk = Gate._trusted
    tl, kl, k3l, cl, vl, xl = t.tolist(), kind.tolist(), k3.tolist(), craw.tolist(), vu.tolist(), xhalf.tolist()
    for i in range(depth):
        ti = tl[i]
        d = dims[ti]
        if kl[i] == 0:
            gates.append(mk((ti,), mats[i], name="haar"))
        elif kl[i] == 1:
            key = (d, k3l[i])
            if key not in fixed:
                fixed[key] = (x_plus(d, 1), z_gen(d), fourier(d))[key[1]]
            gates.append(mk((ti,), fixed[key], name=("X", "Z", "F")[key[1]]))
        else:
            c = cl[i]
            if c >= ti:
                c += 1
            v = int(vl[i] * dims[c])
            if xl[i]:
                key = (d, "x")
                if key not in fixed:
                    fixed[key] = x_plus(d, 1)
                gates.append(mk((ti,), fixed[key], (c,), (v,), name="CX"))
            else:
                gates.append(mk((ti,), mats[i], (c,), (v,), name="CU"))
    return Circuit(dims, gates)


def config0_circuit(seed: int = 0, depth: int = 200) -> Circuit:
    """3 qubits + 3 qutrits (216 amplitudes), ``depth`` gates of the mix."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return random_mixed_circuit((2, 2, 2, 3, 3, 3), depth, rng)


def config1_circuit(seed: int = 1, depth: int = 500) -> Circuit:
    """12 qubits + 8 qutrits in a seeded wire order, Clifford+T-like mix.

    70% single-wire gates (qubit wire: H, S, T uniform; qutrit wire: F_3,
    Z_3, X_3 uniform), 30% two-wire gates (qubit target: CNOT with a qubit
    control; qutrit target: controlled X_3 with any control wire), the
    control value being the control wire's highest level ``d_c - 1``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = tuple(int(x) for x in rng.permutation([2] * 12 + [3] * 8))
    n = len(dims)
    qubits = [i for i in range(n) if dims[i] == 2]
    gates: List[Gate] = []
    H, S, T = fourier(2), qubit_s(), qubit_t()
    F3, Z3, X3 = fourier(3), z_gen(3), x_plus(3, 1)
    for _ in range(depth):
        t = int(rng.integers(n))
        if rng.random() < 0.7:
            k = int(rng.integers(3))
            if dims[t] == 2:
                gates.append(Gate((t,), (H, S, T)[k], name=("H", "S", "T")[k]))
            else:
                gates.append(Gate((t,), (F3, Z3, X3)[k], name=("F3", "Z3", "X3")[k]))
        else:
            if dims[t] == 2:
                pool = [q for q in qubits if q != t]
                c = int(pool[int(rng.integers(len(pool)))])
                gates.append(Gate((t,), x_plus(2, 1), (c,), (1,), name="CNOT"))
            else:
                c = int(rng.integers(n - 1))
                if c >= t:
                    c += 1
                gates.append(Gate((t,), X3, (c,), (dims[c] - 1,), name="CX3"))
    return Circuit(dims, gates)


def config2_circuit(seed: int = 2, depth: int = 200, n_qubits: int = 18,
                    n_qutrits: int = 8) -> Circuit:
    """Large state: 18 qubits + 8 qutrits, 70% Haar single, 30% controlled."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = tuple(int(x) for x in rng.permutation([2] * n_qubits + [3] * n_qutrits))
    n = len(dims)
    gates: List[Gate] = []
    for _ in range(depth):
        t = int(rng.integers(n))
        d = dims[t]
        if rng.random() < 0.7:
            gates.append(Gate((t,), haar(d, rng), name="haar"))
        else:
            c = int(rng.integers(n - 1))
            if c >= t:
                c += 1
            v = int(rng.integers(dims[c]))
            if rng.random() < 0.5:
                gates.append(Gate((t,), x_plus(d, 1), (c,), (v,), name="CX"))
            else:
                gates.append(Gate((t,), haar(d, rng), (c,), (v,), name="CU"))
    return Circuit(dims, gates)


def redraw_haar(circ: Circuit, seed: int) -> Circuit:
    """The same circuit with every gate named "haar" or "CU" given a fresh
    Haar matrix of its size (seeded): the same wires, controls and gate kinds,
    so the same work, with new matrices."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gates = []
    for g in circ.gates:
        U = haar(g.U.shape[0], rng) if g.name in ("haar", "CU") else g.U
        gates.append(Gate(g.wires, U, g.controls, g.values, name=g.name))
    return Circuit(circ.dims, gates)


def prefix_circuit(circ: Circuit, n_prefix: int) -> Circuit:
    """The gates of ``circ`` whose wires all lie in the lowest ``n_prefix`` wires."""
    keep = []
    for g in circ.gates:
        if all(w < n_prefix for w in g.wires + g.controls):
            keep.append(g)
    return Circuit(tuple(circ.dims[:n_prefix]), keep)


def config3_batch(seed: int = 3, n_circuits: int = 8192, wmin: int = 4,
                  wmax: int = 12, dmin: int = 20, dmax: int = 300,
                  dim_choices: Sequence[int] = (2, 3, 4, 5)) -> List[Circuit]:
    """Independent small circuits: width U{wmin..wmax}, dims i.i.d. from
    ``dim_choices``, depth U{dmin..dmax}, gate mix as ``config0_circuit``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_circuits):
        w = int(rng.integers(wmin, wmax + 1))
        dims = tuple(int(dim_choices[int(rng.integers(len(dim_choices)))]) for _ in range(w))
        depth = int(rng.integers(dmin, dmax + 1))
        out.append(random_mixed_circuit(dims, depth, rng))
    return out


def config4_trace(seed: int = 4, rate: float = 2000.0, duration: float = 10.0,
                  wmin: int = 4, wmax: int = 16, dim_choices: Sequence[int] = (2, 3, 4),
                  dmin_amp: int = 16, dmax_amp: int = 16_000_000, depth_min: int = 50,
                  depth_max: int = 500, max_requests: int | None = None
                  ) -> List[Tuple[float, Circuit]]:
    """Poisson arrivals of circuits for the serving loop.

    Widths U{wmin..wmax}, dims i.i.d. from ``dim_choices``, rejection-sampled
    so that ``dmin_amp <= D <= dmax_amp``; depths U{depth_min..depth_max};
    gate mix as ``config0_circuit``.  Returns ``(arrival_seconds, circuit)``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out: List[Tuple[float, Circuit]] = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration or (max_requests is not None and len(out) >= max_requests):
            break
        while True:
            w = int(rng.integers(wmin, wmax + 1))
            dims = tuple(int(dim_choices[int(rng.integers(len(dim_choices)))]) for _ in range(w))
            D = int(np.prod(dims))
            if dmin_amp <= D <= dmax_amp:
                break
        depth = int(rng.integers(depth_min, depth_max + 1))
        out.append((t, random_mixed_circuit(dims, depth, rng)))
    return out


def product_circuit(dims: Sequence[int], depth: int, seed: int = 22) -> Circuit:
    """Uncontrolled single-wire gates only, so that ``|0...0>`` stays a
    product state: one Haar gate on every wire first (so no factor stays a
    basis vector), then ``depth - len(dims)`` gates on uniform wires drawn
    from {Haar, F_d, Z_d, X_{+1}} with probabilities 0.55 / 0.15 / 0.15 /
    0.15."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = tuple(int(x) for x in dims)
    gates: List[Gate] = [Gate((w,), haar(dims[w], rng), name="haar") for w in range(len(dims))]
    for _ in range(max(0, depth - len(dims))):
        t = int(rng.integers(len(dims)))
        d = dims[t]
        k = float(rng.random())
        if k < 0.55:
            gates.append(Gate((t,), haar(d, rng), name="haar"))
        elif k < 0.70:
            gates.append(Gate((t,), fourier(d), name="F"))
        elif k < 0.85:
            gates.append(Gate((t,), z_gen(d), name="Z"))
        else:
            gates.append(Gate((t,), x_plus(d, 1), name="X"))
    return Circuit(dims, gates)


def ghz_circuit(dims: Sequence[int], root: int = 0) -> Circuit:
    """Generalised GHZ preparation: ``F_d`` on ``root``, then for every other
    wire ``t`` and every level ``v = 1 .. d_root - 1`` a controlled
    ``X_{+v}`` on ``t`` conditioned on ``root = v``.

    Requires ``dims[root] <= dims[t]`` for every wire so that the result is
    ``sum_k |k ... k> / sqrt(d_root)``.
    """
    dims = tuple(int(x) for x in dims)
    d = dims[root]
    gates = [Gate((root,), fourier(d), name="F")]
    for t in range(len(dims)):
        if t == root:
            continue
        for v in range(1, d):
            gates.append(Gate((t,), x_plus(dims[t], v), (root,), (v,), name="CX"))
    return Circuit(dims, gates)


def circuit_from_arrays(dims, gates):
    """Build a :class:`Circuit` from plain tuples ``(wires, U, controls, values)``."""
    return Circuit(tuple(int(x) for x in dims),
                   [Gate(tuple(w), U, tuple(c), tuple(v)) for (w, U, c, v) in gates])
