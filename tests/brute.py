"""Independent brute-force constructions used to pin the oracle (tests only).

Two constructions, both unlike the oracle's per-index digit arithmetic:
  * ``kron_unitary``: the full ``D x D`` matrix of a single-target gate
    (optionally controlled) as a Kronecker product of per-wire factors,
    most significant wire first (numpy ``kron`` order), using
    ``I + (x)_w B_w`` with ``B_c = |v_c><v_c|``, ``B_t = U - I``, ``B = I``
    elsewhere;
  * ``tensor_apply``: the state reshaped to a tensor with one axis per wire
    and the gate contracted on its wires with ``numpy.tensordot``; controls
    select a sub-tensor by slicing.
"""
import numpy as np


def kron_unitary(dims, target, U, controls=(), values=()):
    n = len(dims)
    factors = []
    for w in range(n - 1, -1, -1):  # most significant first
        d = dims[w]
        if w == target:
            factors.append(np.asarray(U, dtype=np.complex128) - np.eye(d))
        elif w in controls:
            v = values[list(controls).index(w)]
            p = np.zeros((d, d), dtype=np.complex128)
            p[v, v] = 1.0
            factors.append(p)
        else:
            factors.append(np.eye(d, dtype=np.complex128))
    M = factors[0]
    for f in factors[1:]:
        M = np.kron(M, f)
    return np.eye(M.shape[0], dtype=np.complex128) + M


def tensor_apply(dims, psi, wires, U, controls=(), values=()):
    n = len(dims)
    shape = tuple(dims[w] for w in range(n - 1, -1, -1))
    T = np.array(psi, dtype=np.complex128).reshape(shape)
    ax = lambda w: n - 1 - w
    idx = [slice(None)] * n
    for c, v in zip(controls, values):
        idx[ax(c)] = v
    sub = T[tuple(idx)]
    # axes of the sub-tensor: the original axes minus the control axes
    kept = [a for a in range(n) if a not in {ax(c) for c in controls}]
    sub_ax = {a: i for i, a in enumerate(kept)}
    k = len(wires)
    gdims = [dims[w] for w in wires]
    # local index: first-listed wire least significant -> reshape U with the
    # most significant gate wire first
    Ur = np.asarray(U, dtype=np.complex128).reshape(tuple(gdims[::-1]) * 2)
    in_axes = [sub_ax[ax(w)] for w in wires[::-1]]
    res = np.tensordot(Ur, sub, axes=(list(range(k, 2 * k)), in_axes))
    res = np.moveaxis(res, list(range(k)), in_axes)
    T[tuple(idx)] = res
    return T.reshape(-1)


def tensor_unitary(dims, wires, U, controls=(), values=()):
    D = int(np.prod(dims))
    M = np.zeros((D, D), dtype=np.complex128)
    for j in range(D):
        e = np.zeros(D, dtype=np.complex128)
        e[j] = 1.0
        M[:, j] = tensor_apply(dims, e, wires, U, controls, values)
    return M


def tensor_marginal(dims, psi, wire):
    n = len(dims)
    shape = tuple(dims[w] for w in range(n - 1, -1, -1))
    P = (np.abs(np.asarray(psi).reshape(shape)) ** 2)
    axes = tuple(a for a in range(n) if a != n - 1 - wire)
    return P.sum(axis=axes)
