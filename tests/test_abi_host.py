"""Host-side checks of libqudit.so (no GPU needed, no kernel launched).

The library must load on a machine without a GPU, export every symbol that
``include/qudit.h`` declares, and its planning logic (exact matrix
classification, class enumeration, argument validation) runs on the host.
"""
import os
import re

import numpy as np
import pytest

import __graft_entry__

__graft_entry__.build()
from paper_2410_17876_gb300 import binding as qb  # noqa: E402
from paper_2410_17876_gb300 import inputs as gen  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(qd_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    names = _declared_symbols()
    assert len(names) >= 20
    lib = qb._lib
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_wraps_every_declared_symbol():
    names = _declared_symbols()
    missing = [n for n in sorted(names) if not hasattr(qb, n)]
    assert not missing, f"no binding for: {missing}"


def test_host_index_arithmetic_selftest():
    qb.qd_selftest_host(400)


def test_version():
    assert "sm_103a" in qb.qd_version()


def _plan(dims, wires, U, cw=None, cv=None, prec=qb.QD_C64):
    return qb.qd_plan_gate(dims, prec, wires, U, cw, cv)


def test_classification_is_exact():
    dims = (2, 3, 4, 2)
    assert _plan(dims, [1], gen.z_gen(3))["kind"] == 1          # diagonal
    assert _plan(dims, [1], gen.x_plus(3, 2))["kind"] == 2      # permutation
    assert _plan(dims, [1], gen.fourier(3))["kind"] == 0        # dense
    ph = np.diag(np.exp(1j * np.array([0.1, 0.2, 0.3, 0.4]))) @ gen.x_plus(4, 1)
    assert _plan(dims, [2], ph)["kind"] == 2                     # monomial with phases
    # T touches one of the two rows of each class
    assert _plan(dims, [0], gen.qubit_t())["touched_rows"] == 1
    # a near-diagonal matrix is dense (classification is exact, no tolerance)
    almost = gen.z_gen(3).copy()
    almost[0, 1] = 1e-300
    assert _plan(dims, [1], almost)["kind"] == 0


def test_class_counts_and_runs():
    dims = (2, 3, 4, 2, 3)
    D = int(np.prod(dims))
    b = np.cumprod((1,) + dims[:-1])
    for t in range(len(dims)):
        p = _plan(dims, [t], gen.haar(dims[t], np.random.default_rng(t)))
        assert p["classes"] == D // dims[t]
        assert p["run"] == b[t]
        assert p["vec"] == (2 if b[t] % 2 == 0 else 1)
        p128 = _plan(dims, [t], gen.haar(dims[t], np.random.default_rng(t)), prec=qb.QD_C128)
        assert p128["vec"] == 1
    # controls shrink the visited classes by their dimensions (no O(D M) scan)
    p = _plan(dims, [2], gen.x_plus(4), [0, 4], [1, 2])
    assert p["classes"] == D // (4 * 2 * 3)
    assert p["run"] == 1
    # multi-wire gates and wide single wires go to the tile kernel
    p = _plan(dims, [1, 3], gen.haar(6, np.random.default_rng(0)))
    assert p["family"] == 1 and p["classes"] == D // 6


@pytest.mark.parametrize("bad", [
    dict(wires=[5], U=gen.x_plus(2)),                        # target out of range
    dict(wires=[0], U=gen.x_plus(2), cw=[0], cv=[1]),        # control equals target
    dict(wires=[0], U=gen.x_plus(2), cw=[1, 1], cv=[0, 0]),  # duplicate control
    dict(wires=[0], U=gen.x_plus(2), cw=[1], cv=[3]),        # value >= d_c
    dict(wires=[1, 1], U=gen.haar(9, np.random.default_rng(0))),  # repeated gate wire
])
def test_invalid_gates_rejected(bad):
    dims = (2, 3, 4)
    with pytest.raises(qb.QuditError) as ei:
        _plan(dims, bad["wires"], bad["U"], bad.get("cw"), bad.get("cv"))
    assert ei.value.status == qb.QD_ERR_ARG
    assert qb.qd_last_error()


def test_too_large_gate_unsupported():
    dims = (4, 4, 4, 2)
    with pytest.raises(qb.QuditError) as ei:
        _plan(dims, [0, 1, 2, 3], np.eye(128))
    assert ei.value.status == qb.QD_ERR_UNSUPPORTED


def test_invalid_layouts_rejected():
    for dims in [(1, 2), (2, 65), ()]:
        with pytest.raises(qb.QuditError):
            _plan(dims, [0], np.eye(2))


def test_regular_build_has_no_bounds_checks():
    """qd_bounds_status in the regular build: no checks compiled, nothing recorded (no GPU needed)."""
    from paper_2410_17876_gb300 import binding as qb

    assert qb.qd_bounds_status() == (qb.QD_OK, -1, 0)
