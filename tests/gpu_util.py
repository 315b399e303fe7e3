"""Helpers shared by the GPU parity tests."""
import numpy as np

C128_TOL = 1e-12  # max |delta amp|, complex128
C64_TOL = 1e-5    # max |delta amp|, complex64
C64_INFID = 1e-6  # infidelity, complex64 (depth <= 500)


def infidelity(ref: np.ndarray, got: np.ndarray) -> float:
    """1 - |<ref|got>|^2 / (<ref|ref><got|got>), in binary64."""
    ref = np.asarray(ref, dtype=np.complex128)
    got = np.asarray(got, dtype=np.complex128)
    ov = np.vdot(ref, got)
    return float(1.0 - (abs(ov) ** 2) / (np.vdot(ref, ref).real * np.vdot(got, got).real))


def assert_close(got, ref, prec, what=""):
    from paper_2410_17876_gb300 import binding as qb

    err = float(np.max(np.abs(np.asarray(got, dtype=np.complex128) - ref)))
    if prec == qb.QD_C128:
        assert err <= C128_TOL, f"{what}: max |d amp| = {err:.3e} > {C128_TOL}"
    else:
        inf = infidelity(ref, got)
        assert err <= C64_TOL, f"{what}: max |d amp| = {err:.3e} > {C64_TOL}"
        assert inf <= C64_INFID, f"{what}: infidelity {inf:.3e} > {C64_INFID}"
    return err
