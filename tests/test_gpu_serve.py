"""GPU tests of the serving loop: results against the oracle, the same result
alone and in a mix, admission bounded by the state-byte budget, timed
arrivals, and rejection of a request larger than the budget."""
import time

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


def _requests(gen, seed, n, wmax=14):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        w = int(rng.integers(3, wmax + 1))
        dims = tuple(int(x) for x in rng.choice([2, 3, 4], size=w))
        while np.prod(dims) > 3_000_000:
            dims = dims[:-1]
        c = gen.random_mixed_circuit(dims, int(rng.integers(10, 120)), rng)
        if i % 9 == 4 and len(dims) > 1 and dims[0] * dims[1] <= 64:
            c.gates.append(gen.Gate((0, 1), gen.haar(dims[0] * dims[1], rng)))
        out.append(c)
    return out


def _results(qb, s, n):
    res = {}
    deadline = time.time() + 120
    while len(res) < n and time.time() < deadline:
        for r in qb.qd_server_poll(s):
            res[r["id"]] = r
        time.sleep(0.001)
    return res


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_served_results_match_oracle(qb, gen, prec):
    p = qb.QD_C64 if prec == "c64" else qb.QD_C128
    reqs = _requests(gen, 21, 30)
    s = qb.qd_server_create(p, hbm_budget_bytes=1 << 30)
    ids = [qb.qd_server_submit(s, c, keep_state=True) for c in reqs]
    qb.qd_server_drain(s, 120)
    res = _results(qb, s, len(reqs))
    for rid, c in zip(ids, reqs):
        r = res[rid]
        assert r["status"] == 0 and r["kept"] == 1
        assert r["t_arrival"] <= r["t_admit"] <= r["t_done"]
        got = qb.qd_server_get_amplitudes(s, rid, c.D)
        ref = oracle.run_circuit(c)
        assert_close(got, ref, p, f"served dims={c.dims}")
        assert abs(r["norm"] - 1.0) < (1e-12 if p == qb.QD_C128 else 1e-5)
        qb.qd_server_release(s, rid)
    qb.qd_server_destroy(s)


def test_same_result_alone_and_in_the_mix(qb, gen):
    reqs = _requests(gen, 22, 40)
    probe = [3, 17, 30]
    alone = {}
    s = qb.qd_server_create(qb.QD_C64, hbm_budget_bytes=1 << 30)
    for i in probe:
        rid = qb.qd_server_submit(s, reqs[i], keep_state=True)
        qb.qd_server_drain(s, 60)
        alone[i] = qb.qd_server_get_amplitudes(s, rid, reqs[i].D)
        qb.qd_server_release(s, rid)
    qb.qd_server_destroy(s)
    s = qb.qd_server_create(qb.QD_C64, hbm_budget_bytes=1 << 30)
    ids = [qb.qd_server_submit(s, c, keep_state=(i in probe)) for i, c in enumerate(reqs)]
    qb.qd_server_drain(s, 120)
    for i in probe:
        assert np.array_equal(qb.qd_server_get_amplitudes(s, ids[i], reqs[i].D), alone[i])
    qb.qd_server_destroy(s)


def test_admission_respects_the_byte_budget(qb, gen):
    rng = np.random.Generator(np.random.PCG64(23))
    dims = (2,) * 16  # 65,536 amplitudes = 512 KiB complex64 (> one CTA: runs on a slot)
    reqs = [gen.random_mixed_circuit(dims, 60, rng) for _ in range(24)]
    per = 65536 * 8
    budget = 3 * per + per // 2  # at most 3 resident at once
    s = qb.qd_server_create(qb.QD_C64, hbm_budget_bytes=budget, max_slots=8)
    ids = [qb.qd_server_submit(s, c) for c in reqs]
    qb.qd_server_drain(s, 120)
    res = _results(qb, s, len(reqs))
    assert all(res[i]["status"] == 0 for i in ids)
    events = sorted([(res[i]["t_admit"], 1) for i in ids] + [(res[i]["t_done"], -1) for i in ids],
                    key=lambda e: (e[0], e[1]))
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak <= 3
    admits = [res[i]["t_admit"] for i in ids]
    assert admits == sorted(admits)  # admitted in arrival order
    qb.qd_server_destroy(s)


def test_timed_arrivals(qb, gen):
    reqs = _requests(gen, 24, 6, wmax=8)
    s = qb.qd_server_create(qb.QD_C64, hbm_budget_bytes=1 << 28)
    t0 = qb.qd_server_now(s) + 0.2
    ids = [qb.qd_server_submit_at(s, c, t0 + 0.05 * k) for k, c in enumerate(reqs)]
    qb.qd_server_drain(s, 60)
    res = _results(qb, s, len(reqs))
    for k, rid in enumerate(ids):
        assert abs(res[rid]["t_arrival"] - (t0 + 0.05 * k)) < 1e-9
        assert res[rid]["t_admit"] >= res[rid]["t_arrival"]
    qb.qd_server_destroy(s)


def test_request_larger_than_budget_is_rejected(qb, gen):
    s = qb.qd_server_create(qb.QD_C64, hbm_budget_bytes=1 << 20)
    big = gen.Circuit((2,) * 20, [gen.Gate((0,), gen.fourier(2))])
    with pytest.raises(qb.QuditError) as ei:
        qb.qd_server_submit(s, big)
    assert ei.value.status == qb.QD_ERR_UNSUPPORTED
    qb.qd_server_destroy(s)


def test_large_requests_match_oracle_and_closed_forms(qb, gen):
    """Requests above 2^20 amplitudes (the slot-stream path): two random
    mixed circuits against the oracle, and a GHZ circuit on 15,925,248
    amplitudes against its closed form, served together with small ones."""
    import oracle

    rng = np.random.Generator(np.random.PCG64(808))
    big = [gen.random_mixed_circuit((2, 3, 4, 2, 3, 4, 2, 2, 3, 2, 2, 4, 3, 4), 60, rng),  # 1,327,104 amplitudes
           gen.random_mixed_circuit((4, 3, 2, 2, 4, 3, 2, 4, 3, 2, 4, 2, 4, 3, 3), 50, rng)]  # 7,962,624
    ghz_dims = (2, 2, 3, 4, 2, 3, 4, 4, 2, 3, 2, 4, 3, 2, 2, 2, 3)                    # 15,925,248
    ghz = gen.ghz_circuit(ghz_dims, root=0)
    small = [gen.random_mixed_circuit((2, 3, 2, 3), 80, rng) for _ in range(8)]
    s = qb.qd_server_create(qb.QD_C64, hbm_budget_bytes=4 << 30)
    ids = [qb.qd_server_submit(s, c, keep_state=True) for c in big + [ghz] + small]
    qb.qd_server_drain(s, 600)
    for i, c in enumerate(big):
        got = qb.qd_server_get_amplitudes(s, ids[i], c.D)
        assert_close(got, oracle.run_circuit(c, nthreads=oracle.max_threads()), qb.QD_C64, f"served dims={c.dims}")
    got = qb.qd_server_get_amplitudes(s, ids[len(big)], ghz.D)
    ones = int(np.sum(np.cumprod((1,) + ghz_dims[:-1])))
    ref = np.zeros(ghz.D, dtype=np.complex128)
    ref[0] = ref[ones] = 2 ** -0.5
    assert float(np.max(np.abs(got - ref))) <= 1e-6
    for j, c in enumerate(small):
        got = qb.qd_server_get_amplitudes(s, ids[len(big) + 1 + j], c.D)
        assert_close(got, oracle.run_circuit(c), qb.QD_C64, "small served request")
    qb.qd_server_destroy(s)
