"""Host logic of bench.py: update counting, algorithmic bytes, clock parsing and
the multi-rank aggregation (world size 2 over gloo on CPU)."""
import os
import socket
import subprocess
import sys
import textwrap

import numpy as np

import bench
from paper_2410_17876_gb300 import inputs as gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gate_updates_count_controls():
    dims = (2, 3, 4)
    assert bench.gate_updates(dims, gen.Gate((0,), gen.x_plus(2))) == 24
    assert bench.gate_updates(dims, gen.Gate((0,), gen.x_plus(2), (2,), (1,))) == 6
    assert bench.gate_updates(dims, gen.Gate((0,), gen.x_plus(2), (1, 2), (1, 0))) == 2


def test_config1_updates():
    c = gen.config1_circuit()
    assert c.D == 4096 * 6561
    u = bench.circuit_updates(c)
    # 70% single (D each) and 30% controlled (D / d_c) gates
    assert 0.7 * 500 * c.D * 0.8 < u < 500 * c.D


def test_algorithmic_bytes():
    assert bench.algorithmic_bytes({"classes": 10, "touched_rows": 3}, 8) == 2 * 8 * 30


def test_aggregate_uses_slowest_rank():
    v, t = bench.aggregate([100, 100], [1.0, 2.0])
    assert t == 2.0 and v == 100.0


def test_parse_clocks():
    lines = [
        "0, 1965 MHz, 2070 MHz, 900.5 W, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1800 MHz, 2070 MHz, 1200.0 W, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 300 MHz, 2070 MHz, 100.0 W, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.parse_clocks(lines)
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    assert c["sm_mhz"] in (1965.0, 1800.0, 1882.5)
    assert bench.parse_clocks([])["samples"] == 0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_max_over_ranks_gloo_world_size_2(tmp_path):
    code = textwrap.dedent(f"""
        import os, sys
        sys.path.insert(0, {ROOT!r})
        os.environ["QD_BENCH_BACKEND"] = "gloo"
        import bench
        rank, world, local = bench.dist_setup(2)
        t = bench.max_over_ranks(1.0 + rank, world)
        v, _ = bench.aggregate([10] * world, [t] * world)
        bench.barrier(world)
        print(f"rank={{rank}} t={{t}} v={{v}}")
        import torch.distributed as dist
        dist.destroy_process_group()
    """)
    script = tmp_path / "agg.py"
    script.write_text(code)
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    for o in outs:
        assert "t=2.0 v=10.0" in o, o


def test_reference_arm_non_zero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_method_flops_per_gate_kind():
    """8 P flops per amplitude for dense gates, 6 per changed amplitude for
    phases and phased permutations, 0 for pure permutations; controls divide
    the visited classes."""
    from paper_2410_17876_gb300 import binding as qb

    dims = (2, 3, 4)
    D = 24
    rng = np.random.Generator(np.random.PCG64(3))

    def flops(wires, U, cw=(), cv=()):
        p = qb.qd_plan_gate(dims, qb.QD_C64, wires, U, list(cw) or None, list(cv) or None)
        return bench.method_flops(p, U)

    assert flops((1,), gen.haar(3, rng)) == 8 * 3 * D
    assert flops((1,), gen.haar(3, rng), (2,), (1,)) == 8 * 3 * D // 4
    assert flops((0, 1), gen.haar(6, rng)) == 8 * 6 * D
    assert flops((0,), gen.qubit_s()) == 6 * D // 2          # one non-unit diagonal entry
    assert flops((1,), gen.z_gen(3)) == 6 * D * 2 // 3        # two non-unit entries of three
    assert flops((1,), gen.x_plus(3)) == 0
    assert flops((1,), -gen.x_plus(3)) == 6 * D


def test_config2_method_flops_and_updates():
    from paper_2410_17876_gb300 import binding as qb

    c = gen.config2_circuit()
    assert c.D == 1719926784 and len(c.gates) == 200
    f = bench.circuit_method_flops(qb, c, qb.QD_C64)
    u = bench.circuit_updates(c)
    # dense gates cost 16 (qubit) or 24 (qutrit) flops per touched amplitude
    assert 0.5 * 16 * u < f < 24 * u


def test_end_to_end_circuits_keep_the_workload_shape():
    """The end-to-end steps' circuits: the large workload's wires, controls
    and gate kinds with fresh unitary Haar matrices (seeded), so each step
    does the same updates and method flops on new inputs."""
    from paper_2410_17876_gb300 import binding as qb

    c = gen.config2_circuit()
    a, b, a2 = gen.redraw_haar(c, 1000), gen.redraw_haar(c, 1001), gen.redraw_haar(c, 1000)
    assert bench.circuit_updates(a) == bench.circuit_updates(c)
    assert bench.circuit_method_flops(qb, a, qb.QD_C64) == bench.circuit_method_flops(qb, c, qb.QD_C64)
    redrawn = 0
    for g0, ga, gb, ga2 in zip(c.gates, a.gates, b.gates, a2.gates):
        assert (ga.wires, ga.controls, ga.values, ga.name) == (g0.wires, g0.controls, g0.values, g0.name)
        assert np.array_equal(ga.U, ga2.U)
        assert np.allclose(ga.U @ ga.U.conj().T, np.eye(ga.U.shape[0]), atol=1e-12)
        if g0.name in ("haar", "CU"):
            assert not np.allclose(ga.U, g0.U) and not np.allclose(ga.U, gb.U)
            redrawn += 1
        else:
            assert np.array_equal(ga.U, g0.U)
    assert redrawn > 150
