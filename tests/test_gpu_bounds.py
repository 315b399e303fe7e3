"""The bounds-checked debug build (QD_BOUNDS=1), which stands in for a memory
sanitizer: built in its own directory and loaded in a fresh interpreter, it
runs circuits through every gate path (per gate in both precisions, tile
passes, tensor-core blocks in TF32x3 and through the BF16x3 tile ring, a
multi-wire gate, a batch through the layer
queue and through stream programs) against the oracle with no index
recorded outside its buffer; then the testing hook that hides the last
amplitudes of the state from the per-gate kernels shows that such an index
is recorded, reported as QD_ERR_DEVICE, and its access skipped."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import os, sys
    sys.path.insert(0, {root!r})
    os.environ["QD_BOUNDS"] = "1"
    import numpy as np
    from paper_2410_17876_gb300 import build
    build.build(bounds=True)
    from paper_2410_17876_gb300 import binding as qb, inputs as gen
    import oracle
    from tests.gpu_util import assert_close
    assert qb.LIB_PATH == build.LIB_BOUNDS
    rc, bad, compiled = qb.qd_bounds_status()
    assert compiled == 1 and rc == qb.QD_OK and bad == -1
    rng = np.random.Generator(np.random.PCG64(7))
    dims = (2, 3, 2, 4, 3, 2, 5, 2, 2, 3)
    circ = gen.random_mixed_circuit(dims, 150, rng)
    circ.gates.insert(40, gen.Gate((1, 3, 0), gen.haar(24, rng)))      # multi-wire, tensor cores in complex64
    ref = oracle.run_circuit(circ)
    for prec in (qb.QD_C128, qb.QD_C64):
        for fuse in (False, "tile", "block", "block_bf16x3"):
            if fuse == "block_bf16x3" and prec != qb.QD_C64:
                continue
            st = qb.State(dims, prec=prec)
            if fuse == "block_bf16x3":   # tensor-core blocks through the tile ring
                n0 = qb.qd_test_tc_ring_launches()
                st.run(circ, fuse="block", tc_mode="bf16x3")
                assert qb.qd_test_tc_ring_launches() > n0
            else:
                st.run(circ, fuse=fuse)
            assert_close(st.amplitudes(), ref, prec, f"bounds build prec={{prec}} fuse={{fuse}}")
            st.close()
    circs = [gen.random_mixed_circuit(tuple(int(x) for x in rng.choice([2, 3, 4], size=int(rng.integers(5, 11)))),
                                      int(rng.integers(20, 120)), rng) for _ in range(24)]
    for path in (qb.QD_BATCH_LAYERS, qb.QD_BATCH_STREAMS):
        b = qb.qd_batch_create(qb.QD_C64)
        qb.qd_batch_run(b, circs, small_max_amps=512, path=path)
        for i, c in enumerate(circs):
            assert_close(qb.qd_batch_get_amplitudes(b, i), oracle.run_circuit(c), qb.QD_C64, "bounds build batch")
        qb.qd_batch_destroy(b)
    rc, bad, compiled = qb.qd_bounds_status()
    assert rc == qb.QD_OK and bad == -1, (rc, bad)
    # the hook: the per-gate kernels are told the state is 3 amplitudes shorter
    st = qb.State(dims, prec=qb.QD_C128)
    D = st.D
    qb.qd_test_set_bounds_shrink(3)
    qb.qd_apply_gate(st.handle, 0, gen.fourier(2))
    st.synchronize()
    qb.qd_test_set_bounds_shrink(0)
    rc, bad, compiled = qb.qd_bounds_status()
    assert rc == qb.QD_ERR_DEVICE and D - 3 <= bad < D, (rc, bad, D)
    assert qb.qd_bounds_status()[0] == qb.QD_OK   # read and cleared
    st.close()
    print("bounds build ok")
""")


def test_bounds_checked_build(tmp_path):
    script = tmp_path / "bounds.py"
    script.write_text(SCRIPT.format(root=ROOT))
    env = dict(os.environ)
    env.pop("QD_BOUNDS", None)
    r = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, timeout=1200, env=env, cwd=ROOT)
    assert r.returncode == 0 and "bounds build ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
