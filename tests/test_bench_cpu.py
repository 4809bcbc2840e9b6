"""bench.py pieces that run without a GPU: the shared recursion path of a
workload's nuclei and the reference arm (the oracle timed on the host)."""
import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_shared_path_puts_every_nucleus_on_a_prefix():
    for nuclei in ([(2, 1, 2, None), (2, 2, 2, None)], [(1, 1, 2, None), (2, 1, 2, None), (2, 2, 2, None)],
                   [(0, 1, 4, None), (0, 2, 4, None), (2, 2, 4, None)]):
        path = bench.shared_path(nuclei)
        for n_p, n_n, _, _ in nuclei:
            prefix = path[: n_p + n_n]
            assert prefix.count(0) == n_p and prefix.count(1) == n_n, (nuclei, path)
    with pytest.raises(SystemExit):
        bench.shared_path([(2, 0, 2, None), (0, 2, 2, None)])


@pytest.mark.parametrize("args,metric", [(["--steps", "1", "--warmup", "0"], "sink-site correlators/s"),
                                         (["--workload", "he4two", "--steps", "1", "--warmup", "0"],
                                          "momentum-projected correlators/s")])
def test_reference_arm_prints_one_line(args, metric):
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, timeout=900, env=env, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == metric and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_mixed_roofline_carries_the_operand_bound():
    """The mixed recursion reads 16 B of FP32 complex operands per
    site-operation (8 flops) through a data pipe of 128 B per SM clock: on 152
    SMs at 2070 MHz that is 20.14 TFLOP/s, a quarter of the FP32 peak."""
    import bench
    l1 = bench.l1_operand_bound(152, 2070.0)
    assert abs(l1 - 152 * 2070e6 * 64) < 1.0
    fp32 = 152 * 128 * 2 * 2070e6
    assert abs(l1 / fp32 - 0.25) < 1e-12
    r = bench.roofline_entry(1e12, 1, 100.0, 110.0, 1, fp32, 0.99 * fp32, "fp32", "k", l1)
    assert abs(r["achieved"] - 10.0) < 1e-9 and abs(r["l1_operand_bound"]["frac"] - 1e13 / l1) < 1e-12
    assert "l1_operand_bound" not in bench.roofline_entry(1e12, 1, 100.0, 110.0, 1, fp32, fp32, "fp64", "k")
