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
