"""The two launch forms of the Cholesky QR (Algorithm 4's QR of each sketch):
the fused cooperative launch that single calls use, and the launch per step
that the stream-lane batch uses.

* The launch-per-step form on single calls (HATT_QR_FORM=steps) meets the
  FP64 parity bar against the oracle on the d = 20 benchmark workload, a
  truncating recompression, a TT rounding and four uneven pairs.
* Both forms give bitwise the same result on the d = 20 workload (same row
  partition, same device code); the GEMM tuner is off in both processes so
  that the remaining products take the same plans.
* A grid-barrier wait of the fused form that runs out (HATT_QR_SPIN_CAP=1:
  one poll) ends the kernel with the timeout status, no hang, and the batch
  run afterwards in the same process still matches the oracle.
Each case runs in a fresh process (the hooks are read once)."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TT_ERR_TIMEOUT = 7


def run(script, env_extra, args=()):
    from paper_2410_04385_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "tests", script), *args],
                       capture_output=True, text=True, env=env, timeout=900, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-3000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_launch_per_step_form_parity():
    r = run("gemm_forms_check.py", {"HATT_QR_FORM": "steps"})
    assert r["d20_ranks_equal"] and r["d20_rel"] <= 1e-12
    assert r["trunc_ranks_equal"] and r["trunc_rel"] <= 1e-12
    assert r["round_ranks_equal"] and r["round_rel_to_input"] <= 1e-12
    assert r["uneven_rel_max"] <= 1e-12
    assert r["device_error"] == 0


def test_forms_are_bitwise_equal():
    a = run("gemm_forms_check.py", {"HATT_QR_FORM": "steps"}, ["model"])
    b = run("gemm_forms_check.py", {"HATT_QR_FORM": ""}, ["model"])
    assert a["d20_rel"] <= 1e-12 and b["d20_rel"] <= 1e-12
    assert a["d20_sha"] == b["d20_sha"]


def test_barrier_wait_that_runs_out_reports_timeout():
    r = run("qr_timeout_check.py", {"HATT_QR_SPIN_CAP": "1"})
    assert r["status_after_fused"] == TT_ERR_TIMEOUT
    assert r["batch_rel"] <= 1e-12
    assert r["status_after_batch"] == 0
