"""Both FP64 GEMM forms against the oracle, whatever the tuner would pick:
every product of a workload forced to the paired-column kernel
(HATT_GEMM_FORM=pair), and every product on the model's plan with the
first-use tuner off. Each runs in a fresh process (the form is fixed per
shape for the life of a process): the d = 20 benchmark workload, a truncating
recompression, a TT rounding and four uneven pairs, each within the FP64
parity bar of 1e-12 of the oracle's result for the same sketch."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPT = os.path.join(ROOT, "tests", "gemm_forms_check.py")


def run_check(env_extra, args):
    from paper_2410_04385_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, SCRIPT] + args, capture_output=True, text=True, env=env,
                       timeout=900, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-3000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("env_extra, args", [({"HATT_GEMM_FORM": "pair"}, []),
                                             ({"HATT_GEMM_FORM": ""}, ["model"])],
                         ids=["paired_form", "model_plan"])
def test_gemm_form_parity(env_extra, args):
    r = run_check(env_extra, args)
    assert r["d20_ranks_equal"] and r["d20_rel"] <= 1e-12
    assert r["trunc_ranks_equal"] and r["trunc_rel"] <= 1e-12
    assert r["round_ranks_equal"] and r["round_rel_to_input"] <= 1e-12
    assert r["uneven_rel_max"] <= 1e-12
    assert r["device_error"] == 0
