"""The bounds-checking build (libhelm_check.so, -DHELM_CHECK_BOUNDS) on the GPU.

In that build every bulk copy and the computed global loads and stores of the stage,
interface, Krylov, Gram-Schmidt, tensor-core, HABC and adjoint kernels first check
that the bytes they touch lie inside a live device range (an allocation of the
library, or a caller buffer of the call in progress); a failed check is counted and
the access skipped.  This stands in for a memory checker on the small parity cases:
* the check itself: on a 256-byte allocation the whole range passes, the byte past
  its end and a range straddling its end fail (no access is made);
* the parity, edge-case, HABC and packed-operator test files run against the
  checking build in a child process (HELM_LIBRARY=check); tests/conftest.py makes
  every GPU test there fail if any check failed during it, so each of those cases
  runs with every checked access in bounds and with its usual parity bar.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_edge.py", "tests/test_gpu_habc.py", "tests/test_gpu_sym.py"]


@pytest.fixture(scope="module")
def checking_build():
    from paper_2209_10886_gb300 import build
    return build.build(variant="check")


def child(args, timeout):
    env = dict(os.environ, HELM_LIBRARY="check")
    return subprocess.run([sys.executable] + args, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_check_flags_ranges_outside_the_allocation(checking_build):
    code = ("import torch; torch.cuda.init()\n"
            "from paper_2209_10886_gb300 import helm\n"
            "helm.check_bounds_report(reset=True)\n"
            "print(helm.check_bounds_selftest())\n"
            "r = helm.check_bounds_report(reset=True)\n"
            "print(r['checking_build'], r['violations'], r['first_bytes'])\n")
    r = child(["-c", code], 600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = r.stdout.strip().splitlines()
    print(lines)
    assert lines[-2] == "(True, False, False)"
    assert lines[-1] == "True 2 1"            # two failures, the first one the 1-byte probe


def test_parity_cases_under_the_checking_build(checking_build):
    r = child(["-m", "pytest"] + SUITES + ["-q", "-m", "gpu and not slow", "-p", "no:cacheprovider"], 3000)
    print(r.stdout[-4000:])
    assert r.returncode == 0, r.stdout[-6000:] + r.stderr[-2000:]
