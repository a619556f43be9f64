"""The product path has no CPU fallback: without a CUDA device every entry point of the binding fails
loudly before doing any work, a missing library is an error, and importing the package never loads the
oracle (which is test infrastructure only)."""
import os
import subprocess
import sys

import pytest
import torch

from paper_1406_5802_gb300 import rmge

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(code):
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)


def test_package_never_imports_the_oracle():
    r = _run("import sys\n"
             "import paper_1406_5802_gb300.rmge, paper_1406_5802_gb300.autograd, paper_1406_5802_gb300.batch\n"
             "import paper_1406_5802_gb300.ranks, paper_1406_5802_gb300.workloads\n"
             "bad = sorted(m for m in sys.modules if m == 'oracle' or m.startswith('oracle.'))\n"
             "assert not bad, bad\n")
    assert r.returncode == 0, r.stderr


def test_missing_library_is_an_error():
    r = _run("from paper_1406_5802_gb300 import rmge\n"
             "rmge.load_library('/nonexistent/librmge.so')\n")
    assert r.returncode != 0
    assert "librmge is not built" in r.stderr


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a CUDA device")
def test_entry_points_fail_loudly_without_a_gpu():
    A = torch.eye(8, dtype=torch.float64)
    B = torch.ones(8, 1, dtype=torch.float64)
    calls = [
        lambda: rmge.make_multiplier("gaussian", 8, 1),
        lambda: rmge.apply_multiplier("gaussian", A, A),
        lambda: rmge.factor(A.clone()),
        lambda: rmge.solve("gaussian", A, A, B),
        lambda: rmge.refine("gaussian", A, A, A, B, B.clone()),
        lambda: rmge.lowrank_multiplier("gaussian", 8, 2, 1),
    ]
    for call in calls:
        with pytest.raises(RuntimeError, match="needs a CUDA device"):
            call()
