"""Index-checked build (-DBTRT_DEBUG_BOUNDS): every global access of the sweeps
checks its index and raises flag bit 3 instead of faulting.  Tiny grids in every
kernel form (plain, vector access, TMA-staged, two steps per launch, batched,
D3Q19) raise no flag, and the checked build computes the same results as the
ordinary one."""
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu


def test_tiny_grids_pass_the_index_checks(tmp_path):
    import importlib
    b = importlib.import_module("paper_1902_09813_gb300.build")
    dbg = b.build_debug()
    out = tmp_path / "debug.npz"
    env = dict(os.environ, BTRT_LIBRARY=str(dbg), PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "tiny_runs.py"), str(out)], env=env,
                       capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    checked = np.load(out)
    import tiny_runs
    ref, ref_flags = tiny_runs.run_all()
    for key, v in ref.items():
        assert int(checked["flags__" + key]) == 0, key
        assert ref_flags[key] == 0, key
        assert np.allclose(checked[key], v, rtol=1e-12, atol=1e-14), key
