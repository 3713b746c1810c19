"""The debug build (librc_debug.so, -DRC_DEBUG): every brick index and table
entry index is checked on the device before use, and a failure is reported
as RC_ERR_CUDA at the next synchronising call, with no trap and no access
outside a buffer (the stand-in for a memory checker on this GPU pool).

Every kernel family runs under both builds in separate processes: the debug
build reports no failure and renders what the release build renders. Then
the debug build's test hook moves every brick index out of range: the checks
report it, replace each index by an in-range one, and the context keeps
working once the hook is cleared."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def run(out, debug, poison=False):
    env = dict(os.environ)
    env.pop("RC_DEBUG_POISON", None)
    env["RC_DEBUG"] = "1" if debug else "0"
    cmd = [sys.executable, os.path.join(HERE, "debug_scenarios.py"), out] + (["--poison"] if poison else [])
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.load(out)


def test_debug_build_checks_every_index(tmp_path):
    from paper_1211_5595_gb300 import build
    build.build()
    assert os.path.exists(build.DEBUG_LIB)
    rel = run(str(tmp_path / "release.npz"), debug=False)
    dbg = run(str(tmp_path / "debug.npz"), debug=True)
    assert sorted(rel.files) == sorted(dbg.files) and len(rel.files) >= 18
    for k in rel.files:
        a, b = rel[k], dbg[k]
        assert np.isfinite(b).all(), k
        scale = max(1.0, float(np.abs(a).max()))
        assert np.abs(a - b).max() <= 1e-6 * scale, (k, float(np.abs(a - b).max()))
    assert rel["f32_shaded"][..., 3].max() > 0.3
    # every check fires under the hook; afterwards the same images again
    poi = run(str(tmp_path / "poison.npz"), debug=True, poison=True)
    assert int(poi["poison_caught"]) == 1
    for k in rel.files:
        scale = max(1.0, float(np.abs(rel[k]).max()))
        assert np.abs(rel[k] - poi[k]).max() <= 1e-6 * scale, k
