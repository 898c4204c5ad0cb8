"""The bounds-checked debug build (-DLBIB_DEBUG, liblbib_debug.so): every
population index of the lattice and particle passes is checked against its
buffer and a failed check is reported as LBIB_E_BOUNDS.  The same cases --
FP32, FP16 and FP64 batches with particles and bonds (bulk, near-box and
particle passes), a body-force channel in 16-bit storage, a particle carried
across work tiles and around a periodic boundary (the debug build checks the
bulk pass's per-tile near-box counts), and the copy-engine variants of the
bulk pass -- run under the debug and the release build in fresh processes:
no check fails, and the results are the same bits.
The debug build collides every node on its own, the release build the bulk
nodes of 16-bit storage two at a time in paired FP32 instructions, so the
comparison also checks that the pairs give each node its own bits."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def run(tmp_path, debug):
    from paper_1808_01448_gb300 import build
    build.build()
    out = tmp_path / ("debug.npz" if debug else "release.npz")
    env = dict(os.environ, LBIB_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_debug_cases.py"), str(out)],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out), r.stdout


def test_debug_build_checks_pass_and_match_release(tmp_path):
    dbg, text = run(tmp_path, True)
    assert "bounds-checked" in text
    rel, _ = run(tmp_path, False)
    assert sorted(dbg.files) == sorted(rel.files)
    for k in rel.files:
        np.testing.assert_array_equal(dbg[k], rel[k], err_msg=k)
