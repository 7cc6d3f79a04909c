"""Every data-unit size of the float32 weighting kernel (Eq. 1 over all data
points) against the FP64 oracle.  A stream-K unit is one query tile by one
piece of a 2048-point weighting tile (the whole tile, or 1/2 .. 1/16 of it
for small point sets); the size is chosen per launch, and AIDW_WEIGHT_PIECES
fixes it for a process, so each size runs in a child process that writes
its predictions.  The point counts leave the last piece partial (20,011 and
2,999 points) or make every piece the tile's head (300 points), and the
query counts leave the last query tile ragged."""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_helpers import TOL_FP32
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _workloads():
    return {
        "uniform": inputs.uniform_kilo(n=20011, m=3001, seed=81),
        "clustered": inputs.clustered_kilo(n=2999, m=4097, seed=82),
        "tiny": inputs.uniform_kilo(n=300, m=1500, seed=83),
    }


CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_1601_05904_gb300 as aidw
from paper_1601_05904_gb300 import inputs
ws = {"uniform": inputs.uniform_kilo(n=20011, m=3001, seed=81),
      "clustered": inputs.clustered_kilo(n=2999, m=4097, seed=82),
      "tiny": inputs.uniform_kilo(n=300, m=1500, seed=83)}
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
res = {}
for name, w in ws.items():
    p = aidw.Params(k=w.k)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    z, _ = aidw.aidw_interpolate(g, dev(w.qx), dev(w.qy), p)
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()
    res[name] = z.cpu().numpy()
np.savez(sys.argv[2], **res)
"""


@pytest.fixture(scope="module")
def references(oracle):
    return {name: oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k)
            for name, w in _workloads().items()}


@pytest.mark.parametrize("shift", [0, 1, 2, 3, 4])
def test_piece_size_matches_oracle(aidw, oracle, references, shift, tmp_path):
    out = str(tmp_path / "z.npz")
    env = dict(os.environ, AIDW_WEIGHT_PIECES=str(shift))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, out], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.load(out)
    for name, ref in references.items():
        z = got[name]
        assert np.isfinite(z).all(), f"pieces 1/{1 << shift} {name}: non-finite"
        err = oracle.normalized_error(z, ref["z"], ref["scale"])
        assert err.max() <= TOL_FP32, f"pieces 1/{1 << shift} {name}: {err.max():.3e}"
