"""Every FMA-pipe / SFU split of the float32 weighting kernel (Eq. 1 over all
data points, Sec. 3.3) against the FP64 oracle.  A split moves part of the
exp2 and lg2 evaluations to polynomials on the FMA pipe; the split is chosen
once per process (AIDW_WEIGHT_POLY), so each one runs in a child process
that writes its predictions, and the oracle is evaluated once here.  The data
counts are not multiples of the 64-point chunk, so every split also weights
tile padding (which must stay at weight 0)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_helpers import TOL_FP32
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SPLITS = ["2,0", "0,0", "3,0", "4,0", "0,1", "1,1", "0,2"]
LEVELS = (0.5, 1.0, 2.0, 3.0, 5.0)


def _workloads():
    return {
        "uniform": inputs.uniform_kilo(n=20011, m=3001, seed=71),
        "clustered": inputs.clustered_kilo(n=30005, m=2999, seed=72),
    }


CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_1601_05904_gb300 as aidw
from paper_1601_05904_gb300 import inputs
out = sys.argv[2]
levels = tuple(float(a) for a in sys.argv[3].split(","))
ws = {"uniform": inputs.uniform_kilo(n=20011, m=3001, seed=71),
      "clustered": inputs.clustered_kilo(n=30005, m=2999, seed=72)}
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
res = {}
for name, w in ws.items():
    p = aidw.Params(k=w.k, alpha=levels)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    z, _ = aidw.aidw_interpolate(g, dev(w.qx), dev(w.qy), p)
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()
    res[name] = z.cpu().numpy()
np.savez(out, **res)
"""


@pytest.fixture(scope="module")
def references(oracle):
    return {name: oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k, levels=LEVELS)
            for name, w in _workloads().items()}


@pytest.mark.parametrize("split", SPLITS)
def test_split_matches_oracle(aidw, oracle, references, split, tmp_path):
    out = str(tmp_path / "z.npz")
    env = dict(os.environ, AIDW_WEIGHT_POLY=split)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, out, ",".join(map(str, LEVELS))],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.load(out)
    for name, ref in references.items():
        err = oracle.normalized_error(got[name], ref["z"], ref["scale"])
        assert err.max() <= TOL_FP32, f"split {split} {name}: {err.max():.3e}"
