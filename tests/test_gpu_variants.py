"""Alternative execution paths that environment switches select (read once per
process, so each runs in a subprocess): the SIMT projections instead of the
tensor-core ones (both sides, or the LQ side alone), the one-sweep-per-block bulge chase, the grid-wide panel, the
shared-memory cluster panel, programmatic dependent launch and other sweep-group sizes.  Each must give the same
singular values as the FP64 oracle within the parity tolerance."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
from paper_2608_21227_gb300 import nla, inputs
import oracle
from _util import err_rel, tol_for
out = []
for (m, n, b, dt) in [(300, 260, 16, 1), (512, 512, 32, 1), (257, 200, 16, 0), (640, 640, 64, 1)]:
    A = inputs.gaussian(m, n, 900 + m + b)
    if dt == 1:
        A = A.astype(np.float32).astype(np.float64)
    t = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().to(torch.float32 if dt == 1 else torch.float64)
    S, info = nla.gesvd_vals(t, cfg=nla.Cfg.make(band=b))
    torch.cuda.synchronize()
    e = err_rel(S.double().cpu().numpy(), oracle.svdvals(A))
    out.append({"m": m, "n": n, "b": b, "dt": dt, "info": int(info.item()), "err": e, "tol": tol_for(dt, max(m, n))})
print(json.dumps(out))
"""

VARIANTS = {
    "simt_projections": {"NLA_PROJ_TC": "0"},
    "simt_lq_projection": {"NLA_PROJ_TC": "1"},
    "chase_one_sweep_per_block": {"NLA_CHASE_GROUP": "0"},
    "chase_group_4": {"NLA_CHASE_GROUP": "4"},
    "grid_panel": {"NLA_PANEL_CLUSTER": "0"},
    "shared_memory_cluster_panel": {"NLA_PANEL_REG": "0"},
    "programmatic_dependent_launch": {"NLA_PDL": "1"},
}


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_variant_matches_oracle(name):
    env = dict(os.environ, **VARIANTS[name])
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    for rec in json.loads(r.stdout.strip().splitlines()[-1]):
        assert rec["info"] == 0, rec
        assert rec["err"] <= rec["tol"], rec
