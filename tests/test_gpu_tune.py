"""Launch-shape autotuning of the FP32 z-marching elasticity kernel.  The first FP32 solve
of a context times the candidate run lengths (planes per block) and stores the fastest in
the JSON cache; every run length must give bitwise-identical results, so the choice can
never change an answer.  Checked here, each configuration in a fresh process (the library
reads the cache once per process): a tuning run on an empty cache writes one key per
column count the solver launches, and runs with every key forced to the shortest run
(4 planes), to a single run over the whole z extent, and with tuning off (the built-in
heuristic) reproduce the tuning run's V-cycle, FP32 slab apply and mixed-precision solve
bit for bit, iteration count included."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = (30, 26, 34)  # 61 x 53 x 69 displacement nodes: the z-marching kernel's range, ragged tiles
NODES = "61x53x69"

SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, "tests")
from gpu_common import C2, consolidation_bcs
from paper_1801_04984_gb300 import binding as B
from paper_1801_04984_gb300.inputs import K0, layered_logk, random_vector
n = %r
ubc, fbc = consolidation_bcs(3)
g = layered_logk(n, layer_cells=4, std=1.5, seed=7)
ctx = B.Context(3, n, dict(C2, K=K0 * np.exp(g)), 1, ubc, fbc)
tau = 0.1
rhs = torch.tensor(random_vector(ctx.n_slab, seed=11), device="cuda")
x = torch.zeros_like(rhs)
st = ctx.solve_slab(tau, rhs, x, tol=1e-8, mode=B.MIXED)
v_in = torch.tensor(random_vector(ctx.n_space, seed=12), device="cuda").float()
v_out = torch.empty_like(v_in)
ctx.apply_part(B.PART_VCYCLE, tau, v_in, v_out)
a_in = torch.tensor(random_vector(ctx.n_slab, seed=13), device="cuda").float()
a_out = torch.empty_like(a_in)
ctx.apply_slab(tau, a_in, a_out)
torch.cuda.synchronize()
np.savez(sys.argv[1], x=x.cpu().numpy(), iters=st["iterations"], v=v_out.cpu().numpy(), a=a_out.cpu().numpy())
""" % (N,)


def _run(tmp_path, name, cache, **env):
    out = tmp_path / (name + ".npz")
    e = dict(os.environ, BIOT_TUNE_CACHE=str(cache), **env)
    p = subprocess.run([sys.executable, "-c", SCRIPT, str(out)], cwd=ROOT, env=e, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    return dict(np.load(out))


def test_every_tuned_run_length_gives_bitwise_identical_results(tmp_path):
    cache = tmp_path / "tune.json"
    base = _run(tmp_path, "tuned", cache)
    table = json.load(open(cache))
    keys = sorted(k for k in table if k.startswith("elast3_zrun|") and k.split("|")[2] == NODES)
    # one entry per column count of the solver (dG(1): 1 and 2 columns), each a valid run length
    assert [k.split("|")[3] for k in keys] == ["cols1", "cols2"], table
    assert all(1 <= table[k] <= 69 for k in keys), table
    runs = {}
    for name, z in (("short", 4), ("single", 69)):
        forced = tmp_path / ("forced_%s.json" % name)
        forced.write_text(json.dumps({k: z for k in keys}))
        runs[name] = _run(tmp_path, name, forced)
        assert json.load(open(forced)) == {k: z for k in keys}  # found, so nothing re-measured
    runs["heuristic"] = _run(tmp_path, "heuristic", tmp_path / "absent.json", BIOT_TUNE="0")
    assert not (tmp_path / "absent.json").exists()
    for name, got in runs.items():
        assert int(got["iters"]) == int(base["iters"]), name
        for f in ("x", "v", "a"):
            assert np.array_equal(got[f], base[f]), (name, f, np.abs(got[f] - base[f]).max())
