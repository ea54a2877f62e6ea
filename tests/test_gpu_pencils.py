"""The sliding-stencil kernels (minmod, PPM, WENO-Z, MP5 reconstruction and the UCT edge inputs) walk each pencil
of cells with a stencil carried from one cell to the next; the launch autotuner picks the pencil length (8 or 16
cells) per kernel by timing.  The results must not depend on that choice: two RK4 steps of ragged blocks, run in
separate processes with the autotuner off and the default or the long pencils (ASTERX_PENCIL=16), end bit for bit
equal, state and primitives, for every reconstruction scheme and for a batch of two blocks."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
import torch
from paper_2406_11669_gb300 import asterx as A, workloads as W
out = sys.argv[1]
dev = torch.device("cuda")
res = {}

def upload(w):
    M = torch.from_numpy(np.ascontiguousarray(np.stack([w.metric[k] for k in W.METRIC_NAMES]))).to(dev)
    P = torch.from_numpy(np.ascontiguousarray(np.stack([w.prims[k] for k in W.PRIM_NAMES]))).to(dev)
    U = torch.zeros((9,) + w.shape, dtype=torch.float64, device=dev)
    for v, k in ((5, "Ax"), (6, "Ay"), (7, "Az")):
        U[v] = torch.from_numpy(w.A[k]).to(dev)
    U[8] = torch.from_numpy(w.Psi).to(dev)
    return M, U, P

for recon in (W.RECON_MINMOD, W.RECON_PPM, W.RECON_WENOZ, W.RECON_MP5):
    w = W.smooth_general(n=(37, 29, 33), recon=recon)
    M, U, P = upload(w)
    s = A.Solver.for_workload(w, device=dev)
    s.prepare(M)
    s.fill_ghosts(U)
    s.prim2con(U, P)
    for _ in range(2):
        s.rk4_step(U, P, w.dt)
    torch.cuda.synchronize()
    res[f"U{recon}"] = U.cpu().numpy()
    res[f"P{recon}"] = P.cpu().numpy()

ws = [W.smooth_general(n=(35, 20, 26), seed=208, recon=W.RECON_WENOZ),
      W.smooth_general(n=(19, 33, 24), seed=209, recon=W.RECON_WENOZ)]
blocks = []
for w in ws:
    M, U, P = upload(w)
    blocks.append((w, M, U, P))
b = A.Batch(ws[0].params, [(w.n, w.g, w.x0, w.dx, w.bc, M, U, P) for (w, M, U, P) in blocks])
b.prepare()
b.prim2con()
b.step(ws[0].dt, nsteps=2)
torch.cuda.synchronize()
for i, (w, M, U, P) in enumerate(blocks):
    res[f"batchU{i}"] = U.cpu().numpy()
np.savez(out, **res)
"""


def run(tmp_path, tag, extra_env):
    out = str(tmp_path / f"{tag}.npz")
    env = dict(os.environ, ASTERX_AUTOTUNE="0", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    env.pop("ASTERX_PENCIL", None)
    env.update(extra_env)
    r = subprocess.run([sys.executable, "-c", SCRIPT, out], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


def test_results_do_not_depend_on_the_pencil_length(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    short = run(tmp_path, "short", {})
    long_ = run(tmp_path, "long", {"ASTERX_PENCIL": "16"})
    assert set(short.files) == set(long_.files)
    for k in short.files:
        assert np.all(np.isfinite(short[k])), k
        assert np.array_equal(short[k], long_[k]), k
