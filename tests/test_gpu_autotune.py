"""The tridiagonalisation's autotuner (BHT_AUTOTUNE=1): a process with it on solves the same
eigenproblems to the same results as the fixed launch shape (eigenvalues to 1e-12 of the largest,
orthonormal vectors spanning the same subspaces), before and after its cache is filled."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPT = r"""
import numpy as np, torch, sys
import paper_2412_16544_gb300 as B
rng = np.random.default_rng(5)
out = []
for n in (40, 200, 521):
    M = rng.normal(size=(n, n + 30)) * np.logspace(0, -3, n)[:, None]
    G = M @ M.T
    for rep in range(2):                      # the first call tunes, the second uses the cache
        lam, U = B.bht_sym_eig(torch.from_numpy(G).cuda(), n // 3)
        out.append((lam.cpu().numpy(), U.cpu().numpy()))
np.save(sys.argv[1], np.array(out, dtype=object), allow_pickle=True)
"""


def run(tmp_path, tune):
    env = dict(os.environ, BHT_AUTOTUNE="1" if tune else "0", PYTHONPATH=ROOT)
    f = str(tmp_path / f"out_{int(tune)}.npy")
    subprocess.run([sys.executable, "-c", SCRIPT, f], env=env, check=True, cwd=ROOT)
    return np.load(f, allow_pickle=True)


def test_autotuned_shapes_give_the_same_eigenpairs(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fixed, tuned = run(tmp_path, False), run(tmp_path, True)
    for (l0, u0), (l1, u1) in zip(fixed, tuned):
        assert np.abs(l0 - l1).max() <= 1e-12 * np.abs(l0).max()
        assert np.abs(u1.T @ u1 - np.eye(u1.shape[1])).max() <= 1e-12
        # same subspace: the projector difference
        assert np.linalg.norm(u0 @ u0.T - u1 @ u1.T, 2) <= 1e-9
