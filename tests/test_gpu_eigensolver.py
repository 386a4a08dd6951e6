"""The three forms of the Davidson subspace eigensolver give the same PDEP eigenpairs.

The default form runs the cyclic Jacobi sweeps in one thread-block cluster with the matrix in
distributed shared memory; WDF_NO_CLUSTER_JACOBI selects one cooperative launch with a grid
barrier, and WDF_NO_CLUSTER_JACOBI + WDF_NO_COOP_JACOBI the two-kernels-per-round form. The
switches are read once per process, so each form runs in a subprocess through the C ABI. Same
rotations in the same order: the eigenvalues agree to 1e-12 relative and the eigenvectors span
the same space (|<x_a, y_a>| = 1 to 1e-9).
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, json, numpy as np
sys.path.insert(0, {root!r})
import synth
from paper_2607_14025_gb300 import wdf
s = synth.make_system("small")
guess = synth.make_perturbations(s, 12, 4)
with wdf.Context(s, precision="fp64", cg_tol=1e-12, gs_tol=1e-11) as c:
    lam, vec, st = c.pdep(8, guess, maxiter=100, tol=1e-9)
np.save({out!r}, vec)
print(json.dumps({{"lam": lam.tolist(), "converged": st.converged}}))
"""


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_14025_gb300 import build

    build.build()


def run_form(env_flags, tmp_path):
    out = str(tmp_path / ("vec_" + "_".join(sorted(env_flags)) + ".npy"))
    env = {k: v for k, v in os.environ.items() if k not in ("WDF_NO_CLUSTER_JACOBI", "WDF_NO_COOP_JACOBI")}
    env.update({k: "1" for k in env_flags})
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, out=out)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    return np.array(res["lam"]), np.load(out), res["converged"]


def test_eigensolver_forms_agree(tmp_path):
    from oracle import basis

    lam0, vec0, c0 = run_form([], tmp_path)
    assert c0 == 1
    for flags in (["WDF_NO_CLUSTER_JACOBI"], ["WDF_NO_CLUSTER_JACOBI", "WDF_NO_COOP_JACOBI"]):
        lam, vec, conv = run_form(flags, tmp_path)
        assert conv == 1, flags
        assert np.abs(lam - lam0).max() <= 1e-12 * np.abs(lam0).max(), flags
        overlap = np.abs(np.sum(basis.half_to_real(vec) * basis.half_to_real(vec0), axis=1))
        assert np.abs(overlap - 1.0).max() <= 1e-9, flags
