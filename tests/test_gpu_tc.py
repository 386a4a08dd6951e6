"""Tensor-core (tcgen05, 3xTF32) against CUDA-core projections in the FP32 inner CG.

The backend is chosen per process (tensor cores by default, CUDA cores with WDF_NO_TC in the
environment), so each case runs in a subprocess through the C ABI. Small system: both backends
against the FP64 oracle at the mixed form's bar (1e-8 relative at cg_tol 1e-10). Medium system (192 projection rows, 320 solves: three
128-solve tiles with a ragged tail, 8,455 elements: 67 value tiles with a ragged tail): the two
backends against each other, 1e-8 relative.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from oracle import dfpt, hamiltonian

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, json, numpy as np
sys.path.insert(0, {root!r})
import synth
from paper_2607_14025_gb300 import wdf
s = synth.make_system({name!r})
phi = synth.make_perturbations(s, {npert}, 17)
psi = np.load({psi!r}) if {psi!r} else None
eps = np.load({eps!r}) if {eps!r} else None
with wdf.Context(s, psi=psi, eps=eps, precision="mixed_df", cg_tol=1e-10) as c:
    out, drho, st = c.apply_chi0(phi, want_drho=True)
np.save({out!r}, np.stack([out, drho]))
print(json.dumps(st.as_dict()))
"""


def run_backend(flag, name, npert, tmp_path, psi=None, eps=None, extra_env=None):
    out = str(tmp_path / f"{name}_{flag}_{sorted((extra_env or {}).items())}.npy".replace(" ", ""))
    pp = ep = ""
    if psi is not None:
        pp, ep = str(tmp_path / "psi.npy"), str(tmp_path / "eps.npy")
        np.save(pp, psi)
        np.save(ep, eps)
    env = {k: v for k, v in os.environ.items() if k != "WDF_NO_TC"}
    if flag == "WDF_NO_TC":
        env[flag] = "1"
    env.update(extra_env or {})
    code = SCRIPT.format(root=ROOT, name=name, npert=npert, psi=pp, eps=ep, out=out)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    st = json.loads(r.stdout.strip().splitlines()[-1])
    return np.load(out), st


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_14025_gb300 import build

    build.build()


@pytest.mark.parametrize("flag", ["tensor_cores", "WDF_NO_TC"])
def test_small_system_against_oracle(flag, tmp_path):
    s = synth.make_system("small")
    H = hamiltonian.Hamiltonian(s)
    w, psi = H.ground_state(s.nocc)
    R = dfpt.Response(H, w, psi)
    phi = synth.make_perturbations(s, 6, 17)
    ref = R.apply(phi, tol=1e-13)
    res, st = run_backend(flag, "small", 6, tmp_path, psi, w)
    assert st["converged"] == 1 and st["max_residual"] <= 1e-10
    assert np.abs(res[1] - ref["drho"]).max() <= 1e-8 * np.abs(ref["drho"]).max()
    assert np.abs(res[0] - ref["out"]).max() <= 1e-8 * np.abs(ref["out"]).max()


def test_medium_system_backends_agree(tmp_path):
    a, sa = run_backend("tensor_cores", "medium", 5, tmp_path)
    b, sb = run_backend("WDF_NO_TC", "medium", 5, tmp_path)
    assert sa["converged"] == 1 and sb["converged"] == 1
    assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max()
    # the inner iteration counts differ little: both backends carry FP32 accuracy
    assert abs(sa["cg_iters"] - sb["cg_iters"]) <= 0.05 * sb["cg_iters"]


@pytest.mark.parametrize("variant", ["4", "5"])
def test_plane_kernel_variants_agree_on_the_medium_system(variant, tmp_path):
    # against the one-thread-per-line register plane kernel (64^3): the two-threads-per-line
    # kernel (4) and the persistent kernel with bulk copies and the compile-time disk (5)
    a, sa = run_backend("tensor_cores", "medium", 5, tmp_path, extra_env={"WDF_PLANE_VARIANT": "1"})
    b, sb = run_backend("tensor_cores", "medium", 5, tmp_path, extra_env={"WDF_PLANE_VARIANT": variant})
    assert sa["converged"] == 1 and sb["converged"] == 1
    assert np.abs(a - b).max() <= 1e-8 * np.abs(a).max()
    assert abs(sa["cg_iters"] - sb["cg_iters"]) <= 0.02 * sa["cg_iters"]


def test_double_float_plane_kernel_agrees_on_the_medium_system(tmp_path):
    # the 64 x 64 double-float plane kernel (residual V_loc product, right-hand-side product and
    # density sum, one radix-8 task per thread) against the general Stockham and generic kernels
    a, sa = run_backend("tensor_cores", "medium", 5, tmp_path)
    b, sb = run_backend("tensor_cores", "medium", 5, tmp_path, extra_env={"WDF_NO_DF_PLANE": "1"})
    assert sa["converged"] == 1 and sb["converged"] == 1
    assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max()
    assert abs(sa["cg_iters"] - sb["cg_iters"]) <= 0.02 * sb["cg_iters"]


def test_l2_chunked_fft_passes_are_bitwise_identical(tmp_path):
    # the three FFT kernels of an operator application in chunks of pairs (a 1 MB column-buffer
    # budget: two pairs per chunk on the 64^3 grid) against one pass over all pairs
    a, sa = run_backend("tensor_cores", "medium", 5, tmp_path, extra_env={"WDF_FFT_CHUNK_MB": "0"})
    b, sb = run_backend("tensor_cores", "medium", 5, tmp_path, extra_env={"WDF_FFT_CHUNK_MB": "1"})
    assert sa["converged"] == 1 and sb["converged"] == 1
    assert np.array_equal(a, b)
    assert sa["cg_iters"] == sb["cg_iters"]
