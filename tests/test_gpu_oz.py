"""The residual operator A_v = H - eps_v + alpha P in the residuals' precision, through the C ABI,
against the FP64 oracle (Sec. 2.1).

In the double-float form (mixed_df) the projections on [beta; psi] run on the tensor cores by
exact integer digits: seven 7-bit digits per value against a per-row exponent, products summed
exactly in FP32 chains of 512 values, so the result carries about 48 significant bits like the
CUDA-core double-float kernels. Both the FP64 form and the double-float form are held to 1e-12
relative (largest deviation over the largest magnitude) against the oracle, on the small system
(12 projection rows, 300 vectors: nine 32-vector tiles and a ragged tail, two K chains), the
medium system (192 rows: a full and a ragged 128-row tile, 33 chains) and the 96^3 reduced
precision system (91 chains, K split over CTAs). Edge cases: a pair of zero vectors (two vectors
share one complex FFT) maps to exactly zero, and a pair of vectors scaled by 1e-20 maps to the
scaled images to the same relative accuracy (each row has its own exponent). The CUDA-core double-float path (WDF_NO_OZ) is held to the same bar in a
subprocess.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from oracle import basis, dfpt, hamiltonian

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BAR = 1e-12


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_14025_gb300 import build

    build.build()
    wdf.load()


_cache = {}


def case(name, n):
    """System, the library's FP64 orbitals, vectors (rows 8, 9 zero; rows 6, 7 = 1e-20 x rows 4,
    1) and the oracle's A x with those orbitals."""
    key = (name, n)
    if key not in _cache:
        s = synth.make_system(name)
        with wdf.Context(s, precision="fp64") as c:
            eps, psi = c.orbitals()
        x = synth.make_guess(s, n, 5)
        x[8:10] = 0.0
        x[6] = 1e-20 * x[4]
        x[7] = 1e-20 * x[1]
        vidx = (np.arange(n) % s.nocc).astype(np.int32)
        vidx[6], vidx[7] = vidx[4], vidx[1]
        R = dfpt.Response(hamiltonian.Hamiltonian(s), eps, psi)
        ref = basis.fold(R.shifted(basis.expand(x), eps[vidx]))
        _cache[key] = (s, eps, psi, x, vidx, ref)
    return _cache[key]


@pytest.mark.parametrize("name,n", [("small", 300), ("medium", 320), ("precision_reduced", 40)])
@pytest.mark.parametrize("prec", ["fp64", "mixed_df"])
def test_residual_operator_matches_oracle(name, n, prec):
    s, eps, psi, x, vidx, ref = case(name, n)
    with wdf.Context(s, psi=psi, eps=eps, precision=prec) as c:
        y = c.apply_sternheimer_operator(vidx, x)
    err = rel(y, ref)
    print(f"{name} {prec}: max |A x - ref| / max |ref| = {err:.2e}")
    assert err < BAR
    assert np.all(y[8:10] == 0.0)
    assert rel(y[6], 1e-20 * y[4]) < BAR and rel(y[7], 1e-20 * y[1]) < BAR


SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import synth
from paper_2607_14025_gb300 import wdf
s = synth.make_system({name!r})
d = np.load({inp!r})
with wdf.Context(s, psi=d["psi"], eps=d["eps"], precision="mixed_df") as c:
    y = c.apply_sternheimer_operator(d["vidx"], d["x"])
np.save({out!r}, y)
"""


def test_residual_operator_cuda_core_double_float(tmp_path):
    s, eps, psi, x, vidx, ref = case("medium", 320)
    inp, out = str(tmp_path / "in.npz"), str(tmp_path / "out.npy")
    np.savez(inp, psi=psi, eps=eps, x=x, vidx=vidx)
    env = dict(os.environ, WDF_NO_OZ="1")
    code = SCRIPT.format(root=ROOT, name="medium", inp=inp, out=out)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    y = np.load(out)
    err = rel(y, ref)
    print(json.dumps({"cuda_core_df64_rel": err}))
    assert err < BAR


def test_residual_operator_rejects_bad_input():
    s = synth.make_system("tiny")
    with wdf.Context(s, precision="mixed_df") as c:
        x = synth.make_guess(s, 2, 1)
        with pytest.raises(wdf.WdfError):
            c.apply_sternheimer_operator(np.array([0, s.nocc], dtype=np.int32), x)
        assert c.apply_sternheimer_operator(np.zeros(0, dtype=np.int32), x[:0]).shape == (0, s.npw_h)
