"""Failure paths of the C ABI, each made without faulting the GPU.

* Forced non-convergence: a CG budget of 2 iterations per solve makes wdf_apply_chi0 return
  WDF_ENOCONV with its outputs (the last iterates) and statistics filled.
* An expired device wait: the cooperative subspace eigensolver's grid barrier is given a poll
  limit of one poll (wdf_set_wait_limit), so its blocks give up, flag the error and return; PDEP
  returns WDF_ETIMEOUT and the same context then converges once the limit is restored. The
  cooperative form is chosen by WDF_NO_CLUSTER_JACOBI, which the library reads once per process,
  so this case runs in a child process.
* A capped allocator: with the library's device memory capped at what it already holds
  (wdf_set_device_limit), a call that needs larger workspaces returns WDF_ENOMEM without
  allocating, and the context works again when the cap is lifted.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tiny():
    from paper_2607_14025_gb300 import build

    build.build()
    return synth.make_system("tiny")


@pytest.mark.parametrize("precision", ["fp64", "mixed_df"])
def test_forced_nonconvergence_returns_partial_results(tiny, precision):
    s = tiny
    phi = synth.make_perturbations(s, 4, 7)
    with wdf.Context(s, precision=precision, cg_tol=1e-10, cg_maxiter=2) as c:
        with pytest.raises(wdf.NotConverged) as e:
            c.apply_chi0(phi, want_drho=True)
        assert e.value.code == wdf.WDF_ENOCONV
        out, drho, st = e.value.result
        assert st.converged == 0 and st.nsolve == 4 * s.nocc
        assert 0 < st.cg_iters_max <= 2
        assert st.max_residual > 1e-10
        assert np.isfinite(out).all() and np.isfinite(drho).all() and np.abs(out).max() > 0
        # the context stays usable and is deterministic
        with pytest.raises(wdf.NotConverged) as e2:
            c.apply_chi0(phi, want_drho=True)
        assert np.array_equal(e2.value.result[0], out)


_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import synth
from paper_2607_14025_gb300 import wdf
s = synth.make_system("tiny")
guess = synth.make_perturbations(s, 6, 3)
res = {}
with wdf.Context(s, precision="mixed", cg_tol=1e-11) as c:
    c.set_wait_limit(1)
    try:
        c.pdep(4, guess, maxiter=40, tol=1e-9)
        res["first"] = "returned"
    except wdf.WdfError as e:
        res["first"] = e.code
    c.set_wait_limit(0)
    lam, vec, st = c.pdep(4, guess, maxiter=40, tol=1e-9)
    res["lam"] = [float(v) for v in lam]
    res["converged"] = int(st.converged)
print("RESULT " + json.dumps(res))
"""


def test_expired_wait_returns_timeout_and_context_recovers(tiny):
    env = dict(os.environ, WDF_NO_CLUSTER_JACOBI="1")
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1][7:])
    assert res["first"] == wdf.WDF_ETIMEOUT
    assert res["converged"] == 1
    # the recovered run finds the same eigenvalues as the default eigensolver in this process
    guess = synth.make_perturbations(tiny, 6, 3)
    with wdf.Context(tiny, precision="mixed", cg_tol=1e-11) as c:
        lam, _, st = c.pdep(4, guess, maxiter=40, tol=1e-9)
    assert st.converged == 1
    assert np.abs(np.array(res["lam"]) - lam).max() <= 1e-8 * np.abs(lam).max()


def test_capped_device_memory_returns_enomem(tiny):
    s = tiny
    phi_small = synth.make_perturbations(s, 2, 11)
    phi_big = synth.make_perturbations(s, 32, 12)
    with wdf.Context(s, precision="fp64", cg_tol=1e-10) as ref:
        want, _, _ = ref.apply_chi0(phi_big)
    with wdf.Context(s, precision="fp64", cg_tol=1e-10) as c:
        c.apply_chi0(phi_small)
        n_alloc = wdf.alloc_count()
        try:
            wdf.set_device_limit(wdf.device_bytes())
            with pytest.raises(wdf.WdfError) as e:
                c.apply_chi0(phi_big)
            assert e.value.code == wdf.WDF_ENOMEM
            assert wdf.alloc_count() == n_alloc  # refused before cudaMalloc
            c.apply_chi0(phi_small)  # what fits in the buffers held still runs
        finally:
            wdf.set_device_limit(0)
        out, _, st = c.apply_chi0(phi_big)
    assert st.converged == 1
    assert np.abs(out - want).max() <= 1e-12 * np.abs(want).max()
