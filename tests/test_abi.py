"""The C ABI without a GPU: the library builds, loads, exports every function that include/wdf.h
declares, and fails cleanly (no abort) when no device is present."""

import ctypes

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def lib():
    from paper_2607_14025_gb300 import build, wdf

    build.build()
    return wdf.load()


def test_exports_every_declared_function(lib):
    from paper_2607_14025_gb300 import wdf

    names = wdf.header_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_header(tmp_path):
    # field offsets of the ctypes mirrors against what the C compiler makes of include/wdf.h
    import os
    import shutil
    import subprocess

    from paper_2607_14025_gb300 import wdf

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    probes = []
    mirrors = (("wdf_system", wdf._System), ("wdf_options", wdf._Options), ("wdf_stats", wdf.Stats),
               ("wdf_train_opts", wdf.TrainOpts), ("wdf_train_stats", wdf.TrainStats))
    for cname, py in mirrors:
        probes.append(f'printf("%zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            probes.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"wdf.h\"\nint main(void){" + "".join(probes) + "return 0;}\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for _, py in mirrors:
        want.append(ctypes.sizeof(py))
        want.extend(getattr(py, f).offset for f, _ in py._fields_)
    assert got == want


def test_strerror_and_defaults(lib):
    from paper_2607_14025_gb300 import wdf

    assert lib.wdf_strerror(wdf.WDF_ENOCONV) == b"not converged"
    assert lib.wdf_strerror(99) == b"unknown status"
    o = wdf._Options()
    lib.wdf_default_options(ctypes.byref(o))
    assert o.precision == wdf.WDF_MIXED and o.precond == wdf.WDF_PRECOND_TPA
    assert o.cg_tol == 1e-8 and o.cg_maxiter == 1000 and o.inner_tol == 1e-5 and o.warm_start == 0
    assert o.residual_update == 0  # every refinement recomputes b - A x unless asked
    t = wdf.TrainOpts()
    lib.wdf_default_train_opts(ctypes.byref(t))
    assert t.steps == 600 and t.lr == 3e-3 and t.npert == 8 and t.seed == 0


def test_null_arguments_are_rejected(lib):
    from paper_2607_14025_gb300 import wdf

    assert lib.wdf_setup_hamiltonian(None, None, None) == wdf.WDF_EINVAL
    assert lib.wdf_apply_chi0(None, 1, None, None, None, 0, None) == wdf.WDF_EINVAL
    lib.wdf_destroy(None)  # ignored
    assert lib.wdf_model_num_samples(None) == -1
    assert lib.wdf_model_loss_grad(None, None, None) == wdf.WDF_EINVAL
    assert lib.wdf_set_model(None, None) == wdf.WDF_EINVAL
    assert lib.wdf_model_create(0, 0, None) == wdf.WDF_EINVAL
    assert lib.wdf_plane_variant(None, 32, None) == wdf.WDF_EINVAL
    assert lib.wdf_apply_sternheimer_operator(None, 1, None, None, None, 0) == wdf.WDF_EINVAL
    assert lib.wdf_set_residual_update(None, 1) == wdf.WDF_EINVAL
    lib.wdf_model_free(None)  # ignored


def test_model_layout_constants_match_header():
    import re

    from paper_2607_14025_gb300 import wdf
    from oracle import mlp

    text = open(wdf.HEADER).read()
    assert int(re.search(r"#define WDF_MODEL_NPARAM (\d+)", text).group(1)) == wdf.MODEL_NPARAM == mlp.NPARAM
    assert int(re.search(r"#define WDF_MODEL_FLOATS (\d+)", text).group(1)) == wdf.MODEL_FLOATS == mlp.NMODEL


def test_without_gpu_setup_reports_state_error():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2607_14025_gb300 import wdf

    s = synth.make_system("tiny")
    with pytest.raises(wdf.WdfError) as e:
        wdf.Context(s)
    assert e.value.code == wdf.WDF_ESTATE


@pytest.mark.parametrize("name", ["tiny", "small", "ragged", "medium", "precision"])
def test_half_sphere_matches_the_input_generator(lib, name):
    # host-only entry point: the library's canonical half sphere equals the one the inputs use
    from paper_2607_14025_gb300 import wdf

    sp = synth.spec(name)
    cell = np.eye(3) * sp.L
    got = wdf.half_sphere(cell, sp.ecut)
    want = synth.half_sphere(sp.L, sp.ecut)
    assert np.array_equal(got, want)


def test_half_sphere_of_a_skewed_cell_by_brute_force(lib):
    from paper_2607_14025_gb300 import wdf

    cell = np.array([[9.0, 0.0, 0.0], [2.0, 8.5, 0.0], [1.0, -1.5, 10.0]])
    ecut = 12.0
    got = wdf.half_sphere(cell, ecut)
    B = 2 * np.pi * np.linalg.inv(cell).T
    r = np.arange(-12, 13)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    g2 = np.sum((n @ B) ** 2, axis=1)
    half = (n[:, 2] > 0) | ((n[:, 2] == 0) & (n[:, 1] > 0)) | ((n[:, 2] == 0) & (n[:, 1] == 0) & (n[:, 0] >= 0))
    want = n[(g2 <= ecut) & half]
    assert len(got) == len(want)
    assert {tuple(x) for x in got} == {tuple(x) for x in want}
    gg = np.sum((got @ B) ** 2, axis=1)
    assert np.all(np.diff(gg) >= -1e-9 * ecut)  # ordered by |G|^2
    assert tuple(got[0]) == (0, 0, 0)
