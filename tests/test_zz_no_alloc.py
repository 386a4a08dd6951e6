"""The allocation-free H application against the allocating one.

wdf_apply_hamiltonian_noalloc serves callers that cannot allocate device memory (a process whose
GPU memory belongs to another allocator, or a service with a fixed memory budget): it takes its
temporaries from a fixed device array instead of cudaMalloc. Its results must equal those of
wdf_apply_hamiltonian, call after call, since every call reuses (and must re-clear) that array,
and it must make no device allocation at all. Covered: an FP64 and a double-float context (whose
FP64 transforms are not autotuned), even and odd vector counts (an odd count runs the last
vector with a zero partner in its Gamma pair), an in-place call, and the refusals (a request
larger than the array, buffers of the wrong type or shape, host memory).
This file is collected last so that a run stopping at the first failure has run everything else.
"""

import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def small():
    from paper_2607_14025_gb300 import build

    build.build()
    return synth.make_system("small")


@pytest.mark.parametrize("precision", ["fp64", "mixed_df"])
def test_noalloc_matches_allocating_entry_point(small, precision):
    import torch

    s = small
    with wdf.Context(s, precision=precision) as c:
        refs, xs = [], []
        for call, nvec in enumerate((6, 5)):
            x = synth.make_guess(s, nvec, 21 + call)
            xs.append(torch.from_numpy(x).cuda())
            refs.append(c.apply_hamiltonian(x))
        outs = [torch.empty_like(x) for x in xs]
        torch.cuda.synchronize()
        n_alloc = wdf.alloc_count()
        for x, out, ref in zip(xs, outs, refs):  # two calls in a row reuse the same scratch
            c.apply_hamiltonian_noalloc(x, out)
            torch.cuda.synchronize()
            assert rel(out.cpu().numpy(), ref) < 1e-12
        # in place: out is x itself
        y = xs[0].clone()
        c.apply_hamiltonian_noalloc(y, y)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), refs[0]) < 1e-12
        assert wdf.alloc_count() == n_alloc, "the allocation-free entry point allocated device memory"


def test_noalloc_refusals(small):
    import torch

    s = small
    with wdf.Context(s, precision="fp64") as c:
        # a request larger than the fixed array is refused on the host, before any GPU work
        big = torch.zeros((6000, s.npw_h), dtype=torch.complex128, device="cuda")
        with pytest.raises(wdf.WdfError) as e:
            c.apply_hamiltonian_noalloc(big, torch.empty_like(big))
        assert e.value.code == wdf.WDF_EINVAL
        x = torch.from_numpy(synth.make_guess(s, 2, 5)).cuda()
        with pytest.raises(ValueError):  # wrong element type
            c.apply_hamiltonian_noalloc(x.to(torch.complex64), torch.empty_like(x.to(torch.complex64)))
        with pytest.raises(ValueError):  # rows narrower than the context's plane-wave count
            narrow = x[:, : s.npw_h - 1].contiguous()
            c.apply_hamiltonian_noalloc(narrow, torch.empty_like(narrow))
        # the C entry point itself refuses host memory (checked with cudaPointerGetAttributes)
        h_in = np.zeros((2, s.npw_h), dtype=np.complex128)
        h_out = np.zeros_like(h_in)
        rc = c._lib.wdf_apply_hamiltonian_noalloc(c._ctx, 2, h_in.ctypes.data_as(ctypes.c_void_p), h_out.ctypes.data_as(ctypes.c_void_p))
        assert rc == wdf.WDF_EINVAL
        # the context is still usable afterwards
        out = torch.empty_like(x)
        c.apply_hamiltonian_noalloc(x, out)
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), c.apply_hamiltonian(x.cpu().numpy())) < 1e-12
