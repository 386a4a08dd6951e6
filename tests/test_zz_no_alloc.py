"""The allocation-free H application against the allocating one.

wdf_apply_hamiltonian_noalloc serves callers that cannot allocate device memory (code inside
another component's CUDA graph capture, or under an allocator that owns the GPU): it takes its
temporaries from a fixed device array instead of cudaMalloc. Its results must equal those of
wdf_apply_hamiltonian, call after call, since every call reuses (and must re-clear) that array.
This file is collected last so that a run stopping at the first failure has run everything else.
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_noalloc_matches_allocating_entry_point():
    import torch

    from paper_2607_14025_gb300 import build

    build.build()
    s = synth.make_system("small")
    with wdf.Context(s, precision="fp64") as c:
        for call in range(2):  # two calls in a row reuse the same scratch
            x = synth.make_guess(s, 6, 21 + call)
            ref = c.apply_hamiltonian(x)
            xd = torch.from_numpy(x).cuda()
            out = torch.empty_like(xd)
            c.apply_hamiltonian_noalloc(xd, out)
            torch.cuda.synchronize()
            assert rel(out.cpu().numpy(), ref) < 1e-12
        # a request larger than the fixed array is refused on the host, before any GPU work
        big = torch.zeros((6000, s.npw_h), dtype=torch.complex128, device="cuda")
        with pytest.raises(wdf.WdfError) as e:
            c.apply_hamiltonian_noalloc(big, torch.empty_like(big))
        assert e.value.code == wdf.WDF_EINVAL
