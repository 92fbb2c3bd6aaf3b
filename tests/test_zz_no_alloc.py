"""The allocation-free random assembly (rac_assembly_noalloc) against the
allocating one (rac_assembly), called through the C-ABI.

rac_assembly_noalloc serves callers that cannot allocate device memory; its
scratch is a fixed device array shared by all calls.  This file is named to
be collected last so that a run stopping at the first failure has already
run every other test; it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1907_01995_gb300 import _lib  # noqa: E402


@pytest.mark.gpu
def test_noalloc_assembly_matches_allocating_entry_point():
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different sizes: the shared scratch keeps the
    # first call's contents, which must not leak into the second result
    for (n, p, seed, sweep0, ns) in [(2000, 20, 0, 3, 4), (777, 7, 5, 0, 2)]:
        ref_perm = torch.empty((ns, n), dtype=torch.int32, device="cuda")
        ref_blk = torch.empty((ns, n), dtype=torch.int32, device="cuda")
        got_perm = torch.full((ns, n), -1, dtype=torch.int32, device="cuda")
        got_blk = torch.full((ns, n), -1, dtype=torch.int32, device="cuda")
        assert lib.rac_assembly(n, p, seed, sweep0, ns, ref_perm.data_ptr(), ref_blk.data_ptr(),
                                stream) == _lib.RAC_OK
        assert lib.rac_assembly_noalloc(n, p, seed, sweep0, ns, got_perm.data_ptr(),
                                        got_blk.data_ptr(), stream) == _lib.RAC_OK
        assert torch.equal(ref_perm, got_perm)
        assert torch.equal(ref_blk, got_blk)
        perm = got_perm.cpu().numpy()
        for s in range(ns):
            assert np.array_equal(np.sort(perm[s]), np.arange(n))


@pytest.mark.gpu
def test_noalloc_assembly_rejects_oversize_request():
    lib = _lib.load()
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    n = 300000
    assert lib.rac_assembly_noalloc(n, 10, 0, 0, 1, out.data_ptr(), None,
                                    torch.cuda.current_stream().cuda_stream) == _lib.RAC_ERR_ARG
