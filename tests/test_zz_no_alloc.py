"""The allocation-free row-offset entry point, for callers that may not
allocate device memory (their device memory belongs to another allocator, or
cudaMalloc's device-wide synchronisation would stall their other streams).
Called through the C ABI and checked, on two calls in a row, against the
prefix sum of the counts computed on the host and against the offsets
spgemm_symbolic produces for the same products.  Kept in a file of its own,
collected last."""
import ctypes

import numpy as np
import pytest

from paper_1804_00695_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _products():
    a, p, r = I.galerkin_problem(128)          # 2,097,152 rows: about a thousand tiles
    yield a, p
    g = I.rmat_symmetric(12, 16, seed=3)        # uneven rows, empty rows
    yield g, g
    z = I.Csr(5, 5, np.zeros(6, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0))
    yield z, z


def test_row_offsets_noalloc_matches_symbolic(cuda_lib):
    import torch
    sg = cuda_lib
    lib = sg.load()
    h = sg.Handle()
    stream = torch.cuda.current_stream().cuda_stream
    for a, b in _products():
        A, B = sg.Csr.from_host(a), sg.Csr.from_host(b)
        rp, nnz = h.symbolic(A, B)             # offsets from the existing entry point
        counts = torch.zeros_like(rp)
        counts[1:] = rp[1:] - rp[:-1]
        counts[0] = 12345                      # ignored by the call
        host_counts = counts[1:].cpu().numpy()
        expect = np.concatenate([[0], np.cumsum(host_counts)]).astype(np.int64)
        for _ in range(2):                     # two calls in a row share the scratch
            x = counts.clone()
            rc = lib.spgemm_row_offsets_noalloc(ctypes.c_void_p(x.data_ptr()), a.nrows,
                                                ctypes.c_void_p(stream))
            assert rc == 0, lib.spgemm_last_error()
            torch.cuda.synchronize()
            assert np.array_equal(x.cpu().numpy(), expect)
            assert torch.equal(x, rp)
            assert int(x[-1]) == nnz


def test_row_offsets_noalloc_rejects_oversize(cuda_lib):
    import torch
    sg = cuda_lib
    lib = sg.load()
    limit = lib.spgemm_row_offsets_noalloc_max_rows()
    assert limit >= 100_000_000
    x = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = lib.spgemm_row_offsets_noalloc(ctypes.c_void_p(x.data_ptr()), limit + 1,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1 and b"exceed" in lib.spgemm_last_error()
    assert not x.any()
