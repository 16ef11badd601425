"""The allocation-free Bk-means entry point (bdg_bkmeans_noalloc) gives the same
centres and objective as bdg_bkmeans, on two calls in a row through the C ABI.

It exists for callers that cannot allocate device memory (device memory owned
by an outside manager, loops that must never reach the allocator); its scratch
is a fixed array
inside the library, so the second call also checks that nothing left over from
the first call changes the result. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import datagen

pytestmark = pytest.mark.gpu


def _call(fn, codes, sample, m, iters):
    cent = torch.empty(m, codes.shape[1], dtype=torch.int64, device=codes.device)
    loss = torch.empty(iters + 1, dtype=torch.int64, device=codes.device)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ctypes.c_void_p(codes.data_ptr()), ctypes.c_int64(codes.shape[0]),
            ctypes.c_int32(64 * codes.shape[1]), ctypes.c_void_p(sample.data_ptr()),
            ctypes.c_int64(sample.numel()), ctypes.c_int32(m), ctypes.c_int32(iters),
            ctypes.c_void_p(cent.data_ptr()), ctypes.c_void_p(loss.data_ptr()), st)
    return rc, cent, loss


def test_noalloc_bkmeans_matches_allocating_entry_point_twice():
    from paper_2102_04656_b300 import build as b
    b.build()
    import paper_2102_04656_b300 as bdg
    L = bdg.lib()
    cases = [(datagen.MixtureSpec(20000, 128, 64, 512, seed=501), 256, 16384, 8),
             (datagen.MixtureSpec(9000, 64, 32, 256, seed=502), 40, 2560, 5)]
    for spec, m, S, iters in cases:  # two calls in a row, different sizes
        codes = datagen.make_codes(spec).cuda()
        sample = torch.from_numpy(datagen.sample_ids(spec.n, S, spec.seed + 3)).cuda()
        rc0, c0, l0 = _call(L.bdg_bkmeans, codes, sample, m, iters)
        rc1, c1, l1 = _call(L.bdg_bkmeans_noalloc, codes, sample, m, iters)
        torch.cuda.synchronize()
        assert rc0 == 0 and rc1 == 0, L.bdg_last_error()
        assert torch.equal(c0, c1)
        assert torch.equal(l0, l1)
    # a request beyond the fixed scratch is refused before any work
    huge_S = 1 << 22
    cent = torch.empty(1, codes.shape[1], dtype=torch.int64, device="cuda")
    rc = L.bdg_bkmeans_noalloc(ctypes.c_void_p(codes.data_ptr()), ctypes.c_int64(codes.shape[0]),
                               ctypes.c_int32(64 * codes.shape[1]), ctypes.c_void_p(16),
                               ctypes.c_int64(huge_S), ctypes.c_int32(1), ctypes.c_int32(1),
                               ctypes.c_void_p(cent.data_ptr()), None, None)
    assert rc == -1 and b"fixed scratch" in L.bdg_last_error()
