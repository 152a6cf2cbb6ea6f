"""mp_minplus_mul_noalloc: the dense product for callers that cannot allocate.

Some callers may not call cudaMalloc at all (device memory owned by another
allocator, paths that must not touch the allocator).  The no-allocation entry
point keeps its only scratch, the occupancy masks, in a fixed array inside the
library.  Its results must equal mp_minplus_mul's, bit for bit (the tolerance
of every integer test here), on consecutive calls that share that array.  The
call goes straight through the C ABI.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_17688_gb300 as mp
    L = mp.lib()
    f = L.mp_minplus_mul_noalloc
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    f.restype = ctypes.c_int
    f.argtypes = [P, P, P, I64, I64, I64, I64, I64, I64, ctypes.c_int, P]
    return torch, mp, f


def _call(torch, mp, f, X, Y, Z):
    dtype = mp.MP_I16 if X.dtype == torch.int16 else mp.MP_U8
    M, K = X.shape
    N = Y.shape[1]
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return f(X.data_ptr(), Y.data_ptr(), Z.data_ptr(), M, N, K, X.stride(0), Y.stride(0),
             Z.stride(0), dtype, s)


def test_noalloc_matches_minplus_mul_twice(env):
    torch, mp, f = env
    from paper_2409_17688_gb300 import synth
    # two consecutive calls with different shapes and INF patterns: the second
    # must not see the first call's masks left in the shared array
    cases = [(700, 900, 530, np.int16, 0.6, 11), (1000, 300, 777, np.uint8, 0.2, 12),
             (700, 900, 530, np.int16, 0.1, 13)]
    for M, K, N, dt, frac, seed in cases:
        X = torch.from_numpy(synth.block_inf_matrix(M, K, seed, dt, inf_frac=frac)).cuda()
        Y = torch.from_numpy(synth.block_inf_matrix(K, N, seed + 100, dt, inf_frac=frac)).cuda()
        want = mp.mp_minplus_mul(X, Y)
        got = torch.empty_like(want)
        assert _call(torch, mp, f, X, Y, got) == 0, mp.mp_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, want), (M, K, N, dt)
