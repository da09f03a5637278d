"""The fifth-generation tensor-core building block (tcgen05 MMA from shared memory into TMEM,
commit to an mbarrier, TMEM loads) against a float64 product of the same bfloat16 inputs.
FP32 accumulation of K products of O(1) terms: error below K * 2^-24 of the sum of |terms|."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_03277_gb300 import build
    build.build()
    import paper_2512_03277_gb300 as P
    lib = P.load_library()
    lib.cavmd_tc_selftest.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
    return lib


def _bf16_bits(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def _bf16_value(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("K,N", [(64, 128), (256, 256), (1024, 128)])
def test_tc_bf16_tile_matches_host_product(lib, K, N):
    rng = np.random.default_rng(K + N)
    A = _bf16_bits(rng.uniform(-1, 1, (128, K)))
    B = _bf16_bits(rng.uniform(-1, 1, (N, K)))
    out = np.zeros((128, N), np.float32)
    rc = lib.cavmd_tc_selftest(A.ctypes.data, B.ctypes.data, K, N, out.ctypes.data)
    assert rc == 0, lib.cavmd_last_error(None)
    ref = _bf16_value(A) @ _bf16_value(B).T
    scale = np.abs(_bf16_value(A)) @ np.abs(_bf16_value(B)).T
    assert np.all(np.abs(out - ref) <= K * 2.0 ** -24 * scale + 1e-30)
