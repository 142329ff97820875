"""The allocation-free Response (qpadl_pir_answer_noalloc) agrees with the
handle-based qpadl_pir_answer.

Callers that cannot allocate device memory when they answer (inside a CUDA
graph capture, under a runtime that owns all device memory, or in a loop that
must not take cudaMalloc's device-wide synchronisation) use this entry point;
its scratch is a fixed device array shared by every call.  The test calls it
twice in a row through the C ABI, so the second call runs on whatever the
first left in that array, and compares each answer bit-exactly with the
existing entry point.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_03631_gb300 import inputs, pir

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return pir.load()


def _call(lib, D, R, C, q, ans):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.qpadl_pir_answer_noalloc(ctypes.c_void_p(D.data_ptr()), R, C, ctypes.c_void_p(q.data_ptr()),
                                        ctypes.c_void_p(ans.data_ptr()), stream)


@pytest.mark.parametrize("R,C", [(4099, 32768), (1000, 1008), (77, 1000)])
def test_noalloc_matches_handle_answer_on_two_calls(lib, R, C):
    D = torch.from_numpy(inputs.db_digits(R, C, 256, seed=R)).cuda()
    db = pir.qpadl_pir_setup(pir.params(R, C, 8, seed=R), D)
    for call in range(2):
        q = pir.from_u32(inputs.uniform_u32(C, seed=100 * R + call, tag=inputs.TAG_MISC))
        ref = torch.empty(R, dtype=torch.int32, device="cuda")
        pir.qpadl_pir_answer(db, q, ref)
        got = torch.full((R,), -1, dtype=torch.int32, device="cuda")
        assert _call(lib, D, R, C, q, got) == pir.QPADL_OK
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {call}"
    db.close()


def test_noalloc_rejects_columns_beyond_its_fixed_scratch(lib):
    limit = 262144
    D = torch.zeros(16, dtype=torch.uint8, device="cuda")
    q = torch.zeros(16, dtype=torch.int32, device="cuda")
    ans = torch.zeros(16, dtype=torch.int32, device="cuda")
    assert _call(lib, D, 1, limit + 16, q, ans) == pir.QPADL_EINVAL
