"""The allocation-free Response (qpadl_pir_answer_noalloc) against the oracle
and against the handle-based qpadl_pir_answer.

Some callers cannot allocate device memory when they answer: a runtime whose
own allocator owns all device memory, or a serving loop that must not take
the device-wide synchronisation of cudaMalloc/cudaFree.  They use this entry
point; its scratch is a fixed device array shared by every call.  Each test
calls it twice in a row through the C ABI, so the second call runs on
whatever the first left in that array, compares every answer with the CPU
oracle and with the existing entry point, and then reads the array's status
word, which must report that no bounded wait gave up.  This file is collected
last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2510_03631_gb300 import inputs, pir

pytestmark = pytest.mark.gpu

MAX_COLS = 262144   # QPADL_NOALLOC_MAX_COLS


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


@pytest.mark.parametrize("R,C", [(4099, 32768), (1000, 1008), (77, 1000), (64, MAX_COLS)])
def test_noalloc_matches_oracle_and_handle_answer_on_two_calls(lib, R, C):
    D_np = inputs.db_digits(R, C, 256, seed=R)
    D = torch.from_numpy(D_np).cuda()
    db = pir.qpadl_pir_setup(pir.params(R, C, 8, seed=R), D)
    for call in range(2):
        q_np = inputs.uniform_u32(C, seed=100 * R + call, tag=inputs.TAG_MISC)
        q = pir.from_u32(q_np)
        ref = torch.empty(R, dtype=torch.int32, device="cuda")
        pir.qpadl_pir_answer(db, q, ref)
        got = torch.full((R,), -1, dtype=torch.int32, device="cuda")
        assert _call(lib, D, R, C, q, got) == pir.QPADL_OK
        torch.cuda.synchronize()
        want = oracle.answer(D_np, q_np, threads=8)
        assert np.array_equal(pir.as_u32(got), want), f"call {call}: differs from the oracle"
        assert torch.equal(got, ref), f"call {call}: differs from qpadl_pir_answer"
    db.close()
    assert lib.qpadl_pir_noalloc_status() == pir.QPADL_OK


def test_noalloc_rejects_columns_beyond_its_fixed_scratch(lib):
    D = torch.zeros(16, dtype=torch.uint8, device="cuda")
    q = torch.zeros(16, dtype=torch.int32, device="cuda")
    ans = torch.zeros(16, dtype=torch.int32, device="cuda")
    assert _call(lib, D, 1, MAX_COLS + 16, q, ans) == pir.QPADL_EINVAL
    assert lib.qpadl_pir_noalloc_status() == pir.QPADL_OK
