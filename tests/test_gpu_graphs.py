"""Batched Responses (LWE, Goldberg, Chor) captured in a CUDA graph and replayed with new queries.

The uint8-digit GEMM is launched as the programmatic dependent of the kernel
that makes its limbs and zeroes its output; under stream capture that launch
becomes a programmatic graph edge.  These tests replay such graphs with fresh
query contents (same buffers) and compare every answer with the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_03631_gb300 import inputs, pir

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


def _capture(fn):
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


@pytest.mark.parametrize("B,u8max,pair", [
    (8, 64, 1),      # uint8-digit GEMM, 32-column pair tiles
    (32, 64, 1),     # uint8-digit GEMM, 128-column pair tiles
    (48, 64, 0),     # uint8-digit GEMM, two tiles per row tile, single-SM tiles
    (100, 0, 1),     # fp16-copy pair GEMM with a split tail (memset inside the graph)
])
def test_batched_answers_replayed_in_a_cuda_graph(cuda, B, u8max, pair):
    R, C = 3000, 4096 + 64
    D = inputs.db_digits(R, C, 256, seed=B + 1)
    db = pir.qpadl_pir_setup(pir.params(R, C, 8, seed=1), torch.from_numpy(D).cuda())
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_U8_MAX_BATCH, u8max)
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_PAIR_GEMM, pair)
    Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
    ans = torch.empty(B * R, dtype=torch.int32, device="cuda")
    Q.copy_(pir.from_u32(inputs.uniform_u32(B * C, seed=B, tag=inputs.TAG_MISC)))
    call = lambda: pir.qpadl_pir_answer_batch(db, Q, ans, path=1)
    call()   # builds the lazily made copies and scratch before the capture
    torch.cuda.synchronize()
    g = _capture(call)
    for seed in (B + 100, B + 200):
        Q_np = inputs.uniform_u32(B * C, seed=seed, tag=inputs.TAG_MISC).reshape(B, C)
        Q.copy_(pir.from_u32(Q_np.reshape(-1)))
        ans.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert pir.qpadl_pir_status(db) == pir.QPADL_OK
        got = pir.as_u32(ans).reshape(B, R)
        assert np.array_equal(got, oracle.answer_batch(D, Q_np, threads=oracle.max_threads())), seed
    del g
    db.close()


@pytest.mark.parametrize("B", [40, 200])   # uint8-digit one-row GEMM / one-limb pair GEMM
def test_goldberg_answers_replayed_in_a_cuda_graph(cuda, B):
    R, C, p = 1500, 3000, 257
    D = (inputs.db_digits(R, C, 256, seed=B).astype(np.int64) % p).astype(np.uint8)
    h = pir.qpadl_goldberg_setup(R, C, p, torch.from_numpy(D).cuda())
    Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
    out = torch.empty(B * R, dtype=torch.int32, device="cuda")
    Q.copy_(pir.from_u32(inputs.uniform_u32(B * C, seed=B, tag=inputs.TAG_MISC) % p))
    call = lambda: pir.qpadl_goldberg_answer_batch(h, Q, out)
    call()
    torch.cuda.synchronize()
    g = _capture(call)
    for seed in (B + 7, B + 8):
        Q_np = (inputs.uniform_u32(B * C, seed=seed, tag=inputs.TAG_MISC) % p).reshape(B, C)
        Q.copy_(pir.from_u32(Q_np.reshape(-1)))
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert pir.qpadl_goldberg_status(h) == pir.QPADL_OK
        got = pir.as_u32(out).reshape(B, R)
        assert np.array_equal(got, oracle.goldberg_answer(D, Q_np, p, threads=oracle.max_threads())), seed
    del g
    h.close()


@pytest.mark.parametrize("B,m4rm_min", [(1, 257), (8, 257), (32, 257), (100, 64)])   # scans / four-Russians
def test_chor_answers_replayed_in_a_cuda_graph(cuda, B, m4rm_min):
    rows, bits = 3000, 4096
    DB = inputs.chor_db(rows, bits, seed=B + 3)
    h = pir.qpadl_chor_setup(rows, bits, torch.from_numpy(DB.view(np.int32).reshape(-1)).cuda())
    pir.qpadl_chor_set_option(h, pir.QPADL_CHOR_OPT_M4RM_MIN_BATCH, m4rm_min)
    Q0 = inputs.chor_queries(B, rows, seed=B)
    Q = torch.from_numpy(np.ascontiguousarray(Q0).view(np.int32).reshape(-1)).cuda()
    out = torch.empty(B * h.words, dtype=torch.int32, device="cuda")
    call = lambda: pir.qpadl_chor_answer_batch(h, Q, out)
    call()
    torch.cuda.synchronize()
    g = _capture(call)
    for seed in (B + 11, B + 12):
        Q_np = inputs.chor_queries(B, rows, seed=seed)
        Q.copy_(torch.from_numpy(np.ascontiguousarray(Q_np).view(np.int32).reshape(-1)))
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert pir.qpadl_chor_status(h) == pir.QPADL_OK
        got = pir.as_u32(out).reshape(B, h.words)
        assert np.array_equal(got, oracle.chor_answer(DB, rows, Q_np, threads=oracle.max_threads())), seed
    del g
    h.close()
