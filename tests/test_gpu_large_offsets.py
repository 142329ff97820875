"""Parity on a database larger than 2^32 bytes.

40000 x 131072 digits is 5.24 GB, so every byte offset past row 32768
exceeds 32 bits.  Each path that addresses the database (the streaming
Response and its allocation-free entry point, the uint8-digit and fp16-copy
GEMMs, the hint) is checked on sampled rows on both sides of that boundary
against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_03631_gb300 import inputs, pir

pytestmark = pytest.mark.gpu

R, C, N = 40000, 131072, 64
SEED = 17


@pytest.fixture(scope="module")
def large():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    D_dev = torch.empty(R * C, dtype=torch.uint8, device="cuda")
    band = 4096
    for r0 in range(0, R, band):
        rc = min(band, R - r0)
        blk = inputs.db_digits(R, C, 256, seed=SEED, row_start=r0, row_count=rc)
        D_dev[r0 * C:(r0 + rc) * C].copy_(torch.from_numpy(np.ascontiguousarray(blk).reshape(-1)))
    prm = pir.params(R, C, N, seed=SEED)
    db = pir.qpadl_pir_setup(prm, D_dev)
    rng = np.random.default_rng(SEED)
    first_past = (1 << 32) // C   # first row whose bytes start past 2^32
    rows = sorted(set([0, 1, 127, 128, first_past - 1, first_past, first_past + 1, R - 129, R - 2, R - 1]
                      + rng.integers(0, R, 12).tolist()))
    rows = np.array(rows)
    D_rows = np.stack([inputs.db_digits(R, C, 256, seed=SEED, row_start=int(r), row_count=1)[0] for r in rows])
    yield dict(prm=prm, db=db, D=D_dev, rows=rows, D_rows=D_rows)
    db.close()


def _batch(large, B, path):
    Q_np = inputs.uniform_u32(B * C, seed=B + 3, tag=inputs.TAG_MISC).reshape(B, C)
    ans = torch.empty(B * R, dtype=torch.int32, device="cuda")
    Q = pir.from_u32(Q_np.reshape(-1))
    if B == 1 and path is None:
        pir.qpadl_pir_answer(large["db"], Q, ans)
    else:
        pir.qpadl_pir_answer_batch(large["db"], Q, ans, path=path)
    torch.cuda.synchronize()
    assert pir.qpadl_pir_status(large["db"]) == 0
    got = pir.as_u32(ans).reshape(B, R)[:, large["rows"]]
    exp = oracle.answer_batch(large["D_rows"], Q_np, threads=oracle.max_threads())
    return got, exp


def test_single_query_stream(large):
    got, exp = _batch(large, 1, None)
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("B", [8, 64])
def test_batched_gemms(large, B):
    # 8 queries take the uint8-digit GEMM (blocked copy of the digits), 64 the fp16-copy GEMM
    got, exp = _batch(large, B, 1)
    assert np.array_equal(got, exp)


def test_noalloc_entry_point(large):
    q_np = inputs.uniform_u32(C, seed=5, tag=inputs.TAG_MISC)
    ans = torch.empty(R, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_answer_noalloc(large["D"], R, C, pir.from_u32(q_np), ans)
    torch.cuda.synchronize()
    exp = oracle.answer_batch(large["D_rows"], q_np[None, :], threads=oracle.max_threads())[0]
    assert np.array_equal(pir.as_u32(ans)[large["rows"]], exp)


def test_hint_sampled_rows(large):
    A = torch.empty(C * N, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_gen_a(large["prm"], A)
    H = torch.empty(R * N, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_hint(large["db"], A, H)
    torch.cuda.synchronize()
    assert pir.qpadl_pir_status(large["db"]) == 0
    exp = oracle.hint(large["D_rows"], oracle.gen_a(SEED, C, N), threads=oracle.max_threads())
    assert np.array_equal(pir.as_u32(H).reshape(R, N)[large["rows"]], exp)
