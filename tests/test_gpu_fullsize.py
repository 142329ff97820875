"""Parity at the full sizes of the measured workloads, in the launch
configuration the benchmark times.

The 1 GiB database (32768 x 32768 digits, n = 1024) is too large for the
oracle to redo every product, so each step is checked two ways:
  - sampled rows: the oracle recomputes chosen rows exactly (first, last,
    rows at CTA-band and MMA-tile boundaries, and seeded random rows);
  - a property over every row: Recover(Answer(Query(col))) must return the
    whole column D[:, col] exactly, which fails if any row of the hint or
    the answer is wrong by more than the noise margin.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_03631_gb300 import inputs, pir

pytestmark = pytest.mark.gpu

W = inputs.WORKLOADS["single_1gib"]
R, C, N, P = W["rows"], W["cols"], W["n"], W["p"]
SEED = 1


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    D = inputs.db_digits(R, C, P, seed=SEED)
    prm = pir.params(R, C, N, p=P, seed=SEED)
    db = pir.qpadl_pir_setup(prm, torch.from_numpy(D).cuda())
    A = torch.empty(C * N, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_gen_a(prm, A)
    H = torch.empty(R * N, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_hint(db, A, H)
    torch.cuda.synchronize()
    assert pir.qpadl_pir_status(db) == 0
    rng = np.random.default_rng(SEED)
    rows = sorted(set([0, 1, 7, 8, 127, 128, 215, 216, 4095, 4096, R - 129, R - 2, R - 1]
                      + rng.integers(0, R, 24).tolist()))
    yield dict(D=D, prm=prm, db=db, A=A, H=H, rows=np.array(rows))
    db.close()


def _check_rows(D, rows, got_rows_by_query, Q_np):
    """Oracle answers of the sampled rows for every query."""
    sub = np.ascontiguousarray(D[rows])
    exp = oracle.answer_batch(sub, Q_np, threads=oracle.max_threads())
    assert np.array_equal(got_rows_by_query, exp)


def _queries(big, B, seed):
    S_np = inputs.secrets(B, N, seed=seed)
    E_np = inputs.noise_batch(B, C, seed=seed + 1)
    cols = inputs.target_columns(B, C, seed=seed + 2)
    Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_query_batch(big["prm"], big["A"], pir.from_u32(S_np.reshape(-1)),
                              torch.from_numpy(E_np.reshape(-1)).cuda(),
                              torch.from_numpy(cols.astype(np.int32)).cuda(), Q)
    return S_np, E_np, cols, Q


def test_setup_and_hint_sampled_rows(big):
    A_np = pir.as_u32(big["A"]).reshape(C, N)
    assert np.array_equal(A_np[[0, 1, C - 1]], oracle.gen_a(SEED, C, N)[[0, 1, C - 1]])
    rows = big["rows"][:12]
    H_np = pir.as_u32(big["H"]).reshape(R, N)
    exp = oracle.hint(np.ascontiguousarray(big["D"][rows]), A_np, threads=oracle.max_threads())
    assert np.array_equal(H_np[rows], exp)


def test_single_query_response_full_size(big):
    S_np, E_np, cols, Q = _queries(big, 1, seed=100)
    ans = torch.empty(R, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_answer(big["db"], Q, ans)
    out = torch.empty(R, dtype=torch.uint8, device="cuda")
    pir.qpadl_pir_recover(big["prm"], ans, big["H"], pir.from_u32(S_np[0]), out)
    torch.cuda.synchronize()
    assert pir.qpadl_pir_status(big["db"]) == 0
    ans_np = pir.as_u32(ans)
    rows = big["rows"]
    _check_rows(big["D"], rows, ans_np[rows][None, :], pir.as_u32(Q).reshape(1, C))
    # every row: the recovered column is the database column
    assert np.array_equal(out.cpu().numpy(), big["D"][:, cols[0]])


def test_query_matches_oracle_sampled(big):
    S_np, E_np, cols, Q = _queries(big, 4, seed=200)
    torch.cuda.synchronize()
    A_np = pir.as_u32(big["A"]).reshape(C, N)
    Q_np = pir.as_u32(Q).reshape(4, C)
    for b in range(4):
        assert np.array_equal(Q_np[b], oracle.query(A_np, S_np[b], E_np[b], int(cols[b]), 1 << 24))


# 16: uint8-digit GEMM, 64-column tiles; 64: two 128-column tiles per row tile; 128: the fp16-copy
# pair GEMM with a split tail; 256, 1024: whole tiles
@pytest.mark.parametrize("B", [16, 64, 128, 256, 1024])
def test_batched_response_full_size(big, B):
    S_np, E_np, cols, Q = _queries(big, B, seed=300 + B)
    ans = torch.empty(B * R, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_answer_batch(big["db"], Q, ans)
    out = torch.empty(B * R, dtype=torch.uint8, device="cuda")
    pir.qpadl_pir_recover_batch(big["prm"], ans, big["H"], pir.from_u32(S_np.reshape(-1)), out)
    torch.cuda.synchronize()
    assert pir.qpadl_pir_status(big["db"]) == 0
    ans_np = pir.as_u32(ans).reshape(B, R)
    rows = big["rows"][:16]
    Q_np = pir.as_u32(Q).reshape(B, C)
    _check_rows(big["D"], rows, ans_np[:, rows], Q_np)
    got = out.cpu().numpy().reshape(B, R)
    assert np.array_equal(got, big["D"][:, cols].T)


@pytest.mark.parametrize("B", [2, 4, 8, 32])
def test_small_batches_both_paths_full_size(big, B):
    Q_np = inputs.uniform_u32(B * C, seed=B, tag=inputs.TAG_MISC).reshape(B, C)
    Q = pir.from_u32(Q_np.reshape(-1))
    rows = big["rows"][:8]
    for path in (0, 1):
        ans = torch.empty(B * R, dtype=torch.int32, device="cuda")
        pir.qpadl_pir_answer_batch(big["db"], Q, ans, path=path)
        torch.cuda.synchronize()
        ans_np = pir.as_u32(ans).reshape(B, R)
        _check_rows(big["D"], rows, ans_np[:, rows], Q_np)


def test_client_batch_full_size(big):
    # 1024 queries and recoveries through the tensor-core client context
    B = 1024
    S_np = inputs.secrets(B, N, seed=700)
    E_np = inputs.noise_batch(B, C, seed=701)
    cols = inputs.target_columns(B, C, seed=702)
    S = pir.from_u32(S_np.reshape(-1))
    E = torch.from_numpy(E_np.reshape(-1)).cuda()
    cols_t = torch.from_numpy(cols.astype(np.int32)).cuda()
    cl = pir.qpadl_client_create(big["prm"], big["A"], big["H"], max_batch=B)
    Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
    pir.qpadl_client_query_batch(cl, S, E, cols_t, Q)
    ans = torch.empty(B * R, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_answer_batch(big["db"], Q, ans)
    out = torch.empty(B * R, dtype=torch.uint8, device="cuda")
    pir.qpadl_client_recover_batch(cl, ans, S, out)
    torch.cuda.synchronize()
    assert pir.qpadl_client_status(cl) == pir.QPADL_OK
    A_np = pir.as_u32(big["A"]).reshape(C, N)
    Q_np = pir.as_u32(Q).reshape(B, C)
    for b in (0, 1, 511, B - 1):
        assert np.array_equal(Q_np[b], oracle.query(A_np, S_np[b], E_np[b], int(cols[b]), 1 << 24))
    # Recover(Answer(Query(col))) = D[:, col] for all 1024 queries over every row
    assert np.array_equal(out.cpu().numpy().reshape(B, R), big["D"][:, cols].T)
    cl.close()
