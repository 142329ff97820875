"""Client context: batched Query and Recover on the tensor cores equal the
oracle's Query and Recover (and the CUDA-core batch entry points) bit for
bit, across ragged shapes, chunked batches and limb-boundary values."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_03631_gb300 import inputs, pir

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev_u32(a):
    return pir.from_u32(np.ascontiguousarray(a, dtype=np.uint32).reshape(-1))


# (R, C, n, B, max_batch): ragged C, n not a multiple of 64, batches chunked by max_batch
CASES = [(1024, 1024, 512, 8, 1024), (700, 1000, 64, 37, 16), (300, 4096 + 48, 96, 130, 64),
         (2048, 2048, 1024, 256, 256), (129, 257, 16, 3, 1), (512, 512, 128, 65, 65)]


@pytest.mark.parametrize("pair", [1, 0])
@pytest.mark.parametrize("R,C,n,B,max_batch", CASES)
def test_query_and_recover_match_oracle(cuda, R, C, n, B, max_batch, pair):
    seed = R + C + n + B
    D = inputs.db_digits(R, C, 256, seed=seed)
    A_np = inputs.public_matrix(C, n, seed=seed + 1)
    H_np = oracle.hint(D, A_np, threads=oracle.max_threads())
    S_np = inputs.secrets(B, n, seed=seed + 2)
    E_np = inputs.noise_batch(B, C, seed=seed + 3)
    cols = inputs.target_columns(B, C, seed=seed + 4)
    prm = pir.params(R, C, n, seed=seed)
    A, H, S = _dev_u32(A_np), _dev_u32(H_np), _dev_u32(S_np)
    E = torch.from_numpy(np.ascontiguousarray(E_np).reshape(-1)).cuda()
    cols_t = torch.from_numpy(cols.astype(np.int32)).cuda()
    cl = pir.qpadl_client_create(prm, A, H, max_batch=max_batch)
    pir.qpadl_client_set_option(cl, pir.QPADL_CLIENT_OPT_PAIR_GEMM, pair)
    Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
    pir.qpadl_client_query_batch(cl, S, E, cols_t, Q)
    Q_simt = torch.empty_like(Q)
    pir.qpadl_pir_query_batch(prm, A, S, E, cols_t, Q_simt)
    torch.cuda.synchronize()
    Q_np = pir.as_u32(Q).reshape(B, C)
    for b in range(B):
        assert np.array_equal(Q_np[b], oracle.query(A_np, S_np[b], E_np[b], int(cols[b]), 1 << 24)), b
    assert torch.equal(Q, Q_simt)
    ans_np = oracle.answer_batch(D, Q_np, threads=oracle.max_threads())
    out = torch.empty(B * R, dtype=torch.uint8, device="cuda")
    pir.qpadl_client_recover_batch(cl, _dev_u32(ans_np), S, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(B, R)
    for b in range(B):
        assert np.array_equal(got[b], oracle.recover(ans_np[b], H_np, S_np[b])), b
    assert np.array_equal(got, D[:, cols].T)   # every queried record recovered exactly
    assert pir.qpadl_client_status(cl) == pir.QPADL_OK
    assert pir.qpadl_client_device_bytes(cl) >= 8 * (C + R) * n
    cl.close()


# n a multiple of 512 and B > 8: shift groups of 16, 32 and 64 columns, ragged last tiles, chunked batches
@pytest.mark.parametrize("R,C,n,B,max_batch", [(1000, 1500, 512, 12, 64), (700, 600, 512, 24, 1024),
                                               (300, 2048 + 40, 1024, 37, 1024), (513, 1000, 1024, 150, 70)])
@pytest.mark.parametrize("skip", [0, 1])
@pytest.mark.parametrize("pair", [1, 0])
def test_zero_block_skipping_on_and_off(cuda, R, C, n, B, max_batch, skip, pair):
    seed = 3 * R + C + n + B
    D = inputs.db_digits(R, C, 256, seed=seed)
    A_np = inputs.public_matrix(C, n, seed=seed + 1)
    H_np = oracle.hint(D, A_np, threads=oracle.max_threads())
    S_np = inputs.secrets(B, n, seed=seed + 2)
    E_np = inputs.noise_batch(B, C, seed=seed + 3)
    cols = inputs.target_columns(B, C, seed=seed + 4)
    cl = pir.qpadl_client_create(pir.params(R, C, n, seed=seed), _dev_u32(A_np), _dev_u32(H_np),
                                 max_batch=max_batch)
    pir.qpadl_client_set_option(cl, pir.QPADL_CLIENT_OPT_SKIP_ZERO_BLOCKS, skip)
    pir.qpadl_client_set_option(cl, pir.QPADL_CLIENT_OPT_PAIR_GEMM, pair)
    Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
    pir.qpadl_client_query_batch(cl, _dev_u32(S_np), torch.from_numpy(E_np.reshape(-1)).cuda(),
                                 torch.from_numpy(cols.astype(np.int32)).cuda(), Q)
    torch.cuda.synchronize()
    Q_np = pir.as_u32(Q).reshape(B, C)
    for b in range(B):
        assert np.array_equal(Q_np[b], oracle.query(A_np, S_np[b], E_np[b], int(cols[b]), 1 << 24)), b
    ans_np = oracle.answer_batch(D, Q_np, threads=oracle.max_threads())
    out = torch.empty(B * R, dtype=torch.uint8, device="cuda")
    pir.qpadl_client_recover_batch(cl, _dev_u32(ans_np), _dev_u32(S_np), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(B, R)
    for b in range(0, B, 7):
        assert np.array_equal(got[b], oracle.recover(ans_np[b], H_np, S_np[b])), b
    assert np.array_equal(got, D[:, cols].T)
    assert pir.qpadl_client_status(cl) == pir.QPADL_OK
    cl.close()


@pytest.mark.parametrize("a_word,s_word", [(0x7F7F7F80, 0x7F7F7F80),   # every limb -128: chunks of 2^24 exactly
                                           (0xFFFFFFFF, 0xFFFFFFFF), (0x80808080, 0x80808080),
                                           (0x7F7F7F7F, 0x80808080), (0x80808080, 0x7F7F7F7F),
                                           (0x7F7F7F7F, 0x7F7F7F7F), (0x00800080, 0xFF7FFF80)])
@pytest.mark.parametrize("B", [16, 40])
def test_limb_boundary_values(cuda, a_word, s_word, B):
    # every limb at +-127/-128 pushes each exact chunk to its bound (1024-deep chunks of limb
    # products reach 2^24 when every limb is -128); B = 16 runs 64-wide pair tiles (plain), B = 40
    # planed 256-wide pair tiles
    R, C, n = 256, 512, 1024
    A_np = np.full((C, n), a_word, dtype=np.uint32)
    S_np = np.full((B, n), s_word, dtype=np.uint32)
    H_np = np.full((R, n), a_word, dtype=np.uint32)
    E_np = np.zeros((B, C), dtype=np.int32)
    cols = np.array([0, 1, C - 1, 77] * (B // 4), dtype=np.int32)
    prm = pir.params(R, C, n)
    cl = pir.qpadl_client_create(prm, _dev_u32(A_np), _dev_u32(H_np), max_batch=B)
    Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
    pir.qpadl_client_query_batch(cl, _dev_u32(S_np), torch.from_numpy(E_np.reshape(-1)).cuda(),
                                 torch.from_numpy(cols).cuda(), Q)
    ans_np = inputs.uniform_u32(B * R, seed=5, tag=inputs.TAG_MISC).reshape(B, R)
    out = torch.empty(B * R, dtype=torch.uint8, device="cuda")
    pir.qpadl_client_recover_batch(cl, _dev_u32(ans_np), _dev_u32(S_np), out)
    torch.cuda.synchronize()
    Q_np = pir.as_u32(Q).reshape(B, C)
    got = out.cpu().numpy().reshape(B, R)
    for b in range(B):
        assert np.array_equal(Q_np[b], oracle.query(A_np, S_np[b], E_np[b], int(cols[b]), 1 << 24))
        assert np.array_equal(got[b], oracle.recover(ans_np[b], H_np, S_np[b]))
    cl.close()


def test_other_moduli(cuda):
    for p in (2, 16):
        R, C, n, B = 200, 300, 64, 5
        D = inputs.db_digits(R, C, p, seed=p)
        A_np = inputs.uniform_u32(C * n, seed=p + 1, tag=inputs.TAG_A).reshape(C, n)
        H_np = oracle.hint(D, A_np)
        S_np = inputs.secrets(B, n, seed=p + 2)
        E_np = inputs.noise_batch(B, C, seed=p + 3)
        cols = inputs.target_columns(B, C, seed=p + 4)
        prm = pir.params(R, C, n, p=p)
        cl = pir.qpadl_client_create(prm, _dev_u32(A_np), _dev_u32(H_np), max_batch=8)
        Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
        pir.qpadl_client_query_batch(cl, _dev_u32(S_np), torch.from_numpy(E_np.reshape(-1)).cuda(),
                                     torch.from_numpy(cols.astype(np.int32)).cuda(), Q)
        torch.cuda.synchronize()
        Q_np = pir.as_u32(Q).reshape(B, C)
        delta = oracle.delta_for(p)
        for b in range(B):
            assert np.array_equal(Q_np[b], oracle.query(A_np, S_np[b], E_np[b], int(cols[b]), delta))
        ans_np = oracle.answer_batch(D, Q_np)
        out = torch.empty(B * R, dtype=torch.uint8, device="cuda")
        pir.qpadl_client_recover_batch(cl, _dev_u32(ans_np), _dev_u32(S_np), out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().reshape(B, R), D[:, cols].T)
        cl.close()


def test_errors(cuda):
    prm = pir.params(64, 64, 8)
    A = torch.zeros(64 * 8, dtype=torch.int32, device="cuda")
    with pytest.raises(pir.QpadlError) as e:
        pir.qpadl_client_create(prm, A, None, max_batch=0)
    assert e.value.code == pir.QPADL_EINVAL
    cl = pir.qpadl_client_create(prm, A, None, max_batch=4)
    S = torch.zeros(4 * 8, dtype=torch.int32, device="cuda")
    ans = torch.zeros(4 * 64, dtype=torch.int32, device="cuda")
    out = torch.zeros(4 * 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(pir.QpadlError) as e:   # built without the hint
        pir.qpadl_client_recover_batch(cl, ans, S, out)
    assert e.value.code == pir.QPADL_EINVAL
    for opt, val in ((pir.QPADL_CLIENT_OPT_SKIP_ZERO_BLOCKS, 2), (99, 0)):
        with pytest.raises(pir.QpadlError) as e:
            pir.qpadl_client_set_option(cl, opt, val)
        assert e.value.code == pir.QPADL_EINVAL
    cl.close()
