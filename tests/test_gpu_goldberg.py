"""Goldberg-style Response over Z_p (Sec. 5.2, Alg. 4): both the streaming
path (exact integer sums, then mod p) and the one-limb tensor-core GEMM
(centred queries, mod-p epilogue) equal the oracle element for element, at
the exact-sum bounds too, and the FTR protocol of Sec. 7 recovers records
through them."""
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


def _db(R, C, p, seed):
    return (inputs.db_digits(R, C, 256, seed=seed).astype(np.int64) % p).astype(np.uint8)


def _answer(h, Q_np, gemm_min=None, u8max=None):
    if gemm_min is not None:
        pir.qpadl_goldberg_set_option(h, pir.QPADL_GOLDBERG_OPT_GEMM_MIN_BATCH, gemm_min)
    if u8max is not None:
        pir.qpadl_goldberg_set_option(h, pir.QPADL_GOLDBERG_OPT_U8_MAX_BATCH, u8max)
    B = Q_np.shape[0]
    out = torch.empty(B * h.rows, dtype=torch.int32, device="cuda")
    pir.qpadl_goldberg_answer_batch(h, pir.from_u32(np.ascontiguousarray(Q_np).reshape(-1)), out)
    torch.cuda.synchronize()
    assert pir.qpadl_goldberg_status(h) == pir.QPADL_OK
    return pir.as_u32(out).reshape(B, h.rows)


CASES = [(300, 1000, 257, 1), (257, 513, 251, 4), (1000, 2048, 257, 5), (700, 4096 + 48, 101, 33),
         (129, 300, 257, 64), (2000, 1024, 257, 200), (384, 512, 2, 7), (50, 777, 257, 1100),
         (640, 512, 257, 65), (333, 1500, 101, 300),
         (600, 2048, 2, 100), (520, 1100, 3, 257)]   # p < 4 on the 256-wide one-limb tiles


@pytest.mark.parametrize("R,C,p,B", CASES)
# uint8-digit GEMM up to 32, 64 or 256 queries (on SM pairs or single SMs; above 64 several tiles
# per row tile) / fp16-copy GEMM / streaming
@pytest.mark.parametrize("gemm_min,u8max,pair", [(1, 32, 1), (1, 64, 1), (1, 64, 0), (1, 256, 1), (1, 256, 0),
                                                 (1, 0, 1), (1 << 30, 32, 1)])
def test_goldberg_matches_oracle(cuda, R, C, p, B, gemm_min, u8max, pair):
    D = _db(R, C, p, seed=R + C)
    Q = (inputs.uniform_u32(B * C, seed=B + p, tag=inputs.TAG_MISC) % p).reshape(B, C)
    h = pir.qpadl_goldberg_setup(R, C, p, torch.from_numpy(D).cuda())
    pir.qpadl_goldberg_set_option(h, pir.QPADL_GOLDBERG_OPT_PAIR_GEMM, pair)
    got = _answer(h, Q, gemm_min, u8max)
    assert np.array_equal(got, oracle.goldberg_answer(D, Q, p, threads=oracle.max_threads()))
    h.close()


@pytest.mark.parametrize("B", [40, 100])
def test_many_row_tiles(cuda, B):
    # 313 row tiles: every persistent CTA of the one-limb GEMM (register sums at 40 queries,
    # TMEM-resident residues at 100) walks two or three tiles
    R, C, p = 40000, 1100, 257
    D = _db(R, C, p, seed=B)
    Q = (inputs.uniform_u32(B * C, seed=B + 9, tag=inputs.TAG_MISC) % p).reshape(B, C)
    h = pir.qpadl_goldberg_setup(R, C, p, torch.from_numpy(D).cuda())
    got = _answer(h, Q, 1, 0)
    assert np.array_equal(got, oracle.goldberg_answer(D, Q, p, threads=oracle.max_threads()))
    h.close()


@pytest.mark.parametrize("gemm_min,u8max,B", [(1, 32, 6), (1, 64, 40), (1, 0, 6), (1 << 30, 32, 6), (1, 0, 70)])
@pytest.mark.parametrize("qval", [256, 128, 129])
def test_exact_sum_bounds(cuda, gemm_min, u8max, B, qval):
    # the largest allowed record count with every byte 255: the unsigned sum of the streaming
    # path, the signed sums of the uint8-digit GEMM (6 and 40 queries), the centred register
    # sums of the fp16-copy GEMM (6 queries) and its TMEM-resident residues reduced mod p after
    # every chunk (70 queries) all stay exact
    R, C, p = 128, 65792, 257
    D = np.full((R, C), 255, dtype=np.uint8)
    D[::3, ::7] = 0
    Q = np.full((B, C), qval, dtype=np.uint32)
    h = pir.qpadl_goldberg_setup(R, C, p, torch.from_numpy(D).cuda())
    got = _answer(h, Q, gemm_min, u8max)
    assert np.array_equal(got, oracle.goldberg_answer(D, Q, p, threads=oracle.max_threads()))
    h.close()


@pytest.mark.parametrize("t,ell", [(1, 3), (3, 5)])
def test_ftr_protocol_recovers_the_record(cuda, t, ell):
    p, R, C = 257, 500, 3000
    D = _db(R, C, p, seed=t)
    h = pir.qpadl_goldberg_setup(R, C, p, torch.from_numpy(D).cuda())
    alpha = np.arange(1, ell + 1, dtype=np.uint32)
    for theta in (0, 1234, C - 1):
        coef = (inputs.uniform_u32(C * t, seed=theta, tag=inputs.TAG_MISC) % p).reshape(C, t)
        queries = oracle.goldberg_query(coef, theta, alpha, p)
        responses = _answer(h, queries)   # each server answers its share
        rec = oracle.goldberg_reconstruct(responses[: t + 1], alpha[: t + 1], p)
        assert np.array_equal(rec, D[:, theta].astype(np.uint32))
    h.close()


def test_errors(cuda):
    D = torch.zeros(64 * 64, dtype=torch.uint8, device="cuda")
    for p in (256, 258, 1, 0, 91):
        with pytest.raises(pir.QpadlError) as e:
            pir.qpadl_goldberg_setup(64, 64, p, D)
        assert e.value.code == pir.QPADL_EINVAL
    big = torch.zeros(65793, dtype=torch.uint8, device="cuda")
    with pytest.raises(pir.QpadlError) as e:
        pir.qpadl_goldberg_setup(1, 65793, 257, big)
    assert e.value.code == pir.QPADL_EINVAL
    D2 = torch.full((64 * 64,), 251, dtype=torch.uint8, device="cuda")   # not an element of Z_251
    with pytest.raises(pir.QpadlError) as e:
        pir.qpadl_goldberg_setup(64, 64, 251, D2)
    assert e.value.code == pir.QPADL_EINVAL


@pytest.mark.parametrize("B", [1, 256])
def test_full_size_sampled_rows(cuda, B):
    W = inputs.WORKLOADS["single_1gib"]
    R, C, p = W["rows"], W["cols"], 257
    D = inputs.db_digits(R, C, 256, seed=3)
    Q = (inputs.uniform_u32(B * C, seed=4 + B, tag=inputs.TAG_MISC) % p).reshape(B, C)
    h = pir.qpadl_goldberg_setup(R, C, p, torch.from_numpy(D).cuda())
    got = _answer(h, Q)
    rows = np.array([0, 1, 127, 128, 4095, 16384, R - 1])
    exp = oracle.goldberg_answer(np.ascontiguousarray(D[rows]), Q, p, threads=oracle.max_threads())
    assert np.array_equal(got[:, rows], exp)
    h.close()
