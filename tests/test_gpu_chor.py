"""Chor-style Response over GF(2) (Sec. 5.2, Alg. 3): the batched one-pass
kernel equals the oracle's XOR of selected rows word for word, across ragged
row counts, column tiles and batch sizes (including chunked batches above
256), and the ENS protocol of Sec. 7 recovers the record through it."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32).reshape(-1)).cuda()


def _answer(h, Q_np):
    B = Q_np.shape[0]
    out = torch.empty(B * h.words, dtype=torch.int32, device="cuda")
    pir.qpadl_chor_answer_batch(h, _dev(Q_np), out)
    torch.cuda.synchronize()
    assert pir.qpadl_chor_status(h) == pir.QPADL_OK
    return pir.as_u32(out).reshape(B, h.words)


# (rows, bits, B): rows below one band, ragged bands, words not a multiple of the
# column tile, every kernel shape (1..32 queries per group, 2/4/8 groups), chunked batches
CASES = [(100, 128, 1), (33, 128, 7), (1000, 1024, 3), (777, 4096 + 128, 17), (513, 2048, 32), (64, 256, 33),
         (300, 8192, 100), (2000, 1280, 256), (129, 384, 300), (4097, 32768, 2), (1500, 512, 64), (90, 2560, 129)]


@pytest.mark.parametrize("rows,bits,B", CASES)
@pytest.mark.parametrize("m4rm_min", [257, 1])   # masked-XOR scan only / four-Russians kernel only
def test_chor_matches_oracle(cuda, rows, bits, B, m4rm_min):
    DB = inputs.chor_db(rows, bits, seed=rows + bits)
    Q = inputs.chor_queries(B, rows, seed=rows * 7 + B)
    h = pir.qpadl_chor_setup(rows, bits, _dev(DB))
    pir.qpadl_chor_set_option(h, pir.QPADL_CHOR_OPT_M4RM_MIN_BATCH, m4rm_min)
    assert pir.qpadl_chor_get_option(h, pir.QPADL_CHOR_OPT_M4RM_MIN_BATCH) == m4rm_min
    exp = oracle.chor_answer(DB, rows, Q, threads=oracle.max_threads())
    # every inner-loop form of the masked-XOR scan (4 or 8 words per thread, mask or predicated)
    for form in ((0, 1, 2, 3) if m4rm_min > 256 else (0,)):
        pir.qpadl_chor_set_option(h, pir.QPADL_CHOR_OPT_SCAN_FORM, form)
        assert pir.qpadl_chor_get_option(h, pir.QPADL_CHOR_OPT_SCAN_FORM) == form
        assert np.array_equal(_answer(h, Q), exp), f"form {form}"
    h.close()


@pytest.mark.parametrize("m4rm_min", [257, 1])
def test_padding_bits_are_ignored(cuda, m4rm_min):
    rows, bits = 45, 256
    DB = inputs.chor_db(rows, bits, seed=3)
    Q = inputs.chor_queries(5, rows, seed=4)
    noisy = Q.copy()
    noisy[:, -1] |= np.uint32(0xFFFFFFFF << (rows % 32) & 0xFFFFFFFF)
    h = pir.qpadl_chor_setup(rows, bits, _dev(DB))
    pir.qpadl_chor_set_option(h, pir.QPADL_CHOR_OPT_M4RM_MIN_BATCH, m4rm_min)
    assert np.array_equal(_answer(h, noisy), oracle.chor_answer(DB, rows, Q))
    h.close()


def test_unit_queries_return_the_records(cuda):
    rows, bits = 96, 640
    DB = inputs.chor_db(rows, bits, seed=5)
    Q = np.zeros((rows, 3), dtype=np.uint32)
    for t in range(rows):
        Q[t, t // 32] = np.uint32(1 << (t % 32))
    h = pir.qpadl_chor_setup(rows, bits, _dev(DB))
    assert np.array_equal(_answer(h, Q), DB)
    h.close()


@pytest.mark.parametrize("ell", [2, 4])
def test_ens_protocol_recovers_the_record(cuda, ell):
    rows, bits = 1000, 2048
    DB = inputs.chor_db(rows, bits, seed=6)
    h = pir.qpadl_chor_setup(rows, bits, _dev(DB))
    for theta in (0, 31, 517, rows - 1):
        queries = oracle.chor_query(inputs.chor_queries(ell - 1, rows, seed=theta + 10), theta)
        responses = _answer(h, queries)   # each of the ell servers answers its query
        assert np.array_equal(oracle.chor_reconstruct(responses), DB[theta])
    h.close()


def test_errors(cuda):
    DB = torch.zeros(64 * 8, dtype=torch.int32, device="cuda")
    for rows, bits in ((64, 96), (0, 256), (64, 0)):
        with pytest.raises(pir.QpadlError) as e:
            pir.qpadl_chor_setup(rows, bits, DB)
        assert e.value.code == pir.QPADL_EINVAL
    with pytest.raises(pir.QpadlError) as e:   # misaligned database pointer
        pir.qpadl_chor_setup(8, 128, DB[1:])
    assert e.value.code == pir.QPADL_EINVAL
    h = pir.qpadl_chor_setup(8, 128, DB)
    for opt, val in ((pir.QPADL_CHOR_OPT_M4RM_MIN_BATCH, 0), (pir.QPADL_CHOR_OPT_M4RM_MIN_BATCH, 258), (9, 1)):
        with pytest.raises(pir.QpadlError) as e:
            pir.qpadl_chor_set_option(h, opt, val)
        assert e.value.code == pir.QPADL_EINVAL
    h.close()


@pytest.mark.parametrize("B", [1, 16, 256, 300])
def test_full_size_sampled_columns(cuda, B):
    w = inputs.WORKLOADS["chor_1gib"]
    rows, bits = w["rows"], w["bits"]
    DB = inputs.chor_db(rows, bits, seed=21)
    Q = inputs.chor_queries(B, rows, seed=22 + B)
    h = pir.qpadl_chor_setup(rows, bits, _dev(DB))
    got = _answer(h, Q)
    W = bits // 32
    # word slices at the start, across column-tile boundaries (128..1024 words) and at the end
    for w0 in (0, 96, 1000, 4090, W - 64):
        sl = np.ascontiguousarray(DB[:, w0:w0 + 64])
        exp = oracle.chor_answer(sl, rows, Q, threads=oracle.max_threads())
        assert np.array_equal(got[:, w0:w0 + 64], exp), w0
    h.close()
