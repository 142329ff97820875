"""The autotuner times the exact-path choices of a handle on the device and
keeps the fastest; whatever it picks, every answer still equals the oracle."""
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


def _check_answers(db, D, C, R, batches):
    for B in batches:
        Q_np = inputs.uniform_u32(B * C, seed=300 + B, tag=inputs.TAG_MISC).reshape(B, C)
        ans = torch.empty(B * R, dtype=torch.int32, device="cuda")
        if B == 1:
            pir.qpadl_pir_answer(db, pir.from_u32(np.ascontiguousarray(Q_np[0])), ans)
        else:
            pir.qpadl_pir_answer_batch(db, pir.from_u32(Q_np.reshape(-1)), ans)
        torch.cuda.synchronize()
        assert np.array_equal(pir.as_u32(ans).reshape(B, R), oracle.answer_batch(D, Q_np, threads=oracle.max_threads()))


@pytest.mark.parametrize("R,C,max_batch", [(4096, 8192, 16), (1000, 2048 + 48, 4), (777, 4096, 1)])
def test_autotune_picks_valid_options_and_keeps_answers_exact(cuda, R, C, max_batch):
    D = inputs.db_digits(R, C, 256, seed=R + C)
    db = pir.qpadl_pir_setup(pir.params(R, C, 16, seed=1), torch.from_numpy(D).cuda())
    before = pir.qpadl_pir_get_option(db, pir.QPADL_OPT_TENSOR_MIN_BATCH)
    rep = pir.qpadl_pir_autotune(db, max_batch)
    assert pir.qpadl_pir_status(db) == pir.QPADL_OK
    assert rep["stream_chunk"] in (1024, 2048, 4096) and rep["stream_raw"] in (0, 1)
    assert pir.qpadl_pir_get_option(db, pir.QPADL_OPT_STREAM_CHUNK) == rep["stream_chunk"]
    assert pir.qpadl_pir_get_option(db, pir.QPADL_OPT_STREAM_RAW) == rep["stream_raw"]
    timed = [t for row in rep["single_ms"] for t in row if t > 0]
    assert timed and min(timed) > 0
    if max_batch >= 2:
        assert 2 <= rep["tensor_min_batch"] <= 5
        assert pir.qpadl_pir_get_option(db, pir.QPADL_OPT_TENSOR_MIN_BATCH) == rep["tensor_min_batch"]
        assert all(t > 0 for t in rep["stream_ms"][:1])
        if rep["u8_kstep_ms"][0] > 0:
            # both stage depths were timed; with the pair tiles on (the default) the depth stays at
            # 128, the only one they take
            assert rep["u8_kstep_ms"][1] > 0
            assert pir.qpadl_pir_get_option(db, pir.QPADL_OPT_PAIR_GEMM) == 1
            assert pir.qpadl_pir_get_option(db, pir.QPADL_OPT_U8_KSTEP) == 128 == rep["u8_kstep"]
    else:
        assert pir.qpadl_pir_get_option(db, pir.QPADL_OPT_TENSOR_MIN_BATCH) == before
    _check_answers(db, D, C, R, (1, 2, 3, 5, 16))
    db.close()


def test_autotune_chooses_the_uint8_gemm_limit(cuda):
    # max_batch above 32: the tuner times both batched GEMMs at 64 and 128 queries and keeps the
    # largest batch the uint8-digit GEMM wins; answers on either side of the limit stay exact
    R, C = 2048, 4096
    D = inputs.db_digits(R, C, 256, seed=17)
    db = pir.qpadl_pir_setup(pir.params(R, C, 16, seed=1), torch.from_numpy(D).cuda())
    rep = pir.qpadl_pir_autotune(db, 256)
    assert rep["u8_max_batch"] in (32, 64, 128)
    assert pir.qpadl_pir_get_option(db, pir.QPADL_OPT_U8_MAX_BATCH) == rep["u8_max_batch"]
    assert all(t > 0 for row in rep["u8_vs_f16_ms"] for t in row)
    _check_answers(db, D, C, R, (33, 64, 65, 129))
    db.close()


def test_autotune_rejects_bad_arguments(cuda):
    D = torch.zeros(64 * 64, dtype=torch.uint8, device="cuda")
    db = pir.qpadl_pir_setup(pir.params(64, 64, 8), D)
    with pytest.raises(pir.QpadlError) as e:
        pir.qpadl_pir_autotune(db, 0)
    assert e.value.code == pir.QPADL_EINVAL
    db.close()
