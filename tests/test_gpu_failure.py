"""Failure detection on the GPU without a fault: the bounded wait every
TMA/tcgen05 kernel uses gives up on a barrier that nothing arrives on,
reports the timeout through its status word, and the context stays usable."""
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


def test_bounded_wait_gives_up_and_reports(cuda):
    status, waited = pir.qpadl_selftest_bounded_wait(arrive=False)
    assert status == 1                       # the device code of QPADL_ETIMEOUT
    assert 1.5e9 < waited < 10e9             # the 2 s limit, not a hang
    # the context still works: a Response right after equals the oracle
    R, C = 256, 1024
    D = inputs.db_digits(R, C, 256, seed=5)
    db = pir.qpadl_pir_setup(pir.params(R, C, 8), torch.from_numpy(D).cuda())
    q = inputs.uniform_u32(C, seed=6, tag=inputs.TAG_MISC)
    ans = torch.empty(R, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_answer(db, pir.from_u32(q), ans)
    torch.cuda.synchronize()
    assert np.array_equal(pir.as_u32(ans), oracle.answer(D, q))
    assert pir.qpadl_pir_status(db) == pir.QPADL_OK
    db.close()


def test_completed_barrier_returns_at_once(cuda):
    status, waited = pir.qpadl_selftest_bounded_wait(arrive=True)
    assert status == 0 and waited < 1e8
