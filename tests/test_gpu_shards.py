"""Row shards on one GPU, run one after another: each shard is its own
handle over a band of the database's rows; the shards' Hint, Response
(single and batched, every path) and Recover concatenate to the full
results and to the oracle's."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_03631_gb300 import inputs, pir, replicas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("R,C,world", [(1000, 2048, 3), (1536, 4096 + 48, 2), (640, 1024, 5)])
def test_shards_concatenate(cuda, R, C, world):
    n, seed = 64, 40
    D = inputs.db_digits(R, C, 256, seed=seed)
    D_dev = torch.from_numpy(D).cuda()
    prm_full = pir.params(R, C, n, seed=seed)
    A = torch.empty(C * n, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_gen_a(prm_full, A)
    B = 40
    Q = torch.from_numpy(inputs.uniform_u32(B * C, seed=seed + 1, tag=inputs.TAG_MISC).view(np.int32)).cuda()
    s = torch.from_numpy(inputs.secrets(1, n, seed=seed + 2).reshape(-1).view(np.int32)).cuda()
    e = torch.from_numpy(inputs.noise(C, seed=seed + 3)).cuda()
    col = 17
    q = torch.empty(C, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_query(prm_full, A, s, e, col, q)
    parts = {"hint": [], "one": [], "b8": [], "b40": [], "rec": []}
    for r in range(world):
        r0, r1 = replicas.shard_rows(R, world, r)
        rows = r1 - r0
        assert rows > 0
        h = pir.qpadl_pir_setup(pir.params(rows, C, n, seed=seed), D_dev[r0:r1])
        H = torch.empty(rows * n, dtype=torch.int32, device="cuda")
        pir.qpadl_pir_hint(h, A, H)
        a1 = torch.empty(rows, dtype=torch.int32, device="cuda")
        pir.qpadl_pir_answer(h, q, a1)
        a8 = torch.empty(8 * rows, dtype=torch.int32, device="cuda")
        pir.qpadl_pir_answer_batch(h, Q[: 8 * C], a8)
        a40 = torch.empty(B * rows, dtype=torch.int32, device="cuda")
        pir.qpadl_pir_answer_batch(h, Q, a40)
        out = torch.empty(rows, dtype=torch.uint8, device="cuda")
        pir.qpadl_pir_recover(pir.params(rows, C, n, seed=seed), a1, H, s, out)
        torch.cuda.synchronize()
        parts["hint"].append(pir.as_u32(H).reshape(rows, n))
        parts["one"].append(pir.as_u32(a1))
        parts["b8"].append(pir.as_u32(a8).reshape(8, rows))
        parts["b40"].append(pir.as_u32(a40).reshape(B, rows))
        parts["rec"].append(out.cpu().numpy())
        h.close()
    A_np = pir.as_u32(A).reshape(C, n)
    Q_np = pir.as_u32(Q).reshape(B, C)
    assert np.array_equal(np.concatenate(parts["hint"]), oracle.hint(D, A_np))
    assert np.array_equal(np.concatenate(parts["one"]), oracle.answer(D, pir.as_u32(q)))
    assert np.array_equal(np.concatenate(parts["b8"], axis=1), oracle.answer_batch(D, Q_np[:8]))
    assert np.array_equal(np.concatenate(parts["b40"], axis=1), oracle.answer_batch(D, Q_np))
    assert np.array_equal(np.concatenate(parts["rec"]), D[:, col])
