"""Database compression (Sec. 5.3) on the GPU: the byte width, the compressed
database and the block decoding equal the oracle's bit for bit, and a record
retrieved privately from the compressed database (Query -> Answer -> Recover
on R' = 4 + w (E - 1) rows) decodes to the original entries."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_03631_gb300 import inputs, pir

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pir.load()
    torch.cuda.set_device(0)
    yield


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).cuda()


@pytest.mark.parametrize("n,E,gap", [(1000, 16, 40), (999, 7, 300), (37, 5, 70000), (8, 1, 3), (5, 8, 9),
                                     (40000, 2048, 255), (65537, 4096, 256), (3000, 300, 2 ** 24)])
def test_width_and_encode_match_oracle(n, E, gap):
    x = inputs.sorted_entries(n, seed=n + E, max_gap=gap)
    xd = _dev(x)
    w = pir.qpadl_pir_delta_width(xd, E)
    assert w == oracle.delta_width(x, E)
    C = (n + E - 1) // E
    db = torch.full((pir.delta_rows(E, w) * C,), 0xAB, dtype=torch.uint8, device="cuda")
    pir.qpadl_pir_delta_encode(xd, E, w, db)
    torch.cuda.synchronize()
    assert np.array_equal(db.cpu().numpy().reshape(pir.delta_rows(E, w), C), oracle.delta_encode(x, E, w))


@pytest.mark.parametrize("E,w,B", [(1, 1, 3), (2, 1, 5), (300, 2, 7), (4096, 1, 64), (5000, 3, 2), (257, 4, 300)])
def test_decode_matches_oracle(E, w, B):
    Rp = pir.delta_rows(E, w)
    digits = inputs.uniform_u32((B * Rp + 3) // 4, seed=E + w, tag=inputs.TAG_MISC).view(np.uint8)[:B * Rp]
    digits = np.ascontiguousarray(digits).reshape(B, Rp)
    out = torch.empty(B * E, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_delta_decode(torch.from_numpy(digits).cuda(), B, E, w, out)
    torch.cuda.synchronize()
    exp = np.stack([oracle.delta_decode(digits[b], E, w) for b in range(B)])
    assert np.array_equal(pir.as_u32(out).reshape(B, E), exp)


def test_unsorted_entries_round_trip():
    x = inputs.uniform_u32(5000, seed=9, tag=inputs.TAG_MISC)
    E = 100
    xd = _dev(x)
    w = pir.qpadl_pir_delta_width(xd, E)
    assert w == 4
    C = (x.size + E - 1) // E
    db = torch.empty(pir.delta_rows(E, w) * C, dtype=torch.uint8, device="cuda")
    pir.qpadl_pir_delta_encode(xd, E, w, db)
    cols = db.view(pir.delta_rows(E, w), C).t().contiguous()   # every block's digits as a row
    out = torch.empty(C * E, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_delta_decode(cols, C, E, w, out)
    torch.cuda.synchronize()
    assert np.array_equal(pir.as_u32(out), x)


@pytest.mark.parametrize("E,gap", [(512, 31), (700, 1000)])
def test_private_retrieval_from_the_compressed_database(E, gap):
    # the compressed database is an ordinary R' x C digit matrix: the lattice PIR retrieves block
    # j (a column) and the client decodes it to the original entries
    C, n_lwe = 1024, 512
    n = C * E - 123                                   # a ragged last block
    x = inputs.sorted_entries(n, seed=E, max_gap=gap)
    xd = _dev(x)
    w = pir.qpadl_pir_delta_width(xd, E)
    Rp = pir.delta_rows(E, w)
    db = torch.empty(Rp * C, dtype=torch.uint8, device="cuda")
    pir.qpadl_pir_delta_encode(xd, E, w, db)
    prm = pir.params(Rp, C, n_lwe, seed=E)
    h = pir.qpadl_pir_setup(prm, db)
    A = torch.empty(C * n_lwe, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_gen_a(prm, A)
    H = torch.empty(Rp * n_lwe, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_hint(h, A, H)
    B = 6
    cols_np = np.array([0, 1, C // 2, C - 2, C - 1, 77])
    S = pir.from_u32(inputs.secrets(B, n_lwe, seed=1).reshape(-1))
    Eq = torch.from_numpy(inputs.noise_batch(B, C, seed=2).reshape(-1)).cuda()
    Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_query_batch(prm, A, S, Eq, torch.from_numpy(cols_np.astype(np.int32)).cuda(), Q)
    ans = torch.empty(B * Rp, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_answer_batch(h, Q, ans)
    digits = torch.empty(B * Rp, dtype=torch.uint8, device="cuda")
    pir.qpadl_pir_recover_batch(prm, ans, H, S, digits)
    entries = torch.empty(B * E, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_delta_decode(digits, B, E, w, entries)
    torch.cuda.synchronize()
    assert pir.qpadl_pir_status(h) == 0
    got = pir.as_u32(entries).reshape(B, E)
    padded = np.concatenate([x, np.full(C * E - n, x[-1], dtype=np.uint32)]).reshape(C, E)
    assert np.array_equal(got, padded[cols_np])
    h.close()
