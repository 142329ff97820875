"""Bit-exact parity of every CUDA step with the CPU oracle, through the C ABI.

Sizes here are small enough for the oracle to check every output element
while still spanning several tiles and ragged tails: rows not a multiple of
the 8-row TMA box or the 128-row MMA tile, columns not a multiple of the
256-digit streaming chunk, the 64-element K block or the 512-deep exact
chunk, batch sizes around every limb-tile width, C not a multiple of 16
(the fallback kernel), and the extreme digit/limb values that push the fp32
tensor-core accumulator to its exactness bound.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_03631_gb300 import inputs, pir

pytestmark = pytest.mark.gpu

M32 = (1 << 32) - 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pir.load()
    torch.cuda.set_device(0)
    yield


def _setup(R, C, n=8, p=256, seed=1, D=None, flags=0):
    if D is None:
        D = inputs.db_digits(R, C, p, seed=seed)
    prm = pir.params(R, C, n, p=p, seed=seed, flags=flags)
    db = pir.qpadl_pir_setup(prm, torch.from_numpy(np.ascontiguousarray(D)).cuda())
    return prm, D, db


def _answers(db, Q_np, path=None):
    B = Q_np.shape[0]
    ans = torch.full((B * db.rows,), -1, dtype=torch.int32, device="cuda")
    Q = pir.from_u32(Q_np.reshape(-1))
    if B == 1 and path is None:
        pir.qpadl_pir_answer(db, Q, ans)
    else:
        pir.qpadl_pir_answer_batch(db, Q, ans, path=path)
    torch.cuda.synchronize()
    assert pir.qpadl_pir_status(db) == 0
    return pir.as_u32(ans).reshape(B, db.rows)


# ------------------------------------------------------------------ Setup
@pytest.mark.parametrize("C,n,seed", [(1024, 512, 1), (7, 3, 0), (1000, 33, 2**63 + 5)])
def test_gen_a_matches_oracle(C, n, seed):
    prm = pir.params(16, C, n, seed=seed)
    A = torch.empty(C * n, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_gen_a(prm, A)
    torch.cuda.synchronize()
    assert np.array_equal(pir.as_u32(A).reshape(C, n), oracle.gen_a(seed, C, n))


# ------------------------------------------------------------------ single-query Response
@pytest.mark.parametrize("R,C", [
    (1024, 1024),      # tiny workload
    (1, 16),           # one row, one 16-digit group
    (7, 272),          # rows < box, ragged last chunk
    (1000, 1008),      # ragged rows (not /8) and columns (not /256)
    (2053, 4096),      # more octets than SMs: several per CTA
    (4100, 512),       # several spans per CTA band
    (777, 1000),       # C % 16 != 0 -> generic kernel
    (33, 5),           # tiny ragged generic
])
def test_answer_single(R, C):
    prm, D, db = _setup(R, C, seed=R + C)
    q = inputs.uniform_u32(C, seed=R * C, tag=inputs.TAG_MISC)
    got = _answers(db, q[None, :])
    assert np.array_equal(got[0], oracle.answer(D, q))


@pytest.mark.parametrize("chunk", [512, 1024, 2048, 4096])
@pytest.mark.parametrize("R,C", [
    (1000, 1008), (153, 4096 + 16), (2, 9000 - 8),     # C % 256 != 0: per-row bulk copies
    (640, 512), (1000, 4096), (157, 2304), (9, 33024),  # 3-D boxes, remainder rows, partial last chunk
    (300, 2048 + 48), (17, 4096 + 4080),                 # partial last chunk by row copies
])
def test_answer_single_every_chunk_width(R, C, chunk):
    prm, D, db = _setup(R, C, seed=chunk + R)
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_STREAM_CHUNK, chunk)
    assert pir.qpadl_pir_get_option(db, pir.QPADL_OPT_STREAM_CHUNK) == chunk
    q = inputs.uniform_u32(C, seed=chunk, tag=inputs.TAG_MISC)
    exp = oracle.answer(D, q)
    for raw in (0, 1):
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_STREAM_RAW, raw)
        assert np.array_equal(_answers(db, q[None, :])[0], exp), f"raw={raw}"


@pytest.mark.parametrize("chunk", [1024, 2048, 4096])
@pytest.mark.parametrize("R,C", [
    (1000, 1008), (153, 4096 + 16), (2, 9000 - 8),     # per-row bulk copies
    (640, 512), (1000, 4096), (9, 33024),               # 3-D boxes, remainder rows, partial last chunk
    (300, 2048 + 48), (17, 4096 + 4080),
])
def test_answer_two_queries_one_pass(R, C, chunk):
    # two queries: one streaming pass with both packed in-kernel (raw = 1), or the pack launch first
    prm, D, db = _setup(R, C, seed=chunk + 3 * R)
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_STREAM_CHUNK, chunk)
    Q = inputs.uniform_u32(2 * C, seed=chunk + C, tag=inputs.TAG_MISC).reshape(2, C)
    exp = oracle.answer_batch(D, Q)
    for raw in (0, 1):
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_STREAM_RAW, raw)
        assert np.array_equal(_answers(db, Q, path=0), exp), f"raw={raw}"
    # the largest limb magnitudes in both queries
    Dx = np.full((R, C), 255, dtype=np.uint8)
    prm, Dx, dbx = _setup(R, C, D=Dx)
    pir.qpadl_pir_set_option(dbx, pir.QPADL_OPT_STREAM_RAW, 1)
    Qx = np.stack([np.full(C, 0x7F7F7F80, dtype=np.uint32), np.full(C, 0xFFFFFFFF, dtype=np.uint32)])
    assert np.array_equal(_answers(dbx, Qx, path=0), oracle.answer_batch(Dx, Qx))


def test_options_reject_bad_values():
    prm, D, db = _setup(64, 64, seed=1)
    for opt, val in ((pir.QPADL_OPT_STREAM_CHUNK, 256), (pir.QPADL_OPT_STREAM_CHUNK, 3000),
                     (pir.QPADL_OPT_TENSOR_MIN_BATCH, 0), (99, 1)):
        with pytest.raises(pir.QpadlError):
            pir.qpadl_pir_set_option(db, opt, val)


def test_answer_single_many_rows_per_cta():
    # 40000 rows on a 152-SM grid gives each CTA > 256 rows, i.e. several spans
    R, C = 40000, 256
    prm, D, db = _setup(R, C, seed=5)
    q = inputs.uniform_u32(C, seed=6, tag=inputs.TAG_MISC)
    assert np.array_equal(_answers(db, q[None, :])[0], oracle.answer(D, q, threads=oracle.max_threads()))


def test_answer_extreme_values():
    # all digits 255 against the query words that give the largest limb magnitudes
    R, C = 256, 2048
    D = np.full((R, C), 255, dtype=np.uint8)
    prm, D, db = _setup(R, C, D=D)
    for word in (0x7F7F7F80, 0x7F7F7F7F, 0xFFFFFFFF, 0x80808080, 0x80000000):
        q = np.full(C, word, dtype=np.uint32)
        exp = np.full(R, (255 * C * word) & M32, dtype=np.uint32)
        for path in (None, 0, 1):
            got = _answers(db, np.stack([q, q, q]) if path is not None else q[None, :], path=path)
            for b in range(got.shape[0]):
                assert np.array_equal(got[b], exp), (hex(word), path)


def test_answer_unit_queries_select_columns():
    R, C = 300, 1024
    prm, D, db = _setup(R, C, seed=9)
    cols = [0, 1, 255, 256, 1023]
    Q = np.zeros((len(cols), C), dtype=np.uint32)
    for b, c in enumerate(cols):
        Q[b, c] = 1 << 24
    for path in (0, 1):
        got = _answers(db, Q, path=path)
        for b, c in enumerate(cols):
            assert np.array_equal(got[b], (D[:, c].astype(np.uint64) << np.uint64(24)).astype(np.uint32))


# ------------------------------------------------------------------ batched Response
@pytest.mark.parametrize("B", [1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 32, 33, 64, 65, 100])
def test_answer_batch_both_paths(B):
    R, C = 300, 1000 + 8   # ragged rows vs 128-row tile, columns vs 64/256/512
    prm, D, db = _setup(R, C, seed=B)
    Q = inputs.uniform_u32(B * C, seed=B + 100, tag=inputs.TAG_MISC).reshape(B, C)
    exp = oracle.answer_batch(D, Q)
    for path in (0, 1):
        assert np.array_equal(_answers(db, Q, path=path), exp), f"path {path}"
    assert np.array_equal(_answers(db, Q), exp)


@pytest.mark.parametrize("R,C,B", [(129, 1537, 40), (128, 64, 3), (1, 8, 5), (513, 4100, 70), (1024, 1024, 256),
                                   (64, 256, 4096 + 300)])   # the last one crosses the 4096-query chunk
def test_answer_batch_tensor_ragged(R, C, B):
    prm, D, db = _setup(R, C, seed=R)
    Q = inputs.uniform_u32(B * C, seed=C, tag=inputs.TAG_MISC).reshape(B, C)
    assert np.array_equal(_answers(db, Q, path=1), oracle.answer_batch(D, Q, threads=oracle.max_threads()))


@pytest.mark.parametrize("R,C", [(300, 1008), (129, 4096 + 16), (1000, 2048)])
@pytest.mark.parametrize("B", [1, 3, 8, 17, 32])
def test_answer_batch_u8_and_fp16_gemms_agree_with_oracle(R, C, B):
    # B <= 32 runs the GEMM on the uint8 digits by default; 0 forces the fp16-copy GEMM
    prm, D, db = _setup(R, C, seed=R + B)
    Q = inputs.uniform_u32(B * C, seed=C + B, tag=inputs.TAG_MISC).reshape(B, C)
    exp = oracle.answer_batch(D, Q, threads=oracle.max_threads())
    for u8max, kstep, pair in ((32, 0, 1), (32, 0, 0), (32, 128, 1), (32, 256, 1), (0, 0, 1), (0, 0, 0)):
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_U8_MAX_BATCH, u8max)
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_U8_KSTEP, kstep)
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_PAIR_GEMM, pair)
        assert np.array_equal(_answers(db, Q, path=1), exp), f"u8 max batch {u8max}, k-step {kstep}, pair {pair}"


@pytest.mark.parametrize("B,kstep", [(8, 0), (8, 128), (16, 0), (16, 128), (32, 0), (32, 256), (40, 0)])
def test_answer_batch_many_tiles_per_cta(B, kstep):
    # 48000 rows make 375 row tiles, so every persistent CTA walks several tiles
    # and the stage rings wrap many times
    R, C = 48000, 1024
    prm, D, db = _setup(R, C, seed=B + 7)
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_U8_KSTEP, kstep)
    Q = inputs.uniform_u32(B * C, seed=B, tag=inputs.TAG_MISC).reshape(B, C)
    exp = oracle.answer_batch(D, Q, threads=oracle.max_threads())
    for pair in (1, 0):
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_PAIR_GEMM, pair)
        assert np.array_equal(_answers(db, Q, path=1), exp), f"pair {pair}"


@pytest.mark.parametrize("R,C,B", [(40000, 2100, 70), (20000, 1100, 64), (128, 600, 1024)])
def test_answer_batch_split_tiles(R, C, B):
    # the fp16-copy GEMM deals whole tiles round-robin and splits the last waves' tiles over
    # all SMs (pieces add into a zeroed output): 626 tiles of 5 chunks (the last one 64 deep),
    # 157 tiles of 3 chunks, and 16 tiles of 2 chunks spread over more SMs than tiles
    prm, D, db = _setup(R, C, seed=R + C)
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_PAIR_GEMM, 0)   # the single-SM tiles split their last waves
    Q = inputs.uniform_u32(B * C, seed=B + 5, tag=inputs.TAG_MISC).reshape(B, C)
    got = _answers(db, Q, path=1)
    assert np.array_equal(got, oracle.answer_batch(D, Q, threads=oracle.max_threads()))


@pytest.mark.parametrize("R,C,B", [
    (300, 1000 + 8, 33),     # one pair tile row: the peer's rows partly past R; ragged K
    (257, 640, 64),          # a second pair row of one matrix row
    (1000, 2048, 100),       # ragged vector tile (400 of 512 limb rows)
    (4099, 1536, 200),       # many pair tiles, ragged in rows and vectors
    (128, 64, 40),           # the peer holds no rows at all; K below one k-step
    (20000, 1100, 300),      # several tiles per CTA pair, rings wrapping
    (20000, 2048 + 8, 100),  # two vector tiles per row tile: a whole wave, then a split tail (ragged K)
    (20000, 1100, 160),      # three vector tiles per row tile (the last half full): whole waves, split tail
    (1000, 2048, 256),       # four vector tiles per row tile, tiles filling few clusters: all split
    (600, 512, 17),          # 68 limb columns: 128-wide pair tiles (u8 GEMM off)
    (600, 512, 9),           # 36 limb columns: 64-wide pair tiles (u8 GEMM off)
])
def test_answer_batch_pair_and_single_sm_gemms(R, C, B):
    # the fp16-copy GEMM on tiles of 256 rows over pairs of SMs and on 128-row tiles of one SM
    prm, D, db = _setup(R, C, seed=R + 3 * B)
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_U8_MAX_BATCH, 0)
    Q = inputs.uniform_u32(B * C, seed=C + 7 * B, tag=inputs.TAG_MISC).reshape(B, C)
    exp = oracle.answer_batch(D, Q, threads=oracle.max_threads())
    for pair in (1, 0):
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_PAIR_GEMM, pair)
        assert pir.qpadl_pir_get_option(db, pir.QPADL_OPT_PAIR_GEMM) == pair
        assert np.array_equal(_answers(db, Q, path=1), exp), f"pair {pair}"


@pytest.mark.parametrize("R,C,B", [
    (300, 1000 + 8, 33),     # two vector tiles; the peer's rows partly past R
    (1000, 2048, 100),       # four vector tiles, the last ragged
    (4099, 1536, 200),       # round-robin whole tiles, then a split tail
    (20000, 1100, 300),      # many tiles per CTA: several round-robin waves
    (128, 64, 40),           # the peer holds no rows; K below one stage
    (640, 512, 4096 + 40),   # crosses the 4096-query chunk of the limb scratch
])
def test_answer_batch_u8_gemm_large_batches(R, C, B):
    # the uint8-digit GEMM for batches above 32 (tiles of 128 limb columns, several per row tile)
    prm, D, db = _setup(R, C, seed=R + 5 * B)
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_U8_MAX_BATCH, 1 << 20)
    Q = inputs.uniform_u32(B * C, seed=C + 11 * B, tag=inputs.TAG_MISC).reshape(B, C)
    exp = oracle.answer_batch(D, Q, threads=oracle.max_threads())
    for pair in (1, 0):
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_PAIR_GEMM, pair)
        assert np.array_equal(_answers(db, Q, path=1), exp), f"pair {pair}"


def test_answer_batch_pair_gemm_extreme_values():
    # every digit 255 against limb-extreme query words: each 512-deep chunk at its exactness bound
    R, C, B = 512, 2048, 64
    D = np.full((R, C), 255, dtype=np.uint8)
    prm, D, db = _setup(R, C, D=D)
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_PAIR_GEMM, 1)
    words = np.array([0x7F7F7F80, 0x7F7F7F7F, 0xFFFFFFFF, 0x80808080], dtype=np.uint32)
    Q = np.repeat(words, B // 4)[:, None].repeat(C, axis=1)
    exp = ((255 * C * Q[:, 0].astype(np.uint64)) & M32).astype(np.uint32)
    got = _answers(db, Q, path=1)
    for b in range(B):
        assert np.all(got[b] == exp[b]), hex(int(Q[b, 0]))


@pytest.mark.parametrize("R,C,B", [(512, 2048, 16), (1000, 2048 + 128, 40), (3000, 1024, 32)])
def test_answer_batch_u8_gemm_extreme_values(R, C, B):
    # the uint8-digit GEMM holds digits as fp16 subnormals (d * 2^-24): every digit 255 against
    # limb-extreme words puts each 512-deep chunk at its exactness bound, on tiles split between
    # CTAs (the answers start at -1: the zeroing before the split tiles' adds is part of the call)
    D = np.full((R, C), 255, dtype=np.uint8)
    prm, D, db = _setup(R, C, D=D)
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_U8_MAX_BATCH, 1 << 20)
    words = np.array([0x7F7F7F80, 0x7F7F7F7F, 0xFFFFFFFF, 0x80808080], dtype=np.uint32)
    Q = np.resize(words, B)[:, None].repeat(C, axis=1)
    exp = ((255 * C * Q[:, 0].astype(np.uint64)) & M32).astype(np.uint32)
    for pair in (1, 0):
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_PAIR_GEMM, pair)
        got = _answers(db, Q, path=1)
        for b in range(B):
            assert np.all(got[b] == exp[b]), (pair, hex(int(Q[b, 0])))


def test_answer_batch_linearity_on_device():
    R, C, B = 256, 2048, 8
    prm, D, db = _setup(R, C, seed=3)
    Q1 = inputs.uniform_u32(B * C, seed=1, tag=inputs.TAG_MISC).reshape(B, C)
    Q2 = inputs.uniform_u32(B * C, seed=2, tag=inputs.TAG_MISC).reshape(B, C)
    with np.errstate(over="ignore"):
        lhs = _answers(db, (Q1 + Q2).astype(np.uint32), path=1)
        rhs = (_answers(db, Q1, path=1) + _answers(db, Q2, path=1)).astype(np.uint32)
    assert np.array_equal(lhs, rhs)


def test_small_plaintext_modulus_and_digit_check():
    R, C = 64, 512
    D = inputs.db_digits(R, C, 16, seed=4)
    prm, D, db = _setup(R, C, p=16, D=D)
    q = inputs.uniform_u32(C, seed=5, tag=inputs.TAG_MISC)
    assert np.array_equal(_answers(db, q[None, :])[0], oracle.answer(D, q))
    bad = D.copy()
    bad[3, 7] = 16
    with pytest.raises(pir.QpadlError) as ei:
        _setup(R, C, p=16, D=bad)
    assert ei.value.code == pir.QPADL_EINVAL


# ------------------------------------------------------------------ Hint
@pytest.mark.parametrize("R,C,n", [(1024, 1024, 512), (100, 1000, 17), (129, 520, 1), (300, 64, 70),
                                   (40000, 700, 64)])   # 313 row tiles: whole waves, then a split last wave
@pytest.mark.parametrize("pair", [1, 0])
def test_hint_matches_oracle(R, C, n, pair):
    prm, D, db = _setup(R, C, n=n, seed=n)
    pir.qpadl_pir_set_option(db, pir.QPADL_OPT_PAIR_GEMM, pair)
    A = torch.empty(C * n, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_gen_a(prm, A)
    H = torch.full((R * n,), -1, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_hint(db, A, H)
    torch.cuda.synchronize()
    assert pir.qpadl_pir_status(db) == 0
    exp = oracle.hint(D, oracle.gen_a(n, C, n), threads=oracle.max_threads())
    assert np.array_equal(pir.as_u32(H).reshape(R, n), exp)


# ------------------------------------------------------------------ Query / Recover
@pytest.mark.parametrize("C,n", [(1024, 512), (1000, 33), (64, 1)])
def test_query_single_and_batch(C, n):
    prm = pir.params(8, C, n, seed=C)
    A = torch.empty(C * n, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_gen_a(prm, A)
    A_o = oracle.gen_a(C, C, n)
    B = 19
    S_o = inputs.secrets(B, n, seed=1)
    E_o = inputs.noise_batch(B, C, seed=2)
    cols = inputs.target_columns(B, C, seed=3)
    q = torch.empty(C, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_query(prm, A, pir.from_u32(S_o[0]), torch.from_numpy(E_o[0]).cuda(), int(cols[0]), q)
    Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_query_batch(prm, A, pir.from_u32(S_o.reshape(-1)), torch.from_numpy(E_o.reshape(-1)).cuda(),
                              torch.from_numpy(cols.astype(np.int32)).cuda(), Q)
    torch.cuda.synchronize()
    exp = np.stack([oracle.query(A_o, S_o[b], E_o[b], int(cols[b]), 1 << 24) for b in range(B)])
    assert np.array_equal(pir.as_u32(q), exp[0])
    assert np.array_equal(pir.as_u32(Q).reshape(B, C), exp)


@pytest.mark.parametrize("C,n", [(1000, 128), (777, 132), (4096, 1024), (1, 256), (300, 4000), (9000, 512),
                                 (5000, 2048), (4867, 1024), (80000, 1024), (80001, 2048)])
def test_query_and_recover_matvec_shapes(C, n):
    # n in {512, 1024, 2048} with enough rows takes the register-resident kernel; others the generic one.
    # The last two give each warp of the register kernel more than one run of 32 rows (one or two
    # resident blocks of 8 warps per SM): the runs' gathered epilogue inputs and ragged last run.
    prm = pir.params(C, C, n, seed=n + C)
    A = torch.empty(C * n, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_gen_a(prm, A)
    A_o = oracle.gen_a(n + C, C, n)
    s_o = inputs.secrets(1, n, seed=C)[0]
    e_o = inputs.noise(C, seed=n)
    col = C // 3
    q = torch.empty(C, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_query(prm, A, pir.from_u32(s_o), torch.from_numpy(e_o).cuda(), col, q)
    torch.cuda.synchronize()
    assert np.array_equal(pir.as_u32(q), oracle.query(A_o, s_o, e_o, col, 1 << 24))
    # Recover over H = A (any R x n matrix) with arbitrary answers
    ans_o = inputs.uniform_u32(C, seed=3, tag=inputs.TAG_MISC)
    out = torch.empty(C, dtype=torch.uint8, device="cuda")
    pir.qpadl_pir_recover(prm, pir.from_u32(ans_o), A, pir.from_u32(s_o), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.recover(ans_o, A_o, s_o))
    assert pir.qpadl_pir_client_status() == pir.QPADL_OK


@pytest.mark.parametrize("p", [256, 16, 2])
def test_roundtrip_recover_every_column(p):
    R, C, n = 200, 96, 64
    prm, D, db = _setup(R, C, n=n, p=p, seed=p)
    A = torch.empty(C * n, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_gen_a(prm, A)
    H = torch.empty(R * n, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_hint(db, A, H)
    B = C
    S = pir.from_u32(inputs.secrets(B, n, seed=7).reshape(-1))
    E = torch.from_numpy(inputs.noise_batch(B, C, seed=8).reshape(-1)).cuda()
    cols = torch.arange(C, dtype=torch.int32, device="cuda")
    Q = torch.empty(B * C, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_query_batch(prm, A, S, E, cols, Q)
    ans = torch.empty(B * R, dtype=torch.int32, device="cuda")
    pir.qpadl_pir_answer_batch(db, Q, ans)
    out = torch.empty(B * R, dtype=torch.uint8, device="cuda")
    pir.qpadl_pir_recover_batch(prm, ans, H, S, out)
    out1 = torch.empty(R, dtype=torch.uint8, device="cuda")
    pir.qpadl_pir_recover(prm, ans[:R], H, S[:n], out1)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(B, R)
    assert np.array_equal(got, D.T)
    assert np.array_equal(out1.cpu().numpy(), D[:, 0])


def test_host_buffer_answer():
    R, C = 512, 1024
    prm, D, db = _setup(R, C, seed=12)
    q = inputs.uniform_u32(C, seed=13, tag=inputs.TAG_MISC)
    qh = torch.from_numpy(q.view(np.int32)).pin_memory()
    ah = torch.empty(R, dtype=torch.int32).pin_memory()
    pir.qpadl_pir_answer_host(db, qh, ah)
    assert np.array_equal(ah.numpy().view(np.uint32), oracle.answer(D, q))


def test_tensor_copy_at_setup_and_device_bytes():
    R, C = 256, 512
    prm, D, db = _setup(R, C, seed=14, flags=pir.QPADL_SETUP_TENSOR_COPY)
    assert pir.qpadl_pir_device_bytes(db) >= R * C * 2
    Q = inputs.uniform_u32(4 * C, seed=15, tag=inputs.TAG_MISC).reshape(4, C)
    assert np.array_equal(_answers(db, Q, path=1), oracle.answer_batch(D, Q))
