"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each step of the scheme is checked against something the mathematics or a
published source fixes: published SplitMix64 outputs, exact integer matrix
products from numpy's own int64 routines (no overflow at these sizes), Python
big-integer brute force, closed forms of special queries, linearity, and the
end-to-end identity Recover(Answer(Query(col))) = column col of D.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2510_03631_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M32 = (1 << 32) - 1


def _exact_matmul_mod32(D: np.ndarray, X: np.ndarray) -> np.ndarray:
    """D (uint8) times X (uint32) mod 2^32 via numpy int64 products.

    255 * (2^32 - 1) * C < 2^63 for C < 8.4e6, so the int64 result is exact.
    """
    assert D.shape[1] < 8_000_000
    return ((D.astype(np.int64) @ X.astype(np.int64)) & M32).astype(np.uint32)


def _exact_u32_matvec(A: np.ndarray, s: np.ndarray) -> np.ndarray:
    """A (uint32) times s (uint32) mod 2^32, exact via 16-bit halves of s."""
    A64 = A.astype(np.int64)
    lo = (s & 0xFFFF).astype(np.int64)
    hi = (s >> 16).astype(np.int64)
    # each product < 2^48; n < 2^15 keeps the sums below 2^63
    assert A.shape[1] < (1 << 15)
    r = (A64 @ lo) & M32
    r = (r + (((A64 @ hi) & M32) << 16)) & M32
    return r.astype(np.uint32)


# ---------------------------------------------------------------- Setup / PRG

def test_splitmix64_published_vectors():
    path = os.path.join(GOLDEN, "splitmix64.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 6
    for seed, idx, hexval in rows:
        assert oracle.splitmix64(int(seed), int(idx)) == int(hexval, 16)


def test_gen_a_layout_and_word():
    # A[j][k] is the upper half of output number j*n + k (row-major counter)
    A = oracle.gen_a(0, 3, 1)
    assert [int(x) for x in A[:, 0]] == [0xE220A839, 0x6E789E6A, 0x06C45D18]
    A2 = oracle.gen_a(0, 1, 3)
    assert [int(x) for x in A2[0]] == [0xE220A839, 0x6E789E6A, 0x06C45D18]
    A3 = oracle.gen_a(1234567, 2, 2)
    assert int(A3[0, 1]) == 0x2C73F084 and int(A3[1, 0]) == 0x883EBCE5


def test_gen_a_is_uniform_looking():
    A = oracle.gen_a(7, 256, 64)
    bits = np.unpackbits(A.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.01


# ---------------------------------------------------------------- Hint

@pytest.mark.parametrize("R,C,n", [(7, 13, 5), (64, 200, 33), (128, 1000, 17)])
def test_hint_equals_exact_int64_product(R, C, n):
    D = inputs.db_digits(R, C, 256, seed=R + C)
    A = inputs.public_matrix(C, n, seed=n)
    assert np.array_equal(oracle.hint(D, A), _exact_matmul_mod32(D, A))


def test_hint_identity_public_matrix_returns_db():
    C = 48
    D = inputs.db_digits(20, C, 256, seed=3)
    eye = np.eye(C, dtype=np.uint32)
    assert np.array_equal(oracle.hint(D, eye), D.astype(np.uint32))


def test_hint_linearity():
    D = inputs.db_digits(33, 70, 256, seed=4)
    A1 = inputs.public_matrix(70, 9, seed=10)
    A2 = inputs.public_matrix(70, 9, seed=11)
    with np.errstate(over="ignore"):
        lhs = oracle.hint(D, (A1 + A2).astype(np.uint32))
        rhs = (oracle.hint(D, A1) + oracle.hint(D, A2)).astype(np.uint32)
    assert np.array_equal(lhs, rhs)


def test_hint_threads_match_single_thread():
    D = inputs.db_digits(97, 120, 256, seed=5)
    A = inputs.public_matrix(120, 11, seed=6)
    assert np.array_equal(oracle.hint(D, A, threads=1), oracle.hint(D, A, threads=4))


# ---------------------------------------------------------------- Query

def test_query_bigint_bruteforce():
    C, n = 37, 11
    A = inputs.public_matrix(C, n, seed=21)
    s = inputs.secrets(1, n, seed=22)[0]
    e = inputs.noise(C, seed=23)
    col, delta = 5, 1 << 24
    got = oracle.query(A, s, e, col, delta)
    for j in range(C):
        v = sum(int(A[j, k]) * int(s[k]) for k in range(n)) + int(e[j])
        if j == col:
            v += delta
        assert int(got[j]) == v % (1 << 32), j


def test_query_exact_matvec_and_terms():
    C, n = 500, 64
    A = inputs.public_matrix(C, n, seed=31)
    s = inputs.secrets(1, n, seed=32)[0]
    e = inputs.noise(C, seed=33)
    col, delta = 123, 1 << 24
    got = oracle.query(A, s, e, col, delta).astype(np.int64)
    exp = _exact_u32_matvec(A, s).astype(np.int64) + e.astype(np.int64)
    exp[col] += delta
    assert np.array_equal(got, exp & M32)


def test_query_zero_secret_and_noise_is_scaled_unit_vector():
    C, n = 40, 8
    A = inputs.public_matrix(C, n, seed=41)
    qu = oracle.query(A, np.zeros(n, np.uint32), np.zeros(C, np.int32), 17, 1 << 24)
    exp = np.zeros(C, np.uint32)
    exp[17] = 1 << 24
    assert np.array_equal(qu, exp)


# ---------------------------------------------------------------- Answer

@pytest.mark.parametrize("R,C", [(1, 1), (5, 3), (64, 257), (300, 1000)])
def test_answer_equals_exact_int64_product(R, C):
    D = inputs.db_digits(R, C, 256, seed=R * 7 + C)
    qu = inputs.uniform_u32(C, seed=C, tag=inputs.TAG_MISC)
    assert np.array_equal(oracle.answer(D, qu), _exact_matmul_mod32(D, qu[:, None])[:, 0])


def test_answer_hand_worked_instance():
    # D = [[1, 2, 3], [255, 0, 7]], qu = [2^31, 3, 2^32 - 1]
    # row 0: 2^31 + 6 + 3*(2^32-1) = 2^31 + 3 + 3*2^32  -> 2^31 + 3
    # row 1: 255*2^31 + 0 + 7*(2^32-1) = 127*2^32 + 2^31 + 7*2^32 - 7 -> 2^31 - 7
    D = np.array([[1, 2, 3], [255, 0, 7]], dtype=np.uint8)
    qu = np.array([1 << 31, 3, M32], dtype=np.uint32)
    assert [int(x) for x in oracle.answer(D, qu)] == [(1 << 31) + 3, (1 << 31) - 7]


def test_answer_unit_query_selects_column():
    # qu = Delta * e_j  ->  ans = Delta * D[:, j]  (catches a transposed D)
    D = inputs.db_digits(50, 70, 256, seed=51)
    for j in (0, 13, 69):
        qu = np.zeros(70, np.uint32)
        qu[j] = 1 << 24
        exp = (D[:, j].astype(np.uint64) << np.uint64(24)) & np.uint64(M32)
        assert np.array_equal(oracle.answer(D, qu), exp.astype(np.uint32))


def test_answer_all_ones_is_row_sums_and_half_modulus_is_parity():
    D = inputs.db_digits(40, 333, 256, seed=52)
    rs = D.astype(np.int64).sum(axis=1)
    assert np.array_equal(oracle.answer(D, np.ones(333, np.uint32)), rs.astype(np.uint32))
    half = np.full(333, 1 << 31, np.uint32)
    assert np.array_equal(oracle.answer(D, half), ((rs % 2) << 31).astype(np.uint32))


def test_answer_linearity():
    D = inputs.db_digits(64, 300, 256, seed=53)
    q1 = inputs.uniform_u32(300, seed=1, tag=inputs.TAG_MISC)
    q2 = inputs.uniform_u32(300, seed=2, tag=inputs.TAG_MISC)
    with np.errstate(over="ignore"):
        lhs = oracle.answer(D, (q1 + q2).astype(np.uint32))
        rhs = (oracle.answer(D, q1) + oracle.answer(D, q2)).astype(np.uint32)
    assert np.array_equal(lhs, rhs)


def test_answer_batch_is_per_query():
    D = inputs.db_digits(30, 90, 256, seed=54)
    Q = inputs.uniform_u32(5 * 90, seed=3, tag=inputs.TAG_MISC).reshape(5, 90)
    got = oracle.answer_batch(D, Q, threads=2)
    for b in range(5):
        assert np.array_equal(got[b], _exact_matmul_mod32(D, Q[b][:, None])[:, 0])


# ---------------------------------------------------------------- Recover

def test_recover_rounding_closed_forms():
    # s = 0 removes the mask, so Recover is the rounding of ans alone:
    # Delta*d + t -> d for -Delta/2 <= t < Delta/2, ties round up, wrap mod p.
    R, n, delta = 8, 4, 1 << 24
    H = inputs.public_matrix(R, n, seed=61)
    s = np.zeros(n, np.uint32)
    d = np.array([0, 1, 17, 128, 254, 255, 255, 0], dtype=np.int64)
    t = np.array([0, delta // 2 - 1, -delta // 2, 5, -1, delta // 2 - 1, delta // 2, -3])
    ans = ((d * delta + t) & M32).astype(np.uint32)
    exp = np.array([0, 1, 17, 128, 254, 255, 0, 0], dtype=np.uint8)
    assert np.array_equal(oracle.recover(ans, H, s), exp)


def test_recover_strips_mask():
    R, n = 16, 6
    H = inputs.public_matrix(R, n, seed=62)
    s = inputs.secrets(1, n, seed=63)[0]
    digits = inputs.db_digits(1, R, 256, seed=64)[0].astype(np.int64)
    mask = _exact_u32_matvec(H, s).astype(np.int64)
    ans = ((digits << 24) + mask + 1000) & M32
    assert np.array_equal(oracle.recover(ans.astype(np.uint32), H, s), digits.astype(np.uint8))


@pytest.mark.parametrize("p", [2, 16, 256])
def test_recover_small_plaintext_moduli(p):
    R, n = 12, 3
    H = inputs.public_matrix(R, n, seed=65)
    s = np.zeros(n, np.uint32)
    delta = oracle.delta_for(p)
    d = np.arange(R) % p
    ans = ((d * delta - (delta // 2) + 1) & M32).astype(np.uint32)
    assert np.array_equal(oracle.recover(ans, H, s, p=p), d.astype(np.uint8))


# ---------------------------------------------------------------- end to end

def _roundtrip(R, C, n, p, seed, cols):
    D = inputs.db_digits(R, C, p, seed=seed)
    A = oracle.gen_a(seed, C, n)
    H = oracle.hint(D, A, threads=oracle.max_threads())
    delta = oracle.delta_for(p)
    S = inputs.secrets(len(cols), n, seed=seed + 1)
    E = inputs.noise_batch(len(cols), C, seed=seed + 2)
    Q = np.stack([oracle.query(A, S[b], E[b], int(c), delta) for b, c in enumerate(cols)])
    ans = oracle.answer_batch(D, Q, threads=oracle.max_threads())
    for b, c in enumerate(cols):
        got = oracle.recover(ans[b], H, S[b], p=p)
        assert np.array_equal(got, D[:, c]), f"column {c}"


def test_roundtrip_every_column_small():
    _roundtrip(64, 96, 32, 256, seed=70, cols=list(range(96)))


def test_roundtrip_small_modulus():
    _roundtrip(40, 50, 16, 16, seed=71, cols=list(range(0, 50, 7)))


def test_roundtrip_tiny_workload_sampled_columns():
    w = inputs.WORKLOADS["tiny"]
    cols = inputs.target_columns(24, w["cols"], seed=1).tolist() + [0, w["cols"] - 1]
    _roundtrip(w["rows"], w["cols"], w["n"], w["p"], seed=1, cols=cols)


def test_noise_margin_of_largest_database():
    # |D e| must stay below Delta/2 = 2^23 for exact recovery.  With uniform
    # digits and sigma = 6.4 the standard deviation of D e at C = 32768 is
    # sqrt(C * E[d^2]) * sigma; the bound holds with ~49 standard deviations.
    C, sigma = 32768, 6.4
    ed2 = np.mean(np.arange(256, dtype=np.float64) ** 2)
    sd = np.sqrt(C * ed2) * sigma
    assert (1 << 23) / sd > 45
    # and a sampled row of the real workload stays far inside
    D = inputs.db_digits(32768, C, 256, seed=1, row_start=1234, row_count=2).astype(np.int64)
    e = inputs.noise(C, seed=9).astype(np.int64)
    assert np.abs(D @ e).max() < (1 << 23) // 8


def test_noise_distribution():
    e = inputs.noise(200_000, seed=5)
    assert abs(e.mean()) < 0.1
    assert abs(e.std() - np.sqrt(6.4 ** 2 + 1 / 12)) < 0.1
    assert np.abs(e).max() <= 64


# ----------------------------------------------------------------------------- Chor over GF(2)
# Sec. 5.2 "Parallel Chor-PIR": rho = q . DB over GF(2), the XOR of the rows
# whose query bit is set; Sec. 7 (ENS): ell - 1 random queries plus their XOR
# with e_theta, and D_theta = XOR of the ell responses.

def _bits(words: np.ndarray, nbits: int) -> np.ndarray:
    """Unpack uint32 words (LSB first) into a 0/1 int64 array of nbits."""
    b = ((words[..., :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(*words.shape[:-1], -1)
    return b[..., :nbits].astype(np.int64)


def test_chor_hand_worked_example():
    # three 32-bit rows; query selects rows 0 and 2
    DB = np.array([[0x0000000F], [0x000000F0], [0x00000F0F]], dtype=np.uint32)
    Q = np.array([[0b101]], dtype=np.uint32)
    assert oracle.chor_answer(DB, 3, Q)[0, 0] == 0x0000000F ^ 0x00000F0F == 0x00000F00


def test_chor_brute_force_python_ints():
    rng = np.random.default_rng(11)
    r, w = 37, 3
    DB = rng.integers(0, 2**32, (r, w), dtype=np.uint64).astype(np.uint32)
    Q = rng.integers(0, 2**32, (5, 2), dtype=np.uint64).astype(np.uint32)
    Q[:, 1] &= (1 << (r - 32)) - 1
    got = oracle.chor_answer(DB, r, Q)
    rows = [sum(int(DB[i, c]) << (32 * c) for c in range(w)) for i in range(r)]
    for b in range(5):
        qint = int(Q[b, 0]) | (int(Q[b, 1]) << 32)
        acc = 0
        for i in range(r):
            if (qint >> i) & 1:
                acc ^= rows[i]
        assert sum(int(got[b, c]) << (32 * c) for c in range(w)) == acc


def test_chor_equals_integer_matmul_mod_2():
    # GF(2) product = integer product of the 0/1 matrices, reduced mod 2 (numpy matmul)
    r, bits = 300, 256
    DB = inputs.chor_db(r, bits, seed=5)
    Q = inputs.chor_queries(9, r, seed=6)
    got = oracle.chor_answer(DB, r, Q)
    exp = (_bits(Q, r) @ _bits(DB, bits)) % 2
    assert np.array_equal(_bits(got, bits), exp)


def test_chor_unit_queries_select_rows():
    r, bits = 70, 128
    DB = inputs.chor_db(r, bits, seed=7)
    Q = np.zeros((r, (r + 31) // 32), dtype=np.uint32)
    for t in range(r):
        Q[t, t // 32] = np.uint32(1 << (t % 32))
    assert np.array_equal(oracle.chor_answer(DB, r, Q), DB)


def test_chor_zero_all_ones_linearity_and_padding():
    r, bits = 45, 96
    DB = inputs.chor_db(r, bits, seed=8)
    qw = (r + 31) // 32
    zero = np.zeros((1, qw), dtype=np.uint32)
    assert not oracle.chor_answer(DB, r, zero).any()
    ones = np.full((1, qw), 0xFFFFFFFF, dtype=np.uint32)   # bits past r are ignored
    assert np.array_equal(oracle.chor_answer(DB, r, ones)[0], np.bitwise_xor.reduce(DB, axis=0))
    q1, q2 = inputs.chor_queries(1, r, seed=9), inputs.chor_queries(1, r, seed=10)
    a = oracle.chor_answer(DB, r, np.concatenate([q1, q2, q1 ^ q2]))
    assert np.array_equal(a[2], a[0] ^ a[1])
    garbage = q1.copy()
    garbage[0, -1] |= np.uint32(0xFFFFFFFF << (r % 32) & 0xFFFFFFFF)
    assert np.array_equal(oracle.chor_answer(DB, r, garbage), a[:1])


@pytest.mark.parametrize("ell", [2, 3, 5])
def test_chor_ens_protocol_recovers_the_record(ell):
    r, bits = 200, 160
    DB = inputs.chor_db(r, bits, seed=12)
    qw = (r + 31) // 32
    for theta in (0, 31, 32, 199):
        shares = inputs.chor_queries(ell - 1, r, seed=100 + theta)
        queries = oracle.chor_query(shares, theta)
        assert queries.shape == (ell, qw)
        # the last query differs from the XOR of the others in exactly bit theta
        diff = np.bitwise_xor.reduce(queries, axis=0)
        exp = np.zeros(qw, dtype=np.uint32)
        exp[theta // 32] = np.uint32(1 << (theta % 32))
        assert np.array_equal(diff, exp)
        responses = oracle.chor_answer(DB, r, queries)
        assert np.array_equal(oracle.chor_reconstruct(responses), DB[theta])


def test_chor_thread_count_invariance():
    r, bits = 513, 1024
    DB = inputs.chor_db(r, bits, seed=13)
    Q = inputs.chor_queries(16, r, seed=14)
    assert np.array_equal(oracle.chor_answer(DB, r, Q, threads=1), oracle.chor_answer(DB, r, Q, threads=4))


# ----------------------------------------------------------------------------- Goldberg over Z_p
# Sec. 5.2 "Parallel Goldberg-PIR": rho = q . DB over a field (here Z_p, p prime <= 257);
# Sec. 7 (FTR): Shamir shares f_j(alpha_k) of e_theta, Lagrange reconstruction at 0.

def test_goldberg_hand_worked_example():
    # two records (columns) of three bytes, p = 7: q = (2, 3) -> 2 * col0 + 3 * col1 mod 7
    D = np.array([[1, 4], [6, 6], [0, 5]], dtype=np.uint8)
    got = oracle.goldberg_answer(D, np.array([[2, 3]], dtype=np.uint32), 7)
    assert got.tolist() == [[(2 + 12) % 7, (12 + 18) % 7, 15 % 7]] == [[0, 2, 1]]


@pytest.mark.parametrize("p", [257, 251, 101, 2])
def test_goldberg_equals_integer_matmul_mod_p(p):
    R, C, B = 70, 130, 6
    D = (inputs.db_digits(R, C, 256, seed=p).astype(np.int64) % p).astype(np.uint8)
    Q = (inputs.uniform_u32(B * C, seed=p + 1, tag=inputs.TAG_MISC) % p).reshape(B, C)
    exp = (Q.astype(np.int64) @ D.T.astype(np.int64)) % p
    assert np.array_equal(oracle.goldberg_answer(D, Q, p), exp.astype(np.uint32))


def test_goldberg_brute_force_python_ints():
    p, R, C = 257, 5, 9
    rng = np.random.default_rng(3)
    D = rng.integers(0, 256, (R, C), dtype=np.uint8)
    q = rng.integers(0, p, C).astype(np.uint32)
    got = oracle.goldberg_answer(D, q[None, :], p)[0]
    for i in range(R):
        assert int(got[i]) == sum(int(q[j]) * int(D[i, j]) for j in range(C)) % p


def test_goldberg_unit_queries_linearity_and_ones():
    p, R, C = 257, 40, 33
    D = inputs.db_digits(R, C, 256, seed=9)
    E = np.eye(C, dtype=np.uint32)
    assert np.array_equal(oracle.goldberg_answer(D, E, p), D.T.astype(np.uint32))
    ones = np.ones((1, C), dtype=np.uint32)
    assert np.array_equal(oracle.goldberg_answer(D, ones, p)[0], (D.astype(np.int64).sum(axis=1) % p).astype(np.uint32))
    q1 = (inputs.uniform_u32(C, seed=1, tag=7) % p)[None, :]
    q2 = (inputs.uniform_u32(C, seed=2, tag=7) % p)[None, :]
    a = oracle.goldberg_answer(D, np.concatenate([q1, q2, (q1 + q2) % p]), p)
    assert np.array_equal(a[2], (a[0] + a[1]) % p)


@pytest.mark.parametrize("p,t,ell", [(257, 1, 2), (257, 2, 4), (251, 3, 5), (101, 2, 3)])
def test_goldberg_ftr_protocol_recovers_the_record(p, t, ell):
    R, C = 24, 50
    D = (inputs.db_digits(R, C, 256, seed=p + t).astype(np.int64) % p).astype(np.uint8)
    alpha = np.arange(1, ell + 1, dtype=np.uint32)
    for theta in (0, 17, C - 1):
        coef = (inputs.uniform_u32(C * t, seed=theta + 5, tag=7) % p).reshape(C, t)
        queries = oracle.goldberg_query(coef, theta, alpha, p)
        # query k evaluates every polynomial at alpha_k: f_j(0) = [j == theta] is hidden behind degree t
        x = np.zeros(C, dtype=np.int64)
        x[theta] = 1
        for k in range(ell):
            direct = x.copy()
            for u in range(1, t + 1):
                direct = (direct + coef[:, u - 1].astype(np.int64) * pow(int(alpha[k]), u, p)) % p
            assert np.array_equal(queries[k], direct.astype(np.uint32))
        responses = oracle.goldberg_answer(D, queries, p)
        # any t + 1 of the ell responses interpolate the record
        for sub in (list(range(t + 1)), list(range(ell - t - 1, ell))):
            rec = oracle.goldberg_reconstruct(responses[sub], alpha[sub], p)
            assert np.array_equal(rec, D[:, theta].astype(np.uint32))


# ---------------------------------------------------------------- database compression (Sec. 5.3)
def test_delta_hand_example():
    # entries 5, 7, 300, 301 in blocks of two: differences 2 and 1 fit one byte; each block is its
    # first entry in four little-endian bytes (300 = 1 * 256 + 44), then the difference
    x = np.array([5, 7, 300, 301], dtype=np.uint32)
    assert oracle.delta_width(x, 2) == 1
    db = oracle.delta_encode(x, 2, 1)
    assert db.shape == (5, 2)
    assert db[:, 0].tolist() == [5, 0, 0, 0, 2]
    assert db[:, 1].tolist() == [44, 1, 0, 0, 1]
    assert oracle.delta_decode(db[:, 1], 2, 1).tolist() == [300, 301]
    # a difference of exactly 256 needs a second byte; 255 does not
    assert oracle.delta_width(np.array([0, 256], dtype=np.uint32), 2) == 2
    assert oracle.delta_width(np.array([0, 255], dtype=np.uint32), 2) == 1


def _delta_brute(x, E, w):
    """Independent restatement in Python integers: padded blocks, first entry, differences."""
    n = len(x)
    C = (n + E - 1) // E
    pad = [int(v) for v in x] + [int(x[-1])] * (C * E - n)
    cols = []
    for j in range(C):
        blk = pad[j * E:(j + 1) * E]
        digits = [(blk[0] >> (8 * b)) & 255 for b in range(4)]
        for i in range(1, E):
            d = (blk[i] - blk[i - 1]) % (1 << 32)
            digits += [(d >> (8 * b)) & 255 for b in range(w)]
        cols.append(digits)
    return np.array(cols, dtype=np.uint8).T, pad


@pytest.mark.parametrize("n,E,gap", [(1000, 16, 40), (1000, 7, 300), (37, 5, 70000), (8, 1, 3), (5, 8, 9)])
def test_delta_round_trip_width_and_size(n, E, gap):
    rng = np.random.default_rng(n + E)
    x = np.cumsum(rng.integers(0, gap, n, dtype=np.uint64)).astype(np.uint32)   # sorted unless it wraps
    w = oracle.delta_width(x, E)
    C = (n + E - 1) // E
    _, pad = _delta_brute(x, E, 4)
    diffs = [(pad[j * E + i] - pad[j * E + i - 1]) % (1 << 32) for j in range(C) for i in range(1, E)]
    dmax = max(diffs) if diffs else 0
    assert dmax < 256 ** w and (w == 1 or dmax >= 256 ** (w - 1))   # the fewest bytes that hold them
    db = oracle.delta_encode(x, E, w)
    exp, pad = _delta_brute(x, E, w)
    assert db.shape == (4 + w * (E - 1), C)
    assert np.array_equal(db, exp)
    for j in range(C):
        assert oracle.delta_decode(db[:, j], E, w).tolist() == pad[j * E:(j + 1) * E]


def test_delta_unsorted_entries_wrap():
    # a decreasing pair stores its difference mod 2^32 (four bytes) and still decodes exactly
    x = np.array([10, 3, 2 ** 32 - 1, 0], dtype=np.uint32)
    w = oracle.delta_width(x, 4)
    assert w == 4
    assert oracle.delta_decode(oracle.delta_encode(x, 4, w)[:, 0], 4, w).tolist() == x.tolist()
