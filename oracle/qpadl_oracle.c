/*
 * CPU oracle for the LWE-style PIR of the QPADL spectrum-database query path
 * (arxiv 2510.03631).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the benchmark's CPU-baseline leg are the only code that may load it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Everything is exact integer arithmetic in Z_q with q = 2^32, i.e. uint32_t
 * with wraparound.  Each function is the plain definition, a loop nest in the
 * order the definition is written, with no blocking or reordering; the only
 * concession to speed is an optional OpenMP split over independent output
 * rows, which changes no arithmetic.
 *
 * What the paper fixes and what is read into it:
 *  - Def. 1 (Sec. 3, PIR): Query(theta) -> q ; Response(q) -> rho computed
 *    from the server's local database ; BlockReconst(rho) -> D_theta.
 *  - Sec. 5.2 ("Parallel Chor-PIR", "Parallel Goldberg-PIR", Alg. 3/4): the
 *    server's work is one product of the query with the whole database
 *    matrix, accumulated "mod q" (Alg. 4).
 *  - Sec. 5.3 (offline-online mode): query-independent work moves offline;
 *    here that is the hint H = D * A.
 *  - The lattice instantiation itself (public A, secret s, noise e, scale
 *    Delta = q / p, rounding in Recover) is the standard single-server LWE
 *    PIR; the paper states no formula for it, so the readings are:
 *      Setup   : A[j][k] = hi32(SplitMix64 output number j*n+k, state = seed)
 *      Hint    : H[i][k] = sum_j D[i][j] * A[j][k]                 (mod 2^32)
 *      Query   : qu[j]  = sum_k A[j][k]*s[k] + e[j] + Delta*[j == col]
 *      Answer  : ans[i] = sum_j D[i][j] * qu[j]                    (mod 2^32)
 *      Recover : x = ans[i] - sum_k H[i][k]*s[k];  d = floor((x + Delta/2) / Delta) mod p
 *    A record is a column of D; digits are unsigned in [0, p), p = 2^l.
 */
#include <stdint.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): state advances by the golden gamma, the output
 * is the state passed through the variant-13 finaliser.  Output number i
 * (0-based) from initial state `seed` therefore uses state seed + (i+1)*gamma. */
static uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Exposed so the tests can check the generator against its published vectors. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t i)
{
    return oracle_splitmix64_at(seed, i);
}

/* Setup: the public matrix A in Z_q^{C x n}, row-major, from its seed. */
void oracle_gen_a(uint64_t seed, uint64_t C, uint64_t n, uint32_t *A)
{
    for (uint64_t j = 0; j < C; ++j)
        for (uint64_t k = 0; k < n; ++k)
            A[j * n + k] = (uint32_t)(oracle_splitmix64_at(seed, j * n + k) >> 32);
}

static int oracle_threads(int nthreads)
{
    return nthreads > 0 ? nthreads : 1;
}

/* Hint (offline, Sec. 5.3): H = D * A over Z_q.  D: R x C, A: C x n, H: R x n. */
void oracle_hint(const uint8_t *D, uint64_t R, uint64_t C,
                 const uint32_t *A, uint64_t n, uint32_t *H, int nthreads)
{
    int nt = oracle_threads(nthreads);
    (void)nt;
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < (int64_t)R; ++i) {
        for (uint64_t k = 0; k < n; ++k) {
            uint32_t acc = 0;
            for (uint64_t j = 0; j < C; ++j)
                acc += (uint32_t)D[(uint64_t)i * C + j] * A[j * n + k];
            H[(uint64_t)i * n + k] = acc;
        }
    }
}

/* Query (Def. 1, Client.Query): qu = A*s + e + Delta * u_col over Z_q.
 * e is a signed integer reduced mod 2^32. */
void oracle_query(const uint32_t *A, uint64_t C, uint64_t n, const uint32_t *s,
                  const int32_t *e, uint64_t col, uint32_t delta, uint32_t *qu)
{
    for (uint64_t j = 0; j < C; ++j) {
        uint32_t acc = 0;
        for (uint64_t k = 0; k < n; ++k)
            acc += A[j * n + k] * s[k];
        acc += (uint32_t)e[j];
        if (j == col)
            acc += delta;
        qu[j] = acc;
    }
}

/* Answer (Def. 1, DB.Query.Response; Sec. 5.2 "rho <- q . DB", accumulated
 * mod q as in Alg. 4): ans = D * qu over Z_q, digits read unsigned. */
void oracle_answer(const uint8_t *D, uint64_t R, uint64_t C,
                   const uint32_t *qu, uint32_t *ans, int nthreads)
{
    int nt = oracle_threads(nthreads);
    (void)nt;
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < (int64_t)R; ++i) {
        uint32_t acc = 0;
        for (uint64_t j = 0; j < C; ++j)
            acc += (uint32_t)D[(uint64_t)i * C + j] * qu[j];
        ans[i] = acc;
    }
}

/* Batched answer (Alg. 4's batch of queries): each query answered on its own.
 * Q holds query b at Q[b*C .. b*C+C-1]; answer b goes to ans[b*R .. b*R+R-1]. */
void oracle_answer_batch(const uint8_t *D, uint64_t R, uint64_t C,
                         const uint32_t *Q, uint64_t B, uint32_t *ans, int nthreads)
{
    for (uint64_t b = 0; b < B; ++b)
        oracle_answer(D, R, C, Q + b * C, ans + b * R, nthreads);
}

/* Recover (Def. 1, Client.BlockReconst): strip the mask H*s, then round to
 * the nearest multiple of Delta = 2^32 / p and reduce mod p.  p = 2^l with
 * 1 <= l <= 8, so dividing by Delta is a right shift by 32 - l and the
 * "mod p" is implied by the 32-bit wrap. */
void oracle_recover(const uint32_t *ans, const uint32_t *H, uint64_t R, uint64_t n,
                    const uint32_t *s, uint32_t log2_p, uint8_t *out)
{
    uint32_t shift = 32u - log2_p;
    uint32_t half = 1u << (shift - 1u);
    for (uint64_t i = 0; i < R; ++i) {
        uint32_t mask = 0;
        for (uint64_t k = 0; k < n; ++k)
            mask += H[i * n + k] * s[k];
        uint32_t x = ans[i] - mask;
        out[i] = (uint8_t)((uint32_t)(x + half) >> shift);
    }
}

/* ---------------------------------------------------------------------------
 * Chor-style PIR over GF(2) (Sec. 5.2 "Parallel Chor-PIR", Alg. 3; the ENS
 * instantiation of Sec. 7).  The database is r rows of b bits, a record is a
 * row, and the server's response to an r-bit query q is rho = q . DB over
 * GF(2): the XOR of the rows whose query bit is set.
 * Packing (a reading; the paper fixes none): bit c of row i is bit c % 32 of
 * word db[i * w + c / 32] (w = b / 32 words per row); bit i of a query is bit
 * i % 32 of word q[i / 32] (qw = ceil(r / 32) words); query bits at positions
 * >= r are ignored.  Query b of a batch starts at q + b * qw, its response at
 * out + b * w.
 */
void oracle_chor_answer(const uint32_t *db, uint64_t r, uint64_t w, const uint32_t *q, uint64_t qw,
                        uint64_t B, uint32_t *out, int nthreads)
{
    int nt = oracle_threads(nthreads);
    (void)nt;
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t b = 0; b < (int64_t)B; ++b) {
        uint32_t *rho = out + (uint64_t)b * w;
        const uint32_t *qb = q + (uint64_t)b * qw;
        for (uint64_t c = 0; c < w; ++c)
            rho[c] = 0;
        for (uint64_t i = 0; i < r; ++i) {
            if ((qb[i / 32] >> (i % 32)) & 1u) {
                for (uint64_t c = 0; c < w; ++c)
                    rho[c] ^= db[i * w + c];
            }
        }
    }
}

/* Client query of the ENS instantiation (Sec. 7): given ell - 1 uniformly
 * random r-bit vectors, the last vector is their XOR with the unit vector
 * e_theta.  shares: (ell - 1) x qw words; queries: ell x qw words. */
void oracle_chor_query(const uint32_t *shares, uint64_t ell, uint64_t qw, uint64_t theta, uint32_t *queries)
{
    for (uint64_t k = 0; k < qw; ++k) {
        uint32_t acc = 0;
        for (uint64_t j = 0; j + 1 < ell; ++j) {
            queries[j * qw + k] = shares[j * qw + k];
            acc ^= shares[j * qw + k];
        }
        if (k == theta / 32)
            acc ^= 1u << (theta % 32);
        queries[(ell - 1) * qw + k] = acc;
    }
}

/* Reconstruction of the ENS instantiation (Sec. 7): D_theta = XOR of the ell
 * responses.  responses: ell x w words; out: w words. */
void oracle_chor_reconstruct(const uint32_t *responses, uint64_t ell, uint64_t w, uint32_t *out)
{
    for (uint64_t c = 0; c < w; ++c) {
        uint32_t acc = 0;
        for (uint64_t j = 0; j < ell; ++j)
            acc ^= responses[j * w + c];
        out[c] = acc;
    }
}

/* ---------------------------------------------------------------------------
 * Goldberg-style PIR over a prime field Z_p (Sec. 5.2 "Parallel Goldberg-PIR",
 * Alg. 4; the FTR instantiation of Sec. 7).  The paper names no field; the
 * reading here is a prime p <= 257, so that every byte of the database is a
 * field element when p = 257.  The database keeps the layout of the lattice
 * scheme (R x C bytes, record j = column j), a query is C field elements
 * and the response R field elements:
 *     rho[i] = sum_j q[j] * D[i][j]  mod p.
 * Query b of a batch is q + b * C, its response out + b * R. */
void oracle_goldberg_answer(const uint8_t *D, uint64_t R, uint64_t C, const uint32_t *q, uint64_t B,
                            uint32_t p, uint32_t *out, int nthreads)
{
    int nt = oracle_threads(nthreads);
    (void)nt;
    for (uint64_t b = 0; b < B; ++b) {
        const uint32_t *qb = q + b * C;
#pragma omp parallel for num_threads(nt) schedule(static)
        for (int64_t i = 0; i < (int64_t)R; ++i) {
            uint64_t acc = 0;
            for (uint64_t j = 0; j < C; ++j)
                acc = (acc + (uint64_t)qb[j] * D[(uint64_t)i * C + j]) % p;
            out[b * R + (uint64_t)i] = (uint32_t)acc;
        }
    }
}

static uint32_t oracle_pow_mod(uint32_t x, uint32_t e, uint32_t p)
{
    uint64_t r = 1, b = x % p;
    while (e) {
        if (e & 1u)
            r = r * b % p;
        b = b * b % p;
        e >>= 1;
    }
    return (uint32_t)r;
}

/* FTR client query (Sec. 7): record index j gets a degree-t polynomial
 * f_j(x) = [j == theta] + sum_{u=1..t} coef[j][u-1] x^u over Z_p, and server k
 * (evaluation point alpha[k], distinct and nonzero) receives
 * q_k[j] = f_j(alpha[k]).  coef: C x t (uniform in Z_p); queries: ell x C. */
void oracle_goldberg_query(const uint32_t *coef, uint64_t C, uint64_t t, uint64_t theta, const uint32_t *alpha,
                           uint64_t ell, uint32_t p, uint32_t *queries)
{
    for (uint64_t k = 0; k < ell; ++k) {
        for (uint64_t j = 0; j < C; ++j) {
            /* Horner from the highest coefficient down to the constant term */
            uint64_t v = 0;
            for (uint64_t u = t; u >= 1; --u)
                v = (v * alpha[k] + coef[j * t + (u - 1)]) % p;
            v = (v * alpha[k] + (j == theta ? 1u : 0u)) % p;
            queries[k * C + j] = (uint32_t)v;
        }
    }
}

/* Reconstruction (Sec. 5.1, FTR): Lagrange interpolation at 0 of the
 * responses of k servers, out[i] = sum_s lambda_s * R_s[i] mod p with
 * lambda_s = prod_{m != s} alpha_m / (alpha_m - alpha_s); p prime, so the
 * inverse is x^(p-2).  responses: k x R. */
void oracle_goldberg_reconstruct(const uint32_t *responses, const uint32_t *alpha, uint64_t k, uint64_t R,
                                 uint32_t p, uint32_t *out)
{
    for (uint64_t i = 0; i < R; ++i)
        out[i] = 0;
    for (uint64_t s = 0; s < k; ++s) {
        uint64_t num = 1, den = 1;
        for (uint64_t m = 0; m < k; ++m) {
            if (m == s)
                continue;
            num = num * alpha[m] % p;
            den = den * ((alpha[m] + p - alpha[s]) % p) % p;
        }
        const uint64_t lambda = num * oracle_pow_mod((uint32_t)den, p - 2, p) % p;
        for (uint64_t i = 0; i < R; ++i)
            out[i] = (uint32_t)((out[i] + lambda * responses[s * R + i]) % p);
    }
}

/* ---------------------------------------------------------------------
 * Database compression (Sec. 5.3, "Database Compression Techniques"): the
 * DB entries are sorted and each is stored as its difference from the entry
 * before it, so that close entries take fewer bits.  Reading taken here: the
 * entries are 32-bit unsigned integers x_0 <= x_1 <= ... <= x_{N-1}; block j
 * (one PIR record, a column of the database) holds entries jE .. jE + E - 1,
 * positions past N - 1 repeating x_{N-1}; a block is stored as the first
 * entry in full (4 little-endian bytes) followed by the E - 1 differences
 * x_{jE+i} - x_{jE+i-1} (mod 2^32), each in w little-endian bytes, w the
 * fewest bytes that hold every such difference in the database.  A block is
 * therefore R' = 4 + w (E - 1) digits and decodes on its own by prefix sums.
 * ------------------------------------------------------------------- */

/* Entry k of the padded sequence (positions past n - 1 repeat the last entry). */
static uint32_t oracle_entry(const uint32_t *x, uint64_t n, uint64_t k)
{
    return k < n ? x[k] : x[n - 1];
}

/* The byte width w in 1..4 of the largest within-block difference. */
uint32_t oracle_delta_width(const uint32_t *x, uint64_t n, uint64_t E)
{
    uint32_t dmax = 0;
    const uint64_t blocks = (n + E - 1) / E;
    for (uint64_t j = 0; j < blocks; ++j)
        for (uint64_t i = 1; i < E; ++i) {
            const uint32_t d = oracle_entry(x, n, j * E + i) - oracle_entry(x, n, j * E + i - 1);
            if (d > dmax)
                dmax = d;
        }
    uint32_t w = 1;
    while (w < 4 && dmax >= (1u << (8 * w)))
        ++w;
    return w;
}

/* Compressed database: R' x C digits, row-major (digit k of block j at k * C + j). */
void oracle_delta_encode(const uint32_t *x, uint64_t n, uint64_t E, uint32_t w, uint8_t *db)
{
    const uint64_t C = (n + E - 1) / E;
    for (uint64_t j = 0; j < C; ++j) {
        const uint32_t first = oracle_entry(x, n, j * E);
        for (uint32_t b = 0; b < 4; ++b)
            db[b * C + j] = (uint8_t)(first >> (8 * b));
        for (uint64_t i = 1; i < E; ++i) {
            const uint32_t d = oracle_entry(x, n, j * E + i) - oracle_entry(x, n, j * E + i - 1);
            for (uint32_t b = 0; b < w; ++b)
                db[(4 + (i - 1) * w + b) * C + j] = (uint8_t)(d >> (8 * b));
        }
    }
}

/* One block's E entries from its R' digits (prefix sums of the differences, mod 2^32). */
void oracle_delta_decode(const uint8_t *digits, uint64_t E, uint32_t w, uint32_t *out)
{
    uint32_t v = 0;
    for (uint32_t b = 0; b < 4; ++b)
        v |= (uint32_t)digits[b] << (8 * b);
    out[0] = v;
    for (uint64_t i = 1; i < E; ++i) {
        uint32_t d = 0;
        for (uint32_t b = 0; b < w; ++b)
            d |= (uint32_t)digits[4 + (i - 1) * w + b] << (8 * b);
        v += d;
        out[i] = v;
    }
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
