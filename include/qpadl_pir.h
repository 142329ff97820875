/*
 * qpadl_pir.h - C ABI of the GB300 (sm_103a) LWE-style PIR engine for the
 * private spectrum-database queries of QPADL (arxiv 2510.03631).
 *
 * The scheme.  A database D of R x C digits in Z_p (p = 2^l, l = 1..8) is
 * stored row-major as uint8; a record is a column of D.  All other quantities
 * live in Z_q with q = 2^32, i.e. uint32 with wraparound.  With public
 * A in Z_q^{C x n}, client secret s in Z_q^n, noise e in Z^C and
 * Delta = q / p:
 *     Setup    A       = PRG(seed)                       (C x n)
 *     Hint     H       = D * A                           (R x n, offline)
 *     Query    qu      = A * s + e + Delta * u_col       (C)
 *     Answer   ans     = D * qu                          (R)
 *     Recover  d_i     = round((ans_i - (H s)_i) / Delta) mod p  = D[i][col]
 * The paper's Def. 1 (Sec. 3) fixes the three-call shape (Client.Query,
 * DB.Query.Response, Client.BlockReconst); Sec. 5.2 fixes the server's work
 * as one product of the query with the whole database matrix accumulated
 * mod q (Alg. 3, Alg. 4); Sec. 5.3 moves query-independent work offline
 * (here, the hint).  The lattice instantiation is the standard
 * single-server LWE PIR, which the paper does not spell out.
 *
 * Conventions shared by every call:
 *  - Return value: QPADL_OK (0) or a negative QPADL_E* code.  Nothing throws.
 *  - Pointers named *_dev are device pointers that the CALLER allocates,
 *    owns and frees; the library never frees them.  They must stay valid
 *    until the work enqueued on `stream` has completed.  Pointers named
 *    *_host are host pointers; calls taking them return after the result is
 *    back in host memory.
 *  - `stream` is a cudaStream_t (0 = legacy default stream).  Device calls
 *    are asynchronous on it unless documented otherwise.
 *  - Shapes are validated before any launch; invalid shapes or pointers
 *    return QPADL_EINVAL and enqueue nothing.
 *  - A handle (qpadl_db) is library-owned and freed by qpadl_pir_destroy.
 *    Device work that fails inside a kernel (a bounded wait that ran out)
 *    records a code in the handle's device status word; qpadl_pir_status
 *    reads it.
 *  - Calls on one handle must not overlap on different streams: the
 *    handle's scratch buffers are shared by its calls.
 */
#ifndef QPADL_PIR_H
#define QPADL_PIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *qpadl_stream_t; /* identical to cudaStream_t */

enum {
    QPADL_OK = 0,
    QPADL_EINVAL = -1,   /* bad argument, shape, alignment or digit >= p */
    QPADL_ENOMEM = -2,   /* device allocation failed / over memory budget */
    QPADL_ECUDA = -3,    /* a CUDA runtime call or launch failed */
    QPADL_ETIMEOUT = -4, /* a kernel's bounded wait ran out (see qpadl_pir_status) */
    QPADL_EBUSY = -5,    /* serving admission refused the request */
    QPADL_EAGAIN = -6    /* serving: result not ready yet */
};

/* Setup flags. */
#define QPADL_SETUP_TENSOR_COPY 0x1u /* build the tensor-core operand copy of D
                                        at setup (else: on first batched call) */

/* Scheme parameters (Setup).  Digits of D must be < p. */
typedef struct qpadl_params {
    uint64_t rows;   /* R: database rows (> 0) */
    uint64_t cols;   /* C: database columns = number of records (> 0) */
    uint32_t n;      /* LWE dimension (> 0, <= 16384) */
    uint32_t log_q;  /* must be 32 */
    uint32_t p;      /* plaintext modulus, a power of two in [2, 256] */
    uint32_t flags;  /* QPADL_SETUP_* */
    double sigma;    /* noise standard deviation (informational: noise is an input) */
    uint64_t seed;   /* seed of the public matrix A (qpadl_pir_gen_a) */
} qpadl_params;

typedef struct qpadl_db qpadl_db;

/* Human-readable name of a QPADL_* code (static storage). */
const char *qpadl_strerror(int code);

/* Version of this ABI (major * 10000 + minor * 100 + patch). */
int qpadl_version(void);

/* Tuning options of a handle (qpadl_pir_set_option / qpadl_pir_get_option).
 * They change speed only, never results. */
#define QPADL_OPT_STREAM_CHUNK 1     /* digits per row per pipeline stage of the streaming
                                        Response: 512, 1024, 2048 (default) or 4096 */
#define QPADL_OPT_TENSOR_MIN_BATCH 2 /* smallest batch that qpadl_pir_answer_batch sends to
                                        the tensor-core GEMM (>= 1; default 3) */
#define QPADL_OPT_STREAM_RAW 3       /* 1: one or two queries are packed inside the streaming
                                        kernel (one launch, no scratch; two queries share one
                                        pass over D); 0 (default): a separate packing launch
                                        first */
#define QPADL_OPT_U8_MAX_BATCH 4     /* batches of up to this many queries (0..2^30, default 64)
                                        run the tensor-core GEMM on the uint8 digits as stored;
                                        larger ones use the handle's fp16 operand copy, and so
                                        does the hint when n is larger.  A value at or above
                                        every batch and n keeps no fp16 copy at all (the lean
                                        layout: D plus one blocked copy of the same size) */
#define QPADL_OPT_U8_KSTEP 5         /* digits per row per pipeline stage of that GEMM: 128 or 256;
                                        0 (default) = 128 */
#define QPADL_OPT_PAIR_GEMM 6        /* batches on the fp16 operand copy and the hint: 1 (default)
                                        = tiles of 256 rows over pairs of SMs (tcgen05
                                        cta_group::2, each SM loads half of the vector tile);
                                        0 = tiles of 128 rows on one SM each (stream-K split
                                        of the last wave) */

/*
 * Setup (server side; Def. 1's server holds D).  Validates `prm`, records
 * the shape and binds the caller's resident database `db_dev` (R*C bytes,
 * row-major, not copied; it must outlive the handle).  When p < 256 the
 * digits are checked on the device (this call then synchronises `stream`)
 * and a digit >= p returns QPADL_EINVAL.  With QPADL_SETUP_TENSOR_COPY the
 * library also allocates and fills its tensor-core operand copy of D
 * (2 * R * roundup(C, 8) bytes, library-owned) on `stream`.
 * On success *out receives the handle.
 */
int qpadl_pir_setup(const qpadl_params *prm, const uint8_t *db_dev,
                    qpadl_stream_t stream, qpadl_db **out);

/* Synchronises the device, then frees the handle and all library-owned
 * device memory it holds.  NULL is accepted. */
int qpadl_pir_destroy(qpadl_db *db);

/* Synchronises the device, then reads and clears the handle's device
 * status word: QPADL_OK, or QPADL_ETIMEOUT when a kernel's bounded wait ran
 * out since the last call. */
int qpadl_pir_status(qpadl_db *db);

/* Bytes of device memory the handle currently owns (operand copy + scratch). */
uint64_t qpadl_pir_device_bytes(const qpadl_db *db);

/* Shape of a handle's database: *rows = R, *cols = C. */
int qpadl_pir_shape(const qpadl_db *db, uint64_t *rows, uint64_t *cols);

/*
 * Row shard of a database for one of `world` GPUs (host only; no device
 * access).  Answer row i depends on database row i alone (ans = D qu, Def. 1
 * DB.Query.Response), so rank r may hold rows [*r0, *r1) of D and of H,
 * answer every query on them, and the ranks' answers concatenate in rank
 * order with no reduction.  Shards are whole 128-row tiles (the GEMM tile
 * height) except the last, as even as that allows; a rank may get an empty
 * shard when rows < 128 * world.  A shard is set up as its own handle:
 * qpadl_pir_setup with rows = *r1 - *r0 and db_dev + *r0 * C.
 * QPADL_EINVAL if world == 0, rank >= world or an output pointer is NULL.
 */
int qpadl_pir_shard_rows(uint64_t rows, uint32_t world, uint32_t rank, uint64_t *r0, uint64_t *r1);

/* Pre-sizes the handle's scratch so that later Response calls with batches
 * of up to max_batch queries allocate nothing (tensor-core operand copy of D
 * and limb scratch when max_batch reaches the tensor-core threshold).  May
 * call cudaMalloc; synchronises the device.  Use before a stream capture. */
int qpadl_pir_reserve(qpadl_db *db, uint32_t max_batch, qpadl_stream_t stream);

/* Sets / reads a tuning option (QPADL_OPT_*).  QPADL_EINVAL for an unknown
 * option or an unsupported value.  Host-only; enqueues nothing. */
int qpadl_pir_set_option(qpadl_db *db, int option, int64_t value);
int qpadl_pir_get_option(const qpadl_db *db, int option, int64_t *value);

/* Autotuner: times this handle's exact-path choices on the device with CUDA
 * events (uniform synthetic queries, answers discarded) and keeps the
 * fastest; every choice gives the same results.  Tunes, in order:
 *  - one query: QPADL_OPT_STREAM_CHUNK in {1024, 2048, 4096} x
 *    QPADL_OPT_STREAM_RAW in {0, 1};
 *  - if max_batch >= 2: QPADL_OPT_U8_KSTEP in {128, 256} at
 *    min(max(max_batch, 4), 16) queries (when that batch takes the uint8-
 *    digit GEMM; both are timed, but with QPADL_OPT_PAIR_GEMM on the depth
 *    stays 128, the only one the pair tiles take), then
 *    QPADL_OPT_TENSOR_MIN_BATCH = the first B in 2..4 at
 *    which the tensor path beats the streaming kernel (5 if none does);
 *  - if max_batch > 32: QPADL_OPT_U8_MAX_BATCH = 128 if the uint8-digit GEMM
 *    beats the fp16-copy GEMM at 128 queries, else 64 if it does at 64, else
 *    32 (the two GEMMs, so the fp16 copy is built).
 * Allocates and frees scratch for up to 128 queries and answers, may build the
 * blocked digit copy, and synchronises the stream.  report (may be NULL)
 * receives the times in ms (-1 where a choice does not apply). */
typedef struct qpadl_tune_report {
    double single_ms[3][2];     /* [chunk 1024, 2048, 4096][raw 0, 1] */
    double u8_kstep_ms[2];      /* [128, 256] at tuned_batch queries */
    double stream_ms[3];        /* B = 2, 3, 4 on the streaming kernel */
    double tensor_ms[3];        /* B = 2, 3, 4 on the tensor path */
    uint32_t tuned_batch;
    int32_t stream_chunk, stream_raw, u8_kstep;   /* the chosen settings */
    uint32_t tensor_min_batch;
    double u8_vs_f16_ms[2][2];  /* [B = 64, 128][uint8-digit GEMM, fp16-copy GEMM] */
    uint32_t u8_max_batch;      /* the chosen QPADL_OPT_U8_MAX_BATCH */
} qpadl_tune_report;
int qpadl_pir_autotune(qpadl_db *db, uint32_t max_batch, qpadl_stream_t stream, qpadl_tune_report *report);

/*
 * Setup, public matrix: A_dev[j*n + k] = upper 32 bits of output number
 * j*n + k of SplitMix64 started from state prm->seed (C x n, row-major).
 * A_dev: C*n uint32, 4-byte aligned.
 */
int qpadl_pir_gen_a(const qpadl_params *prm, uint32_t *A_dev, qpadl_stream_t stream);

/*
 * Hint (offline; Sec. 5.3's offline precomputation): H = D * A mod 2^32.
 * A_dev: C x n uint32 row-major; H_dev: R x n uint32 row-major.  Runs the
 * exact byte-limb tensor-core GEMM; allocates the handle's operand copy of
 * D on first use and a library-owned scratch of 8 * n * roundup(C, 8) bytes
 * (kept for reuse).
 */
int qpadl_pir_hint(qpadl_db *db, const uint32_t *A_dev, uint32_t *H_dev,
                   qpadl_stream_t stream);

/*
 * Query (Def. 1, Client.Query): q_dev[j] = sum_k A[j][k] s[k] + e[j]
 * + (j == col ? Delta : 0) mod 2^32, Delta = 2^32 / p.
 * A_dev: C x n uint32; s_dev: n uint32; e_dev: C int32 (reduced mod 2^32);
 * q_dev: C uint32.  col < C.
 */
int qpadl_pir_query(const qpadl_params *prm, const uint32_t *A_dev,
                    const uint32_t *s_dev, const int32_t *e_dev, uint64_t col,
                    uint32_t *q_dev, qpadl_stream_t stream);

/*
 * Batched Query: B queries.  S_dev: B x n (secret b in row b); E_dev: B x C;
 * cols_dev: B uint32 target columns (each < C, not checked on the host);
 * Q_dev: B x C (query b in row b).
 */
int qpadl_pir_query_batch(const qpadl_params *prm, const uint32_t *A_dev,
                          const uint32_t *S_dev, const int32_t *E_dev,
                          const uint32_t *cols_dev, uint32_t B, uint32_t *Q_dev,
                          qpadl_stream_t stream);

/*
 * Answer (Def. 1, DB.Query.Response; Sec. 5.2's product of the query with
 * the database, accumulated mod q as in Alg. 4): ans_dev[i] = sum_j D[i][j]
 * q[j] mod 2^32.  q_dev: C uint32; ans_dev: R uint32.  One streaming pass
 * over D (HBM bound).  Allocates nothing.
 */
int qpadl_pir_answer(qpadl_db *db, const uint32_t *q_dev, uint32_t *ans_dev,
                     qpadl_stream_t stream);

/*
 * Batched Answer (Alg. 4's batch of q-bar queries): for b < B,
 * ans_dev[b*R + i] = sum_j D[i][j] Q[b*C + j] mod 2^32.  Q_dev: B x C
 * (query b in row b); ans_dev: B x R (answer b in row b).  B >= 1.
 * Small B runs the streaming kernel; larger B the exact byte-limb
 * tensor-core GEMM: on the uint8 digits as stored for B <= 32
 * (QPADL_OPT_U8_MAX_BATCH), otherwise on the handle's fp16 operand copy of D
 * (allocated on first use).  Both use a library-owned limb scratch of
 * 8 * B * roundup(C, 8) bytes, kept and grown as needed.
 */
int qpadl_pir_answer_batch(qpadl_db *db, const uint32_t *Q_dev, uint32_t B,
                           uint32_t *ans_dev, qpadl_stream_t stream);

/* As qpadl_pir_answer_batch, forcing the path: 0 = streaming kernel,
 * 1 = tensor-core GEMM.  For tests and measurement. */
int qpadl_pir_answer_batch_path(qpadl_db *db, const uint32_t *Q_dev, uint32_t B,
                                uint32_t *ans_dev, int path, qpadl_stream_t stream);

/*
 * Answer with host buffers (the end-to-end call): copies q_host (C uint32)
 * to the device, answers, copies ans_host (R uint32) back and synchronises
 * `stream`.  Uses a handle-owned device staging buffer.
 */
int qpadl_pir_answer_host(qpadl_db *db, const uint32_t *q_host, uint32_t *ans_host,
                          qpadl_stream_t stream);

/*
 * Allocation-free Response.  The paper has no counterpart: this is a
 * deployment variant of qpadl_pir_answer for callers that cannot allocate
 * device memory at the moment they answer - a runtime whose own allocator
 * owns all device memory and forbids side allocations, or a serving loop
 * that must not take the device-wide synchronisation that cudaMalloc and
 * cudaFree imply.
 *
 * Computes ans_dev[i] = sum_j D[i][j] q_dev[j] mod 2^32 for the caller's
 * resident database db_dev (rows x cols digits, row-major uint8) with no
 * handle and no allocation of any kind.  Its scratch (the packed query limbs
 * and a status word) is one fixed file-scope device array of 1 MiB + 256
 * bytes, which every GPU that loads this library holds until process exit.
 *  - cols > QPADL_NOALLOC_MAX_COLS returns QPADL_EINVAL (and says why on
 *    stderr); nothing is enqueued.
 *  - The first call on each device does a one-time host-side set-up with
 *    that device current (resolving the array's device address, setting
 *    kernel attributes).  Make that first call before any stream capture.
 *  - All calls on a device share the array and it keeps the last call's
 *    contents: calls whose work overlaps on the GPU (e.g. on two streams)
 *    race and can return wrong answers.  Serialise them.
 *  - Asynchronous on `stream`.  If a kernel's bounded wait runs out, ans_dev
 *    is incomplete and the array's status word is set; it stays set across
 *    later calls until qpadl_pir_noalloc_status reads it.
 */
#define QPADL_NOALLOC_MAX_COLS 262144u
int qpadl_pir_answer_noalloc(const uint8_t *db_dev, uint64_t rows, uint64_t cols,
                             const uint32_t *q_dev, uint32_t *ans_dev, qpadl_stream_t stream);

/*
 * Status of the allocation-free Response on the current device (no paper
 * counterpart; see qpadl_pir_answer_noalloc).  Waits for all work on the
 * device (cudaDeviceSynchronize), then reads the fixed array's status word:
 * QPADL_OK if no call since the last read gave up on a bounded wait,
 * QPADL_ETIMEOUT if one did (some answer since the last read is incomplete;
 * the word is cleared), QPADL_ECUDA if the device cannot be read.  Returns
 * QPADL_OK when no allocation-free call has run on the device.  Allocates
 * nothing.
 */
int qpadl_pir_noalloc_status(void);

/*
 * Recover (Def. 1, Client.BlockReconst): out_dev[i] = ((ans[i] - sum_k
 * H[i][k] s[k]) + Delta/2 mod 2^32) >> (32 - log2 p), i.e. the nearest
 * multiple of Delta, reduced mod p.  ans_dev: R uint32; H_dev: R x n;
 * s_dev: n; out_dev: R bytes.  prm gives R, n and p.
 */
int qpadl_pir_recover(const qpadl_params *prm, const uint32_t *ans_dev,
                      const uint32_t *H_dev, const uint32_t *s_dev, uint8_t *out_dev,
                      qpadl_stream_t stream);

/* Batched Recover: ans_dev B x R, S_dev B x n, out_dev B x R. */
int qpadl_pir_recover_batch(const qpadl_params *prm, const uint32_t *ans_dev,
                            const uint32_t *H_dev, const uint32_t *S_dev, uint32_t B,
                            uint8_t *out_dev, qpadl_stream_t stream);

/* ======================================================================
 * Database compression (Sec. 5.3, "Database Compression Techniques"): the
 * DB entries are sorted and stored as differences between successive
 * entries, so that close entries take fewer bits and each Response scans
 * fewer bytes.  Layout: entries are uint32 x_0 <= ... <= x_{n-1} (device);
 * block j (one record = one column of the database) holds entries
 * jE .. jE + E - 1, positions past n - 1 repeating x_{n-1}.  A block is its
 * first entry (4 little-endian bytes) followed by its E - 1 differences
 * x_{jE+i} - x_{jE+i-1} mod 2^32 in w little-endian bytes each, so the
 * compressed database is R' = 4 + w (E - 1) rows by C = ceil(n / E) columns
 * of digits (row-major uint8, p = 256), on which qpadl_pir_setup, hint,
 * Query, Answer and Recover run unchanged.  Unsorted entries still round-trip
 * exactly (the differences wrap mod 2^32) but need a larger w.
 * All three calls: QPADL_EINVAL for a NULL pointer, n or E of 0, w outside
 * 1..4, or R' or C at or above 2^31.
 * ==================================================================== */

/* The fewest bytes w (1..4) holding every within-block difference of the n
 * entries.  Synchronises `stream` (the result is returned on the host) and
 * allocates nothing: the reduction uses one library word per device, and
 * concurrent calls take turns on a host lock. */
int qpadl_pir_delta_width(const uint32_t *entries_dev, uint64_t n, uint32_t E, uint32_t *w_out,
                          qpadl_stream_t stream);

/* Writes the compressed database: db_dev receives R' x C digits (caller-
 * owned, R' * C bytes).  Asynchronous on `stream`; allocates nothing.  Also
 * QPADL_EINVAL for blocks of more than 4,194,241 entries (E - 1 > 64 * 65535). */
int qpadl_pir_delta_encode(const uint32_t *entries_dev, uint64_t n, uint32_t E, uint32_t w,
                           uint8_t *db_dev, qpadl_stream_t stream);

/* Decodes B recovered blocks: digits_dev B x R' (block b's digits at
 * b * R', as qpadl_pir_recover[_batch] writes them), entries_dev B x E
 * (entry i of block b at b * E + i).  Asynchronous; allocates nothing. */
int qpadl_pir_delta_decode(const uint8_t *digits_dev, uint32_t B, uint32_t E, uint32_t w,
                           uint32_t *entries_dev, qpadl_stream_t stream);

/*
 * Status of the handle-free single-vector Query and Recover kernels.  For
 * n in {512, 1024, 2048} (with 16-byte aligned matrix and secret) those two
 * calls stream the matrix through shared memory behind barrier waits that
 * give up after a bounded time; a wait that gives up leaves that call's
 * output incomplete and records QPADL_ETIMEOUT in one status word per
 * device.  This call waits for the current device (cudaDeviceSynchronize),
 * returns the word (QPADL_OK or QPADL_ETIMEOUT; QPADL_ECUDA if the device
 * cannot be read) and clears it.
 */
int qpadl_pir_client_status(void);

/* ======================================================================
 * Client context: batched Query and Recover on the tensor cores
 * (Def. 1 Client.Query and Client.BlockReconst for many secrets at once).
 *
 * X s mod 2^32 (X = A or H, uint32) needs only the byte-limb products
 * x_u s_l with u + l <= 3.  The context keeps X's four balanced byte-limb
 * planes (fp16, side by side along K: rows x 4n) on the device; each call
 * expands the secrets into shifted limb rows and runs one exact tcgen05 GEMM
 * whose epilogue is Query's (+ e_b + Delta at col_b) or Recover's
 * (round((ans_b - .)/Delta) mod p).  Results equal qpadl_pir_query_batch /
 * qpadl_pir_recover_batch bit for bit.
 * ==================================================================== */
typedef struct qpadl_client qpadl_client;

/* Builds the context on the current device from A_dev (C x n uint32) and,
 * if H_dev is not NULL, the hint H_dev (R x n uint32); both are read only
 * during the call (the context keeps limb-plane copies: 8 C n and 8 R n
 * bytes) plus a workspace for max_batch secrets (32 n max_batch bytes;
 * larger calls run in chunks of max_batch).  prm gives R, C, n and p.
 * QPADL_EINVAL for bad parameters, a NULL A_dev or max_batch outside
 * 1..65536; QPADL_ENOMEM if device memory runs out.  Calls on one context
 * share its workspace: issue them on one stream (or order them). */
int qpadl_client_create(const qpadl_params *prm, const uint32_t *A_dev, const uint32_t *H_dev,
                        uint32_t max_batch, qpadl_stream_t stream, qpadl_client **out);

/* B queries: S_dev B x n (secret b in row b), E_dev B x C int32, cols_dev B
 * target columns (each < C, not checked on the host), Q_dev B x C. */
int qpadl_client_query_batch(qpadl_client *c, const uint32_t *S_dev, const int32_t *E_dev,
                             const uint32_t *cols_dev, uint32_t B, uint32_t *Q_dev,
                             qpadl_stream_t stream);

/* B recoveries: ans_dev B x R, S_dev B x n, out_dev B x R digits.
 * QPADL_EINVAL if the context was built without H. */
int qpadl_client_recover_batch(qpadl_client *c, const uint32_t *ans_dev, const uint32_t *S_dev,
                               uint32_t B, uint8_t *out_dev, qpadl_stream_t stream);

/* Synchronises the device; QPADL_ETIMEOUT (and clears it) if a kernel of
 * this context gave up a bounded wait since the last call. */
int qpadl_client_status(qpadl_client *c);

/* Bytes of device memory the context owns. */
uint64_t qpadl_client_device_bytes(const qpadl_client *c);

/* Client options (every setting gives the same results):
 * QPADL_CLIENT_OPT_SKIP_ZERO_BLOCKS (default 1): when n is a multiple of 512
 *   and a call carries more than 8 secrets, skip the (plane u, shift t)
 *   blocks with u > t, whose secret limbs are zero (10 of 16 blocks run);
 *   0 runs all 16.  QPADL_EINVAL for an unknown option or value. */
#define QPADL_CLIENT_OPT_SKIP_ZERO_BLOCKS 1
/* QPADL_CLIENT_OPT_PAIR_GEMM (default 1): run the batches on tiles of 256 rows
 *   over pairs of SMs (tcgen05 cta_group::2: each SM loads its own matrix
 *   rows and half of the secret rows); 0: tiles of 128 rows on one SM each. */
#define QPADL_CLIENT_OPT_PAIR_GEMM 2
int qpadl_client_set_option(qpadl_client *c, int option, int64_t value);

/* Waits for the device and frees the context (NULL is fine). */
int qpadl_client_destroy(qpadl_client *c);

/* ======================================================================
 * Goldberg-style Response over Z_p (Sec. 5.2 "Parallel Goldberg-PIR",
 * Alg. 4; the FTR instantiation of Sec. 7): the server's answer to a query
 * q in Z_p^C is rho = D q mod p.  The paper names no field; here p is a
 * prime <= 257 (p = 257 takes every byte as a field element).  The database
 * keeps the layout of the lattice scheme: R x C bytes, record j = column j;
 * the client's queries are Shamir shares of e_theta (degree-t polynomials
 * at distinct points) and Lagrange interpolation of t + 1 answers at 0
 * gives record theta.
 * ==================================================================== */
typedef struct qpadl_goldberg qpadl_goldberg;

/* Binds a resident database (db_dev: rows x cols bytes, each < p, caller-
 * owned, kept until destroy).  QPADL_EINVAL if p is not a prime in [2, 257],
 * cols is 0 or above 65792 (the exact-sum bound), a byte is >= p (checked on
 * the device when p < 256), or db_dev is NULL. */
int qpadl_goldberg_setup(uint64_t rows, uint64_t cols, uint32_t p, const uint8_t *db_dev,
                         qpadl_stream_t stream, qpadl_goldberg **out);

/* Answers B queries: Q_dev B x cols field elements (uint32, each < p; larger
 * values give unspecified answers), out_dev B x rows elements in [0, p).
 * Below the GEMM threshold the streaming kernel computes the exact integer
 * sums and a second kernel reduces them mod p; up to 64 queries the
 * uint8-digit GEMM does the same with each query as one centred fp16 row
 * (builds the blocked digit copy on first use); above, one exact tcgen05 GEMM
 * over the fp16 operand copy with the same rows and a mod-p epilogue (builds
 * that copy on first use). */
int qpadl_goldberg_answer_batch(qpadl_goldberg *h, const uint32_t *Q_dev, uint32_t B, uint32_t *out_dev,
                                qpadl_stream_t stream);

/* QPADL_GOLDBERG_OPT_GEMM_MIN_BATCH (default 3): smallest batch on a GEMM.
 * QPADL_GOLDBERG_OPT_U8_MAX_BATCH (0..256, default 128): largest batch on the
 *   uint8-digit GEMM (one centred fp16 row per query, exact signed sums, then
 *   mod p; 64-wide tiles, several per row tile above 64 queries); larger batches
 *   take the one-limb fp16 GEMM.  EINVAL outside the range. */
#define QPADL_GOLDBERG_OPT_GEMM_MIN_BATCH 1
#define QPADL_GOLDBERG_OPT_U8_MAX_BATCH 2
/* QPADL_GOLDBERG_OPT_PAIR_GEMM (0/1, default 1): the uint8-digit GEMM, and the
 * one-limb fp16 GEMM's 256-wide tiles, on tiles of 256 rows over pairs of SMs
 * (see QPADL_OPT_PAIR_GEMM). */
#define QPADL_GOLDBERG_OPT_PAIR_GEMM 3
int qpadl_goldberg_set_option(qpadl_goldberg *h, int option, int64_t value);

/* As qpadl_pir_status, for the handle's kernels. */
int qpadl_goldberg_status(qpadl_goldberg *h);

/* Waits for the device and frees the handle (not the database). */
int qpadl_goldberg_destroy(qpadl_goldberg *h);

/* ======================================================================
 * Chor-style Response over GF(2) (Sec. 5.2 "Parallel Chor-PIR", Alg. 3;
 * the ENS instantiation of Sec. 7): the database is `rows` records of `bits`
 * bits, the server's answer to an rows-bit query q is rho = q . DB over
 * GF(2), the XOR of the records whose query bit is set.  The client XORs
 * the answers of ell servers to its ell queries (ell - 1 random, the last
 * their XOR with the unit vector e_theta) and obtains record theta.
 *
 * Packing: bit c of record i is bit c % 32 of word i * (bits/32) + c / 32;
 * bit i of a query is bit i % 32 of its word i / 32 (ceil(rows/32) words per
 * query; bits at positions >= rows are ignored).
 * ==================================================================== */
typedef struct qpadl_chor qpadl_chor;

/* Binds a resident database (db_dev: rows x bits/32 uint32 words, caller-
 * owned, 16-byte aligned, kept until destroy) on the current device and
 * allocates the handle's scratch (32 bytes per row).  QPADL_EINVAL if rows
 * is 0 or >= 2^31, bits is not a positive multiple of 128, or db_dev is
 * NULL or misaligned. */
int qpadl_chor_setup(uint64_t rows, uint64_t bits, const uint32_t *db_dev, qpadl_stream_t stream,
                     qpadl_chor **out);

/* Answers B queries (Q_dev: B x ceil(rows/32) words, query b in row b) in
 * one pass over the database per 256 queries; out_dev: B x bits/32 words
 * (answer b in row b), overwritten.  Calls on one handle share its scratch:
 * issue them on one stream (or order them). */
int qpadl_chor_answer_batch(qpadl_chor *h, const uint32_t *Q_dev, uint32_t B, uint32_t *out_dev,
                            qpadl_stream_t stream);

/* Options (every setting gives the same results):
 * QPADL_CHOR_OPT_M4RM_MIN_BATCH (1..257, default 48): batches (per chunk of
 *   256) of at least this many queries use the four-Russians kernel (4-row
 *   XOR tables in shared memory, looked up by 4 query bits); smaller ones the
 *   masked-XOR scan.  257 disables the four-Russians kernel. */
#define QPADL_CHOR_OPT_M4RM_MIN_BATCH 1
/* QPADL_CHOR_OPT_SCAN_FORM (-1..3, default -1): inner loop of the masked-XOR
 * scan.  Bit 1: each thread covers 8 database words per row (at most 16
 * queries) instead of 4 (at most 32), so one selector test serves twice the
 * words; bit 0: a query's row words are XORed in under its selector bit
 * instead of through an all-ones/all-zeros mask.  -1 picks by batch size:
 * 0 up to 8 queries, 1 up to 16, 3 above.  Every form gives the same bits. */
#define QPADL_CHOR_OPT_SCAN_FORM 2
int qpadl_chor_set_option(qpadl_chor *h, int option, int64_t value);
int qpadl_chor_get_option(qpadl_chor *h, int option, int64_t *value);

/* Synchronises the device; QPADL_ETIMEOUT (and clears it) if a kernel of this
 * handle gave up a bounded wait since the last call. */
int qpadl_chor_status(qpadl_chor *h);

/* Waits for the device and frees the handle (not the database). */
int qpadl_chor_destroy(qpadl_chor *h);

/* ======================================================================
 * Failure-detection self-test.  Every wait of the library's TMA/tcgen05
 * kernels on an mbarrier is bounded (2 s of %globaltimer): a kernel that
 * gives up raises its CTA's abort flag, lets its own copies land, frees its
 * TMEM and records QPADL_ETIMEOUT in a status word, so the host learns of
 * the failure and the CUDA context stays usable; nothing traps.
 * ==================================================================== */

/* Runs that same bounded wait in a one-warp kernel on a barrier that nothing
 * arrives on (arrive = 0: it must give up after about 2 s and write
 * QPADL_ETIMEOUT's device code 1 to *status_dev) or on one completed first
 * (arrive != 0: it must return at once and write 0).  *waited_ns_dev gets
 * the time the wait took.  Both pointers are device memory (int32, uint64).
 * Asynchronous on stream; QPADL_EINVAL for NULL pointers. */
int qpadl_selftest_bounded_wait(int arrive, int32_t *status_dev, uint64_t *waited_ns_dev,
                                qpadl_stream_t stream);

/* ======================================================================
 * Serving: a continuous-batching request loop over several resident
 * databases (the paper's server answering q-bar queries per database,
 * Sec. 5.2, run as a long-lived service).  Requests arrive from any host
 * thread; whenever a launch stream is free, one loop thread forms a launch
 * from up to max_batch queued requests of the database holding the oldest
 * request and of every other database within group_size_ratio of its size,
 * so new arrivals start while earlier launches are still on the GPU.  One
 * launch answers all its databases together in one grouped tensor-core GEMM
 * over their uint8 digits, however uneven their counts (up to each handle's
 * QPADL_OPT_U8_MAX_BATCH queries; a database with more takes the fp16-copy
 * GEMM); a launch of a lone database with 1 or 2 queries uses the streaming
 * kernel.  Admission is by
 * memory: each request's query and answer live in a mapped pinned host
 * arena of host_budget_bytes; each launch's workspace (queries, answers,
 * query limbs) comes from a device arena of device_budget_bytes, and a
 * launch whose workspace would not fit takes fewer requests.
 * ==================================================================== */
typedef struct qpadl_server qpadl_server;

typedef struct qpadl_server_config {
    uint64_t host_budget_bytes;   /* pinned host arena for queued/in-flight requests (admission) */
    uint64_t device_budget_bytes; /* device arena for per-launch batch buffers */
    uint32_t max_inflight;        /* requests admitted and not yet polled */
    uint32_t max_batch;           /* requests of one database per launch (1..65535); a launch holds
                                     at most min(max_inflight, 65535) requests in all */
    uint32_t num_streams;         /* launches in flight at once (1..8); while a launch that
                                     carries a batched GEMM (3 or more requests of a database)
                                     is in flight, at most 2 launches run */
    uint32_t test_drop_completion_launch; /* test hook: 0 = off; k = the k-th launch's completion
                                             is not reported, so its requests run into the watchdog */
    double hold_us;               /* a lone request may wait this long for company while other
                                     launches run (0 = launch as soon as a stream is free) */
    double watchdog_ms;           /* requests whose launch has not completed after this fail
                                     with QPADL_ETIMEOUT (<= 0: 10000) */
    double group_size_ratio;      /* databases whose R*C is within this factor of the leading
                                     database's join its launch; < 1: one database per launch */
} qpadl_server_config;

typedef struct qpadl_request_times {
    double submit_s, launch_s, done_s; /* steady-clock seconds */
} qpadl_request_times;

typedef struct qpadl_server_stats_t {
    uint64_t launches, completed, failed, refused;
    uint32_t inflight, queued;
    double mean_launch_requests;
    uint64_t host_bytes_used, device_bytes_used;
    uint64_t grouped_launches;    /* launches that answered two or more databases */
    double mean_enqueue_us;       /* host time per launch spent enqueueing its kernels */
    uint64_t stream_kernels;      /* streaming Response kernels enqueued (one pass over a
                                     database answers its 1 or 2 queries of a launch) */
    uint64_t gemm_kernels;        /* batched-GEMM Response kernels enqueued */
} qpadl_server_stats_t;

/* Creates a server on the current device (allocates both arenas and the
 * launch streams).  QPADL_EINVAL for a bad config, QPADL_ENOMEM if an arena
 * cannot be allocated. */
int qpadl_server_create(const qpadl_server_config *cfg, qpadl_server **out);

/* Registers a database handle (before qpadl_server_start) and builds the
 * read-only operand copies its launches use (the blocked digit copy if
 * max_batch >= 3, the fp16 copy if max_batch > 32), so launches never
 * allocate.  QPADL_ENOMEM if a copy cannot be allocated or one request's
 * workspace exceeds device_budget_bytes.  The handle must outlive the
 * server. */
int qpadl_server_add_db(qpadl_server *srv, qpadl_db *db, int *db_id);

/* Starts the request loop thread. */
int qpadl_server_start(qpadl_server *srv);

/* Admits one query (C uint32 words in host memory, copied before return)
 * for database db_id.  Requests submitted before qpadl_server_start stay
 * queued and form the first launch.  QPADL_EBUSY if admission refuses (in-flight limit or
 * host arena full): retry later.  *ticket identifies the request. */
int qpadl_server_submit(qpadl_server *srv, int db_id, const uint32_t *q_host, uint64_t *ticket);

/* QPADL_EAGAIN while the request is queued or running; otherwise copies the
 * answer (R words) to ans_host (may be NULL), fills *times (may be NULL),
 * forgets the ticket and returns QPADL_OK, QPADL_ETIMEOUT (watchdog) or
 * QPADL_ECUDA.  Unknown ticket: QPADL_EINVAL. */
int qpadl_server_poll(qpadl_server *srv, uint64_t ticket, uint32_t *ans_host,
                      qpadl_request_times *times);

int qpadl_server_stats(qpadl_server *srv, qpadl_server_stats_t *st);

/* Stops the loop, waits for launches in flight, frees everything. */
int qpadl_server_destroy(qpadl_server *srv);

/* Open-loop load replay: submits request i at arrival_s[i] seconds after
 * the call starts (retrying while admission refuses), waits for all, and
 * writes latency_s[i] = completion - scheduled arrival (-1 on failure) and
 * status[i].  ans_host may be NULL (answers discarded).  arrival_s must be
 * non-decreasing (QPADL_EINVAL otherwise).  Up to four client threads share
 * the requests round-robin, each submitting and polling its own.  times
 * (may be NULL) receives, per completed request, its submit, launch and
 * completion times in seconds after its scheduled arrival. */
int qpadl_server_replay(qpadl_server *srv, uint64_t n, const double *arrival_s,
                        const int32_t *db_ids, const uint32_t *const *q_host,
                        uint32_t *const *ans_host, double *latency_s, int32_t *status,
                        qpadl_request_times *times);

#ifdef __cplusplus
}
#endif

#endif /* QPADL_PIR_H */
