// Chor-style PIR Response over GF(2) (Sec. 5.2 "Parallel Chor-PIR", Alg. 3):
//   rho_b = q_b . DB over GF(2), the XOR of the database rows whose bit in
//   query b is set.  DB: r rows x W words (bit c of row i is bit c % 32 of
//   word i * W + c / 32); query b: qw = ceil(r / 32) words, bit i of word
//   i / 32 selects row i; response b: W words.
//
// One pass over the database answers a whole batch (the paper's kernel runs
// one block row per query and so reads the database once per query):
//  1. chor_transpose_kernel turns the batch's query bits around: bit j of
//     QT[i][g] is bit i of query 32 g + j, so one word gives a thread the
//     selector bits of 32 queries for row i.
//  2. chor_answer_kernel<QB, QG>: persistent CTAs (one per SM) walk units =
//     (column tile of TW words, band of RB rows) in tile-major order, split
//     evenly over the grid.  A producer warp streams each unit's database
//     tile (2-D TMA boxes of up to 256 words x RB rows, 32 KB per stage) and
//     its QT rows into a 4-stage shared-memory ring.  256 consumer threads:
//     thread = (4 consecutive words of the tile, one group of QB queries)
//     keeps acc[QB][4] in registers; per row it does one 16-byte shared load
//     of database words and one selector load, and per query builds a mask
//     (all ones when the query's bit is set) and XORs row & mask into its
//     four accumulators (one LOP3 each).
//  3. When a CTA leaves a column tile it folds its partial XORs into the
//     zeroed response with 32-bit atomic XORs: XOR is exact, associative and
//     commutative, so the split over CTAs changes nothing.
//  4. Large batches take chor_m4rm_kernel instead (the method of four
//     Russians): per band of 64 rows the CTA builds, for each group of 4
//     rows, the 16 XOR combinations of those rows over its 64-word column
//     tile in shared memory, and each query then adds one table entry per
//     4 rows, indexed by its 4 selector bits: 4 XORs per 4 rows x 4 words
//     instead of 16 masked XORs, at one 16-byte shared load per lookup.
//     Thread = (word quad, group of 16 queries), 256 queries per pass.
// Every mbarrier wait is bounded (2 s of %globaltimer); a CTA that gives up
// raises the status word and leaves, no kernel traps.
#include <algorithm>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "chor.cuh"
#include "ptx.cuh"

namespace qpadl {

constexpr int kChorThreads = 256;          // consumer threads
constexpr int kChorStages = 4;
constexpr uint32_t kChorStageWords = 8192;  // 32 KB of database words per stage

// Column tile width and band height for QG query groups per CTA, WPT words per thread.
__host__ __device__ constexpr uint32_t chor_tw(int qg, int wpt) {
    return static_cast<uint32_t>(kChorThreads / qg * wpt);
}
__host__ __device__ constexpr uint32_t chor_rb(int qg, int wpt) { return kChorStageWords / chor_tw(qg, wpt); }

// QT words per row as stored (at least 4, so a TMA box row is 16 bytes).
__host__ __device__ constexpr uint32_t chor_qtw(uint32_t qbw) { return qbw < 4 ? 4u : qbw; }

__global__ void chor_transpose_kernel(const uint32_t *__restrict__ Q, uint64_t qw, uint32_t B, uint64_t r,
                                      uint32_t qtw, uint32_t *__restrict__ QT) {
    // one warp per (32-row word k, query group g): lane j holds query 32 g + j's word k
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t groups = (B + 31) / 32;
    const uint64_t tasks = qw * qtw;
    for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < tasks; t += warps) {
        const uint64_t k = t / qtw;
        const uint32_t g = static_cast<uint32_t>(t - k * qtw);
        const uint64_t b = 32ull * g + lane;
        const uint32_t x = (g < groups && b < B) ? Q[b * qw + k] : 0u;
        uint32_t mine = 0;
#pragma unroll
        for (int bit = 0; bit < 32; ++bit) {
            const uint32_t v = __ballot_sync(0xffffffffu, (x >> bit) & 1u);
            if (lane == static_cast<uint32_t>(bit)) mine = v;
        }
        const uint64_t row = 32ull * k + lane;
        if (row < r) QT[row * qtw + g] = mine;
    }
}

// WPT: database words per thread per row (4 or 8: a mask or selector test serves WPT words).
// PRED: per query, test its selector bit and XOR the row words in under that (warp-uniform)
// condition, instead of building an all-ones/all-zeros mask and AND-ing it in.
template <int QB, int QG, int WPT = 4, bool PRED = false>
__global__ void __launch_bounds__(kChorThreads + 32, 1)
    chor_answer_kernel(const __grid_constant__ CUtensorMap db_map, const __grid_constant__ CUtensorMap qt_map,
                       uint64_t r, uint32_t W, uint32_t B, uint32_t qtw, uint32_t *__restrict__ out,
                       int *__restrict__ status) {
    constexpr uint32_t TW = chor_tw(QG, WPT);
    constexpr uint32_t RB = chor_rb(QG, WPT);
    constexpr uint32_t BOXW = TW < 256 ? TW : 256;   // words per TMA box row
    constexpr uint32_t NBOX = TW / BOXW;
    constexpr uint32_t QUADS = TW / WPT;             // threads per query group
    static_assert(QUADS * QG == kChorThreads, "one thread per (WPT words, query group)");
    static_assert(WPT == 4 || WPT == 8, "words per thread");
    static_assert(QB <= 32 && 32 % QB == 0, "a query group lies inside one selector word");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t qt_stage_bytes = RB * qtw * 4u;
    uint32_t *db_st = reinterpret_cast<uint32_t *>(smem);                                   // [stage][NBOX][RB][BOXW]
    uint32_t *qt_st = reinterpret_cast<uint32_t *>(smem + kChorStages * kChorStageWords * 4);  // [stage][RB][qtw]
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kChorStages * (kChorStageWords * 4 + 2048));
    uint64_t *empty = full + kChorStages;
    volatile int *abort = reinterpret_cast<volatile int *>(empty + kChorStages);

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kChorStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kChorThreads / 32);
        }
        *abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    const uint64_t n_tiles = (W + TW - 1) / TW;
    const uint64_t n_bands = (r + RB - 1) / RB;
    const uint64_t units = n_tiles * n_bands;
    const uint64_t u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
    bool failed = false;

    if (warp == kChorThreads / 32) {
        // ---------------- producer
        if (lane == 0) {
            tma_prefetch_desc(&db_map);
            tma_prefetch_desc(&qt_map);
            uint32_t it = 0;
            for (uint64_t u = u0; u < u1; ++u, ++it) {
                const uint32_t st = it % kChorStages, ph = (it / kChorStages) & 1u;
                if (!mbar_wait(&empty[st], ph ^ 1u, abort)) {
                    failed = true;
                    break;
                }
                const uint64_t tile = u / n_bands, band = u - tile * n_bands;
                mbar_arrive_expect_tx(&full[st], kChorStageWords * 4u + qt_stage_bytes);
#pragma unroll
                for (uint32_t bx = 0; bx < NBOX; ++bx)
                    tma_load_2d(db_st + st * kChorStageWords + bx * RB * BOXW, &db_map, &full[st],
                                static_cast<int32_t>(tile * TW + bx * BOXW), static_cast<int32_t>(band * RB));
                tma_load_2d(qt_st + st * (2048 / 4), &qt_map, &full[st], 0, static_cast<int32_t>(band * RB));
            }
            // let every copy this thread issued land before the CTA can exit
            const uint32_t inflight = it < (uint32_t)kChorStages ? it : (uint32_t)kChorStages;
            for (uint32_t j = it - inflight; j < it; ++j) {
                const uint64_t t0 = global_ns();
                while (!mbar_test(&full[j % kChorStages], (j / kChorStages) & 1u))
                    if (global_ns() - t0 > QPADL_WAIT_NS) {
                        failed = true;
                        break;
                    }
            }
        }
    } else {
        // ---------------- consumers
        const uint32_t quad = threadIdx.x % QUADS, g = threadIdx.x / QUADS;
        const uint32_t bx = (quad * WPT) / BOXW, wx = (quad * WPT) % BOXW;
        // the group's QB selector bits: bits sh .. sh + QB - 1 of selector word g * QB / 32
        const uint32_t sw = (g * QB) / 32, sh = (g * QB) % 32;
        uint32_t acc[QB][WPT];
#pragma unroll
        for (int j = 0; j < QB; ++j)
#pragma unroll
            for (int k = 0; k < WPT; ++k) acc[j][k] = 0u;
        uint64_t cur_tile = u0 < u1 ? u0 / n_bands : 0;
        auto flush = [&](uint64_t tile) {
            const uint64_t w0 = tile * TW + quad * WPT;
#pragma unroll
            for (int j = 0; j < QB; ++j) {
                const uint32_t b = g * QB + j;
                if (b < B) {
                    uint32_t *o = out + (uint64_t)b * W + w0;
#pragma unroll
                    for (int k = 0; k < WPT; ++k)
                        if (w0 + k < W && acc[j][k]) atomicXor(o + k, acc[j][k]);
                }
#pragma unroll
                for (int k = 0; k < WPT; ++k) acc[j][k] = 0u;
            }
        };
        uint32_t it = 0;
        for (uint64_t u = u0; u < u1; ++u, ++it) {
            const uint64_t tile = u / n_bands, band = u - tile * n_bands;
            if (tile != cur_tile) {
                flush(cur_tile);
                cur_tile = tile;
            }
            const uint32_t st = it % kChorStages, ph = (it / kChorStages) & 1u;
            const bool ok = mbar_wait(&full[st], ph, abort);
            if (__any_sync(0xffffffffu, !ok)) {
                failed = true;
                break;
            }
            const uint32_t *rows = db_st + st * kChorStageWords + bx * RB * BOXW + wx;
            const uint32_t *sel = qt_st + st * (2048 / 4) + sw;
            const uint64_t row0 = band * RB;
            const uint32_t nrows = static_cast<uint32_t>(r - row0 < RB ? r - row0 : RB);
            for (uint32_t i = 0; i < nrows; ++i) {
                uint32_t d[WPT];
#pragma unroll
                for (int k = 0; k < WPT; k += 4) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(rows + i * BOXW + k);
                    d[k] = v.x;
                    d[k + 1] = v.y;
                    d[k + 2] = v.z;
                    d[k + 3] = v.w;
                }
                const uint32_t s = sel[i * qtw] >> sh;
#pragma unroll
                for (int j = 0; j < QB; ++j) {
                    if constexpr (PRED) {
                        if ((s >> j) & 1u) {
#pragma unroll
                            for (int k = 0; k < WPT; ++k) acc[j][k] ^= d[k];
                        }
                    } else {
                        const uint32_t m = static_cast<uint32_t>(static_cast<int32_t>(s << (31 - j)) >> 31);
#pragma unroll
                        for (int k = 0; k < WPT; ++k) acc[j][k] ^= d[k] & m;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
        if (!failed && u0 < u1) flush(cur_tile);
    }
    if (failed) {
        *abort = 1;
        *status = kDevTimeout;
    }
}

// ------------------------------------------------------------------ four Russians
constexpr uint32_t kM4TW = 64;                    // column tile (words)
constexpr uint32_t kM4RB = 64;                    // band (rows) = two query words
constexpr uint32_t kM4Tables = kM4RB / 4;         // 4-row tables per band
constexpr uint32_t kM4Quads = kM4TW / 4;          // 16: half a warp spans a tile row
constexpr int kM4QB = 16;                         // queries per thread
constexpr uint32_t kM4StageBytes = kM4RB * kM4TW * 4;          // 16 KB of database words
constexpr uint32_t kM4QWords = kM4RB / 32;                     // query words per band
constexpr uint32_t kM4QBytes = kM4QWords * kChorMaxBatch * 4;   // 2 KB of query words
constexpr uint32_t kM4TableBytes = kM4Tables * 16 * kM4TW * 4;  // 64 KB: [table][entry][quad] of uint4

// Q (B x qw words) -> QS (roundup(qw, 2) x 256 words): QS[k][b] = word k of
// query b (zero for b >= B or k >= qw; bits at positions >= r cleared).
__global__ void chor_words_kernel(const uint32_t *__restrict__ Q, uint64_t qw, uint32_t B, uint64_t r,
                                  uint32_t *__restrict__ QS) {
    const uint64_t total = (qw + kM4QWords - 1) / kM4QWords * kM4QWords * kChorMaxBatch;
    const uint32_t tail = static_cast<uint32_t>(r % 32);
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = e / kChorMaxBatch;
        const uint32_t b = static_cast<uint32_t>(e - k * kChorMaxBatch);
        uint32_t v = (b < B && k < qw) ? Q[(uint64_t)b * qw + k] : 0u;
        if (tail && k == qw - 1) v &= (1u << tail) - 1u;
        QS[e] = v;
    }
}

__global__ void __launch_bounds__(kChorThreads + 32, 1)
    chor_m4rm_kernel(const __grid_constant__ CUtensorMap db_map, const uint32_t *__restrict__ QS, uint64_t r,
                     uint32_t W, uint32_t B, uint32_t *__restrict__ out, int *__restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *db_st = smem;                                               // [stage] 32 rows x 128 words
    uint8_t *q_st = db_st + kChorStages * kM4StageBytes;                 // [stage] 256 query words
    uint8_t *tab = q_st + kChorStages * kM4QBytes;                       // [2][table][entry][quad] uint4
    uint64_t *full = reinterpret_cast<uint64_t *>(tab + 2 * kM4TableBytes);
    uint64_t *empty = full + kChorStages;
    uint64_t *built = empty + kChorStages;   // [2]: every consumer warp has written its part of table buffer b
    volatile int *abort = reinterpret_cast<volatile int *>(built + 2);

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kChorStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kChorThreads / 32);
        }
        mbar_init(&built[0], kChorThreads / 32);
        mbar_init(&built[1], kChorThreads / 32);
        *abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    const uint64_t n_tiles = (W + kM4TW - 1) / kM4TW;
    const uint64_t n_bands = (r + kM4RB - 1) / kM4RB;
    const uint64_t units = n_tiles * n_bands;
    const uint64_t u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
    bool failed = false;

    if (warp == kChorThreads / 32) {
        // ---------------- producer: database tile band + the band's query words
        if (lane == 0) {
            tma_prefetch_desc(&db_map);
            uint32_t it = 0;
            for (uint64_t u = u0; u < u1; ++u, ++it) {
                const uint32_t st = it % kChorStages, ph = (it / kChorStages) & 1u;
                if (!mbar_wait(&empty[st], ph ^ 1u, abort)) {
                    failed = true;
                    break;
                }
                const uint64_t tile = u / n_bands, band = u - tile * n_bands;
                mbar_arrive_expect_tx(&full[st], kM4StageBytes + kM4QBytes);
                tma_load_2d(db_st + st * kM4StageBytes, &db_map, &full[st], static_cast<int32_t>(tile * kM4TW),
                            static_cast<int32_t>(band * kM4RB));
                bulk_load(q_st + st * kM4QBytes, QS + band * kM4QWords * kChorMaxBatch, kM4QBytes, &full[st]);
            }
            const uint32_t inflight = it < (uint32_t)kChorStages ? it : (uint32_t)kChorStages;
            for (uint32_t j = it - inflight; j < it; ++j) {
                const uint64_t t0 = global_ns();
                while (!mbar_test(&full[j % kChorStages], (j / kChorStages) & 1u))
                    if (global_ns() - t0 > QPADL_WAIT_NS) {
                        failed = true;
                        break;
                    }
            }
        }
    } else {
        // ---------------- consumers: thread = (word quad of the tile, group of 16 queries)
        const uint32_t quad = lane & 15, g = warp * 2 + (lane >> 4);
        // table parts built by this thread: tables bt + 8 i, word quad bq, entries 8 hh .. 8 hh + 7
        const uint32_t bt = warp, bq = lane & 15, hh = lane >> 4;
        uint32_t acc[kM4QB][4];
#pragma unroll
        for (int j = 0; j < kM4QB; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0u;
        const bool active = g * kM4QB < B;
        uint64_t cur_tile = u0 < u1 ? u0 / n_bands : 0;
        auto flush = [&](uint64_t tile) {
            const uint64_t w0 = tile * kM4TW + quad * 4;
#pragma unroll
            for (int j = 0; j < kM4QB; ++j) {
                const uint32_t b = g * kM4QB + j;
                if (b < B) {
                    uint32_t *o = out + (uint64_t)b * W + w0;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (w0 + k < W && acc[j][k]) atomicXor(o + k, acc[j][k]);
                }
                acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0u;
            }
        };
        auto X = [](uint4 a, uint4 b) { return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w); };
        uint32_t it = 0;
        for (uint64_t u = u0; u < u1; ++u, ++it) {
            const uint64_t tile = u / n_bands;
            if (tile != cur_tile) {
                flush(cur_tile);
                cur_tile = tile;
            }
            const uint32_t st = it % kChorStages, ph = (it / kChorStages) & 1u;
            const bool ok = mbar_wait(&full[st], ph, abort);
            if (__any_sync(0xffffffffu, !ok)) {
                failed = true;
                break;
            }
#pragma unroll
            for (uint32_t half = 0; half < kM4Tables / 8; ++half) {
                // table bt + 8 half: entry m = XOR of the rows whose bit is set in m; entries 8..15 add row 3
                const uint32_t tb = bt + 8 * half;
                const uint4 *rows = reinterpret_cast<const uint4 *>(db_st + st * kM4StageBytes) + bq;
                const uint4 x0 = rows[(4 * tb + 0) * kM4Quads], x1 = rows[(4 * tb + 1) * kM4Quads];
                const uint4 x2 = rows[(4 * tb + 2) * kM4Quads];
                const uint4 z = hh ? rows[(4 * tb + 3) * kM4Quads] : make_uint4(0u, 0u, 0u, 0u);
                uint4 *Tq = reinterpret_cast<uint4 *>(tab + (it & 1u) * kM4TableBytes) + (tb * 16 + 8 * hh) * kM4Quads + bq;
                const uint4 x01 = X(x0, x1);
                Tq[0 * kM4Quads] = z;
                Tq[1 * kM4Quads] = X(z, x0);
                Tq[2 * kM4Quads] = X(z, x1);
                Tq[3 * kM4Quads] = X(z, x01);
                Tq[4 * kM4Quads] = X(z, x2);
                Tq[5 * kM4Quads] = X(X(z, x0), x2);
                Tq[6 * kM4Quads] = X(X(z, x1), x2);
                Tq[7 * kM4Quads] = X(X(z, x01), x2);
            }
            // query 32 warp + lane's words for the band's rows
            static_assert(kM4QWords == 2, "two query words per band");
            uint32_t qwd[kM4QWords];
#pragma unroll
            for (uint32_t k = 0; k < kM4QWords; ++k)
                qwd[k] = reinterpret_cast<const uint32_t *>(q_st + st * kM4QBytes)[k * kChorMaxBatch + warp * 32 + lane];
            // every warp's part of the tables must be written before any warp reads them; a bounded
            // mbarrier wait instead of a CTA barrier, so a warp that gave up cannot hang the others.
            // Buffer b = it & 1 completes a phase every second iteration.
            __syncwarp();
            if (lane == 0) mbar_arrive(&built[it & 1u]);
            const bool tok = mbar_wait(&built[it & 1u], (it >> 1) & 1u, abort);
            if (__any_sync(0xffffffffu, !tok)) {
                failed = true;
                break;
            }
            if (__any_sync(0xffffffffu, active)) {
                const uint4 *T0 = reinterpret_cast<const uint4 *>(tab + (it & 1u) * kM4TableBytes) + quad;
#pragma unroll 1
                for (uint32_t k = 0; k < kM4QWords; ++k) {
                    const uint32_t qk = k ? qwd[1] : qwd[0];
#pragma unroll
                    for (int j = 0; j < kM4QB; ++j) {
                        const uint32_t qv = __shfl_sync(0xffffffffu, qk, (lane & 16u) | static_cast<uint32_t>(j));
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            const uint4 v = T0[((8 * k + t) * 16 + ((qv >> (4 * t)) & 15u)) * kM4Quads];
                            acc[j][0] ^= v.x;
                            acc[j][1] ^= v.y;
                            acc[j][2] ^= v.z;
                            acc[j][3] ^= v.w;
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
        if (!failed && u0 < u1) flush(cur_tile);
    }
    if (failed) {
        *abort = 1;
        *status = kDevTimeout;
    }
}

// ------------------------------------------------------------------ host side
// Queries per thread (qb) and query groups per CTA (qg) for a batch; form bit 1 selects 8
// words per thread (then at most 16 queries per thread, for the registers), bit 0 the
// predicated XOR.
static bool chor_pick(uint32_t B, int form, int *qb, int *qg, int *wpt) {
    if (B == 0 || B > kChorMaxBatch || form < 0 || form > 3) return false;
    *wpt = (form & 2) ? 8 : 4;
    if (*wpt == 8) {
        int q = 1;
        while (q < static_cast<int>(B) && q < 16) q <<= 1;
        *qb = q;
        const uint32_t groups = (B + q - 1) / q;
        int g = 1;
        while (static_cast<uint32_t>(g) < groups) g <<= 1;
        *qg = g;
        return true;
    }
    if (B <= 32) {
        int q = 1;
        while (q < static_cast<int>(B)) q <<= 1;
        *qb = q;
        *qg = 1;
    } else {
        const uint32_t groups = (B + 31) / 32;
        int g = 2;
        while (static_cast<uint32_t>(g) < groups) g <<= 1;
        *qb = 32;
        *qg = g;
    }
    return true;
}

static int chor_smem_bytes() {
    return kChorStages * (kChorStageWords * 4 + 2048) + 2 * kChorStages * 8 + 16 + 1024;
}

template <int QB, int QG, int WPT, bool PRED>
static cudaError_t chor_attr1() {
    return cudaFuncSetAttribute(chor_answer_kernel<QB, QG, WPT, PRED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                chor_smem_bytes());
}

template <int QB, int QG>
static cudaError_t chor_attr() {
    cudaError_t e;
    if ((e = chor_attr1<QB, QG, 4, false>()) != cudaSuccess) return e;
    return chor_attr1<QB, QG, 4, true>();
}

template <int QB, int QG>
static cudaError_t chor_attr8() {
    cudaError_t e;
    if ((e = chor_attr1<QB, QG, 8, false>()) != cudaSuccess) return e;
    return chor_attr1<QB, QG, 8, true>();
}

static int chor_m4rm_smem_bytes() {
    return kChorStages * (kM4StageBytes + kM4QBytes) + 2 * kM4TableBytes + (2 * kChorStages + 2) * 8 + 16 + 1024;
}

cudaError_t prepare_chor_kernels() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(chor_m4rm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  chor_m4rm_smem_bytes())) != cudaSuccess)
        return e;
    if ((e = chor_attr<1, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<2, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<4, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<8, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<16, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<32, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<32, 2>()) != cudaSuccess) return e;
    if ((e = chor_attr<32, 4>()) != cudaSuccess) return e;
    if ((e = chor_attr<32, 8>()) != cudaSuccess) return e;
    if ((e = chor_attr8<1, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr8<2, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr8<4, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr8<8, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr8<16, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr8<16, 2>()) != cudaSuccess) return e;
    if ((e = chor_attr8<16, 4>()) != cudaSuccess) return e;
    if ((e = chor_attr8<16, 8>()) != cudaSuccess) return e;
    return chor_attr8<16, 16>();
}

bool chor_launch_shape(uint32_t B, int form, uint32_t *tw, uint32_t *rb, uint32_t *box_words, uint32_t *qtw) {
    int qb = 0, qg = 0, wpt = 0;
    if (!chor_pick(B, form, &qb, &qg, &wpt)) return false;
    *tw = chor_tw(qg, wpt);
    *rb = chor_rb(qg, wpt);
    *box_words = *tw < 256 ? *tw : 256;
    *qtw = chor_qtw(static_cast<uint32_t>((qg * qb + 31) / 32));
    return true;
}

cudaError_t launch_chor_transpose(const uint32_t *Q, uint64_t qw, uint32_t B, uint64_t r, uint32_t qtw, uint32_t *QT,
                                  int num_sms, cudaStream_t stream) {
    const uint64_t warps = qw * qtw;
    const uint64_t blocks = (warps + 7) / 8;
    const unsigned grid = static_cast<unsigned>(blocks < (uint64_t)num_sms * 16 ? (blocks ? blocks : 1) : num_sms * 16);
    chor_transpose_kernel<<<grid, 256, 0, stream>>>(Q, qw, B, r, qtw, QT);
    return cudaGetLastError();
}

template <int QB, int QG, int WPT, bool PRED>
static cudaError_t launch_qbg1(const CUtensorMap &db_map, const CUtensorMap &qt_map, uint64_t r, uint32_t W,
                               uint32_t B, uint32_t qtw, uint32_t *out, int num_sms, int *status,
                               cudaStream_t stream) {
    constexpr uint32_t TW = chor_tw(QG, WPT), RB = chor_rb(QG, WPT);
    const uint64_t units = ((W + TW - 1) / TW) * ((r + RB - 1) / RB);
    const int grid = static_cast<int>(units < (uint64_t)num_sms ? units : (uint64_t)num_sms);
    chor_answer_kernel<QB, QG, WPT, PRED><<<grid, kChorThreads + 32, chor_smem_bytes(), stream>>>(
        db_map, qt_map, r, W, B, qtw, out, status);
    return cudaGetLastError();
}

template <int QB, int QG, int WPT>
static cudaError_t launch_qbg(bool pred, const CUtensorMap &db_map, const CUtensorMap &qt_map, uint64_t r,
                              uint32_t W, uint32_t B, uint32_t qtw, uint32_t *out, int num_sms, int *status,
                              cudaStream_t stream) {
    return pred ? launch_qbg1<QB, QG, WPT, true>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream)
                : launch_qbg1<QB, QG, WPT, false>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream);
}

cudaError_t launch_chor_answer(const CUtensorMap &db_map, const CUtensorMap &qt_map, uint64_t r, uint32_t W,
                               uint32_t B, uint32_t qtw, uint32_t *out, int num_sms, int *status,
                               cudaStream_t stream, int form) {
    int qb = 0, qg = 0, wpt = 0;
    if (!chor_pick(B, form, &qb, &qg, &wpt)) return cudaErrorInvalidValue;
    const bool pred = (form & 1) != 0;
#define QPADL_CHOR_L(QB_, QG_, WPT_) \
    launch_qbg<QB_, QG_, WPT_>(pred, db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream)
    if (wpt == 8) {
        if (qg == 1) {
            switch (qb) {
                case 1: return QPADL_CHOR_L(1, 1, 8);
                case 2: return QPADL_CHOR_L(2, 1, 8);
                case 4: return QPADL_CHOR_L(4, 1, 8);
                case 8: return QPADL_CHOR_L(8, 1, 8);
                default: return QPADL_CHOR_L(16, 1, 8);
            }
        }
        switch (qg) {
            case 2: return QPADL_CHOR_L(16, 2, 8);
            case 4: return QPADL_CHOR_L(16, 4, 8);
            case 8: return QPADL_CHOR_L(16, 8, 8);
            default: return QPADL_CHOR_L(16, 16, 8);
        }
    }
    if (qg == 1) {
        switch (qb) {
            case 1: return QPADL_CHOR_L(1, 1, 4);
            case 2: return QPADL_CHOR_L(2, 1, 4);
            case 4: return QPADL_CHOR_L(4, 1, 4);
            case 8: return QPADL_CHOR_L(8, 1, 4);
            case 16: return QPADL_CHOR_L(16, 1, 4);
            default: return QPADL_CHOR_L(32, 1, 4);
        }
    }
    switch (qg) {
        case 2: return QPADL_CHOR_L(32, 2, 4);
        case 4: return QPADL_CHOR_L(32, 4, 4);
        default: return QPADL_CHOR_L(32, 8, 4);
    }
#undef QPADL_CHOR_L
}

cudaError_t launch_chor_words(const uint32_t *Q, uint64_t qw, uint32_t B, uint64_t r, uint32_t *QS, int num_sms,
                              cudaStream_t stream) {
    chor_words_kernel<<<num_sms * 4, 256, 0, stream>>>(Q, qw, B, r, QS);
    return cudaGetLastError();
}

cudaError_t launch_chor_m4rm(const CUtensorMap &db_map, const uint32_t *QS, uint64_t r, uint32_t W, uint32_t B,
                             uint32_t *out, int num_sms, int *status, cudaStream_t stream) {
    if (B == 0 || B > kChorMaxBatch) return cudaErrorInvalidValue;
    const uint64_t units = ((W + kM4TW - 1) / kM4TW) * ((r + kM4RB - 1) / kM4RB);
    const int grid = static_cast<int>(units < (uint64_t)num_sms ? units : (uint64_t)num_sms);
    chor_m4rm_kernel<<<grid, kChorThreads + 32, chor_m4rm_smem_bytes(), stream>>>(db_map, QS, r, W, B, out, status);
    return cudaGetLastError();
}

}  // namespace qpadl
