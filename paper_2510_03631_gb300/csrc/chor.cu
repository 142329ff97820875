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
// Every mbarrier wait is bounded (2 s of %globaltimer); a CTA that gives up
// raises the status word and leaves, no kernel traps.
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "chor.cuh"
#include "ptx.cuh"

namespace qpadl {

constexpr int kChorThreads = 256;          // consumer threads
constexpr int kChorStages = 4;
constexpr uint32_t kChorStageWords = 8192;  // 32 KB of database words per stage

// Column tile width and band height for QG query groups per CTA.
__host__ __device__ constexpr uint32_t chor_tw(int qg) { return 1024u / static_cast<uint32_t>(qg); }
__host__ __device__ constexpr uint32_t chor_rb(int qg) { return kChorStageWords / chor_tw(qg); }

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

template <int QB, int QG>
__global__ void __launch_bounds__(kChorThreads + 32, 1)
    chor_answer_kernel(const __grid_constant__ CUtensorMap db_map, const __grid_constant__ CUtensorMap qt_map,
                       uint64_t r, uint32_t W, uint32_t B, uint32_t qtw, uint32_t *__restrict__ out,
                       int *__restrict__ status) {
    constexpr uint32_t TW = chor_tw(QG);
    constexpr uint32_t RB = chor_rb(QG);
    constexpr uint32_t BOXW = TW < 256 ? TW : 256;   // words per TMA box row
    constexpr uint32_t NBOX = TW / BOXW;
    constexpr uint32_t QUADS = TW / 4;               // threads per query group
    static_assert(QUADS * QG == kChorThreads, "one thread per (word quad, query group)");
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
        const uint32_t bx = (quad * 4) / BOXW, wx = (quad * 4) % BOXW;
        uint32_t acc[QB][4];
#pragma unroll
        for (int j = 0; j < QB; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0u;
        uint64_t cur_tile = u0 < u1 ? u0 / n_bands : 0;
        auto flush = [&](uint64_t tile) {
            const uint64_t w0 = tile * TW + quad * 4;
#pragma unroll
            for (int j = 0; j < QB; ++j) {
                const uint32_t b = g * QB + j;
                if (b < B) {
                    uint32_t *o = out + (uint64_t)b * W + w0;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (w0 + k < W && acc[j][k]) atomicXor(o + k, acc[j][k]);
                }
                acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0u;
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
            const uint32_t *sel = qt_st + st * (2048 / 4) + g;
            const uint64_t row0 = band * RB;
            const uint32_t nrows = static_cast<uint32_t>(r - row0 < RB ? r - row0 : RB);
            for (uint32_t i = 0; i < nrows; ++i) {
                const uint4 d = *reinterpret_cast<const uint4 *>(rows + i * BOXW);
                const uint32_t s = sel[i * qtw];
#pragma unroll
                for (int j = 0; j < QB; ++j) {
                    const uint32_t m = static_cast<uint32_t>(static_cast<int32_t>(s << (31 - j)) >> 31);
                    acc[j][0] ^= d.x & m;
                    acc[j][1] ^= d.y & m;
                    acc[j][2] ^= d.z & m;
                    acc[j][3] ^= d.w & m;
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
static bool chor_pick(uint32_t B, int *qb, int *qg) {
    if (B == 0 || B > kChorMaxBatch) return false;
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

template <int QB, int QG>
static int chor_smem_bytes() {
    return kChorStages * (kChorStageWords * 4 + 2048) + 2 * kChorStages * 8 + 16 + 1024;
}

template <int QB, int QG>
static cudaError_t chor_attr() {
    return cudaFuncSetAttribute(chor_answer_kernel<QB, QG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                chor_smem_bytes<QB, QG>());
}

cudaError_t prepare_chor_kernels() {
    cudaError_t e;
    if ((e = chor_attr<1, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<2, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<4, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<8, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<16, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<32, 1>()) != cudaSuccess) return e;
    if ((e = chor_attr<32, 2>()) != cudaSuccess) return e;
    if ((e = chor_attr<32, 4>()) != cudaSuccess) return e;
    return chor_attr<32, 8>();
}

bool chor_launch_shape(uint32_t B, uint32_t *tw, uint32_t *rb, uint32_t *box_words, uint32_t *qtw) {
    int qb = 0, qg = 0;
    if (!chor_pick(B, &qb, &qg)) return false;
    *tw = chor_tw(qg);
    *rb = chor_rb(qg);
    *box_words = *tw < 256 ? *tw : 256;
    *qtw = chor_qtw(static_cast<uint32_t>(qg));
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

template <int QB, int QG>
static cudaError_t launch_qbg(const CUtensorMap &db_map, const CUtensorMap &qt_map, uint64_t r, uint32_t W,
                              uint32_t B, uint32_t qtw, uint32_t *out, int num_sms, int *status, cudaStream_t stream) {
    const uint64_t units = ((W + chor_tw(QG) - 1) / chor_tw(QG)) * ((r + chor_rb(QG) - 1) / chor_rb(QG));
    const int grid = static_cast<int>(units < (uint64_t)num_sms ? units : (uint64_t)num_sms);
    chor_answer_kernel<QB, QG><<<grid, kChorThreads + 32, chor_smem_bytes<QB, QG>(), stream>>>(db_map, qt_map, r, W, B,
                                                                                              qtw, out, status);
    return cudaGetLastError();
}

cudaError_t launch_chor_answer(const CUtensorMap &db_map, const CUtensorMap &qt_map, uint64_t r, uint32_t W,
                               uint32_t B, uint32_t qtw, uint32_t *out, int num_sms, int *status,
                               cudaStream_t stream) {
    int qb = 0, qg = 0;
    if (!chor_pick(B, &qb, &qg)) return cudaErrorInvalidValue;
    if (qg == 1) {
        switch (qb) {
            case 1: return launch_qbg<1, 1>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream);
            case 2: return launch_qbg<2, 1>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream);
            case 4: return launch_qbg<4, 1>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream);
            case 8: return launch_qbg<8, 1>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream);
            case 16: return launch_qbg<16, 1>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream);
            default: return launch_qbg<32, 1>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream);
        }
    }
    switch (qg) {
        case 2: return launch_qbg<32, 2>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream);
        case 4: return launch_qbg<32, 4>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream);
        default: return launch_qbg<32, 8>(db_map, qt_map, r, W, B, qtw, out, num_sms, status, stream);
    }
}

}  // namespace qpadl
