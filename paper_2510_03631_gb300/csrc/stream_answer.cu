// Streaming Response: ans = D * qu mod 2^32 for one (or a few) queries.
//
// This is the server's product of the query with the whole database matrix
// (QPADL Sec. 5.2; Def. 1 DB.Query.Response), accumulated mod q as in Alg. 4.
// It reads every byte of D once and is bound by HBM bandwidth, so the design
// is about keeping enough bytes in flight and spending few instructions per
// byte:
//  - Persistent grid, one CTA per SM.  Each CTA owns a contiguous band of
//    rows (8-row granularity, so bands differ by at most 8 rows) and streams
//    it chunk by chunk (256 columns) through a 3-stage shared-memory ring
//    filled by TMA (one 2-D box per 8 rows) from a single producer thread.
//  - The query is pre-split into byte limbs: for each group of 4 columns,
//    limb plane k holds byte k of the 4 query words.  A database word (4
//    digits) times a limb word is one dp4a, so 16 digits x 4 limbs = 16 dp4a
//    and no byte unpacking.  Per row the four limb sums recombine exactly
//    as sum_k 2^{8k} acc_k (mod 2^32): D*q = sum_k 2^{8k} (D*limb_k).
//  - 16 consumer warps: thread (row-lane rl, column group cg) covers 16
//    digits of up to 8 rows per stage and keeps its partial sums in
//    registers for the whole band; at the end one 16-lane shuffle reduction
//    per row gives the row total.  No atomics, no second pass.
#include <cstdint>
#include <cuda_runtime.h>

#include "ptx.cuh"
#include "stream_answer.cuh"

namespace qpadl {

template <int NQ>
struct StreamCfg {
    static constexpr int kRowsPerThread = 8 / NQ;
    static constexpr int kSpan = kStreamRowLanes * kRowsPerThread;   // rows per band span
    static constexpr int kDbStageBytes = kSpan * kStreamChunkCols;
    static constexpr int kQStageBytes = NQ * kStreamChunkCols * 4;
    static constexpr int kSmemBytes = kStreamStages * (kDbStageBytes + kQStageBytes) + 256 + 1024;
};

// byte-limb packing of the query: see the file comment
__global__ void pack_query_kernel(const uint32_t *__restrict__ q, uint64_t q_ld, uint32_t C, uint32_t nchunks,
                                  uint32_t *__restrict__ qpack, uint64_t pack_ld) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;   // group of 4 columns
    const uint32_t b = blockIdx.y;
    if (g >= nchunks * (kStreamChunkCols / 4)) return;
    const uint32_t *qb = q + b * q_ld;
    const uint32_t c = 4 * g;
    uint32_t a0 = c + 0 < C ? qb[c + 0] : 0u;
    uint32_t a1 = c + 1 < C ? qb[c + 1] : 0u;
    uint32_t a2 = c + 2 < C ? qb[c + 2] : 0u;
    uint32_t a3 = c + 3 < C ? qb[c + 3] : 0u;
    // t01 = [a.b0 b.b0 a.b1 b.b1], t23 = [c.b0 d.b0 c.b1 d.b1], ...
    const uint32_t lo01 = __byte_perm(a0, a1, 0x5140);
    const uint32_t lo23 = __byte_perm(a2, a3, 0x5140);
    const uint32_t hi01 = __byte_perm(a0, a1, 0x7362);
    const uint32_t hi23 = __byte_perm(a2, a3, 0x7362);
    const uint32_t L0 = __byte_perm(lo01, lo23, 0x5410);
    const uint32_t L1 = __byte_perm(lo01, lo23, 0x7632);
    const uint32_t L2 = __byte_perm(hi01, hi23, 0x5410);
    const uint32_t L3 = __byte_perm(hi01, hi23, 0x7632);
    const uint32_t chunk = g / (kStreamChunkCols / 4);
    const uint32_t gi = g % (kStreamChunkCols / 4);
    uint32_t *dst = qpack + b * pack_ld + chunk * kStreamChunkCols + gi;
    dst[0 * (kStreamChunkCols / 4)] = L0;
    dst[1 * (kStreamChunkCols / 4)] = L1;
    dst[2 * (kStreamChunkCols / 4)] = L2;
    dst[3 * (kStreamChunkCols / 4)] = L3;
}

__device__ __forceinline__ bool drain_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > QPADL_WAIT_NS) return false;
    }
    return true;
}

template <int NQ>
__global__ void __launch_bounds__(kStreamThreads, 1)
    stream_answer_kernel(const __grid_constant__ CUtensorMap db_map, const uint32_t *__restrict__ qpack,
                         uint64_t pack_ld, uint32_t *__restrict__ ans, uint64_t ans_ld, uint32_t R,
                         uint32_t nchunks, int *__restrict__ status) {
    using Cfg = StreamCfg<NQ>;
    constexpr int RPT = Cfg::kRowsPerThread;
    constexpr int SPAN = Cfg::kSpan;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *db_st = smem;                                                   // [stages][SPAN*256]
    uint32_t *q_st = reinterpret_cast<uint32_t *>(smem + kStreamStages * Cfg::kDbStageBytes);  // [stages][NQ][256]
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStreamStages * (Cfg::kDbStageBytes + Cfg::kQStageBytes));
    uint64_t *empty = full + kStreamStages;
    volatile int *abort = reinterpret_cast<volatile int *>(empty + kStreamStages);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStreamStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kStreamConsumerWarps);
        }
        *abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    // this CTA's band of rows, in 8-row octets
    const uint32_t n_oct = (R + 7) / 8;
    const uint32_t oct0 = static_cast<uint32_t>((uint64_t)blockIdx.x * n_oct / gridDim.x);
    const uint32_t oct1 = static_cast<uint32_t>((uint64_t)(blockIdx.x + 1) * n_oct / gridDim.x);
    const uint32_t band_oct = oct1 - oct0;
    const uint32_t nspan = (band_oct * 8 + SPAN - 1) / SPAN;

    if (warp == 0) {
        // ---------------- producer
        if (lane == 0) {
            tma_prefetch_desc(&db_map);
            uint32_t it = 0;
            bool ok = true;
            for (uint32_t sp = 0; sp < nspan && ok; ++sp) {
                const uint32_t so0 = oct0 + sp * band_oct / nspan;
                const uint32_t so1 = oct0 + (sp + 1) * band_oct / nspan;
                for (uint32_t c = 0; c < nchunks; ++c, ++it) {
                    const uint32_t st = it % kStreamStages;
                    const uint32_t ph = (it / kStreamStages) & 1u;
                    if (!mbar_wait(&empty[st], ph ^ 1u, abort)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bytes = (so1 - so0) * 8u * kStreamChunkCols + NQ * kStreamChunkCols * 4u;
                    mbar_arrive_expect_tx(&full[st], bytes);
                    uint8_t *dst = db_st + st * Cfg::kDbStageBytes;
                    for (uint32_t o = so0; o < so1; ++o)
                        tma_load_2d(dst + (o - so0) * 8 * kStreamChunkCols, &db_map, &full[st],
                                    static_cast<int32_t>(c * kStreamChunkCols), static_cast<int32_t>(o * 8));
                    uint32_t *qdst = q_st + st * (Cfg::kQStageBytes / 4);
#pragma unroll
                    for (int b = 0; b < NQ; ++b)
                        bulk_load(qdst + b * kStreamChunkCols, qpack + b * pack_ld + (uint64_t)c * kStreamChunkCols,
                                  kStreamChunkCols * 4u, &full[st]);
                }
            }
            // never leave while copies issued by this thread are still landing
            const uint32_t inflight = it < (uint32_t)kStreamStages ? it : (uint32_t)kStreamStages;
            for (uint32_t j = it - inflight; j < it; ++j) {
                if (!drain_wait(&full[j % kStreamStages], (j / kStreamStages) & 1u)) ok = false;
            }
            if (!ok) *status = kDevTimeout;
        }
        return;
    }

    // ---------------- consumers
    const int ct = threadIdx.x - 32;
    const int cg = ct % kStreamColGroups;   // 16-digit column group within the chunk
    const int rl = ct / kStreamColGroups;   // row lane
    uint32_t it = 0;
    for (uint32_t sp = 0; sp < nspan; ++sp) {
        const uint32_t so0 = oct0 + sp * band_oct / nspan;
        const uint32_t so1 = oct0 + (sp + 1) * band_oct / nspan;
        const uint32_t span_rows = (so1 - so0) * 8;
        uint32_t acc[RPT][NQ][4];
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int b = 0; b < NQ; ++b)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[r][b][k] = 0u;

        for (uint32_t c = 0; c < nchunks; ++c, ++it) {
            const uint32_t st = it % kStreamStages;
            const uint32_t ph = (it / kStreamStages) & 1u;
            if (!mbar_wait(&full[st], ph, abort)) {
                *status = kDevTimeout;
                return;
            }
            const uint32_t *qs = q_st + st * (Cfg::kQStageBytes / 4);
            const uint8_t *ds = db_st + st * Cfg::kDbStageBytes + cg * 16;
#pragma unroll
            for (int b = 0; b < NQ; ++b) {
                uint4 L[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    L[k] = *reinterpret_cast<const uint4 *>(qs + b * kStreamChunkCols + k * (kStreamChunkCols / 4) +
                                                            cg * 4);
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const uint32_t row = rl + r * kStreamRowLanes;
                    if (row < span_rows) {
                        const uint4 w = *reinterpret_cast<const uint4 *>(ds + row * kStreamChunkCols);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            uint32_t a = acc[r][b][k];
                            a = __dp4a(w.x, L[k].x, a);
                            a = __dp4a(w.y, L[k].y, a);
                            a = __dp4a(w.z, L[k].z, a);
                            a = __dp4a(w.w, L[k].w, a);
                            acc[r][b][k] = a;
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }

        // recombine limbs, reduce over the 16 column groups of each row, store
        const uint32_t row_base = so0 * 8;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
#pragma unroll
            for (int b = 0; b < NQ; ++b) {
                uint32_t v = acc[r][b][0] + (acc[r][b][1] << 8) + (acc[r][b][2] << 16) + (acc[r][b][3] << 24);
                v += __shfl_xor_sync(0xffffffffu, v, 8, 16);
                v += __shfl_xor_sync(0xffffffffu, v, 4, 16);
                v += __shfl_xor_sync(0xffffffffu, v, 2, 16);
                v += __shfl_xor_sync(0xffffffffu, v, 1, 16);
                const uint32_t row = row_base + rl + r * kStreamRowLanes;
                if (cg == 0 && rl + r * kStreamRowLanes < span_rows && row < R) ans[b * ans_ld + row] = v;
            }
        }
    }
}

// Generic fallback for shapes/alignments the TMA path cannot take (C not a
// multiple of 16, unaligned pointers): one warp per row, plain loads.
__global__ void rowwise_answer_kernel(const uint8_t *__restrict__ D, uint64_t R, uint64_t C,
                                      const uint32_t *__restrict__ Q, uint64_t q_ld, uint32_t B,
                                      uint32_t *__restrict__ ans, uint64_t ans_ld) {
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < R; i += warps) {
        const uint8_t *row = D + i * C;
        for (uint32_t b = 0; b < B; ++b) {
            const uint32_t *q = Q + b * q_ld;
            uint32_t acc = 0;
            for (uint64_t j = lane; j < C; j += 32) acc += static_cast<uint32_t>(row[j]) * q[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) ans[b * ans_ld + i] = acc;
        }
    }
}

// ------------------------------------------------------------------ host side
int stream_smem_bytes(int nq) {
    switch (nq) {
        case 1: return StreamCfg<1>::kSmemBytes;
        case 2: return StreamCfg<2>::kSmemBytes;
        case 4: return StreamCfg<4>::kSmemBytes;
        default: return -1;
    }
}

cudaError_t launch_pack_query(const uint32_t *q, uint64_t q_ld, uint32_t C, uint32_t nq, uint32_t *qpack,
                              uint64_t pack_ld, cudaStream_t stream) {
    const uint32_t nchunks = (C + kStreamChunkCols - 1) / kStreamChunkCols;
    const uint32_t groups = nchunks * (kStreamChunkCols / 4);
    dim3 grid((groups + 255) / 256, nq);
    pack_query_kernel<<<grid, 256, 0, stream>>>(q, q_ld, C, nchunks, qpack, pack_ld);
    return cudaGetLastError();
}

template <int NQ>
static cudaError_t set_stream_attr() {
    return cudaFuncSetAttribute(stream_answer_kernel<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                StreamCfg<NQ>::kSmemBytes);
}

cudaError_t prepare_stream_kernels() {
    cudaError_t e;
    if ((e = set_stream_attr<1>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<2>()) != cudaSuccess) return e;
    return set_stream_attr<4>();
}

template <int NQ>
static cudaError_t launch_stream_nq(const CUtensorMap &map, const uint32_t *qpack, uint64_t pack_ld, uint32_t *ans,
                                    uint64_t ans_ld, uint32_t R, uint32_t C, int grid, int *status,
                                    cudaStream_t stream) {
    const uint32_t nchunks = (C + kStreamChunkCols - 1) / kStreamChunkCols;
    stream_answer_kernel<NQ><<<grid, kStreamThreads, StreamCfg<NQ>::kSmemBytes, stream>>>(
        map, qpack, pack_ld, ans, ans_ld, R, nchunks, status);
    return cudaGetLastError();
}

cudaError_t launch_stream_answer(int nq, const CUtensorMap &map, const uint32_t *qpack, uint64_t pack_ld,
                                 uint32_t *ans, uint64_t ans_ld, uint32_t R, uint32_t C, int num_sms, int *status,
                                 cudaStream_t stream) {
    const uint32_t n_oct = (R + 7) / 8;
    const int grid = static_cast<int>(n_oct < (uint32_t)num_sms ? n_oct : (uint32_t)num_sms);
    switch (nq) {
        case 1: return launch_stream_nq<1>(map, qpack, pack_ld, ans, ans_ld, R, C, grid, status, stream);
        case 2: return launch_stream_nq<2>(map, qpack, pack_ld, ans, ans_ld, R, C, grid, status, stream);
        case 4: return launch_stream_nq<4>(map, qpack, pack_ld, ans, ans_ld, R, C, grid, status, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rowwise_answer(const uint8_t *D, uint64_t R, uint64_t C, const uint32_t *Q, uint64_t q_ld,
                                  uint32_t B, uint32_t *ans, uint64_t ans_ld, int num_sms, cudaStream_t stream) {
    uint64_t blocks = (R + 7) / 8;
    const uint64_t cap = (uint64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    rowwise_answer_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(D, R, C, Q, q_ld, B, ans, ans_ld);
    return cudaGetLastError();
}

}  // namespace qpadl
