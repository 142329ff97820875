// Streaming Response: ans = D * qu mod 2^32 for one (or a few) queries.
//
// This is the server's product of the query with the whole database matrix
// (QPADL Sec. 5.2; Def. 1 DB.Query.Response), accumulated mod q as in Alg. 4.
// It reads every byte of D once and is bound by HBM bandwidth, so the design
// is about a DRAM-friendly access pattern, enough bytes in flight, and few
// instructions per byte:
//  - Persistent grid, one CTA per SM.  CTA b owns rows [b R / G, (b+1) R / G)
//    (bands differ by at most one row) and streams them in spans of up to
//    SR rows.  A stage is SR rows x CCH contiguous digits per row (CCH =
//    512..4096 bytes) in a shared-memory ring filled by one producer thread.
//    The copy engine is limited by copy instructions rather than bytes
//    (about 100 cycles per copy), so the producer moves 16 KB per
//    instruction (16384/CCH rows x CCH digits) with a 3-D tensor map
//    (256 digits x C/256 x R) and uses one plain bulk copy per row only for
//    rows left over below a whole box, or when C is not a multiple of 256.
//  - The query is pre-split into byte limbs: for each group of 4 columns,
//    limb plane k holds byte k of the 4 query words.  A database word (4
//    digits) times a limb word is one dp4a, so 16 digits x 4 limbs = 16 dp4a
//    and no byte unpacking.  Per row the four limb sums recombine exactly as
//    sum_k 2^{8k} acc_k (mod 2^32), since D*q = sum_k 2^{8k} (D*limb_k).
//  - 16 consumer warps: thread (row lane rl, column group cg) covers 16
//    digits of up to RPT rows per stage and keeps its partial sums in
//    registers for the whole span; at the end of a span a warp shuffle and
//    a small shared-memory step reduce each row.  No atomics, no second pass.
#include <cstdint>
#include <cstring>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "ptx.cuh"
#include "stream_answer.cuh"

namespace qpadl {

// Where a stage's query operand comes from.
constexpr int kQPacked = 0;   // NQ queries pre-packed into byte-limb planes (pack_query_kernel)
constexpr int kQRaw = 1;      // NQ (1 or 2) raw queries (uint32 words); limbs are packed per thread

template <int NQ, int CCH, int QM = kQPacked>
struct StreamCfg {
    static constexpr int kGroups = CCH / 16;                       // 16-digit groups per row chunk
    static constexpr int kRowLanes = 32 * kStreamConsumerWarps / kGroups;
    static constexpr int kRowsPerThread = 8 / NQ;
    static constexpr int kSpan = kRowLanes * kRowsPerThread;       // rows per span (= per stage)
    static constexpr int kWarpsPerRow = kGroups / 32;
    static constexpr int kBoxRows = 16384 / CCH;                   // every 3-D box moves 16 KB
    static constexpr int kDbStageBytes = kSpan * CCH;
    // packed limbs or raw words of NQ queries (4 bytes per digit either way)
    static constexpr int kQStageBytes = NQ * CCH * 4;
    static constexpr int kStageBytes = kDbStageBytes + kQStageBytes;
    static constexpr int kStages = (220 * 1024) / kStageBytes > 4 ? 4 : (220 * 1024) / kStageBytes;
    static constexpr int kRedBytes = NQ * kSpan * kWarpsPerRow * 4;
    static constexpr int kSmemBytes = kStages * kStageBytes + kRedBytes + 256 + 1024;
    static_assert(kGroups % 32 == 0, "a warp must cover one row lane");
    static_assert(kSpan % kBoxRows == 0, "spans hold whole boxes");
    static_assert(kStages >= 2, "need at least double buffering");
};

// byte-limb packing of the query: chunk c of CCH columns holds 4 planes of
// CCH/4 words; word g of plane k = byte k of the 4 query words of columns
// 4g..4g+3 of the chunk.  Columns >= C are packed as zero.
__global__ void pack_query_kernel(const uint32_t *__restrict__ q, uint64_t q_ld, uint32_t C, uint32_t cch,
                                  uint32_t nchunks, uint32_t *__restrict__ qpack, uint64_t pack_ld) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;   // group of 4 columns
    const uint32_t b = blockIdx.y;
    const uint32_t gpc = cch / 4;                                 // groups per chunk
    if (g >= nchunks * gpc) return;
    const uint32_t *qb = q + b * q_ld;
    const uint32_t c = 4 * g;
    const uint32_t a0 = c + 0 < C ? qb[c + 0] : 0u;
    const uint32_t a1 = c + 1 < C ? qb[c + 1] : 0u;
    const uint32_t a2 = c + 2 < C ? qb[c + 2] : 0u;
    const uint32_t a3 = c + 3 < C ? qb[c + 3] : 0u;
    // lo01 = [a0.b0 a1.b0 a0.b1 a1.b1], lo23 likewise; hi* hold bytes 2 and 3
    const uint32_t lo01 = __byte_perm(a0, a1, 0x5140);
    const uint32_t lo23 = __byte_perm(a2, a3, 0x5140);
    const uint32_t hi01 = __byte_perm(a0, a1, 0x7362);
    const uint32_t hi23 = __byte_perm(a2, a3, 0x7362);
    uint32_t *dst = qpack + b * pack_ld + (g / gpc) * cch + (g % gpc);
    dst[0 * gpc] = __byte_perm(lo01, lo23, 0x5410);
    dst[1 * gpc] = __byte_perm(lo01, lo23, 0x7632);
    dst[2 * gpc] = __byte_perm(hi01, hi23, 0x5410);
    dst[3 * gpc] = __byte_perm(hi01, hi23, 0x7632);
}

__device__ __forceinline__ bool drain_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > QPADL_WAIT_NS) return false;
    }
    return true;
}

// Epilogues: what happens to the finished row total v of row `row` (vector b).
struct AnswerEpi {   // Response: store the answer word
    uint32_t *ans;
    uint64_t ld;
    __device__ __forceinline__ void operator()(uint32_t row, int b, uint32_t v) const { ans[b * ld + row] = v; }
};
__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kStreamConsumerWarps) : "memory");
}

// D: R rows of C digits.
//  kQPacked: NQ packed queries (pack_ld words apart).
//  kQRaw:    NQ (1 or 2) raw queries (pack_ld words apart); each thread
//            byte-permutes its 16 words of each query into the 4 limb words
//            of each 4-digit group.
// Launched with programmatic dependent launch: the kernel lets its successor
// be scheduled at once and waits (griddepcontrol.wait) for its predecessor
// before it reads anything the predecessor may have written.  The database
// of a Response is immutable while bound to a handle, so the Response
// producer issues its first stages of database loads before that wait.
template <int NQ, int CCH, int QM, class Epi>
__global__ void __launch_bounds__(kStreamThreads, 1)
    stream_answer_kernel(const __grid_constant__ CUtensorMap map, int use_map, const uint8_t *__restrict__ D,
                         uint32_t R, uint32_t C, const uint32_t *__restrict__ qsrc, uint64_t pack_ld, Epi epi,
                         int *__restrict__ status) {
    using Cfg = StreamCfg<NQ, CCH, QM>;
    static_assert(QM == kQPacked || NQ <= 2, "the raw form serves one or two queries");
    constexpr int RPT = Cfg::kRowsPerThread;
    constexpr int SR = Cfg::kSpan;
    constexpr int ST = Cfg::kStages;
    constexpr int G = Cfg::kGroups;
    constexpr int RL = Cfg::kRowLanes;
    constexpr int WPR = Cfg::kWarpsPerRow;
    constexpr uint32_t BR = Cfg::kBoxRows;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *db_st = smem;                                                           // [ST][SR][CCH]
    uint32_t *q_st = reinterpret_cast<uint32_t *>(smem + ST * Cfg::kDbStageBytes);   // [ST][kQStageBytes]
    uint32_t *red = reinterpret_cast<uint32_t *>(smem + ST * Cfg::kStageBytes);      // [NQ][SR][WPR]
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + ST * Cfg::kStageBytes + Cfg::kRedBytes);
    uint64_t *empty = full + ST;
    volatile int *abort = reinterpret_cast<volatile int *>(empty + ST);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kStreamConsumerWarps);
        }
        *abort = 0;
        fence_barrier_init();
        griddep_launch_dependents();
    }
    __syncthreads();

    const uint32_t r0 = static_cast<uint32_t>((uint64_t)blockIdx.x * R / gridDim.x);
    const uint32_t r1 = static_cast<uint32_t>((uint64_t)(blockIdx.x + 1) * R / gridDim.x);
    const uint32_t band = r1 - r0;
    const uint32_t nspan = (band + SR - 1) / SR;
    const uint32_t nchunks = (C + CCH - 1) / CCH;

    if (warp == 0) {
        // ---------------- producer
        if (lane == 0) {
            if (use_map) tma_prefetch_desc(&map);
            bool waited = false;
            uint32_t pend_st[ST], pend_c[ST], npend = 0;   // stages whose query load waits for the dependency
            const uint32_t total = nspan * nchunks;
            uint32_t it = 0;
            bool ok = true;
            auto load_query = [&](uint32_t st, uint32_t c) {
                const uint32_t c0 = c * CCH;
                const uint32_t bytes = (C - c0) < (uint32_t)CCH ? (C - c0) : (uint32_t)CCH;
                uint32_t *qdst = q_st + st * (Cfg::kQStageBytes / 4);
                if (QM == kQRaw) {
#pragma unroll
                    for (int b = 0; b < NQ; ++b)
                        bulk_load(qdst + b * CCH, qsrc + b * pack_ld + c0, bytes * 4u, &full[st]);
                } else {
#pragma unroll
                    for (int b = 0; b < NQ; ++b)
                        bulk_load(qdst + b * CCH, qsrc + b * pack_ld + (uint64_t)c * CCH, CCH * 4u, &full[st]);
                }
            };
            for (uint32_t sp = 0; sp < nspan && ok; ++sp) {
                const uint32_t s0 = r0 + sp * SR;
                const uint32_t s1 = (s0 + SR < r1) ? s0 + SR : r1;
                const uint32_t nbox = use_map ? (s1 - s0) / BR : 0;
                for (uint32_t c = 0; c < nchunks; ++c, ++it) {
                    const uint32_t st = it % ST;
                    const uint32_t ph = (it / ST) & 1u;
                    if (!mbar_wait(&empty[st], ph ^ 1u, abort)) {
                        ok = false;
                        break;
                    }
                    const uint32_t c0 = c * CCH;
                    const uint32_t bytes = (C - c0) < (uint32_t)CCH ? (C - c0) : (uint32_t)CCH;
                    const uint32_t qbytes = QM == kQRaw ? NQ * bytes * 4u : NQ * CCH * 4u;
                    mbar_arrive_expect_tx(&full[st], nbox * BR * CCH + (s1 - s0 - BR * nbox) * bytes + qbytes);
                    uint8_t *dst = db_st + st * Cfg::kDbStageBytes;
                    for (uint32_t b = 0; b < nbox; ++b)
                        tma_load_3d(dst + b * BR * CCH, &map, &full[st], 0, static_cast<int32_t>(c0 / 256),
                                    static_cast<int32_t>(s0 + BR * b));
                    const uint8_t *src = D + (uint64_t)s0 * C + c0;
                    for (uint32_t r = BR * nbox; r < s1 - s0; ++r)
                        bulk_load(dst + r * CCH, src + (uint64_t)r * C, bytes, &full[st]);
                    if (waited) {
                        load_query(st, c);
                    } else {
                        pend_st[npend] = st;
                        pend_c[npend] = c;
                        ++npend;
                        if (npend == (uint32_t)ST || it + 1 == total) {
                            griddep_wait();
                            waited = true;
                            for (uint32_t j = 0; j < npend; ++j) load_query(pend_st[j], pend_c[j]);
                            npend = 0;
                        }
                    }
                }
            }
            if (!waited) {   // aborted before the first query loads: their stages are owed bytes
                griddep_wait();
                for (uint32_t j = 0; j < npend; ++j) load_query(pend_st[j], pend_c[j]);
            }
            // never leave while copies issued by this thread are still landing
            const uint32_t inflight = it < (uint32_t)ST ? it : (uint32_t)ST;
            for (uint32_t j = it - inflight; j < it; ++j)
                if (!drain_wait(&full[j % ST], (j / ST) & 1u)) ok = false;
            if (!ok && status) *status = kDevTimeout;
        }
        return;
    }

    // ---------------- consumers
    griddep_wait();
    const int ct = threadIdx.x - 32;
    const int cg = ct % G;           // 16-digit column group within the chunk
    const int rl = ct / G;           // row lane
    const int wir = cg / 32;         // warp index within its row lane
    uint32_t it = 0;
    for (uint32_t sp = 0; sp < nspan; ++sp) {
        const uint32_t s0 = r0 + sp * SR;
        const uint32_t span_rows = (s0 + SR < r1) ? SR : r1 - s0;
        uint32_t acc[RPT][NQ][4];
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int b = 0; b < NQ; ++b)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[r][b][k] = 0u;

        for (uint32_t c = 0; c < nchunks; ++c, ++it) {
            const uint32_t st = it % ST;
            const uint32_t ph = (it / ST) & 1u;
            if (!mbar_wait(&full[st], ph, abort)) {
                if (status) *status = kDevTimeout;
                return;
            }
            const uint32_t *qs = q_st + st * (Cfg::kQStageBytes / 4);
            const uint8_t *ds = db_st + st * Cfg::kDbStageBytes + cg * 16;
#pragma unroll
            for (int b = 0; b < NQ; ++b) {
                uint4 L[4];
                if (QM == kQRaw) {
                    // 16 query words of this thread's digits -> limb word k of each 4-digit group
                    // (groups past column C hold stale words: use zero limbs there)
                    const bool valid = c * CCH + cg * 16 < C;
                    uint32_t l[4][4];   // [group][limb]
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        uint4 a = make_uint4(0u, 0u, 0u, 0u);
                        if (valid) a = *reinterpret_cast<const uint4 *>(qs + b * CCH + cg * 16 + 4 * i);
                        const uint32_t lo01 = __byte_perm(a.x, a.y, 0x5140);
                        const uint32_t lo23 = __byte_perm(a.z, a.w, 0x5140);
                        const uint32_t hi01 = __byte_perm(a.x, a.y, 0x7362);
                        const uint32_t hi23 = __byte_perm(a.z, a.w, 0x7362);
                        l[i][0] = __byte_perm(lo01, lo23, 0x5410);
                        l[i][1] = __byte_perm(lo01, lo23, 0x7632);
                        l[i][2] = __byte_perm(hi01, hi23, 0x5410);
                        l[i][3] = __byte_perm(hi01, hi23, 0x7632);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) L[k] = make_uint4(l[0][k], l[1][k], l[2][k], l[3][k]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        L[k] = *reinterpret_cast<const uint4 *>(qs + b * CCH + k * (CCH / 4) + cg * 4);
                }
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const uint32_t row = rl + r * RL;
                    if (row < span_rows) {
                        const uint4 w = *reinterpret_cast<const uint4 *>(ds + row * CCH);
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

        // recombine limbs, reduce each row over its column groups, store
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
#pragma unroll
            for (int b = 0; b < NQ; ++b) {
                uint32_t v = acc[r][b][0] + (acc[r][b][1] << 8) + (acc[r][b][2] << 16) + (acc[r][b][3] << 24);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (WPR == 1) {
                    // one warp covers the whole chunk: the row total is complete
                    const uint32_t row = rl + r * RL;
                    if (lane == 0 && row < span_rows) epi(s0 + row, b, v);
                } else if (lane == 0) {
                    red[(b * SR + rl + r * RL) * WPR + wir] = v;
                }
            }
        }
        if (WPR == 1) continue;
        consumer_sync();
        for (int t = ct; t < NQ * SR; t += 32 * kStreamConsumerWarps) {
            const int b = t / SR, row = t % SR;
            if (row < (int)span_rows) {
                uint32_t v = 0;
#pragma unroll
                for (int w = 0; w < WPR; ++w) v += red[t * WPR + w];
                epi(s0 + row, b, v);
            }
        }
        consumer_sync();
    }
}

// Generic fallback for shapes the bulk-copy path cannot take (C not a
// multiple of 16 or an unaligned database): one warp per row, plain loads.
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
template <int NQ, int CCH, int QM, class Epi>
static cudaError_t set_stream_attr() {
    return cudaFuncSetAttribute(stream_answer_kernel<NQ, CCH, QM, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                StreamCfg<NQ, CCH, QM>::kSmemBytes);
}

cudaError_t prepare_stream_kernels() {
    cudaError_t e;
    if ((e = set_stream_attr<1, 512, kQPacked, AnswerEpi>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<1, 1024, kQPacked, AnswerEpi>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<1, 2048, kQPacked, AnswerEpi>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<1, 4096, kQPacked, AnswerEpi>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<2, 1024, kQPacked, AnswerEpi>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<4, 1024, kQPacked, AnswerEpi>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<1, 512, kQRaw, AnswerEpi>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<1, 1024, kQRaw, AnswerEpi>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<1, 2048, kQRaw, AnswerEpi>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<1, 4096, kQRaw, AnswerEpi>()) != cudaSuccess) return e;
    if ((e = set_stream_attr<2, 1024, kQRaw, AnswerEpi>()) != cudaSuccess) return e;
    return set_stream_attr<2, 2048, kQRaw, AnswerEpi>();
}

bool stream_config_valid(int nq, int cch) {
    if (nq == 1) return cch == 512 || cch == 1024 || cch == 2048 || cch == 4096;
    return (nq == 2 || nq == 4) && cch == 1024;
}

cudaError_t launch_pack_query(const uint32_t *q, uint64_t q_ld, uint32_t C, uint32_t cch, uint32_t nq,
                              uint32_t *qpack, uint64_t pack_ld, cudaStream_t stream) {
    const uint32_t nchunks = (C + cch - 1) / cch;
    const uint32_t groups = nchunks * (cch / 4);
    dim3 grid((groups + 255) / 256, nq);
    pack_query_kernel<<<grid, 256, 0, stream>>>(q, q_ld, C, cch, nchunks, qpack, pack_ld);
    return cudaGetLastError();
}

// Launch with programmatic dependent launch allowed (see the kernel comment).
template <int NQ, int CCH, int QM, class Epi>
static cudaError_t launch_cfg(const CUtensorMap *map, const uint8_t *D, uint32_t R, uint32_t C,
                              const uint32_t *qsrc, uint64_t pack_ld, const Epi &epi, int grid, int *status,
                              cudaStream_t stream) {
    CUtensorMap m;
    if (map) m = *map;
    else std::memset(&m, 0, sizeof(m));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kStreamThreads);
    cfg.dynamicSmemBytes = StreamCfg<NQ, CCH, QM>::kSmemBytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, stream_answer_kernel<NQ, CCH, QM, Epi>, m, map ? 1 : 0, D, R, C, qsrc, pack_ld,
                              epi, status);
}

static int stream_grid(uint32_t R, int num_sms) { return static_cast<int>(R < (uint32_t)num_sms ? R : (uint32_t)num_sms); }

cudaError_t launch_stream_answer(int nq, int cch, const CUtensorMap *map, const uint8_t *D, uint32_t R, uint32_t C,
                                 const uint32_t *qpack, uint64_t pack_ld, uint32_t *ans, uint64_t ans_ld,
                                 int num_sms, int *status, cudaStream_t stream) {
    const int grid = stream_grid(R, num_sms);
    const AnswerEpi epi{ans, ans_ld};
    if (nq == 1) {
        switch (cch) {
            case 512: return launch_cfg<1, 512, kQPacked>(map, D, R, C, qpack, pack_ld, epi, grid, status, stream);
            case 1024: return launch_cfg<1, 1024, kQPacked>(map, D, R, C, qpack, pack_ld, epi, grid, status, stream);
            case 2048: return launch_cfg<1, 2048, kQPacked>(map, D, R, C, qpack, pack_ld, epi, grid, status, stream);
            case 4096: return launch_cfg<1, 4096, kQPacked>(map, D, R, C, qpack, pack_ld, epi, grid, status, stream);
            default: return cudaErrorInvalidValue;
        }
    }
    if (cch != 1024) return cudaErrorInvalidValue;
    if (nq == 2) return launch_cfg<2, 1024, kQPacked>(map, D, R, C, qpack, pack_ld, epi, grid, status, stream);
    if (nq == 4) return launch_cfg<4, 1024, kQPacked>(map, D, R, C, qpack, pack_ld, epi, grid, status, stream);
    return cudaErrorInvalidValue;
}

cudaError_t launch_stream_answer_raw(int cch, const CUtensorMap *map, const uint8_t *D, uint32_t R, uint32_t C,
                                     const uint32_t *q, uint32_t *ans, int num_sms, int *status,
                                     cudaStream_t stream) {
    const int grid = stream_grid(R, num_sms);
    const AnswerEpi epi{ans, 0};
    switch (cch) {
        case 512: return launch_cfg<1, 512, kQRaw>(map, D, R, C, q, 0, epi, grid, status, stream);
        case 1024: return launch_cfg<1, 1024, kQRaw>(map, D, R, C, q, 0, epi, grid, status, stream);
        case 2048: return launch_cfg<1, 2048, kQRaw>(map, D, R, C, q, 0, epi, grid, status, stream);
        case 4096: return launch_cfg<1, 4096, kQRaw>(map, D, R, C, q, 0, epi, grid, status, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stream_answer_raw2(int cch, const CUtensorMap *map, const uint8_t *D, uint32_t R, uint32_t C,
                                      const uint32_t *q, uint64_t q_ld, uint32_t *ans, uint64_t ans_ld, int num_sms,
                                      int *status, cudaStream_t stream) {
    const int grid = stream_grid(R, num_sms);
    const AnswerEpi epi{ans, ans_ld};
    switch (cch) {
        case 1024: return launch_cfg<2, 1024, kQRaw>(map, D, R, C, q, q_ld, epi, grid, status, stream);
        case 2048: return launch_cfg<2, 2048, kQRaw>(map, D, R, C, q, q_ld, epi, grid, status, stream);
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
