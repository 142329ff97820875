// Exact mod-2^32 product of the database with many Z_q vectors on the
// tcgen05 tensor cores:  OUT[i][b] = sum_j D[i][j] * X[b][j]  (mod 2^32).
//
// Used for the batched Response (X = a batch of queries; QPADL Alg. 4's
// q-bar queries against one database) and for the offline hint
// H = D * A (X = columns of A; Sec. 5.3 offline precomputation).
//
// Exactness.  Each X word is split into four balanced byte limbs
// x = sum_k 2^{8k} c_k with c_k in [-128, 127] (low byte, minus 256 and a
// carry when >= 128; the last carry is a multiple of 2^32 and is dropped).
// Digits d in [0, 255] and limbs are small integers, exactly representable
// in fp16, and every product d*c is an integer of magnitude <= 32640.  A run
// of 512 such products sums to less than 2^24 in magnitude, so the fp32
// tensor-core accumulator holds every partial sum of a 512-deep K-chunk
// exactly.  After each chunk the epilogue converts the four limb sums to
// int32 (exact), recombines them as sum_k 2^{8k} s_k in uint32 arithmetic
// (that is, mod 2^32) and adds them into per-thread running sums.  No value
// is ever rounded.  (tcgen05 has no integer kind on sm_103a, so the byte
// limbs ride in fp16 operands.)
//
// Kernel shape (one CTA per SM, persistent over output tiles):
//   warp 0      TMA producer: 128x64 tile of D16 and BNx64 tile of limbs per
//               stage, 128-byte swizzle, mbarrier ring of 4 (BN = 256) to 8 stages.
//   warp 1      allocates TMEM (two BN-column fp32 accumulators) and one
//               thread issues tcgen05.mma M=128, N=BN, K=16 (4 per stage).
//   warps 2..5  epilogue: drain one accumulator per 512-deep K-chunk while
//               the MMA fills the other.
// Output element (row i, vector b) goes through an epilogue functor: a plain
// store for the Response and the hint, the Query or Recover epilogue when the
// matrix operand is the limb planes of A or H (client batches, below).
//
// Client batches (Def. 1 Client.Query / Client.BlockReconst for B secrets).
// For a uint32 matrix X (A or H) and secrets S, (X s_b)[i] mod 2^32 needs
// the limb products a_u * s_l with u + l <= 3 only (the others are multiples
// of 2^32).  The matrix operand holds X's limb planes side by side along K
// (row i: [x_0[i][.], x_1[i][.], x_2[i][.], x_3[i][.]], 4n entries) and the
// vector operand holds, for secret b and shift t, the row
// [s_t, s_{t-1}, .., s_0, 0, ..] (limb t-u of s_b under plane u, zero for
// u > t).  Their product is sum_{u <= t} x_u . s_{t-u}, the coefficient of
// 2^{8t}, and the usual recombination sum_t 2^{8t} (.) gives X s_b mod 2^32.
// Every product is at most 128 * 128 in magnitude, so a 512-deep chunk is
// exact in fp32 here as well.
//
// Planed mode (n a multiple of 512, BN >= 64) skips the zero blocks: each
// 512-deep chunk lies inside one limb plane u, and only the shifts t >= u
// need it.  A tile's vector rows are then ordered by descending shift (row
// (3 - t) * BN/4 + q for vector q of the tile), so the active shifts of
// plane u are the first (4 - u) * BN/4 rows: each MMA of the chunk takes
// N = (4 - u) * BN/4 and the epilogue drains only those columns, adding
// each shift times 2^{8t}.  That runs 10 of the 16 (plane, shift) blocks
// with MMAs no narrower than BN/4.
#include <cstdint>
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "epilogues.cuh"
#include "limb_gemm.cuh"
#include "ptx.cuh"

namespace qpadl {

constexpr int kBM = 128;
constexpr int kBK = 64;          // fp16 elements per 128-byte swizzled row
constexpr int kChunkKB = 8;      // 8 x 64 = 512-deep exact K-chunks
constexpr int kGemmThreads = 192;

template <int BN>
struct GemmCfg {
    static constexpr uint32_t kABytes = kBM * kBK * 2;
    static constexpr uint32_t kBBytes = BN * kBK * 2;
    static constexpr uint32_t kStageBytes = kABytes + kBBytes;
    static constexpr uint32_t kTmemCols = (2 * BN < 32) ? 32 : 2 * BN;
    // as many stages as fit in about 192 KB, at most 8: narrow tiles (small batches, one-limb
    // vectors) get a deeper ring, since each of their stages carries little MMA work
    static constexpr int kStages = (192 * 1024 / kStageBytes) < 8 ? (192 * 1024 / kStageBytes) : 8;
    static constexpr int kSmemBytes = kStages * kStageBytes + 256 + 1024;
    static constexpr int kQPT = BN / 4;   // vectors per tile
};

__device__ __forceinline__ bool drain_wait_g(uint64_t *bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > QPADL_WAIT_NS) return false;
    }
    return true;
}

// Work schedule of one CTA.  Tiles [0, dp_tiles) are whole-tile work dealt
// round-robin (tile b, b + G, ...: neighbouring CTAs share the rows of D).
// The remaining tiles are split stream-K style: their chunks (tile-major)
// form one range that the G CTAs cut into G contiguous, nearly equal
// pieces, so the last wave ends evenly.  A piece is tile t, chunks [c0, c1).
struct Piece {
    uint32_t t, c0, c1;
};
struct PieceIter {
    uint32_t t, u, u_end;
    __device__ __forceinline__ PieceIter(uint32_t tiles, uint32_t dp_tiles, uint32_t nchunks) {
        t = blockIdx.x;
        const uint64_t U = (uint64_t)(tiles - dp_tiles) * nchunks;
        u = static_cast<uint32_t>((uint64_t)blockIdx.x * U / gridDim.x);
        u_end = static_cast<uint32_t>((uint64_t)(blockIdx.x + 1) * U / gridDim.x);
    }
    __device__ __forceinline__ bool next(Piece &p, uint32_t dp_tiles, uint32_t nchunks) {
        if (t < dp_tiles) {
            p = Piece{t, 0u, nchunks};
            t += gridDim.x;
            return true;
        }
        if (u >= u_end) return false;
        const uint32_t c0 = u % nchunks;
        const uint32_t c1 = nchunks - c0 < u_end - u ? nchunks : c0 + (u_end - u);
        p = Piece{dp_tiles + u / nchunks, c0, c1};
        u += c1 - c0;
        return true;
    }
};

template <int BN, class Epi, bool PLANED>
__global__ void __launch_bounds__(kGemmThreads, 1)
    limb_gemm_kernel(const __grid_constant__ CUtensorMap a_map, const __grid_constant__ CUtensorMap b_map,
                     Epi epi, uint32_t M, uint32_t NV, uint32_t KB, uint32_t plane_chunks, uint32_t dp_tiles_arg,
                     int *__restrict__ status) {
    static_assert(!PLANED || BN >= 64, "a shift group needs N = BN/4 >= 16");
    using Cfg = GemmCfg<BN>;
    constexpr int kGemmStages = Cfg::kStages;
    constexpr int LPV = Epi::kLimbs;   // limb rows per vector
    static_assert(LPV == 4 || (LPV == 1 && !PLANED), "one-limb vectors: plain mode");
    constexpr int QPT = BN / LPV;      // vectors per tile
    // one-limb tiles wider than 64 keep their running sums in TMEM, reduced mod p after every
    // chunk (a representative |r| <= 1.5 p plus one chunk stays below 2^24, so fp32 stays exact)
    constexpr bool TMEMSUM = LPV == 1 && BN > 64;
    static_assert(!TMEMSUM || BN % 128 == 0, "the mod-p pass takes 128 columns per load batch");
    constexpr int RUN = TMEMSUM ? 1 : QPT;   // running sums kept in registers
    // K-steps per exact chunk: digits times limbs or centred vector entries (|product| <=
    // 255 * 128) sum to at most 16,711,680 over 512, and with a reduced representative
    // (|r| <= 1.5 p <= 386) added still below 2^24
    constexpr uint32_t CKB = static_cast<uint32_t>(kChunkKB);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kGemmStages * Cfg::kStageBytes);
    uint64_t *empty = full + kGemmStages;
    uint64_t *acc_full = empty + kGemmStages;   // [2]
    uint64_t *acc_empty = acc_full + 2;          // [2]
    uint64_t *mma_done = acc_empty + 2;          // [1]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGemmStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        mbar_init(mma_done, 1);
        *abort = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, Cfg::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const uint32_t m_tiles = (M + kBM - 1) / kBM;
    const uint32_t n_tiles = (NV * LPV + BN - 1) / BN;
    const uint32_t tiles = m_tiles * n_tiles;
    const uint32_t nchunks = (KB + CKB - 1) / CKB;
    // only a plain store can take split tiles (their pieces add into a zeroed output)
    constexpr bool kSplit = std::is_same<Epi, StoreEpi>::value;
    const uint32_t dp_tiles = kSplit && dp_tiles_arg < tiles ? dp_tiles_arg : tiles;
    bool failed = false;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            tma_prefetch_desc(&a_map);
            tma_prefetch_desc(&b_map);
            uint32_t it = 0;
            PieceIter pit(tiles, dp_tiles, nchunks);
            Piece pc;
            while (!failed && pit.next(pc, dp_tiles, nchunks)) {
                const uint32_t t = pc.t;
                const uint32_t kb0 = pc.c0 * CKB, kb1 = pc.c1 * CKB < KB ? pc.c1 * CKB : KB;
                const int32_t m0 = static_cast<int32_t>((t / n_tiles) * kBM);
                const int32_t n0 = static_cast<int32_t>((t % n_tiles) * BN);
                {
                    // what this tile's epilogue will read (Query noise, Recover answers) into L2 now
                    const uint32_t v0 = (t % n_tiles) * QPT;
                    const uint32_t nv = v0 < NV ? (NV - v0 < (uint32_t)QPT ? NV - v0 : (uint32_t)QPT) : 0u;
                    if (static_cast<uint32_t>(m0) + kBM <= M) epi.prefetch(static_cast<uint64_t>(m0), v0, nv);
                }
                for (uint32_t kb = kb0; kb < kb1; ++kb, ++it) {
                    const uint32_t st = it % kGemmStages;
                    const uint32_t ph = (it / kGemmStages) & 1u;
                    if (!mbar_wait(&empty[st], ph ^ 1u, abort)) {
                        failed = true;
                        break;
                    }
                    uint8_t *sa = smem + st * Cfg::kStageBytes;
                    mbar_arrive_expect_tx(&full[st], Cfg::kStageBytes);
                    tma_load_2d(sa, &a_map, &full[st], static_cast<int32_t>(kb * kBK), m0);
                    tma_load_2d(sa + Cfg::kABytes, &b_map, &full[st], static_cast<int32_t>(kb * kBK), n0);
                }
            }
            const uint32_t inflight = it < (uint32_t)kGemmStages ? it : (uint32_t)kGemmStages;
            for (uint32_t j = it - inflight; j < it; ++j)
                if (!drain_wait_g(&full[j % kGemmStages], (j / kGemmStages) & 1u)) failed = true;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: the whole warp walks the loop (warp-uniform descriptors),
        // one elected lane issues; wait outcomes are made warp-uniform
        constexpr uint32_t idesc = umma_idesc_f16(kBM, BN);
        uint32_t it = 0, ci = 0;
        bool issued = false;
        PieceIter pit(tiles, dp_tiles, nchunks);
        Piece pc;
        while (!failed && pit.next(pc, dp_tiles, nchunks)) {
            const uint32_t kb0 = pc.c0 * CKB, kb1 = pc.c1 * CKB < KB ? pc.c1 * CKB : KB;
            uint32_t d_tmem = tmem_base;
            for (uint32_t kb = kb0; kb < kb1; ++kb, ++it) {
                if (kb % CKB == 0) {
                    const uint32_t buf = ci & 1u;
                    const bool ok = mbar_wait(&acc_empty[buf], ((ci >> 1) & 1u) ^ 1u, abort);
                    if (__any_sync(0xffffffffu, !ok)) {
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                    d_tmem = tmem_base + buf * BN;
                }
                const uint32_t st = it % kGemmStages;
                const uint32_t ph = (it / kGemmStages) & 1u;
                const bool ok = mbar_wait(&full[st], ph, abort);
                if (__any_sync(0xffffffffu, !ok)) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_addr(smem + st * Cfg::kStageBytes);
                const uint64_t adesc = umma_desc_sw128(sa);
                const uint64_t bdesc = umma_desc_sw128(sa + Cfg::kABytes);
                if (elect_one()) {
                    if constexpr (PLANED) {
                        // limb plane u of this chunk: the active shifts are the first (4 - u) * BN/4 rows
                        const uint32_t u = (kb / CKB) / plane_chunks;
                        const uint32_t idesc_u = umma_idesc_f16(kBM, (4u - u) * (BN / 4));
#pragma unroll
                        for (int k = 0; k < kBK / 16; ++k)
                            umma_f16(d_tmem, adesc + 2u * k, bdesc + 2u * k, idesc_u,
                                     (kb % CKB != 0 || k != 0) ? 1u : 0u);
                    } else {
#pragma unroll
                        for (int k = 0; k < kBK / 16; ++k) {
                            // advance the start address by 16 elements (32 bytes) inside the swizzle atom
                            umma_f16(d_tmem, adesc + 2u * k, bdesc + 2u * k, idesc,
                                     ((TMEMSUM && kb >= 2u * CKB) || kb % CKB != 0 || k != 0) ? 1u
                                                                                                         : 0u);
                        }
                    }
                    umma_commit(&empty[st]);
                    if (kb % CKB == CKB - 1 || kb == kb1 - 1) umma_commit(&acc_full[ci & 1u]);
                }
                __syncwarp();
                issued = true;
                if (kb % CKB == CKB - 1 || kb == kb1 - 1) ++ci;
            }
        }
        // every MMA this warp issued must finish before TMEM is released
        if (issued) {
            if (elect_one()) umma_commit(mma_done);
            __syncwarp();
            if (!drain_wait_g(mma_done, 0)) failed = true;
        }
    } else {
        // ---------------- epilogue (warps 2..5; TMEM lane quarter = warp % 4)
        const uint32_t quarter = static_cast<uint32_t>(warp & 3);
        const uint32_t lane_addr = (quarter * 32u) << 16;
        uint32_t ci = 0;
        PieceIter pit(tiles, dp_tiles, nchunks);
        Piece pc;
        while (!failed && pit.next(pc, dp_tiles, nchunks)) {
            const uint32_t t = pc.t;
            const uint32_t m0 = (t / n_tiles) * kBM;
            const uint32_t v0 = (t % n_tiles) * QPT;
            uint32_t run[RUN];
#pragma unroll
            for (int q = 0; q < RUN; ++q) run[q] = 0u;
            // planed (client) tiles are short in K: their epilogue inputs (Query noise, Recover
            // answers) are loaded when the tile starts, so the loads overlap its MMAs
            constexpr int EARLY = PLANED ? QPT : 1;
            uint32_t early[EARLY];
            if constexpr (PLANED) {
                const uint32_t erow = m0 + quarter * 32u + static_cast<uint32_t>(lane);
#pragma unroll
                for (int q = 0; q < QPT; ++q) early[q] = (erow < M && v0 + q < NV) ? epi.pre(erow, v0 + q) : 0u;
            }
            for (uint32_t c = pc.c0; c < pc.c1; ++c, ++ci) {
                const uint32_t buf = ci & 1u;
                if (!mbar_wait(&acc_full[buf], (ci >> 1) & 1u, abort)) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                if constexpr (TMEMSUM) {
                    const float pf = static_cast<float>(epi.p), inv = 1.0f / pf;
                    const uint32_t cur = tmem_base + lane_addr + buf * BN;
                    if (c + 1 < nchunks) {
                        // replace this buffer's running sums by small representatives of their
                        // residues mod p: q = x / p rounded to an integer through the 1.5 * 2^23
                        // rounding constant (off by at most one where |x / p| >= 2^22, i.e. p < 4),
                        // r = x - q p with |r| <= 1.5 p.  q p and r are integers below 2^24, so the
                        // fused multiply-add is exact.  Four 32-column loads per wait.
                        constexpr float kRound = 12582912.0f;
#pragma unroll 1
                        for (int j0 = 0; j0 < BN / 32; j0 += 4) {
                            uint32_t v[4][32];
#pragma unroll
                            for (int g = 0; g < 4; ++g) tmem_ld32(cur + 32u * (j0 + g), v[g]);
                            tmem_wait_ld();
#pragma unroll
                            for (int g = 0; g < 4; ++g) {
#pragma unroll
                                for (int q = 0; q < 32; ++q) {
                                    const float x = __uint_as_float(v[g][q]);
                                    const float qf = __fsub_rn(__fmaf_rn(x, inv, kRound), kRound);
                                    v[g][q] = __float_as_uint(__fmaf_rn(-qf, pf, x));
                                }
                                tmem_st32(cur + 32u * (j0 + g), v[g]);
                            }
                        }
                        tmem_wait_st();
                        if (c + 2 < nchunks) {
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&acc_empty[buf]);
                        }
                        // the second-to-last chunk's buffer is held for the final combine
                        continue;
                    }
                    // last chunk: its buffer plus the other buffer's residue, mod p, to the output.  Each
                    // buffer is first cut to a representative |r| <= 1.5 p as in the pass above, so
                    // their sum is an exact float of at most 3 p; q = floor(sum / p) is then off by at
                    // most one, which the two compares put right, and the residue stays exact.
                    const uint32_t oth = tmem_base + lane_addr + (buf ^ 1u) * BN;
                    const uint32_t row = m0 + quarter * 32u + static_cast<uint32_t>(lane);
                    constexpr float kRound = 12582912.0f;
#pragma unroll 1
                    for (int j = 0; j < BN / 32; ++j) {
                        uint32_t v[32], w[32];
                        tmem_ld32(cur + 32u * j, v);
                        if (nchunks >= 2) tmem_ld32(oth + 32u * j, w);
                        tmem_wait_ld();
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            float x = __uint_as_float(v[q]);
                            x = __fmaf_rn(-__fsub_rn(__fmaf_rn(x, inv, kRound), kRound), pf, x);
                            if (nchunks >= 2) {
                                float y = __uint_as_float(w[q]);
                                y = __fmaf_rn(-__fsub_rn(__fmaf_rn(y, inv, kRound), kRound), pf, y);
                                x = __fadd_rn(x, y);
                            }
                            float r = __fmaf_rn(-floorf(x * inv), pf, x);
                            if (r < 0.0f) r = __fadd_rn(r, pf);
                            if (r >= pf) r = __fsub_rn(r, pf);
                            const uint32_t vi = v0 + 32u * j + q;
                            if (row < M && vi < NV) epi.store(row, vi, static_cast<uint32_t>(r));
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(&acc_empty[buf]);
                        if (nchunks >= 2) mbar_arrive(&acc_empty[buf ^ 1u]);
                    }
                    continue;
                } else if constexpr (PLANED) {
                    // active shifts of this chunk's plane; column (3 - t)*QPT + q holds shift t of vector q
                    const uint32_t u = c / plane_chunks;
                    for (uint32_t t = u; t < 4; ++t) {
                        const uint32_t col0 = tmem_base + lane_addr + buf * BN + (3u - t) * QPT;
                        if constexpr (QPT >= 32) {
#pragma unroll
                            for (int j = 0; j < QPT / 32; ++j) {
                                uint32_t v[32];
                                tmem_ld32(col0 + 32u * j, v);
                                tmem_wait_ld();
#pragma unroll
                                for (int q = 0; q < 32; ++q)
                                    run[32 * j + q] +=
                                        static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[q]))) << (8u * t);
                            }
                        } else {
                            uint32_t v[16];
                            tmem_ld16(col0, v);
                            tmem_wait_ld();
#pragma unroll
                            for (int q = 0; q < QPT; ++q)
                                run[q] += static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[q]))) << (8u * t);
                        }
                    }
                } else if constexpr (LPV == 1) {
                    // every column is its own vector; all loads before one wait
                    uint32_t v[BN / 32][32];
#pragma unroll
                    for (int j = 0; j < BN / 32; ++j) tmem_ld32(tmem_base + lane_addr + buf * BN + 32u * j, v[j]);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < BN / 32; ++j)
#pragma unroll
                        for (int q = 0; q < 32; ++q)
                            run[32 * j + q] += static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[j][q])));
                } else {
                    // two 32-column loads per wait
                    constexpr int JB = BN / 32 < 2 ? BN / 32 : 2;
#pragma unroll
                    for (int j0 = 0; j0 < BN / 32; j0 += JB) {
                        uint32_t v[JB][32];
#pragma unroll
                        for (int g = 0; g < JB; ++g) tmem_ld32(tmem_base + lane_addr + buf * BN + 32u * (j0 + g), v[g]);
                        tmem_wait_ld();
#pragma unroll
                        for (int g = 0; g < JB; ++g)
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const uint32_t s0 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[g][4 * q + 0])));
                                const uint32_t s1 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[g][4 * q + 1])));
                                const uint32_t s2 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[g][4 * q + 2])));
                                const uint32_t s3 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[g][4 * q + 3])));
                                run[8 * (j0 + g) + q] += s0 + (s1 << 8) + (s2 << 16) + (s3 << 24);
                            }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[buf]);
            }
            if (failed) break;
            if constexpr (TMEMSUM) continue;   // the last chunk already wrote the tile
            const uint32_t row = m0 + quarter * 32u + static_cast<uint32_t>(lane);
            if constexpr (kSplit) {
                if (row < M && !(pc.c0 == 0 && pc.c1 == nchunks)) {
                    // part of a split tile: exact, since addition mod 2^32 commutes
#pragma unroll
                    for (int q = 0; q < QPT; ++q)
                        if (v0 + q < NV) epi.add(row, v0 + q, run[q]);
                    continue;
                }
            }
            if constexpr (PLANED) {
                if (row < M) {
#pragma unroll
                    for (int q = 0; q < QPT; ++q)
                        if (v0 + q < NV) epi.put(row, v0 + q, run[q], early[q]);
                }
                continue;
            }
            if (row < M) {
                // groups of up to 16 outputs: all their loads first, then all their stores
                constexpr int G = QPT < 16 ? QPT : 16;
#pragma unroll
                for (int g = 0; g < QPT; g += G) {
                    uint32_t pre_v[G];
#pragma unroll
                    for (int q = 0; q < G; ++q) pre_v[q] = (v0 + g + q < NV) ? epi.pre(row, v0 + g + q) : 0u;
#pragma unroll
                    for (int q = 0; q < G; ++q)
                        if (v0 + g + q < NV) epi.put(row, v0 + g + q, run[g + q], pre_v[q]);
                }
            }
        }
    }

    if (failed) {
        *abort = 1;
        *status = kDevTimeout;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, Cfg::kTmemCols);
    }
}

// D (uint8, R x C) -> D16 (fp16, R x pitch), digits as exact small integers.
// One block per row at a time; 16 digits per thread step when rows are aligned.
__global__ void db_to_f16_kernel(const uint8_t *__restrict__ D, uint64_t R, uint64_t C, __half *__restrict__ D16,
                                 uint64_t pitch) {
    const bool vec = (C % 16 == 0) && ((reinterpret_cast<uintptr_t>(D) & 15u) == 0) && (pitch % 8 == 0);
    for (uint64_t i = blockIdx.x; i < R; i += gridDim.x) {
        const uint8_t *src = D + i * C;
        __half *dst = D16 + i * pitch;
        if (vec) {
            for (uint64_t j = 16ull * threadIdx.x; j < C; j += 16ull * blockDim.x) {
                const uint4 w = *reinterpret_cast<const uint4 *>(src + j);
                const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
                uint32_t h[8];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const __half2 lo = __halves2half2(__ushort2half_rn(ws[t] & 255u), __ushort2half_rn((ws[t] >> 8) & 255u));
                    const __half2 hi = __halves2half2(__ushort2half_rn((ws[t] >> 16) & 255u), __ushort2half_rn(ws[t] >> 24));
                    h[2 * t] = *reinterpret_cast<const uint32_t *>(&lo);
                    h[2 * t + 1] = *reinterpret_cast<const uint32_t *>(&hi);
                }
                uint4 *d4 = reinterpret_cast<uint4 *>(dst + j);
                d4[0] = make_uint4(h[0], h[1], h[2], h[3]);
                d4[1] = make_uint4(h[4], h[5], h[6], h[7]);
            }
        } else {
            for (uint64_t j = threadIdx.x; j < C; j += blockDim.x)
                dst[j] = __ushort2half_rn(static_cast<unsigned short>(src[j]));
        }
    }
}

__device__ __forceinline__ void balanced_limbs(uint32_t x, float (&c)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int byte = static_cast<int>(x & 255u);
        if (byte >= 128) {
            c[k] = static_cast<float>(byte - 256);
            x = (x >> 8) + 1u;
        } else {
            c[k] = static_cast<float>(byte);
            x >>= 8;
        }
    }
}

// X (uint32, NV x C, vector v in row v) -> limbs (fp16, 4*NV x pitch),
// limb k of vector v in row 4v + k.  One block per vector at a time.
__global__ void vec_limbs_kernel(const uint32_t *__restrict__ X, uint64_t x_ld, uint32_t NV, uint64_t C,
                                 __half *__restrict__ L, uint64_t pitch, uint32_t *__restrict__ Z, uint64_t z_words) {
    // a GEMM launched as this kernel's programmatic dependent may start now: it waits for this
    // grid's completion (griddepcontrol.wait) before it reads the limbs or writes its output
    griddep_launch_dependents();
    if (Z != nullptr) {   // zero the dependent GEMM's output block (its split tiles add into it)
        const uint64_t nthreads = (uint64_t)gridDim.x * gridDim.y * blockDim.x;
        for (uint64_t i = ((uint64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x; i < z_words;
             i += nthreads)
            Z[i] = 0u;
    }
    // block (x, y): vector y, columns [2048 x, 2048 x + 2048), 8 consecutive columns per thread,
    // so even a handful of vectors spreads over the whole GPU
    constexpr uint32_t kCols = 8;
    const uint32_t v = blockIdx.y;
    const uint32_t *src = X + (uint64_t)v * x_ld;
    __half *dst = L + 4ull * v * pitch;
    const bool vec = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && (pitch % 8 == 0) &&
                     ((reinterpret_cast<uintptr_t>(L) & 15u) == 0);
    const uint64_t j0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * kCols;
    if (j0 >= C) return;
    if (vec && j0 + kCols <= C) {
        const uint4 a = *reinterpret_cast<const uint4 *>(src + j0);
        const uint4 b = *reinterpret_cast<const uint4 *>(src + j0 + 4);
        const uint32_t x[kCols] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        __align__(16) __half h[4][kCols];
#pragma unroll
        for (uint32_t i = 0; i < kCols; ++i) {
            float c[4];
            balanced_limbs(x[i], c);
#pragma unroll
            for (int k = 0; k < 4; ++k) h[k][i] = __float2half_rn(c[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) *reinterpret_cast<uint4 *>(dst + k * pitch + j0) = *reinterpret_cast<const uint4 *>(h[k]);
    } else {
        for (uint64_t j = j0; j < C && j < j0 + kCols; ++j) {
            float c[4];
            balanced_limbs(src[j], c);
#pragma unroll
            for (int k = 0; k < 4; ++k) dst[k * pitch + j] = __float2half_rn(c[k]);
        }
    }
}

// A (uint32, C x n row-major) -> limbs of its columns (fp16, 4n x pitch):
// limb l of column k (over j) in row 4k + l.  32x32 tiles through shared memory.
__global__ void mat_col_limbs_kernel(const uint32_t *__restrict__ A, uint64_t C, uint32_t n,
                                     __half *__restrict__ L, uint64_t pitch) {
    __shared__ uint32_t tile[32][33];
    const uint64_t j0 = (uint64_t)blockIdx.x * 32;
    const uint32_t k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const uint64_t j = j0 + r;
        const uint32_t k = k0 + threadIdx.x;
        tile[r][threadIdx.x] = (j < C && k < n) ? A[j * n + k] : 0u;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const uint32_t k = k0 + r;
        const uint64_t j = j0 + threadIdx.x;
        if (k < n && j < C) {
            float c[4];
            balanced_limbs(tile[threadIdx.x][r], c);
#pragma unroll
            for (int l = 0; l < 4; ++l) L[(4ull * k + l) * pitch + j] = __float2half_rn(c[l]);
        }
    }
}

// X (uint32, rows x n row-major) -> its limb planes side by side (fp16,
// rows x pitch): L[i][u * n + k] = limb u of X[i][k].  Entries past 4n are
// never read (the tensor map ends at 4n).
__global__ void mat_row_limbs_kernel(const uint32_t *__restrict__ X, uint64_t rows, uint32_t n,
                                     __half *__restrict__ L, uint64_t pitch) {
    const uint64_t total = rows * n;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = e / n;
        const uint32_t k = static_cast<uint32_t>(e - i * n);
        float c[4];
        balanced_limbs(X[e], c);
        __half *dst = L + i * pitch + k;
#pragma unroll
        for (int u = 0; u < 4; ++u) dst[(uint64_t)u * n] = __float2half_rn(c[u]);
    }
}

// S (uint32, B x n, secret b in row b) -> shifted limb rows (fp16, 4B x
// pitch): row 4b + t holds limb t-u of s_b under plane u (u <= t), zero
// under planes u > t.
__global__ void secret_limbs_kernel(const uint32_t *__restrict__ S, uint32_t B, uint32_t n,
                                    __half *__restrict__ V, uint64_t pitch) {
    const uint64_t total = (uint64_t)B * n;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = e / n;
        const uint32_t k = static_cast<uint32_t>(e - b * n);
        float c[4];
        balanced_limbs(S[e], c);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            __half *row = V + (4 * b + t) * pitch + k;
#pragma unroll
            for (int u = 0; u < 4; ++u) row[(uint64_t)u * n] = __float2half_rn(u <= t ? c[t - u] : 0.0f);
        }
    }
}

// Planed layout of the same rows for tiles of BN = 4 * qpt rows: vector b
// (of Bp = B rounded up to qpt; vectors >= B are zero) and shift t go to row
// (b / qpt) * 4 qpt + (3 - t) * qpt + b % qpt.
__global__ void secret_limbs_planed_kernel(const uint32_t *__restrict__ S, uint32_t B, uint32_t Bp, uint32_t n,
                                           uint32_t qpt, __half *__restrict__ V, uint64_t pitch) {
    const uint64_t total = (uint64_t)Bp * n;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t b = static_cast<uint32_t>(e / n);
        const uint32_t k = static_cast<uint32_t>(e - (uint64_t)b * n);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        if (b < B) balanced_limbs(S[e], c);
        const uint64_t row0 = (uint64_t)(b / qpt) * 4 * qpt + b % qpt;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            __half *row = V + (row0 + (uint64_t)(3 - t) * qpt) * pitch + k;
#pragma unroll
            for (int u = 0; u < 4; ++u) row[(uint64_t)u * n] = __float2half_rn(u <= t ? c[t - u] : 0.0f);
        }
    }
}

// ------------------------------------------------------------------ host side
template <int BN, class Epi, bool PLANED>
static cudaError_t set_gemm_attr() {
    return cudaFuncSetAttribute(limb_gemm_kernel<BN, Epi, PLANED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                GemmCfg<BN>::kSmemBytes);
}

template <class Epi>
static cudaError_t set_gemm_attrs() {
    cudaError_t e;
    if ((e = set_gemm_attr<32, Epi, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_attr<64, Epi, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_attr<128, Epi, false>()) != cudaSuccess) return e;
    return set_gemm_attr<256, Epi, false>();
}

template <class Epi>
static cudaError_t set_planed_attrs() {
    cudaError_t e;
    if ((e = set_gemm_attr<64, Epi, true>()) != cudaSuccess) return e;
    if ((e = set_gemm_attr<128, Epi, true>()) != cudaSuccess) return e;
    return set_gemm_attr<256, Epi, true>();
}

cudaError_t prepare_limb_gemm_kernels() {
    cudaError_t e;
    if ((e = set_gemm_attrs<StoreEpi>()) != cudaSuccess) return e;
    if ((e = set_gemm_attrs<QueryNoiseEpi>()) != cudaSuccess) return e;
    if ((e = set_gemm_attrs<RecoverEpi>()) != cudaSuccess) return e;
    if ((e = set_planed_attrs<QueryNoiseEpi>()) != cudaSuccess) return e;
    if ((e = set_planed_attrs<RecoverEpi>()) != cudaSuccess) return e;
    if ((e = set_gemm_attr<32, ModPEpi, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_attr<64, ModPEpi, false>()) != cudaSuccess) return e;
    return set_gemm_attr<256, ModPEpi, false>();
}

int limb_gemm_bn_for(uint32_t nv) {
    const uint32_t cols = 4 * nv;
    if (cols <= 32) return 32;
    if (cols <= 64) return 64;
    if (cols <= 128) return 128;
    return 256;
}

template <int BN, class Epi, bool PLANED>
static void launch_one(int grid, const CUtensorMap &a_map, const CUtensorMap &b_map, const Epi &epi, uint32_t M,
                       uint32_t NV, uint32_t KB, uint32_t plane_chunks, int *status, cudaStream_t stream,
                       uint32_t dp_tiles = 0xffffffffu) {
    limb_gemm_kernel<BN, Epi, PLANED><<<grid, kGemmThreads, GemmCfg<BN>::kSmemBytes, stream>>>(
        a_map, b_map, epi, M, NV, KB, plane_chunks, dp_tiles, status);
}

// Schedule of a plain-store GEMM over `tiles` tiles (n_tiles per row tile) on
// `num_sms` SMs: the grid and the number of whole (data-parallel) tiles; the
// rest are split stream-K style.  Whole waves stay whole except the last full
// one, which joins the remainder so that every CTA ends with about the same
// share.  Whole tiles dealt round-robin let the CTAs on the n_tiles tiles of a
// row tile share its rows of D through L2; split pieces run at different K
// offsets and lose that sharing, which measured slower on the 1 GiB database
// once a row tile spans 4 or more tiles.  So splitting is used when there are
// fewer tiles than SMs, or for at most 3 tiles per row tile.  Returns false
// when no tile is split.
static bool store_schedule(uint64_t tiles, uint64_t n_tiles, uint32_t nchunks, int num_sms, int *grid,
                           uint32_t *dp_tiles) {
    const uint64_t G = static_cast<uint64_t>(num_sms);
    *grid = static_cast<int>(tiles < G ? tiles : G);
    *dp_tiles = static_cast<uint32_t>(tiles);
    if (tiles % G == 0 || nchunks < 2) return false;
    if (tiles > G) {
        if (n_tiles > 3) return false;
        *dp_tiles = static_cast<uint32_t>((tiles / G - 1) * G);
    } else {
        *dp_tiles = 0;
        const uint64_t units = tiles * nchunks;
        *grid = static_cast<int>(units < G ? units : G);
    }
    return true;
}

// plane_chunks > 0 selects planed mode (then bn >= 64 and K = 4 * 512 * plane_chunks).
template <class Epi>
static cudaError_t launch_epi(int bn, const CUtensorMap &a_map, const CUtensorMap &b_map, const Epi &epi, uint32_t M,
                              uint32_t NV, uint64_t K, uint32_t plane_chunks, int num_sms, int *status,
                              cudaStream_t stream) {
    const uint32_t KB = static_cast<uint32_t>((K + kBK - 1) / kBK);
    const uint64_t tiles = (uint64_t)((M + kBM - 1) / kBM) * (((uint64_t)Epi::kLimbs * NV + bn - 1) / bn);
    if constexpr (Epi::kLimbs == 1) {
        const int grid1 = static_cast<int>(tiles < (uint64_t)num_sms ? tiles : (uint64_t)num_sms);
        if (plane_chunks) return cudaErrorInvalidValue;
        switch (bn) {
            case 32: launch_one<32, Epi, false>(grid1, a_map, b_map, epi, M, NV, KB, 1, status, stream); break;
            case 64: launch_one<64, Epi, false>(grid1, a_map, b_map, epi, M, NV, KB, 1, status, stream); break;
            case 256: launch_one<256, Epi, false>(grid1, a_map, b_map, epi, M, NV, KB, 1, status, stream); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    } else {
    int grid = static_cast<int>(tiles < (uint64_t)num_sms ? tiles : (uint64_t)num_sms);
    uint32_t dp = 0xffffffffu;
    if constexpr (std::is_same<Epi, StoreEpi>::value) {
        // split tiles add into the output, so it is zeroed first; only a dense output
        // (every element of the M x NV block, in either order) can be zeroed in one piece
        const bool dense = (epi.ld_m == 1 && epi.ld_b == M) || (epi.ld_b == 1 && epi.ld_m == NV);
        int g2 = grid;
        uint32_t dp2 = 0;
        const uint64_t n_tiles = ((uint64_t)Epi::kLimbs * NV + bn - 1) / bn;
        if (dense && store_schedule(tiles, n_tiles, (KB + kChunkKB - 1) / kChunkKB, num_sms, &g2, &dp2)) {
            cudaError_t e = cudaMemsetAsync(epi.out, 0, 4ull * M * NV, stream);
            if (e != cudaSuccess) return e;
            grid = g2;
            dp = dp2;
        }
    }
    if (plane_chunks == 0) {
        switch (bn) {
            case 32: launch_one<32, Epi, false>(grid, a_map, b_map, epi, M, NV, KB, 1, status, stream, dp); break;
            case 64: launch_one<64, Epi, false>(grid, a_map, b_map, epi, M, NV, KB, 1, status, stream, dp); break;
            case 128: launch_one<128, Epi, false>(grid, a_map, b_map, epi, M, NV, KB, 1, status, stream, dp); break;
            case 256: launch_one<256, Epi, false>(grid, a_map, b_map, epi, M, NV, KB, 1, status, stream, dp); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        if constexpr (std::is_same<Epi, StoreEpi>::value) {
            return cudaErrorInvalidValue;
        } else {
            if (K != 4ull * 512 * plane_chunks) return cudaErrorInvalidValue;
            switch (bn) {
                case 64: launch_one<64, Epi, true>(grid, a_map, b_map, epi, M, NV, KB, plane_chunks, status, stream); break;
                case 128:
                    launch_one<128, Epi, true>(grid, a_map, b_map, epi, M, NV, KB, plane_chunks, status, stream);
                    break;
                case 256:
                    launch_one<256, Epi, true>(grid, a_map, b_map, epi, M, NV, KB, plane_chunks, status, stream);
                    break;
                default: return cudaErrorInvalidValue;
            }
        }
    }
    return cudaGetLastError();
    }
}

cudaError_t launch_limb_gemm(int bn, const CUtensorMap &a_map, const CUtensorMap &b_map, uint32_t *out,
                             uint64_t ld_m, uint64_t ld_b, uint32_t M, uint32_t NV, uint64_t K, int num_sms,
                             int *status, cudaStream_t stream) {
    return launch_epi(bn, a_map, b_map, StoreEpi{out, ld_m, ld_b}, M, NV, K, 0, num_sms, status, stream);
}

cudaError_t launch_limb_gemm_query(int bn, const CUtensorMap &a_map, const CUtensorMap &b_map, const QueryNoiseEpi &epi,
                                   uint32_t M, uint32_t NV, uint64_t K, uint32_t plane_chunks, int num_sms,
                                   int *status, cudaStream_t stream) {
    return launch_epi(bn, a_map, b_map, epi, M, NV, K, plane_chunks, num_sms, status, stream);
}

__global__ void add_delta_kernel(uint32_t *__restrict__ Q, uint64_t q_ld, const uint32_t *__restrict__ cols,
                                 uint32_t B, uint32_t delta) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) Q[b * q_ld + cols[b]] += delta;
}

cudaError_t launch_add_delta(uint32_t *Q, uint64_t q_ld, const uint32_t *cols, uint32_t B, uint32_t delta,
                             cudaStream_t stream) {
    if (B == 0) return cudaSuccess;
    add_delta_kernel<<<(B + 255) / 256, 256, 0, stream>>>(Q, q_ld, cols, B, delta);
    return cudaGetLastError();
}

cudaError_t launch_limb_gemm_recover(int bn, const CUtensorMap &a_map, const CUtensorMap &b_map,
                                     const RecoverEpi &epi, uint32_t M, uint32_t NV, uint64_t K,
                                     uint32_t plane_chunks, int num_sms, int *status, cudaStream_t stream) {
    return launch_epi(bn, a_map, b_map, epi, M, NV, K, plane_chunks, num_sms, status, stream);
}

cudaError_t launch_limb_gemm_modp(int bn, const CUtensorMap &a_map, const CUtensorMap &b_map, const ModPEpi &epi,
                                  uint32_t M, uint32_t NV, uint64_t K, int num_sms, int *status, cudaStream_t stream) {
    return launch_epi(bn, a_map, b_map, epi, M, NV, K, 0, num_sms, status, stream);
}

cudaError_t launch_db_to_f16(const uint8_t *D, uint64_t R, uint64_t C, __half *D16, uint64_t pitch, int num_sms,
                             cudaStream_t stream) {
    const uint64_t blocks = R < (uint64_t)num_sms * 8 ? R : (uint64_t)num_sms * 8;
    db_to_f16_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(D, R, C, D16, pitch);
    return cudaGetLastError();
}

cudaError_t launch_vec_limbs(const uint32_t *X, uint64_t x_ld, uint32_t NV, uint64_t C, __half *L, uint64_t pitch,
                             int num_sms, cudaStream_t stream, uint32_t *zero, uint64_t zero_words) {
    (void)num_sms;
    if (NV == 0 || C == 0) {
        if (zero != nullptr && zero_words > 0) return cudaMemsetAsync(zero, 0, 4ull * zero_words, stream);
        return cudaSuccess;
    }
    for (uint32_t v0 = 0; v0 < NV; v0 += 65535) {   // grid.y limit
        const uint32_t nv = NV - v0 < 65535 ? NV - v0 : 65535;
        const dim3 grid(static_cast<unsigned>((C + 2047) / 2048), nv);
        vec_limbs_kernel<<<grid, 256, 0, stream>>>(X + (uint64_t)v0 * x_ld, x_ld, nv, C, L + 4ull * v0 * pitch,
                                                    pitch, v0 == 0 ? zero : nullptr, v0 == 0 ? zero_words : 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_mat_col_limbs(const uint32_t *A, uint64_t C, uint32_t n, __half *L, uint64_t pitch,
                                 cudaStream_t stream) {
    dim3 grid(static_cast<unsigned>((C + 31) / 32), (n + 31) / 32);
    mat_col_limbs_kernel<<<grid, dim3(32, 8), 0, stream>>>(A, C, n, L, pitch);
    return cudaGetLastError();
}

cudaError_t launch_mat_row_limbs(const uint32_t *X, uint64_t rows, uint32_t n, __half *L, uint64_t pitch, int num_sms,
                                 cudaStream_t stream) {
    mat_row_limbs_kernel<<<num_sms * 8, 256, 0, stream>>>(X, rows, n, L, pitch);
    return cudaGetLastError();
}

cudaError_t launch_secret_limbs(const uint32_t *S, uint32_t B, uint32_t n, __half *V, uint64_t pitch, int num_sms,
                                cudaStream_t stream) {
    secret_limbs_kernel<<<num_sms * 4, 256, 0, stream>>>(S, B, n, V, pitch);
    return cudaGetLastError();
}

cudaError_t launch_secret_limbs_planed(const uint32_t *S, uint32_t B, uint32_t n, uint32_t qpt, __half *V,
                                       uint64_t pitch, int num_sms, cudaStream_t stream, uint32_t Bp) {
    if (Bp == 0) Bp = (B + qpt - 1) / qpt * qpt;
    if (Bp < B || Bp % qpt != 0) return cudaErrorInvalidValue;
    secret_limbs_planed_kernel<<<num_sms * 4, 256, 0, stream>>>(S, B, Bp, n, qpt, V, pitch);
    return cudaGetLastError();
}

// Goldberg queries (B x C field elements < p) -> one fp16 row per query,
// centred: q if q <= p / 2, else q - p (|value| <= 128 for p <= 257).
__global__ void centred_rows_kernel(const uint32_t *__restrict__ Q, uint32_t B, uint64_t C, uint32_t p,
                                    __half *__restrict__ L, uint64_t pitch, uint32_t *__restrict__ Z,
                                    uint64_t z_words) {
    // as in vec_limbs_kernel: a GEMM launched as this kernel's programmatic dependent may start now,
    // and its output block is zeroed here
    griddep_launch_dependents();
    if (Z != nullptr) {
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < z_words;
             i += (uint64_t)gridDim.x * blockDim.x)
            Z[i] = 0u;
    }
    const uint64_t total = (uint64_t)B * C;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = e / C, j = e - b * C;
        const uint32_t q = Q[e];
        const int v = q <= p / 2 ? static_cast<int>(q) : static_cast<int>(q) - static_cast<int>(p);
        L[b * pitch + j] = __int2half_rn(v);
    }
}

// x[i] = x[i] mod p for n words (uint32, the exact non-negative sums of the streaming path).
__global__ void mod_p_kernel(uint32_t *__restrict__ x, uint64_t n, uint32_t p) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x)
        x[e] %= p;
}

// x[i] = x[i] mod p in [0, p) for n words holding exact signed 32-bit sums.
__global__ void mod_p_signed_kernel(uint32_t *__restrict__ x, uint64_t n, int32_t p) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
        int32_t r = static_cast<int32_t>(x[e]) % p;
        if (r < 0) r += p;
        x[e] = static_cast<uint32_t>(r);
    }
}

cudaError_t launch_mod_p_signed(uint32_t *x, uint64_t n, uint32_t p, int num_sms, cudaStream_t stream) {
    mod_p_signed_kernel<<<num_sms * 4, 256, 0, stream>>>(x, n, static_cast<int32_t>(p));
    return cudaGetLastError();
}

cudaError_t launch_centred_rows(const uint32_t *Q, uint32_t B, uint64_t C, uint32_t p, __half *L, uint64_t pitch,
                                int num_sms, cudaStream_t stream, uint32_t *zero, uint64_t zero_words) {
    centred_rows_kernel<<<num_sms * 4, 256, 0, stream>>>(Q, B, C, p, L, pitch, zero, zero_words);
    return cudaGetLastError();
}

cudaError_t launch_mod_p(uint32_t *x, uint64_t n, uint32_t p, int num_sms, cudaStream_t stream) {
    mod_p_kernel<<<num_sms * 4, 256, 0, stream>>>(x, n, p);
    return cudaGetLastError();
}

}  // namespace qpadl
