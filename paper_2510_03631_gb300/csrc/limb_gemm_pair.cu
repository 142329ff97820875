// Exact mod-2^32 limb GEMM on CTA pairs: the same product as limb_gemm.cu,
//     OUT[i][b] = sum_j X[i][j] * V[b][j]   (mod 2^32),
// with one tile of 256 matrix rows per pair of SMs (tcgen05 cta_group::2).
//
// Why pairs.  A 128 x BN tile on one SM moves 128 + BN operand rows from L2
// into shared memory per k-step.  A pair tile of 256 x BN lets each SM load
// its own 128 matrix rows but only half of the BN vector rows: the pair MMA
// (M = 256) reads the other half from the peer's shared memory.  At BN = 256
// each SM receives 32 KB per 64-deep k-step instead of 48 KB for the same
// tensor work, which is what bounds the short-K client batches (Query over A,
// Recover over H: K = 4n) and the long-K batched Response and hint.
//
// Exactness is that of limb_gemm.cu: balanced byte limbs in fp16, drained to
// int32 after every exact chunk and recombined as sum_k 2^{8k} s_k in uint32
// arithmetic.  The chunk depth follows the products' bound: digits times limbs
// (Response, hint; magnitude <= 255 * 128) take 512-deep chunks, whose sums
// stay below 2^24; limbs times limbs (client Query/Recover; magnitude <= 2^14)
// take 1024-deep chunks, whose partial sums never exceed 2^24 in magnitude.
// Every integer of magnitude <= 2^24 is an fp32 value, so no partial sum is
// ever rounded either way.
//
// Pair protocol (cluster of 2 CTAs; rank 0 leads):
//   producers (warps 0 and 6 of each CTA)  wait their own `empty` slot; warp
//       0 loads the CTA's A rows and warp 6 its half of the vector rows with
//       TMA; every copy completes on the leader's `full` barrier (the leader's
//       warp 0 expects the bytes of both CTAs).
//   MMA (warp 1 of the leader)  waits `full`, issues the pair MMAs, and
//       commits to `empty` of both CTAs (the stage may be refilled) and, at
//       the end of a chunk, to `acc_full` of both CTAs.
//   epilogue (warps 2..5 of each CTA)  drains its own TMEM (its 128 rows x
//       all N columns of the pair tile) and arrives on the leader's
//       `acc_empty` (count 8: four warps of each CTA).
// TMEM is allocated and freed by warp 1 of both CTAs together.  A CTA that
// gives up on a bounded wait raises its own and its peer's abort flag; both
// leave their loops, the leader's producer waits (bounded) for copies in
// flight, and a cluster barrier keeps either CTA from exiting while the other
// may still touch its shared memory.
//
// Column order.  The pair MMA's N columns take the leader's N/2 vector rows
// first, then the peer's.  Plain mode: the vector rows of a tile are
// consecutive (row n0 + n is column n).  Planed mode (client batches, n a
// multiple of 512): a tile holds QPT = bn/4 secrets; the leader holds secrets
// 0..QPT/2-1 of the tile and the peer the rest, each as 4 shift groups in
// descending shift order (launch_secret_limbs_planed with qpt = QPT/2).  A
// chunk of limb plane u needs shifts t >= u only: each CTA loads the first
// (4 - u) QPT/2 rows of its block and the MMA runs N = (4 - u) QPT; column
// (3 - t) QPT/2 + q is shift t of leader secret q and column N/2 + (3 - t)
// QPT/2 + q shift t of peer secret q.
//
// Schedule.  Whole pair tiles go round-robin to the clusters.  A plain store may split its last
// wave stream-K style (PairPieceIter: clusters grouped by vector tile so the clusters on one row
// tile read its rows together), the split pieces adding into a zeroed output.
//
// One-row mode (ModPEpi: Z_p vectors as single centred fp16 rows, 256-wide tiles).  The running
// sums stay in TMEM: after every 512-deep chunk the epilogue replaces its accumulator buffer by
// small representatives of the sums mod p, and the MMA accumulates the chunk after next on top;
// the last two buffers are combined mod p at the end of the tile.
#include <cstdint>
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "epilogues.cuh"
#include "limb_gemm_pair.cuh"
#include "ptx.cuh"

namespace qpadl {

namespace {

constexpr int kPM = 128;          // matrix rows per CTA (256 per pair)
constexpr int kPK = 64;           // fp16 elements per 128-byte swizzled row
constexpr int kPThreads = 224;   // warps: 0 matrix-tile producer, 1 MMA, 2..5 epilogue, 6 vector-tile producer

template <int BN>
struct PairCfg {
    static constexpr uint32_t kABytes = kPM * kPK * 2;           // 16 KB
    static constexpr uint32_t kBBytes = (BN / 2) * kPK * 2;      // this CTA's half of the vector rows
    static constexpr uint32_t kStageBytes = kABytes + kBBytes;
    // as many stages as the 227 KB of shared memory hold (7 at 32 KB): the ring is bound by
    // bytes in flight over the round trip of a stage, not by bandwidth
    static constexpr int kFit = (227 * 1024 - 2048) / kStageBytes;
    static constexpr int kStages = kFit < 8 ? kFit : 8;
    static constexpr uint32_t kTmemCols = 2 * BN;                 // two accumulators
    static constexpr int kSmemBytes = kStages * kStageBytes + 256 + 1024;
    static_assert(kSmemBytes <= 227 * 1024, "shared memory");
    static_assert(kStages >= 4, "pipeline depth");
};

__device__ __forceinline__ bool drain_wait_p(uint64_t *bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > QPADL_WAIT_NS) return false;
    }
    return true;
}

// One piece of a cluster's work: chunks [c0, c1) of pair tile t.  Tiles below dp_tiles are dealt
// whole, round-robin (tile c, c + nclusters, ...), so the clusters on the n_tiles tiles of one row
// tile run together and share its rows through L2.  The remaining tiles (whole row tiles) are
// split by chunks (stream-K), so the last wave ends evenly: the first tail_parts * n_tiles
// clusters form n_tiles groups, group n takes vector tile n of every tail row tile, and cluster p
// of each group takes the same contiguous share of the (row tile, chunk) units, so the n_tiles
// clusters that read one row tile's rows still read them together.
struct PairPiece {
    uint32_t t, c0, c1;
};
struct PairPieceIter {
    uint32_t t, step, n, u, u_end;
    __device__ __forceinline__ PairPieceIter(uint32_t tiles, uint32_t dp_tiles, uint32_t n_tiles, uint32_t nchunks,
                                             uint32_t tail_parts, uint32_t part, uint32_t nparts) {
        t = part;
        step = nparts;
        n = part % n_tiles;
        u = u_end = 0;
        const uint32_t p = part / n_tiles;
        if (p < tail_parts) {
            const uint64_t U = (uint64_t)((tiles - dp_tiles) / n_tiles) * nchunks;
            u = static_cast<uint32_t>((uint64_t)p * U / tail_parts);
            u_end = static_cast<uint32_t>((uint64_t)(p + 1) * U / tail_parts);
        }
    }
    __device__ __forceinline__ bool next(PairPiece &pc, uint32_t dp_tiles, uint32_t n_tiles, uint32_t nchunks) {
        if (t < dp_tiles) {
            pc = PairPiece{t, 0u, nchunks};
            t += step;
            return true;
        }
        if (u >= u_end) return false;
        const uint32_t c0 = u % nchunks;
        const uint32_t c1 = nchunks - c0 < u_end - u ? nchunks : c0 + (u_end - u);
        pc = PairPiece{dp_tiles + (u / nchunks) * n_tiles + n, c0, c1};
        u += c1 - c0;
        return true;
    }
};

}  // namespace

template <int BN, class Epi, bool PLANED>
__global__ void __launch_bounds__(kPThreads, 1)
    limb_gemm_pair_kernel(const __grid_constant__ CUtensorMap a_map, const __grid_constant__ PairBMaps bm, Epi epi,
                          uint32_t M, uint32_t NV, uint32_t KB, uint32_t ckb, uint32_t plane_chunks,
                          uint32_t dp_tiles_arg, uint32_t tail_parts, int *__restrict__ status) {
    using Cfg = PairCfg<BN>;
    static_assert(BN == 64 || BN == 128 || BN == 256, "tile width");
    static_assert(!PLANED || BN >= 128, "a planed shift group needs N/2 >= 16 rows per CTA");
    constexpr int ST = Cfg::kStages;
    constexpr int LPV = Epi::kLimbs;   // vector-operand rows per vector
    static_assert(LPV == 4 || (LPV == 1 && BN == 256 && !PLANED), "one-row vectors: 256-wide plain tiles");
    constexpr int QPT = BN / LPV;      // vectors per pair tile
    // one-row tiles (Z_p vectors, ModPEpi) keep their running sums in TMEM, reduced mod p after
    // every chunk: a representative |r| <= 1.5 p plus one chunk (digits times centred entries,
    // |product| <= 255 * 128, 512 deep) stays below 2^24, so fp32 stays exact
    constexpr bool TMEMSUM = LPV == 1;
    constexpr int HQ = QPT / 2;   // planed: secrets per CTA block
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + ST * Cfg::kStageBytes);   // [ST], leader's counts
    uint64_t *empty = full + ST;                                                     // [ST], own
    uint64_t *acc_full = empty + ST;                                                 // [2], own
    uint64_t *acc_empty = acc_full + 2;                                              // [2], leader's counts
    uint64_t *mma_done = acc_empty + 2;                                              // [1], leader
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 8);
        }
        mbar_init(mma_done, 1);
        *abort = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc_pair(tmem_slot, Cfg::kTmemCols);
        tmem_relinquish_pair();
    }
    // both CTAs' barriers exist before either touches the other's
    tc_fence_before();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t full_c = cluster_addr(full, 0);          // the leader's full barriers
    const uint32_t acc_empty_c = cluster_addr(acc_empty, 0);
    const uint32_t peer_abort = cluster_addr(const_cast<int *>(abort), rank ^ 1u);

    const uint32_t m_tiles = (M + 2 * kPM - 1) / (2 * kPM);
    const uint32_t n_tiles = (NV + QPT - 1) / QPT;
    const uint32_t tiles = m_tiles * n_tiles;
    const uint32_t cluster = blockIdx.x >> 1, nclusters = gridDim.x >> 1;   // clusters are CTAs 2c, 2c + 1
    const uint32_t nchunks = (KB + ckb - 1) / ckb;
    // only a plain store takes split tiles (their pieces add into a zeroed output)
    constexpr bool kSplit = std::is_same<Epi, StoreEpi>::value;
    const uint32_t dp_tiles = kSplit && dp_tiles_arg < tiles ? dp_tiles_arg : tiles;
    const uint32_t tparts = dp_tiles < tiles ? tail_parts : 0u;
    bool failed = false;
    auto fail_both = [&]() {
        failed = true;
        *abort = 1;
        st_cluster_u32(peer_abort, 1u);
    };

    if (warp == 0 || warp == 6) {
        if (lane == 0) {
            // ---------------- TMA producers (both CTAs): warp 0 loads the matrix tiles (and, in the
            // leader, arms each stage for the bytes of both CTAs), warp 6 the vector tiles; the two
            // copy streams issue in parallel
            const bool mat = warp == 0;
            if (mat) tma_prefetch_desc(&a_map);
            else {
#pragma unroll
                for (int u = 0; u < (PLANED ? 4 : 1); ++u) tma_prefetch_desc(&bm.m[u]);
            }
            const uint32_t kpp = PLANED ? ckb * plane_chunks : KB;   // k-steps per limb plane
            uint32_t it = 0, st = 0, ph = 0;
            PairPieceIter pit(tiles, dp_tiles, n_tiles, nchunks, tparts, cluster, nclusters);
            PairPiece pc;
            while (!failed && pit.next(pc, dp_tiles, n_tiles, nchunks)) {
                const uint32_t t = pc.t;
                const uint32_t kb0 = pc.c0 * ckb, kb1 = pc.c1 * ckb < KB ? pc.c1 * ckb : KB;
                const int32_t m0 = static_cast<int32_t>((t / n_tiles) * 2 * kPM + rank * kPM);
                const int32_t r0 = static_cast<int32_t>((t % n_tiles) * BN + rank * (BN / 2));
                if (mat) {
                    const uint32_t v0 = (t % n_tiles) * QPT;
                    const uint32_t nv = v0 < NV ? (NV - v0 < (uint32_t)QPT ? NV - v0 : (uint32_t)QPT) : 0u;
                    if (static_cast<uint32_t>(m0) + kPM <= M) epi.prefetch(static_cast<uint64_t>(m0), v0, nv);
                }
                uint32_t u = 0, kin = 0;   // limb plane of k-step kb, and kb's place in it (planed: whole tiles)
                for (uint32_t kb = kb0; kb < kb1; ++kb, ++it) {
                    if (!mbar_wait(&empty[st], ph ^ 1u, abort)) {
                        fail_both();
                        break;
                    }
                    uint8_t *sa = smem + st * Cfg::kStageBytes;
                    if (mat) {
                        if (leader) {
                            const uint32_t brows = pair_b_box_rows(BN, PLANED, static_cast<int>(u));
                            mbar_arrive_expect_tx(&full[st], 2u * (Cfg::kABytes + brows * kPK * 2u));
                        }
                        tma_load_2d_pair(sa, &a_map, full_c + 8u * st, static_cast<int32_t>(kb * kPK), m0);
                    } else {
                        tma_load_2d_pair(sa + Cfg::kABytes, &bm.m[u], full_c + 8u * st,
                                         static_cast<int32_t>(kb * kPK), r0);
                    }
                    if (++st == (uint32_t)ST) {
                        st = 0;
                        ph ^= 1u;
                    }
                    if (++kin == kpp) {
                        kin = 0;
                        ++u;
                    }
                }
            }
            if (leader && mat) {
                // the stages still owed bytes (both producers' and the peer's copies) must land before exit
                const uint32_t inflight = it < (uint32_t)ST ? it : (uint32_t)ST;
                for (uint32_t j = it - inflight; j < it; ++j)
                    if (!drain_wait_p(&full[j % ST], (j / ST) & 1u)) failed = true;
            }
        }
    } else if (warp == 1) {
        if (leader) {
            // ---------------- MMA issuer (leader only): the whole warp walks the loop, one lane issues
            uint32_t ci = 0, st = 0, ph = 0;
            const uint32_t kpp = PLANED ? ckb * plane_chunks : KB;
            bool issued = false;
            PairPieceIter pit(tiles, dp_tiles, n_tiles, nchunks, tparts, cluster, nclusters);
            PairPiece pc;
            while (!failed && pit.next(pc, dp_tiles, n_tiles, nchunks)) {
                const uint32_t kb0 = pc.c0 * ckb, kb1 = pc.c1 * ckb < KB ? pc.c1 * ckb : KB;
                uint32_t d_tmem = tmem_base;
                uint32_t u = 0, kin = 0, kc = 0;   // limb plane, place in the plane, place in the chunk
                for (uint32_t kb = kb0; kb < kb1; ++kb) {
                    if (kc == 0) {
                        const uint32_t buf = ci & 1u;
                        const bool ok = mbar_wait(&acc_empty[buf], ((ci >> 1) & 1u) ^ 1u, abort);
                        if (__any_sync(0xffffffffu, !ok)) {
                            fail_both();
                            break;
                        }
                        tc_fence_after();
                        d_tmem = tmem_base + buf * BN;
                    }
                    const bool ok = mbar_wait(&full[st], ph, abort);
                    if (__any_sync(0xffffffffu, !ok)) {
                        fail_both();
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_addr(smem + st * Cfg::kStageBytes);
                    const uint64_t adesc = umma_desc_sw128(sa);
                    const uint64_t bdesc = umma_desc_sw128(sa + Cfg::kABytes);
                    const uint32_t idesc = umma_idesc_f16(2 * kPM, PLANED ? (4u - u) * (BN / 4) : BN);
                    const bool last_of_chunk = kc == ckb - 1 || kb == kb1 - 1;
                    if (elect_one()) {
#pragma unroll
                        for (int k = 0; k < kPK / 16; ++k)
                            umma_f16_pair(d_tmem, adesc + 2u * k, bdesc + 2u * k, idesc,
                                          (kc != 0 || k != 0 || (TMEMSUM && kb >= 2u * ckb)) ? 1u : 0u);
                        umma_commit_pair(&empty[st], 3);
                        if (last_of_chunk) umma_commit_pair(&acc_full[ci & 1u], 3);
                    }
                    __syncwarp();
                    issued = true;
                    if (last_of_chunk) ++ci;
                    if (++st == (uint32_t)ST) {
                        st = 0;
                        ph ^= 1u;
                    }
                    if (++kc == ckb) kc = 0;
                    if (++kin == kpp) {
                        kin = 0;
                        ++u;
                    }
                }
            }
            // every pair MMA must finish before TMEM is released
            if (issued) {
                if (elect_one()) umma_commit_pair(mma_done, 1);
                __syncwarp();
                if (!drain_wait_p(mma_done, 0)) failed = true;
            }
        }
    } else {
        // ---------------- epilogue (warps 2..5 of both CTAs; TMEM lane quarter = warp % 4)
        const uint32_t quarter = static_cast<uint32_t>(warp & 3);
        const uint32_t lane_addr = (quarter * 32u) << 16;
        uint32_t ci = 0;
        PairPieceIter pit(tiles, dp_tiles, n_tiles, nchunks, tparts, cluster, nclusters);
        PairPiece pc;
        while (!failed && pit.next(pc, dp_tiles, n_tiles, nchunks)) {
            const uint32_t t = pc.t;
            const uint32_t row = (t / n_tiles) * 2 * kPM + rank * kPM + quarter * 32u + static_cast<uint32_t>(lane);
            const uint32_t v0 = (t % n_tiles) * QPT;
            constexpr int RUN = TMEMSUM ? 1 : QPT;   // running sums kept in registers
            uint32_t run[RUN];
#pragma unroll
            for (int q = 0; q < RUN; ++q) run[q] = 0u;
            // client tiles are short in K: their epilogue inputs are loaded as the tile starts
            constexpr int EARLY = PLANED ? QPT : 1;
            uint32_t early[EARLY];
            if constexpr (PLANED) {
#pragma unroll
                for (int q = 0; q < QPT; ++q) early[q] = (row < M && v0 + q < NV) ? epi.pre(row, v0 + q) : 0u;
            }
            for (uint32_t c = pc.c0; c < pc.c1; ++c, ++ci) {
                const uint32_t buf = ci & 1u;
                const bool ok = mbar_wait(&acc_full[buf], (ci >> 1) & 1u, abort);
                if (__any_sync(0xffffffffu, !ok)) {   // the TMEM loads below are warp-collective
                    fail_both();
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem_base + lane_addr + buf * BN;
                if constexpr (TMEMSUM) {
                    const float pf = static_cast<float>(epi.p), inv = 1.0f / pf;
                    if (c + 1 < nchunks) {
                        // replace this buffer's running sums by small representatives of their
                        // residues mod p: q = x / p rounded to an integer through the 1.5 * 2^23
                        // rounding constant, r = x - q p with |r| <= 1.5 p; q p and r are integers
                        // below 2^24, so the fused multiply-add is exact.  Four 32-column loads per
                        // wait; the next MMAs into this buffer accumulate on top.
                        constexpr float kRound = 12582912.0f;
#pragma unroll 1
                        for (int j0 = 0; j0 < BN / 32; j0 += 4) {
                            uint32_t v[4][32];
#pragma unroll
                            for (int g = 0; g < 4; ++g) tmem_ld32(acc + 32u * (j0 + g), v[g]);
                            tmem_wait_ld();
#pragma unroll
                            for (int g = 0; g < 4; ++g) {
#pragma unroll
                                for (int q = 0; q < 32; ++q) {
                                    const float x = __uint_as_float(v[g][q]);
                                    const float qf = __fsub_rn(__fmaf_rn(x, inv, kRound), kRound);
                                    v[g][q] = __float_as_uint(__fmaf_rn(-qf, pf, x));
                                }
                                tmem_st32(acc + 32u * (j0 + g), v[g]);
                            }
                        }
                        tmem_wait_st();
                        if (c + 2 < nchunks) {
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive_cluster(acc_empty_c + 8u * buf);
                        }
                        // the second-to-last chunk's buffer is held for the final combine
                        continue;
                    }
                    // last chunk: its buffer plus the other buffer's residue, mod p, to the output.  Each
                    // buffer is first cut to a representative |r| <= 1.5 p as in the pass above, so
                    // their sum is an exact float of at most 3 p; q = floor(sum / p) is then off by at
                    // most one, which the two compares put right, and the residue stays exact.
                    const uint32_t oth = tmem_base + lane_addr + (buf ^ 1u) * BN;
                    constexpr float kRound = 12582912.0f;
#pragma unroll 1
                    for (int j = 0; j < BN / 32; ++j) {
                        uint32_t v[32], w[32];
                        tmem_ld32(acc + 32u * j, v);
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
                        mbar_arrive_cluster(acc_empty_c + 8u * buf);
                        if (nchunks >= 2) mbar_arrive_cluster(acc_empty_c + 8u * (buf ^ 1u));
                    }
                    continue;
                } else if constexpr (PLANED) {
                    const uint32_t u = c / plane_chunks;
                    const uint32_t half = (4u - u) * HQ;   // N / 2
                    for (uint32_t s = u; s < 4; ++s) {
                        const uint32_t col = (3u - s) * HQ;
                        if constexpr (HQ == 32) {
                            uint32_t v[2][32];
                            tmem_ld32(acc + col, v[0]);
                            tmem_ld32(acc + half + col, v[1]);
                            tmem_wait_ld();
#pragma unroll
                            for (int h = 0; h < 2; ++h)
#pragma unroll
                                for (int q = 0; q < 32; ++q)
                                    run[32 * h + q] += static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[h][q])))
                                                       << (8u * s);
                        } else {
                            uint32_t v[2][16];
                            tmem_ld16(acc + col, v[0]);
                            tmem_ld16(acc + half + col, v[1]);
                            tmem_wait_ld();
#pragma unroll
                            for (int h = 0; h < 2; ++h)
#pragma unroll
                                for (int q = 0; q < 16; ++q)
                                    run[16 * h + q] += static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[h][q])))
                                                       << (8u * s);
                        }
                    }
                } else {
                    // two 32-column loads per wait; column 4q + k is limb k of vector q
                    constexpr int NJ = BN / 32;
                    constexpr int JB = NJ < 2 ? NJ : 2;
#pragma unroll
                    for (int j0 = 0; j0 < NJ; j0 += JB) {
                        uint32_t v[JB][32];
#pragma unroll
                        for (int g = 0; g < JB; ++g) tmem_ld32(acc + 32u * (j0 + g), v[g]);
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
                if (lane == 0) mbar_arrive_cluster(acc_empty_c + 8u * buf);
            }
            if (failed) break;
            if constexpr (TMEMSUM) continue;   // the last chunk already wrote the tile
            if constexpr (kSplit) {
                if (row < M && !(pc.c0 == 0 && pc.c1 == nchunks)) {
                    // part of a split tile: exact, since addition mod 2^32 commutes
#pragma unroll
                    for (int q = 0; q < QPT; ++q)
                        if (v0 + q < NV) epi.add(row, v0 + q, run[q]);
                    continue;
                }
            }
            if (row < M) {
                if constexpr (PLANED) {
#pragma unroll
                    for (int q = 0; q < QPT; ++q)
                        if (v0 + q < NV) epi.put(row, v0 + q, run[q], early[q]);
                } else {
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
    }

    if (failed) {
        *abort = 1;
        *status = kDevTimeout;
        // a copy this CTA issued may still be landing (after an abort its stage is never
        // consumed): give it a bounded moment before the CTA can exit
        const uint64_t t0 = global_ns();
        while (global_ns() - t0 < 200000ull) {
        }
    }
    // no CTA leaves (or frees TMEM) while its peer may still reach its shared memory or TMEM
    __syncwarp();
    tc_fence_before();
    cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, Cfg::kTmemCols);
    }
}

// ------------------------------------------------------------------ host side
template <int BN, class Epi, bool PLANED>
static cudaError_t set_pair_attr() {
    return cudaFuncSetAttribute(limb_gemm_pair_kernel<BN, Epi, PLANED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                PairCfg<BN>::kSmemBytes);
}

cudaError_t prepare_limb_gemm_pair_kernels() {
    cudaError_t e;
    if ((e = set_pair_attr<64, StoreEpi, false>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<128, StoreEpi, false>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<256, StoreEpi, false>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<64, QueryNoiseEpi, false>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<128, QueryNoiseEpi, false>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<256, QueryNoiseEpi, false>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<64, RecoverEpi, false>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<128, RecoverEpi, false>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<256, RecoverEpi, false>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<128, QueryNoiseEpi, true>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<256, QueryNoiseEpi, true>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<128, RecoverEpi, true>()) != cudaSuccess) return e;
    if ((e = set_pair_attr<256, RecoverEpi, true>()) != cudaSuccess) return e;
    return set_pair_attr<256, ModPEpi, false>();
}

int limb_gemm_pair_bn_for(uint32_t nv) {
    const uint32_t cols = 4 * nv;
    if (cols <= 64) return 64;
    if (cols <= 128) return 128;
    return 256;
}

// Launch configuration of a pair kernel: clusters of 2 CTAs, one CTA per SM.
template <int BN>
static cudaLaunchConfig_t pair_config(unsigned clusters, cudaStream_t stream, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(kPThreads);
    cfg.dynamicSmemBytes = PairCfg<BN>::kSmemBytes;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// CTA pairs that fit on the GPU at once (a GPC with an odd number of free SMs leaves one
// idle), per device; the persistent grid is never larger, so no cluster waits for a second wave.
template <int BN, class Epi, bool PLANED>
static int resident_pairs(int num_sms) {
    static int cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return num_sms / 2;
    if (cache[dev] > 0) return cache[dev];
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config<BN>(static_cast<unsigned>(num_sms / 2), nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, limb_gemm_pair_kernel<BN, Epi, PLANED>, &cfg) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return num_sms / 2;
    }
    n = n < num_sms / 2 ? n : num_sms / 2;
    cache[dev] = n;
    return n;
}

// k-steps (64 deep) per exact chunk: 8 for digits times limbs (StoreEpi), 16 for limbs times limbs.
template <class Epi>
constexpr uint32_t pair_chunk_kb() {
    return (std::is_same<Epi, StoreEpi>::value || std::is_same<Epi, ModPEpi>::value) ? 8u : 16u;
}

// Schedule of a plain-store launch over `tiles` pair tiles (n_tiles per row tile, nchunks exact
// chunks each) on `pairs` resident clusters.  Measured in tile times, whole tiles take
// ceil(tiles / pairs); a split keeps dp whole tiles (all waves but the last full one, rounded down
// to whole row tiles) and cuts the rest over tail_parts * n_tiles clusters (the grouping of
// PairPieceIter).  The split is taken when it saves at least 8% of that count, and never when
// every cluster is busy on a one-tile-wide batch: that launch reads the fp16 copy of the database
// at the HBM rate whatever the balance, and split pieces only add their atomics.  Nor is it taken
// for more than 3 tiles per row tile unless the tiles fill at most half of the clusters: the
// clusters of a group drift apart over a long tail, and the more of them read one row tile, the
// more of its rows they read from DRAM again (8192 rows, 256 queries: 1.48 GB read instead of
// 0.67 GB, 326 us instead of 306 us).  Returns false when no tile is split; otherwise the
// cluster count, dp and tail_parts.
static bool pair_split_schedule(uint64_t tiles, uint64_t n_tiles, uint32_t nchunks, uint64_t pairs,
                                uint64_t *clusters, uint32_t *dp_tiles, uint32_t *tail_parts) {
    if (pairs == 0 || nchunks < 2 || tiles % pairs == 0 || n_tiles > pairs) return false;
    if (tiles > pairs && n_tiles == 1) return false;
    if (n_tiles > 3 && 2 * tiles > pairs) return false;
    uint64_t dp = 0;
    if (tiles > pairs) dp = ((tiles / pairs - 1) * pairs) / n_tiles * n_tiles;
    const uint64_t tail_units = (tiles - dp) / n_tiles * nchunks;
    uint64_t P = pairs / n_tiles;
    if (P > tail_units) P = tail_units;
    const double whole = static_cast<double>((tiles + pairs - 1) / pairs);
    const double split = static_cast<double>(dp) / pairs + static_cast<double>(tiles - dp) / (P * n_tiles);
    if (split > 0.92 * whole) return false;
    *clusters = dp > 0 ? pairs : P * n_tiles;
    *dp_tiles = static_cast<uint32_t>(dp);
    *tail_parts = static_cast<uint32_t>(P);
    return true;
}

template <int BN, class Epi, bool PLANED>
static cudaError_t launch_pair_t(const CUtensorMap &a_map, const PairBMaps &bm, const Epi &epi, uint32_t M,
                                 uint32_t NV, uint32_t KB, uint32_t ckb, uint32_t plane_chunks, int num_sms,
                                 int *status, cudaStream_t stream) {
    const uint64_t m_tiles = (M + 2ull * kPM - 1) / (2ull * kPM);
    constexpr uint64_t qpt = BN / Epi::kLimbs;   // vectors per pair tile
    const uint64_t n_tiles = (NV + qpt - 1) / qpt;
    const uint64_t tiles = m_tiles * n_tiles;
    const uint64_t pairs = static_cast<uint64_t>(resident_pairs<BN, Epi, PLANED>(num_sms));
    uint64_t clusters = tiles < pairs ? tiles : pairs;
    uint32_t dp = 0xffffffffu, tail_parts = 0;
    if constexpr (std::is_same<Epi, StoreEpi>::value) {
        // split tiles add into the output, so it is zeroed first; only a dense output (every
        // element of the M x NV block, in either order) can be zeroed in one piece
        const bool dense = (epi.ld_m == 1 && epi.ld_b == M) || (epi.ld_b == 1 && epi.ld_m == NV);
        uint64_t c2 = clusters;
        uint32_t dp2 = 0, tp2 = 0;
        if (dense && pair_split_schedule(tiles, n_tiles, (KB + ckb - 1) / ckb, pairs, &c2, &dp2, &tp2)) {
            const cudaError_t e = cudaMemsetAsync(epi.out, 0, 4ull * M * NV, stream);
            if (e != cudaSuccess) return e;
            clusters = c2;
            dp = dp2;
            tail_parts = tp2;
        }
    }
    if (clusters == 0) return cudaSuccess;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config<BN>(static_cast<unsigned>(clusters), stream, attr);
    return cudaLaunchKernelEx(&cfg, limb_gemm_pair_kernel<BN, Epi, PLANED>, a_map, bm, epi, M, NV, KB, ckb,
                              plane_chunks, dp, tail_parts, status);
}

template <class Epi>
static cudaError_t launch_pair_epi(int bn, const CUtensorMap &a_map, const PairBMaps &bm, const Epi &epi, uint32_t M,
                                   uint32_t NV, uint64_t K, uint32_t plane_chunks, int num_sms, int *status,
                                   cudaStream_t stream) {
    if (M == 0 || NV == 0 || K == 0 || num_sms < 2) return cudaErrorInvalidValue;
    const uint32_t KB = static_cast<uint32_t>((K + kPK - 1) / kPK);
    if constexpr (Epi::kLimbs == 1) {   // one row per vector: 256-wide plain tiles only
        if (bn != 256 || plane_chunks != 0) return cudaErrorInvalidValue;
        return launch_pair_t<256, Epi, false>(a_map, bm, epi, M, NV, KB, pair_chunk_kb<Epi>(), 0, num_sms, status,
                                             stream);
    } else {
        if (plane_chunks == 0) {
            constexpr uint32_t ckb = pair_chunk_kb<Epi>();
            switch (bn) {
                case 64:
                    return launch_pair_t<64, Epi, false>(a_map, bm, epi, M, NV, KB, ckb, 0, num_sms, status, stream);
                case 128:
                    return launch_pair_t<128, Epi, false>(a_map, bm, epi, M, NV, KB, ckb, 0, num_sms, status, stream);
                case 256:
                    return launch_pair_t<256, Epi, false>(a_map, bm, epi, M, NV, KB, ckb, 0, num_sms, status, stream);
                default: return cudaErrorInvalidValue;
            }
        }
        if constexpr (std::is_same<Epi, StoreEpi>::value) {
            return cudaErrorInvalidValue;
        } else {
            // every chunk lies inside one limb plane of n = K / 4 columns: 1024-deep chunks when n is a
            // multiple of 1024, else 512-deep (plane_chunks = n / 512 then)
            if (K != 4ull * 512 * plane_chunks) return cudaErrorInvalidValue;
            const uint32_t ckb = plane_chunks % 2 == 0 ? 16u : 8u;
            const uint32_t pc = ckb == 16u ? plane_chunks / 2 : plane_chunks;
            switch (bn) {
                case 128:
                    return launch_pair_t<128, Epi, true>(a_map, bm, epi, M, NV, KB, ckb, pc, num_sms, status, stream);
                case 256:
                    return launch_pair_t<256, Epi, true>(a_map, bm, epi, M, NV, KB, ckb, pc, num_sms, status, stream);
                default: return cudaErrorInvalidValue;
            }
        }
    }
}

cudaError_t launch_limb_gemm_pair(int bn, const CUtensorMap &a_map, const PairBMaps &bm, uint32_t *out,
                                  uint64_t ld_m, uint64_t ld_b, uint32_t M, uint32_t NV, uint64_t K, int num_sms,
                                  int *status, cudaStream_t stream) {
    return launch_pair_epi(bn, a_map, bm, StoreEpi{out, ld_m, ld_b}, M, NV, K, 0, num_sms, status, stream);
}

cudaError_t launch_limb_gemm_pair_query(int bn, const CUtensorMap &a_map, const PairBMaps &bm,
                                        const QueryNoiseEpi &epi,
                                        uint32_t M, uint32_t NV, uint64_t K, uint32_t plane_chunks, int num_sms,
                                        int *status, cudaStream_t stream) {
    return launch_pair_epi(bn, a_map, bm, epi, M, NV, K, plane_chunks, num_sms, status, stream);
}

cudaError_t launch_limb_gemm_pair_recover(int bn, const CUtensorMap &a_map, const PairBMaps &bm,
                                          const RecoverEpi &epi, uint32_t M, uint32_t NV, uint64_t K,
                                          uint32_t plane_chunks, int num_sms, int *status, cudaStream_t stream) {
    return launch_pair_epi(bn, a_map, bm, epi, M, NV, K, plane_chunks, num_sms, status, stream);
}

cudaError_t launch_limb_gemm_pair_modp(const CUtensorMap &a_map, const PairBMaps &bm, const ModPEpi &epi, uint32_t M,
                                       uint32_t NV, uint64_t K, int num_sms, int *status, cudaStream_t stream) {
    return launch_pair_epi(256, a_map, bm, epi, M, NV, K, 0, num_sms, status, stream);
}

}  // namespace qpadl
