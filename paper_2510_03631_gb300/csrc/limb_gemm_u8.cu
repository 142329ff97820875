// Exact mod-2^32 product of one or several databases with batches of Z_q
// vectors, reading the databases as stored (uint8 digits):
//     OUT_g[i][b] = sum_j D_g[i][j] * X_g[b][j]   (mod 2^32), g < ngroups.
// A one-row mode (LPV = 1) takes vectors of small signed integers (|x| <=
// 128, e.g. centred Z_p elements) as single fp16 rows and stores their exact
// signed sums; the Goldberg Response over Z_p uses it.
//
// Same exact byte-limb algebra as limb_gemm.cu (balanced limbs in fp16,
// fp32 accumulation over 512-deep K-chunks, int32 recombination; see there),
// but the A operand never exists as fp16 in memory: TMA brings 128-row digit
// tiles (128 or 256 digits per row) into shared memory from a blocked copy of
// the digits (128 x 128 tiles stored contiguously, so each stage is one
// contiguous 16-32 KB read), converter warps turn each row
// into fp16 (one byte permute per two digits: the byte under a zero exponent
// is the subnormal d * 2^-24, exact; the epilogue scales sums back by 2^24)
// and store it into tensor memory, and the MMA reads A from tensor memory
// (tcgen05.mma with A in TMEM).  Half the HBM traffic of the fp16 copy, and
// shared memory carries only the digit tile (128-byte swizzled, so the row-
// per-thread reads are free of bank conflicts) and the limb tile.
//
// One launch can serve several databases with their own batches (the
// serving loop's grouped launch).  The work of all groups is one list of
// units (one tile's one pipeline stage) that the persistent CTAs split into
// equal contiguous shares across tile boundaries (stream-K), so the last
// wave is never partial; tiles shared by two CTAs are summed with atomic
// adds, which is exact because the result is taken mod 2^32.
//
// Three rings decouple the stages (a stage = KS digits of a 128-row tile):
//   digit tiles in shared memory (freed as soon as they are converted),
//   limb tiles in shared memory (freed when the MMA that reads them completes),
//   fp16 A slots in TMEM (freed when the MMA that reads them completes),
// so the digit loads run ahead of the MMA instead of waiting for it.
//
// Pair form (PAIR = true): a tile is 256 rows over a cluster of two CTAs on
// two SMs (tcgen05 cta_group::2).  Each CTA keeps its own digit ring and
// converters and writes its own 128 rows of fp16 digits into its own TMEM A
// slots; each loads half of the limb rows.  The leader CTA issues the pair
// MMAs (M = 256, A from both CTAs' TMEM, B from both CTAs' shared memory):
// one instruction drives both SMs' tensor cores, and each SM loads only half
// of every limb tile.  Both CTAs' converters arrive on the
// leader's `aready`, both CTAs' limb copies complete on the leader's `lfull`,
// both epilogues arrive on the leader's `acc_empty`; the leader's MMA commits
// to `afree`, `lfree` and `acc_full` of both CTAs.  A cluster barrier keeps
// either CTA from leaving while its peer may still reach its shared memory.
//
// Warp roles (480 threads, one CTA per SM):
//   warp 0       TMA producer of the digit tiles (wider tiles: the first ring's worth issued before
//                setup ends; 32-column tiles: the digits pulled into L2 a few stages ahead)
//   warp 1       TMEM allocation; one thread issues the MMAs
//   warps 2..5   epilogue: drain one of two BN-column accumulators per chunk
//   warps 6..13  converters, two groups of four, each owning every other stage:
//                digits -> fp16 A tiles in TMEM (one row per thread)
//   warp 14      TMA producer of the limb tiles
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "limb_gemm_u8.cuh"
#include "ptx.cuh"

namespace qpadl {

namespace {

constexpr int kBM = 128;
constexpr int kThreads = 480;
constexpr int kConvGroups = 2;
constexpr uint32_t kTmemCols = 512;
// The A operand holds each digit d as the fp16 subnormal d * 2^-24, so an accumulator holds
// 2^-24 times an exact integer sum (|sum| <= 2^24: the fp32 significand keeps it exact); the
// epilogue scales it back by 2^24 (exact) before rounding to an integer.
constexpr float kUnscale = 16777216.0f;

// BN: limb columns per tile; KS: digits per row per pipeline stage (a
// multiple of 128: each digit tile is 128 rows x 128 bytes, 128-byte swizzle).
template <int BN, int KS, bool PAIR = false>
struct U8Cfg {
    static constexpr int kSubA = KS / 128;                          // digit boxes per stage
    static constexpr int kSubB = KS / 64;                           // limb boxes per stage
    static constexpr uint32_t kDigBytes = kBM * KS;                 // one digit slot
    static constexpr uint32_t kBBoxBytes = (PAIR ? BN / 2 : BN) * 128;   // this CTA's limb rows
    static constexpr uint32_t kLimbBytes = kSubB * kBBoxBytes;      // one limb slot
    static constexpr uint32_t kSlotCols = KS / 2;                   // fp16 pairs per row per stage
    // Digit and A-slot counts are even: converter group g owns the stages with it % 2 == g and
    // so every phase of the slots with index % 2 == g (a parity wait never falls two phases behind).
    static constexpr int kSA = (((kTmemCols - 2 * BN) / kSlotCols) / 2) * 2;
    // pair tiles halve a CTA's limb slots, which leaves room for a deeper digit ring
    static constexpr int kSD = KS == 128 ? (PAIR ? (BN == 128 ? 8 : 10) : (BN == 128 ? 6 : 8)) : (BN == 128 ? 2 : 4);
    static constexpr int kRingBytes = PAIR ? 224 * 1024 : 192 * 1024;
    static constexpr int kSLfit = (kRingBytes - kSD * kDigBytes) / kLimbBytes;
    static constexpr int kSL = kSLfit < 8 ? kSLfit : 8;
    static constexpr uint32_t kAColBase = 2 * BN;                   // A slots after the accumulators
    static constexpr int kChunkStages = 512 / KS;                   // stages per exact 512-deep K-chunk
    static constexpr uint32_t kLimbBase = kSD * kDigBytes;
    static constexpr uint32_t kBarBase = kLimbBase + kSL * kLimbBytes;
    static constexpr int kSmemUsed = kBarBase + (2 * kSD + 2 * kSL + 2 * kSA + 5) * 8 + 16 + 1024;
    // padded so that only one CTA fits per SM (it allocates all of TMEM)
    static constexpr int kSmemBytes = kSmemUsed > 120 * 1024 ? kSmemUsed : 120 * 1024;
    static_assert(kSA >= 2 && kSD >= 2 && kSD % 2 == 0 && kSL >= 2, "ring sizes");
    static_assert(KS % 128 == 0 && 512 % KS == 0, "stage depth must divide the exact chunk");
    static_assert(kSmemUsed <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ bool drain_wait_u(uint64_t *bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > QPADL_WAIT_NS) return false;
    }
    return true;
}

// One CTA's piece of one tile: stages [ks0, ks1) of tile (m0, n0) of group g.
struct Seg {
    uint32_t g, m0, n0, ks0, ks1, ns;
};

// The next piece of this CTA's unit range [u, u_end); advances u.
__device__ __forceinline__ bool next_seg(const GroupedGemmArgs &a, uint32_t &u, uint32_t u_end, uint32_t bn,
                                         Seg &s, uint32_t tile_rows = kBM) {
    if (u >= u_end) return false;
    uint32_t g = 0;
    while (g + 1 < a.ngroups && u >= a.g[g + 1].unit_begin) ++g;
    const uint32_t ns = a.g[g].KB;
    const uint32_t local = u - a.g[g].unit_begin;
    const uint32_t tile = local / ns;
    s.g = g;
    s.m0 = (tile / a.g[g].n_tiles) * tile_rows;
    s.n0 = (tile % a.g[g].n_tiles) * bn;
    s.ks0 = local % ns;
    s.ks1 = (ns - s.ks0 < u_end - u) ? ns : s.ks0 + (u_end - u);
    s.ns = ns;
    u += s.ks1 - s.ks0;
    return true;
}

// A CTA's (pair form: a cluster's) pieces: whole tiles part, part + nparts, ... below
// dp_tiles, then its even share of the units from dp_units on.
struct SegIter {
    uint32_t t, u, u_end;
    __device__ __forceinline__ SegIter(const GroupedGemmArgs &a, uint32_t part, uint32_t nparts) {
        t = part;
        const uint32_t tail = a.total_units - a.dp_units;
        u = a.dp_units + static_cast<uint32_t>((uint64_t)part * tail / nparts);
        u_end = a.dp_units + static_cast<uint32_t>((uint64_t)(part + 1) * tail / nparts);
    }
    __device__ __forceinline__ bool next(const GroupedGemmArgs &a, uint32_t bn, uint32_t tile_rows, uint32_t nparts,
                                         Seg &s) {
        if (t < a.dp_tiles) {
            uint32_t g = 0;
            while (g + 1 < a.ngroups && t >= a.g[g + 1].tile_begin) ++g;
            const uint32_t local = t - a.g[g].tile_begin;
            s.g = g;
            s.m0 = (local / a.g[g].n_tiles) * tile_rows;
            s.n0 = (local % a.g[g].n_tiles) * bn;
            s.ks0 = 0;
            s.ks1 = s.ns = a.g[g].KB;
            t += nparts;
            return true;
        }
        return next_seg(a, u, u_end, bn, s, tile_rows);
    }
};

}  // namespace

// LPV: vector-operand rows per vector.  4 = the four byte limbs of 32-bit vectors, recombined
// mod 2^32; 1 = one row per vector (small signed integers, e.g. centred field elements), whose
// exact 32-bit signed sums are stored.
template <int BN, int KS, int LPV = 4, bool PAIR = false>
__global__ void __launch_bounds__(kThreads, 1)
    limb_gemm_u8_kernel(const __grid_constant__ GroupedGemmArgs args, int *__restrict__ status) {
    using Cfg = U8Cfg<BN, KS, PAIR>;
    static_assert(!PAIR || BN >= 32, "a pair MMA needs N >= 32 (16 limb rows per CTA)");
    constexpr uint32_t TM = PAIR ? 2 * kBM : kBM;   // rows per tile
    static_assert(LPV == 4 || (LPV == 1 && BN <= 64), "one-row vectors: at most 64 running sums per thread");
    constexpr int QPT = BN / LPV;
    constexpr int SD = Cfg::kSD, SL = Cfg::kSL, SA = Cfg::kSA;
    constexpr int CS = Cfg::kChunkStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *dig = smem;                       // [SD] digit slots, each kSubA 16 KB boxes
    uint8_t *limb = smem + Cfg::kLimbBase;     // [SL] limb slots, each kSubB boxes, 1024-aligned
    uint64_t *dfull = reinterpret_cast<uint64_t *>(smem + Cfg::kBarBase);
    uint64_t *dfree = dfull + SD;
    uint64_t *lfull = dfree + SD;
    uint64_t *lfree = lfull + SL;
    uint64_t *aready = lfree + SL;
    uint64_t *afree = aready + SA;
    uint64_t *acc_full = afree + SA;   // [2]
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *mma_done = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const uint32_t roff = rank * kBM;   // this CTA's first row within a tile
    // this CTA's (pair: cluster's) pieces: round-robin whole tiles, then a share of the rest
    const uint32_t part = PAIR ? (blockIdx.x >> 1) : blockIdx.x;
    const uint32_t nparts = PAIR ? (gridDim.x >> 1) : gridDim.x;
    uint32_t early = 0;   // digit stages the producer (thread 0) issued before the setup barrier

    if (threadIdx.x == 0) {
        for (int s = 0; s < SD; ++s) {
            mbar_init(&dfull[s], 1);
            mbar_init(&dfree[s], 4);   // the four warps of the converter group that owns the slot
        }
        for (int s = 0; s < SL; ++s) {
            mbar_init(&lfull[s], 1);
            mbar_init(&lfree[s], 1);
        }
        for (int s = 0; s < SA; ++s) {
            mbar_init(&aready[s], PAIR ? 8 : 4);   // the owning converter group (of both CTAs)
            mbar_init(&afree[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], PAIR ? 8 : 4);
        }
        mbar_init(mma_done, 1);
        *abort = 0;
        fence_barrier_init();
        // the first ring's digit loads need only this CTA's own barriers and shared memory: they
        // go out now, while TMEM is allocated and the CTAs meet at the setup barrier (tiles wider
        // than 32 columns; the narrowest ones measured faster with their L2 prefetch prologue first)
        if constexpr (BN > 32) {
            Seg tr;
            SegIter sit(args, part, nparts);
            while (early < static_cast<uint32_t>(SD) && sit.next(args, BN, TM, nparts, tr)) {
                for (uint32_t ks = tr.ks0; ks < tr.ks1 && early < static_cast<uint32_t>(SD); ++ks, ++early) {
                    mbar_arrive_expect_tx(&dfull[early], Cfg::kDigBytes);
                    tma_load_4d(dig + early * Cfg::kDigBytes, &args.a[tr.g], &dfull[early], 0, 0,
                                static_cast<int32_t>(ks * KS / 128), static_cast<int32_t>((tr.m0 + roff) / kBM));
                }
            }
        }
    }
    if (warp == 1) {
        if constexpr (PAIR) {
            tmem_alloc_pair(tmem_slot, kTmemCols);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(tmem_slot, kTmemCols);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    if constexpr (PAIR) cluster_sync();   // both CTAs' barriers exist before either touches the other's
    else __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const bool leader = rank == 0;
    // shared::cluster addresses of the leader's barriers that both CTAs signal (pair form)
    const uint32_t lfull_c = PAIR ? cluster_addr(lfull, 0) : 0u;
    const uint32_t aready_c = PAIR ? cluster_addr(aready, 0) : 0u;
    const uint32_t acc_empty_c = PAIR ? cluster_addr(acc_empty, 0) : 0u;
    const uint32_t peer_abort = PAIR ? cluster_addr(const_cast<int *>(abort), rank ^ 1u) : 0u;
    bool failed = false;
    auto fail_here = [&]() {
        failed = true;
        *abort = 1;
        if constexpr (PAIR) st_cluster_u32(peer_abort, 1u);
    };

    // waits until every copy this thread issued into `ring` has landed (so the CTA can exit)
    auto drain_ring = [&](uint64_t *ring, int slots, uint32_t issued) {
        const uint32_t inflight = issued < (uint32_t)slots ? issued : (uint32_t)slots;
        for (uint32_t j = issued - inflight; j < issued; ++j)
            if (!drain_wait_u(&ring[j % slots], (j / slots) & 1u)) failed = true;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- digit producer (thread 0; stages below `early` are already issued)
            // For the narrowest tiles, whose stages stream fastest, a second walker over the same
            // stage sequence pulls each digit box into L2 kPrefetch stages before its load; wider
            // tiles measured faster without it (each prefetch costs the issuing thread ~0.1 us).
            constexpr int kPrefetch = BN <= 32 ? 8 : 0;
            uint32_t pks = 0;
            Seg ps;
            SegIter pit(args, part, nparts);
            bool pvalid = kPrefetch > 0 && pit.next(args, BN, TM, nparts, ps);
            if (pvalid) pks = ps.ks0;
            auto walk = [&](bool issue) {
                if (!pvalid) return;
                if (issue)
                    tma_prefetch_l2_4d(&args.a[ps.g], 0, 0, static_cast<int32_t>(pks * KS / 128),
                                       static_cast<int32_t>((ps.m0 + roff) / kBM));
                if (++pks >= ps.ks1) {
                    pvalid = pit.next(args, BN, TM, nparts, ps);
                    if (pvalid) pks = ps.ks0;
                }
            };
            if constexpr (kPrefetch > 0) {
                for (uint32_t i = 0; i < early; ++i) walk(false);
                for (int i = 0; i < kPrefetch; ++i) walk(true);
            }
            uint32_t it = 0;
            Seg tr;
            SegIter sit(args, part, nparts);
            while (!failed && sit.next(args, BN, TM, nparts, tr)) {
                for (uint32_t ks = tr.ks0; ks < tr.ks1; ++ks, ++it) {
                    if (it < early) continue;
                    const uint32_t sd = it % SD;
                    if constexpr (kPrefetch > 0) walk(true);
                    if (!mbar_wait(&dfree[sd], ((it / SD) & 1u) ^ 1u, abort)) {
                        fail_here();
                        break;
                    }
                    mbar_arrive_expect_tx(&dfull[sd], Cfg::kDigBytes);
                    // the digits are stored blocked (128 x 128 tiles, each 16 KB contiguous), so the
                    // kSubA tiles of this stage are one contiguous read
                    tma_load_4d(dig + sd * Cfg::kDigBytes, &args.a[tr.g], &dfull[sd], 0, 0,
                                static_cast<int32_t>(ks * KS / 128), static_cast<int32_t>((tr.m0 + roff) / kBM));
                }
            }
            drain_ring(dfull, SD, it > early ? it : early);
        }
    } else if (warp == 14) {
        if (lane == 0) {
            // ---------------- limb producer
            griddep_wait();   // the limbs may come from the kernel this one overlaps (programmatic launch)
            uint32_t it = 0;
            Seg tr;
            SegIter sit(args, part, nparts);
            while (!failed && sit.next(args, BN, TM, nparts, tr)) {
                for (uint32_t ks = tr.ks0; ks < tr.ks1; ++ks, ++it) {
                    const uint32_t sl = it % SL;
                    if (!mbar_wait(&lfree[sl], ((it / SL) & 1u) ^ 1u, abort)) {
                        fail_here();
                        break;
                    }
                    const int32_t k0 = static_cast<int32_t>(ks * KS);
                    if constexpr (PAIR) {
                        // this CTA's half of the limb rows; both halves complete on the leader's barrier
                        if (leader) mbar_arrive_expect_tx(&lfull[sl], 2u * Cfg::kLimbBytes);
#pragma unroll
                        for (int b = 0; b < Cfg::kSubB; ++b)
                            tma_load_2d_pair(limb + sl * Cfg::kLimbBytes + b * Cfg::kBBoxBytes, &args.b[tr.g],
                                             lfull_c + 8u * sl, k0 + 64 * b,
                                             static_cast<int32_t>(tr.n0 + rank * (BN / 2)));
                    } else {
                        mbar_arrive_expect_tx(&lfull[sl], Cfg::kLimbBytes);
#pragma unroll
                        for (int b = 0; b < Cfg::kSubB; ++b)
                            tma_load_2d(limb + sl * Cfg::kLimbBytes + b * Cfg::kBBoxBytes, &args.b[tr.g], &lfull[sl],
                                        k0 + 64 * b, static_cast<int32_t>(tr.n0));
                    }
                }
            }
            // the leader's limb ring counts both CTAs' copies: it waits for them before exit
            if (!PAIR || leader) drain_ring(lfull, SL, it);
        }
    } else if (warp == 1) {
        if (PAIR && !leader) {
            // the peer's MMA warp only holds TMEM with its leader
        } else {
        // ---------------- MMA issuer: the whole warp walks the loop so the descriptors and
        // TMEM addresses stay warp-uniform; one elected lane issues each instruction
        constexpr uint32_t idesc = umma_idesc_f16(TM, BN);
        uint32_t it = 0, ci = 0;
        bool issued = false;
        Seg sg;
        SegIter sit(args, part, nparts);
        while (!failed && sit.next(args, BN, TM, nparts, sg)) {
            uint32_t d_tmem = tmem_base;
            for (uint32_t ks = sg.ks0; ks < sg.ks1; ++ks, ++it) {
                const uint32_t kr = ks - sg.ks0;   // exact chunks restart at every piece
                // every wait outcome is made warp-uniform before the elected issue
                if (kr % CS == 0) {
                    const uint32_t buf = ci & 1u;
                    const bool ok = mbar_wait(&acc_empty[buf], ((ci >> 1) & 1u) ^ 1u, abort);
                    if (__any_sync(0xffffffffu, !ok)) {
                        fail_here();
                        break;
                    }
                    tc_fence_after();
                    d_tmem = tmem_base + buf * BN;
                }
                const uint32_t sa = it % SA, sl = it % SL;
                bool ok = mbar_wait(&aready[sa], (it / SA) & 1u, abort);
                ok = ok && mbar_wait(&lfull[sl], (it / SL) & 1u, abort);
                if (__any_sync(0xffffffffu, !ok)) {
                    fail_here();
                    break;
                }
                tc_fence_after();
                const uint32_t sb = smem_addr(limb + sl * Cfg::kLimbBytes);
                const uint32_t a_tmem = tmem_base + Cfg::kAColBase + sa * Cfg::kSlotCols;
                if (elect_one()) {
#pragma unroll
                    for (int kk = 0; kk < KS / 16; ++kk) {
                        const uint64_t bdesc = umma_desc_sw128(sb + (kk / 4) * Cfg::kBBoxBytes) + 2u * (kk % 4);
                        if constexpr (PAIR)
                            umma_f16_ts_pair(d_tmem, a_tmem + 8u * kk, bdesc, idesc,
                                             (kr % CS != 0 || kk != 0) ? 1u : 0u);
                        else
                            umma_f16_ts(d_tmem, a_tmem + 8u * kk, bdesc, idesc, (kr % CS != 0 || kk != 0) ? 1u : 0u);
                    }
                    if constexpr (PAIR) {
                        umma_commit_pair(&afree[sa], 3);   // both CTAs' TMEM A slots and
                        umma_commit_pair(&lfree[sl], 3);   // limb slots are free once these MMAs complete
                        if (kr % CS == CS - 1 || ks == sg.ks1 - 1) umma_commit_pair(&acc_full[ci & 1u], 3);
                    } else {
                        umma_commit(&afree[sa]);   // the TMEM A slot and
                        umma_commit(&lfree[sl]);   // the limb slot are free once these MMAs complete
                        if (kr % CS == CS - 1 || ks == sg.ks1 - 1) umma_commit(&acc_full[ci & 1u]);
                    }
                }
                __syncwarp();
                issued = true;
                if (kr % CS == CS - 1 || ks == sg.ks1 - 1) ++ci;
            }
        }
        if (issued) {
            if (elect_one()) {
                if constexpr (PAIR) umma_commit_pair(mma_done, 1);
                else umma_commit(mma_done);
            }
            __syncwarp();
            if (!drain_wait_u(mma_done, 0)) failed = true;
        }
        }
    } else if (warp < 6) {
        // ---------------- epilogue (warps 2..5)
        griddep_wait();   // the output may be zeroed by the kernel this one overlaps
        const uint32_t quarter = static_cast<uint32_t>(warp & 3);
        const uint32_t lane_addr = (quarter * 32u) << 16;
        uint32_t ci = 0;
        Seg tr;
        SegIter sit(args, part, nparts);
        while (!failed && sit.next(args, BN, TM, nparts, tr)) {
            const GroupDesc &gd = args.g[tr.g];
            uint32_t run[QPT];
#pragma unroll
            for (int q = 0; q < QPT; ++q) run[q] = 0u;
            const uint32_t nchunks = (tr.ks1 - tr.ks0 + CS - 1) / CS;
            for (uint32_t c = 0; c < nchunks; ++c, ++ci) {
                const uint32_t buf = ci & 1u;
                const bool ok = mbar_wait(&acc_full[buf], (ci >> 1) & 1u, abort);
                if (__any_sync(0xffffffffu, !ok)) {   // the TMEM loads below are warp-collective
                    fail_here();
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int j = 0; j < BN / 16; ++j) {
                    uint32_t v[16];
                    tmem_ld16(tmem_base + lane_addr + buf * BN + 16u * j, v);
                    tmem_wait_ld();
                    if constexpr (LPV == 1) {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            run[16 * j + q] += static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[q]) * kUnscale));
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t s0 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[4 * q + 0]) * kUnscale));
                            const uint32_t s1 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[4 * q + 1]) * kUnscale));
                            const uint32_t s2 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[4 * q + 2]) * kUnscale));
                            const uint32_t s3 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[4 * q + 3]) * kUnscale));
                            run[4 * j + q] += s0 + (s1 << 8) + (s2 << 16) + (s3 << 24);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (PAIR) mbar_arrive_cluster(acc_empty_c + 8u * buf);
                    else mbar_arrive(&acc_empty[buf]);
                }
            }
            if (failed) break;
            const uint32_t row = tr.m0 + roff + quarter * 32u + static_cast<uint32_t>(lane);
            const bool whole = tr.ks0 == 0 && tr.ks1 == tr.ns;   // no other CTA touches this tile
            if (row < gd.M) {
                const uint32_t v0 = tr.n0 / LPV;
#pragma unroll
                for (int q = 0; q < QPT; ++q) {
                    const uint32_t vi = v0 + q;
                    if (vi < gd.NV) {
                        uint32_t *dst = gd.out + (uint64_t)row * gd.ld_m + (uint64_t)vi * gd.ld_b;
                        if (whole) *dst = run[q];
                        else atomicAdd(dst, run[q]);   // exact: addition mod 2^32 commutes
                    }
                }
            }
        }
    } else {
        // ---------------- converters (warps 6..13): digits -> fp16 A in TMEM
        const uint32_t quarter = static_cast<uint32_t>(warp & 3);
        const uint32_t group = static_cast<uint32_t>(warp - 6) / 4;   // owns the stages it % 2 == group
        const uint32_t row = quarter * 32u + static_cast<uint32_t>(lane);
        const uint32_t lane_addr = (quarter * 32u) << 16;
        uint32_t it = 0;
        Seg sg;
        SegIter sit(args, part, nparts);
        while (!failed && sit.next(args, BN, TM, nparts, sg)) {
            for (uint32_t ks = sg.ks0; ks < sg.ks1; ++ks, ++it) {
                if (it % kConvGroups != group) continue;   // this group owns every phase of its slots
                const uint32_t sd = it % SD, sa = it % SA;
                bool ok = mbar_wait(&dfull[sd], (it / SD) & 1u, abort);
                ok = ok && mbar_wait(&afree[sa], ((it / SA) & 1u) ^ 1u, abort);
                if (__any_sync(0xffffffffu, !ok)) {
                    fail_here();
                    break;
                }
                tc_fence_after();   // the MMA that last read this A slot has completed
                const uint32_t a_tmem = tmem_base + lane_addr + Cfg::kAColBase + sa * Cfg::kSlotCols;
#pragma unroll
                for (int b = 0; b < Cfg::kSubA; ++b) {
                    const uint8_t *tile = dig + sd * Cfg::kDigBytes + b * 16384 + row * 128;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        // 128-byte swizzle: logical 16-byte chunk j of row r sits at chunk j ^ (r & 7),
                        // so the eight rows of a quarter-warp read distinct banks
                        const uint32_t phys = static_cast<uint32_t>(j) ^ (row & 7u);
                        const uint4 w = *reinterpret_cast<const uint4 *>(tile + 16u * phys);
                        const uint32_t x[4] = {w.x, w.y, w.z, w.w};
                        uint32_t o[8];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            // [d0, 0, d1, 0]: a byte under a zero exponent is the fp16 subnormal
                            // d * 2^-24, exact, so each pair of digits is one byte permute
                            o[2 * q] = __byte_perm(x[q], 0u, 0x4140);
                            o[2 * q + 1] = __byte_perm(x[q], 0u, 0x4342);
                        }
                        tmem_st8(a_tmem + 64u * b + 8u * j, o);   // warp-uniform TMEM address
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&dfree[sd]);   // the digit slot has been read
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (PAIR) mbar_arrive_cluster(aready_c + 8u * sa);   // the leader's MMA reads both slots
                    else mbar_arrive(&aready[sa]);
                }
            }
        }
    }

    if (failed) {
        *abort = 1;
        *status = kDevTimeout;
        if constexpr (PAIR) {
            // a copy this CTA issued may still be landing (after an abort its stage is never
            // consumed): give it a bounded moment before the CTA can exit
            const uint64_t t0 = global_ns();
            while (global_ns() - t0 < 200000ull) {
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    if constexpr (PAIR) cluster_sync();   // no CTA leaves while its peer may still reach it
    else __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        if constexpr (PAIR) tmem_dealloc_pair(tmem_base, kTmemCols);
        else tmem_dealloc(tmem_base, kTmemCols);
    }
}

// Blocked copy of the digits: tile (rb, cb) of 128 x 128 digits is stored
// contiguously at (rb * CB + cb) * 16384, rows of 128 bytes; zero beyond R, C.
__global__ void block_digits_kernel(const uint8_t *__restrict__ D, uint64_t R, uint64_t C, uint64_t CB,
                                    uint8_t *__restrict__ blk) {
    const uint64_t tile = blockIdx.x;   // rb * CB + cb
    const uint64_t rb = tile / CB, cb = tile % CB;
    const bool full = (rb * 128 + 128 <= R) && (cb * 128 + 128 <= C) && (C % 16 == 0) &&
                      ((reinterpret_cast<uintptr_t>(D) & 15u) == 0);
    uint8_t *dst = blk + tile * 16384;
    for (uint32_t ch = threadIdx.x; ch < 1024; ch += blockDim.x) {   // 16-byte chunks of the tile
        const uint32_t r = ch / 8, k = (ch % 8) * 16;
        const uint64_t row = rb * 128 + r, col = cb * 128 + k;
        uint4 v;
        if (full) {
            v = *reinterpret_cast<const uint4 *>(D + row * C + col);
        } else {
            uint8_t b[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) b[i] = (row < R && col + i < C) ? D[row * C + col + i] : 0;
            v = *reinterpret_cast<const uint4 *>(b);
        }
        *reinterpret_cast<uint4 *>(dst + r * 128 + k) = v;
    }
}

cudaError_t launch_block_digits(const uint8_t *D, uint64_t R, uint64_t C, uint8_t *blk, cudaStream_t stream) {
    const uint64_t RB = (R + 127) / 128, CB = (C + 127) / 128;
    block_digits_kernel<<<static_cast<unsigned>(RB * CB), 256, 0, stream>>>(D, R, C, CB, blk);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host side
template <int BN, int KS, int LPV = 4, bool PAIR = false>
static cudaError_t set_attr() {
    return cudaFuncSetAttribute(limb_gemm_u8_kernel<BN, KS, LPV, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                U8Cfg<BN, KS, PAIR>::kSmemBytes);
}

cudaError_t prepare_limb_gemm_u8_kernels() {
    cudaError_t e;
    if ((e = set_attr<32, 128>()) != cudaSuccess) return e;
    if ((e = set_attr<32, 256>()) != cudaSuccess) return e;
    if ((e = set_attr<64, 128>()) != cudaSuccess) return e;
    if ((e = set_attr<64, 256>()) != cudaSuccess) return e;
    if ((e = set_attr<128, 128>()) != cudaSuccess) return e;
    if ((e = set_attr<128, 256>()) != cudaSuccess) return e;
    if ((e = set_attr<32, 128, 1>()) != cudaSuccess) return e;
    if ((e = set_attr<64, 128, 1>()) != cudaSuccess) return e;
    if ((e = set_attr<32, 128, 4, true>()) != cudaSuccess) return e;
    if ((e = set_attr<64, 128, 4, true>()) != cudaSuccess) return e;
    if ((e = set_attr<128, 128, 4, true>()) != cudaSuccess) return e;
    if ((e = set_attr<32, 128, 1, true>()) != cudaSuccess) return e;
    return set_attr<64, 128, 1, true>();
}

// 128-digit stages for every tile width: with 256 the TMEM A slots allow only two stages in flight
int limb_gemm_u8_default_ks(int) { return 128; }

// Clusters of two CTAs (pair form), one CTA per SM.
template <int BN, int KS, int LPV>
static cudaLaunchConfig_t u8_pair_config(unsigned clusters, cudaStream_t stream, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = U8Cfg<BN, KS, true>::kSmemBytes;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Adds the programmatic-dependent-launch attribute to a launch configuration (attr has room).
static void add_pdl(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr) {
    attr[cfg.numAttrs].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[cfg.numAttrs].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    ++cfg.numAttrs;
}

// CTA pairs resident at once, per device (a GPC with an odd number of free SMs leaves one idle).
template <int BN, int KS, int LPV>
static int u8_resident_pairs(int num_sms) {
    static int cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return num_sms / 2;
    if (cache[dev] > 0) return cache[dev];
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = u8_pair_config<BN, KS, LPV>(static_cast<unsigned>(num_sms / 2), nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, limb_gemm_u8_kernel<BN, KS, LPV, true>, &cfg) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return num_sms / 2;
    }
    n = n < num_sms / 2 ? n : num_sms / 2;
    cache[dev] = n;
    return n;
}

// Numbers the tiles across groups and chooses the schedule for `parts` CTAs (pair form:
// clusters): whole tiles round-robin for every full wave but the last, so the CTAs on the
// tiles of one row tile read its digits together; the last full wave and the remainder are
// split evenly by units, so every CTA ends at about the same time.
static void u8_schedule(GroupedGemmArgs &a, uint32_t tile_rows, uint32_t parts) {
    uint32_t tiles = 0;
    for (uint32_t g = 0; g < a.ngroups; ++g) {
        a.g[g].tile_begin = tiles;
        tiles += (a.g[g].M + tile_rows - 1) / tile_rows * a.g[g].n_tiles;
    }
    a.dp_tiles = tiles >= 2 * parts ? (tiles / parts - 1) * parts : 0;
    a.dp_units = 0;
    for (uint32_t g = 0; g < a.ngroups; ++g) {
        const uint32_t t0 = a.g[g].tile_begin;
        const uint32_t t1 = g + 1 < a.ngroups ? a.g[g + 1].tile_begin : tiles;
        if (a.dp_tiles > t0) a.dp_units += ((a.dp_tiles < t1 ? a.dp_tiles : t1) - t0) * a.g[g].KB;
    }
}

template <int BN, int KS, int LPV = 4>
static cudaError_t launch_u8(const GroupedGemmArgs &args_in, int num_sms, bool pair, int *status,
                             cudaStream_t stream, bool pdl) {
    if (args_in.total_units == 0) return cudaSuccess;
    GroupedGemmArgs args = args_in;
    cudaLaunchAttribute attr[2];
    if (pair) {
        const uint32_t pairs = static_cast<uint32_t>(u8_resident_pairs<BN, KS, LPV>(num_sms));
        const unsigned clusters = args.total_units < pairs ? args.total_units : pairs;
        u8_schedule(args, 2 * kBM, clusters);
        cudaLaunchConfig_t cfg = u8_pair_config<BN, KS, LPV>(clusters, stream, attr);
        if (pdl) add_pdl(cfg, attr);
        return cudaLaunchKernelEx(&cfg, limb_gemm_u8_kernel<BN, KS, LPV, true>, args, status);
    }
    const int grid = static_cast<int>(args.total_units < (uint32_t)num_sms ? args.total_units : (uint32_t)num_sms);
    u8_schedule(args, kBM, static_cast<uint32_t>(grid));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = U8Cfg<BN, KS>::kSmemBytes;
    cfg.stream = stream;
    if (pdl) add_pdl(cfg, attr);
    return cudaLaunchKernelEx(&cfg, limb_gemm_u8_kernel<BN, KS, LPV, false>, args, status);
}

bool limb_gemm_u8_pair_ok(int bn, int ks) { return ks == 128 && bn >= 32 && bn <= 128; }

cudaError_t launch_limb_gemm_u8(int bn, int ks, const GroupedGemmArgs &args, int num_sms, int *status,
                                cudaStream_t stream, bool pair, bool pdl) {
    if (pair && !limb_gemm_u8_pair_ok(bn, ks)) return cudaErrorInvalidValue;
    if (bn == 32 && ks == 128) return launch_u8<32, 128>(args, num_sms, pair, status, stream, pdl);
    if (bn == 32 && ks == 256) return launch_u8<32, 256>(args, num_sms, false, status, stream, pdl);
    if (bn == 64 && ks == 128) return launch_u8<64, 128>(args, num_sms, pair, status, stream, pdl);
    if (bn == 64 && ks == 256) return launch_u8<64, 256>(args, num_sms, false, status, stream, pdl);
    if (bn == 128 && ks == 128) return launch_u8<128, 128>(args, num_sms, pair, status, stream, pdl);
    if (bn == 128 && ks == 256) return launch_u8<128, 256>(args, num_sms, false, status, stream, pdl);
    return cudaErrorInvalidValue;
}

cudaError_t launch_limb_gemm_u8_rows(int bn, const GroupedGemmArgs &args, int num_sms, int *status,
                                     cudaStream_t stream, bool pair, bool pdl) {
    if (bn == 32) return launch_u8<32, 128, 1>(args, num_sms, pair, status, stream, pdl);
    if (bn == 64) return launch_u8<64, 128, 1>(args, num_sms, pair, status, stream, pdl);
    return cudaErrorInvalidValue;
}

}  // namespace qpadl
