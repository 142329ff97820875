// Exact mod-2^32 product of one or several databases with batches of Z_q
// vectors, reading the databases as stored (uint8 digits):
//     OUT_g[i][b] = sum_j D_g[i][j] * X_g[b][j]   (mod 2^32), g < ngroups.
//
// Same exact byte-limb algebra as limb_gemm.cu (balanced limbs in fp16,
// fp32 accumulation over 512-deep K-chunks, int32 recombination; see there),
// but the A operand never exists as fp16 in memory: TMA brings 128 x 64
// digit tiles (8 KB) into shared memory, four converter warps turn each row
// into fp16 (byte-permute next to 0x64 gives 1024 + d exactly, minus 1024)
// and store it into tensor memory, and the MMA reads A from tensor memory
// (tcgen05.mma with A in TMEM).  Half the HBM traffic of the fp16 copy, and
// shared memory carries only the digit tile (64-byte swizzled, so the row-
// per-thread reads are free of bank conflicts) and the limb tile.
//
// One launch can serve several databases with their own batches (the
// serving loop's grouped launch): output tiles of all groups form one list
// that persistent CTAs walk.
//
// Warp roles (320 threads, one CTA per SM):
//   warp 0      TMA producer (digit tile + limb tile per stage, 4 stages)
//   warp 1      TMEM allocation; one thread issues the MMAs
//   warps 2..5  epilogue: drain one of two BN-column accumulators per chunk
//   warps 6..9  converters: digits -> fp16 A tiles in TMEM (one row per thread)
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "limb_gemm_u8.cuh"
#include "ptx.cuh"

namespace qpadl {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kStages = 4;
constexpr int kChunkKB = 8;               // 512-deep exact K-chunks
constexpr int kThreads = 320;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAColBase = 256;       // A slots live after the (<= 256) accumulator columns
constexpr uint32_t kASlotCols = kBK / 2;  // 64 fp16 per row = 32 columns

template <int BN>
struct U8Cfg {
    static constexpr uint32_t kABytes = kBM * kBK;        // digits
    static constexpr uint32_t kBBytes = BN * kBK * 2;     // fp16 limbs
    static constexpr uint32_t kStageBytes = kABytes + kBBytes;
    // padded so that only one CTA fits per SM (it allocates all of TMEM)
    static constexpr int kSmemUsed = kStages * kStageBytes + 512 + 1024;
    static constexpr int kSmemBytes = kSmemUsed > 120 * 1024 ? kSmemUsed : 120 * 1024;
    static constexpr int kQPT = BN / 4;
};

__device__ __forceinline__ bool drain_wait_u(uint64_t *bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > QPADL_WAIT_NS) return false;
    }
    return true;
}

struct TileRef {
    uint32_t g, m0, n0;
};

__device__ __forceinline__ TileRef locate(const GroupedGemmArgs &a, uint32_t t, uint32_t bn) {
    uint32_t g = 0;
    while (g + 1 < a.ngroups && t >= a.g[g + 1].tile_begin) ++g;
    const uint32_t lt = t - a.g[g].tile_begin;
    return TileRef{g, (lt / a.g[g].n_tiles) * kBM, (lt % a.g[g].n_tiles) * bn};
}

}  // namespace

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    limb_gemm_u8_kernel(const __grid_constant__ GroupedGemmArgs args, int *__restrict__ status) {
    using Cfg = U8Cfg<BN>;
    constexpr int QPT = Cfg::kQPT;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // stage s: [digits 8 KB][limbs BN*128 B]; the limb tile stays 1024-aligned
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * Cfg::kStageBytes);
    uint64_t *conv = full + kStages;
    uint64_t *empty = conv + kStages;
    uint64_t *acc_full = empty + kStages;   // [2]
    uint64_t *acc_empty = acc_full + 2;     // [2]
    uint64_t *mma_done = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], 4);
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
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t tiles = args.total_tiles;
    bool failed = false;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            uint32_t it = 0;
            for (uint32_t t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
                const TileRef tr = locate(args, t, BN);
                const uint32_t KB = args.g[tr.g].KB;
                for (uint32_t kb = 0; kb < KB; ++kb, ++it) {
                    const uint32_t st = it % kStages;
                    const uint32_t ph = (it / kStages) & 1u;
                    if (!mbar_wait(&empty[st], ph ^ 1u, abort)) {
                        failed = true;
                        break;
                    }
                    uint8_t *sa = smem + st * Cfg::kStageBytes;
                    mbar_arrive_expect_tx(&full[st], Cfg::kStageBytes);
                    tma_load_2d(sa, &args.a[tr.g], &full[st], static_cast<int32_t>(kb * kBK),
                                static_cast<int32_t>(tr.m0));
                    tma_load_2d(sa + Cfg::kABytes, &args.b[tr.g], &full[st], static_cast<int32_t>(kb * kBK),
                                static_cast<int32_t>(tr.n0));
                }
            }
            const uint32_t inflight = it < (uint32_t)kStages ? it : (uint32_t)kStages;
            for (uint32_t j = it - inflight; j < it; ++j)
                if (!drain_wait_u(&full[j % kStages], (j / kStages) & 1u)) failed = true;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            constexpr uint32_t idesc = umma_idesc_f16(kBM, BN);
            uint32_t it = 0, ci = 0;
            bool issued = false;
            for (uint32_t t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
                const uint32_t KB = args.g[locate(args, t, BN).g].KB;
                uint32_t d_tmem = tmem_base;
                for (uint32_t kb = 0; kb < KB; ++kb, ++it) {
                    if (kb % kChunkKB == 0) {
                        const uint32_t buf = ci & 1u;
                        if (!mbar_wait(&acc_empty[buf], ((ci >> 1) & 1u) ^ 1u, abort)) {
                            failed = true;
                            break;
                        }
                        tc_fence_after();
                        d_tmem = tmem_base + buf * BN;
                    }
                    const uint32_t st = it % kStages;
                    const uint32_t ph = (it / kStages) & 1u;
                    if (!mbar_wait(&conv[st], ph, abort)) {   // implies the limb tile has landed too
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t bdesc = umma_desc_sw128(smem_addr(smem + st * Cfg::kStageBytes + Cfg::kABytes));
                    const uint32_t a_tmem = tmem_base + kAColBase + st * kASlotCols;
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k)
                        umma_f16_ts(d_tmem, a_tmem + 8u * k, bdesc + 2u * k, idesc,
                                    (kb % kChunkKB != 0 || k != 0) ? 1u : 0u);
                    issued = true;
                    umma_commit(&empty[st]);   // frees the shared-memory stage and the TMEM A slot
                    if (kb % kChunkKB == kChunkKB - 1 || kb == KB - 1) {
                        umma_commit(&acc_full[ci & 1u]);
                        ++ci;
                    }
                }
            }
            if (issued) {
                umma_commit(mma_done);
                if (!drain_wait_u(mma_done, 0)) failed = true;
            }
        }
    } else if (warp < 6) {
        // ---------------- epilogue (warps 2..5)
        const uint32_t quarter = static_cast<uint32_t>(warp & 3);
        const uint32_t lane_addr = (quarter * 32u) << 16;
        uint32_t ci = 0;
        for (uint32_t t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
            const TileRef tr = locate(args, t, BN);
            const GroupDesc &gd = args.g[tr.g];
            uint32_t run[QPT];
#pragma unroll
            for (int q = 0; q < QPT; ++q) run[q] = 0u;
            const uint32_t nchunks = (gd.KB + kChunkKB - 1) / kChunkKB;
            for (uint32_t c = 0; c < nchunks; ++c, ++ci) {
                const uint32_t buf = ci & 1u;
                if (!mbar_wait(&acc_full[buf], (ci >> 1) & 1u, abort)) {
                    failed = true;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int j = 0; j < BN / 32; ++j) {
                    uint32_t v[32];
                    tmem_ld32(tmem_base + lane_addr + buf * BN + 32u * j, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const uint32_t s0 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[4 * q + 0])));
                        const uint32_t s1 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[4 * q + 1])));
                        const uint32_t s2 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[4 * q + 2])));
                        const uint32_t s3 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[4 * q + 3])));
                        run[8 * j + q] += s0 + (s1 << 8) + (s2 << 16) + (s3 << 24);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[buf]);
            }
            if (failed) break;
            const uint32_t row = tr.m0 + quarter * 32u + static_cast<uint32_t>(lane);
            if (row < gd.M) {
                const uint32_t v0 = tr.n0 / 4;
#pragma unroll
                for (int q = 0; q < QPT; ++q) {
                    const uint32_t vi = v0 + q;
                    if (vi < gd.NV) gd.out[(uint64_t)row * gd.ld_m + (uint64_t)vi * gd.ld_b] = run[q];
                }
            }
        }
    } else {
        // ---------------- converters (warps 6..9): digits -> fp16 A in TMEM
        const uint32_t quarter = static_cast<uint32_t>(warp & 3);
        const uint32_t row = quarter * 32u + static_cast<uint32_t>(lane);
        const uint32_t lane_addr = (quarter * 32u) << 16;
        const __half2 k1024 = __floats2half2_rn(1024.0f, 1024.0f);
        uint32_t it = 0;
        for (uint32_t t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
            const uint32_t KB = args.g[locate(args, t, BN).g].KB;
            for (uint32_t kb = 0; kb < KB; ++kb, ++it) {
                const uint32_t st = it % kStages;
                const uint32_t ph = (it / kStages) & 1u;
                if (!mbar_wait(&full[st], ph, abort)) {
                    failed = true;
                    break;
                }
                const uint8_t *tile = smem + st * Cfg::kStageBytes + row * kBK;
                const uint32_t a_tmem = tmem_base + lane_addr + kAColBase + st * kASlotCols;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // the digit tile arrives with 64-byte swizzling: logical 16-byte chunk j of row r
                    // sits at chunk j ^ ((r >> 1) & 3), so a quarter-warp reads distinct banks
                    const uint32_t phys = static_cast<uint32_t>(j) ^ ((row >> 1) & 3u);
                    const uint4 w = *reinterpret_cast<const uint4 *>(tile + 16u * phys);
                    const uint32_t x[4] = {w.x, w.y, w.z, w.w};
                    uint32_t o[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        // [d0, 0x64, d1, 0x64] is the fp16 pair (1024 + d0, 1024 + d1)
                        uint32_t lo = __byte_perm(x[q], 0x64646464u, 0x4140);
                        uint32_t hi = __byte_perm(x[q], 0x64646464u, 0x4342);
                        __half2 hl = __hsub2(*reinterpret_cast<__half2 *>(&lo), k1024);
                        __half2 hh = __hsub2(*reinterpret_cast<__half2 *>(&hi), k1024);
                        o[2 * q] = *reinterpret_cast<uint32_t *>(&hl);
                        o[2 * q + 1] = *reinterpret_cast<uint32_t *>(&hh);
                    }
                    tmem_st8(a_tmem + 8u * j, o);   // the TMEM address is warp-uniform
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&conv[st]);
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
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// ------------------------------------------------------------------ host side
template <int BN>
static cudaError_t set_attr() {
    return cudaFuncSetAttribute(limb_gemm_u8_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                U8Cfg<BN>::kSmemBytes);
}

cudaError_t prepare_limb_gemm_u8_kernels() {
    cudaError_t e;
    if ((e = set_attr<32>()) != cudaSuccess) return e;
    if ((e = set_attr<64>()) != cudaSuccess) return e;
    return set_attr<128>();
}

cudaError_t launch_limb_gemm_u8(int bn, const GroupedGemmArgs &args, int num_sms, int *status, cudaStream_t stream) {
    const int grid = static_cast<int>(args.total_tiles < (uint32_t)num_sms ? args.total_tiles : (uint32_t)num_sms);
    if (grid <= 0) return cudaSuccess;
    switch (bn) {
        case 32:
            limb_gemm_u8_kernel<32><<<grid, kThreads, U8Cfg<32>::kSmemBytes, stream>>>(args, status);
            break;
        case 64:
            limb_gemm_u8_kernel<64><<<grid, kThreads, U8Cfg<64>::kSmemBytes, stream>>>(args, status);
            break;
        case 128:
            limb_gemm_u8_kernel<128><<<grid, kThreads, U8Cfg<128>::kSmemBytes, stream>>>(args, status);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace qpadl
