// Launch interface of the grouped byte-limb GEMM over uint8 databases (limb_gemm_u8.cu).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace qpadl {

constexpr int kMaxGemmGroups = 4;

// One group: a database (rows M, K columns) times NV vectors.
struct GroupDesc {
    uint32_t *out;          // out[i * ld_m + v * ld_b]
    uint64_t ld_m, ld_b;
    uint32_t M, NV, KB;     // rows, vectors, 64-wide K blocks
    uint32_t tile_begin;    // first index of this group in the launch's tile list
    uint32_t n_tiles;       // BN-wide tiles per 128-row tile
    uint32_t pad;
};

struct GroupedGemmArgs {
    CUtensorMap a[kMaxGemmGroups];   // uint8 digits, 2-D {C, R}, box {64, 128}, 64-byte swizzle
    CUtensorMap b[kMaxGemmGroups];   // fp16 limbs, 2-D {C, 4 NV}, box {64, BN}, 128-byte swizzle
    GroupDesc g[kMaxGemmGroups];
    uint32_t ngroups, total_tiles;
};

cudaError_t prepare_limb_gemm_u8_kernels();

// bn in {32, 64, 128}: limb columns per tile (the same for every group).
cudaError_t launch_limb_gemm_u8(int bn, const GroupedGemmArgs &args, int num_sms, int *status, cudaStream_t stream);

}  // namespace qpadl
