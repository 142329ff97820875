// Launch interface of the grouped byte-limb GEMM over uint8 databases (limb_gemm_u8.cu).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace qpadl {

constexpr int kMaxGemmGroups = 8;

// One group: a database (rows M, K columns) times NV vectors.
struct GroupDesc {
    uint32_t *out;          // out[i * ld_m + v * ld_b]; must be zero where tiles are split (see below)
    uint64_t ld_m, ld_b;
    uint32_t M, NV, KB;     // rows, vectors, pipeline stages per tile (ceil(K / ks))
    uint32_t unit_begin;    // first work unit (tile x stage) of this group in the launch
    uint32_t n_tiles;       // BN-wide tiles per row tile (128 rows; 256 in the pair form)
    uint32_t tile_begin;    // first tile of this group in the launch (set by the launch)
};

struct GroupedGemmArgs {
    CUtensorMap a[kMaxGemmGroups];   // blocked uint8 digits: 4-D {128, 128, C/128, R/128},
                                     // box {128, 128, ks/128, 1}, 128-byte swizzle
    CUtensorMap b[kMaxGemmGroups];   // fp16 limbs, 2-D {C, 4 NV} ({C, NV} for one row per vector),
                                     // box {64, BN}, 128-byte swizzle
    GroupDesc g[kMaxGemmGroups];
    uint32_t ngroups, total_units;   // units = sum over groups of tiles x stages
    // Schedule (set by the launch): tiles [0, dp_tiles) (numbered across groups, each group's
    // tiles row tile by row tile) are dealt whole, round-robin, so the CTAs on the tiles of one
    // row tile run together and share its digits through L2; the units from dp_units on are
    // split evenly (stream-K).
    uint32_t dp_tiles, dp_units;
};

cudaError_t prepare_limb_gemm_u8_kernels();

// Blocked copy of D: 128 x 128 digit tiles, tile (rb, cb) at (rb * ceil(C/128) + cb) * 16384.
// blk holds ceil(R/128) * ceil(C/128) * 16384 bytes.
cudaError_t launch_block_digits(const uint8_t *D, uint64_t R, uint64_t C, uint8_t *blk, cudaStream_t stream);

// Whole tiles go round-robin to the CTAs for all but the last full wave; the
// rest is split evenly by units (one tile's one pipeline stage), across tile
// boundaries (stream-K): a tile wholly inside one CTA's share is stored, a
// tile shared by CTAs is accumulated with atomic adds (exact mod 2^32), so the
// output must be zeroed before the launch.
// bn in {32, 64, 128}, ks in {128, 256}: limb columns per
// tile (the same for every group) and digits per row per pipeline stage.
int limb_gemm_u8_default_ks(int bn);
// Pair form (pair = true): tiles of 256 rows over clusters of two CTAs (tcgen05 cta_group::2),
// each CTA loading half of the limb rows.  Then a group's units count 256-row tiles
// (ceil(M / 256) x n_tiles x KB) and its b map has box {64, bn / 2}.  bn in {32, 64, 128}, ks = 128.
bool limb_gemm_u8_pair_ok(int bn, int ks);
// pdl: launch as the programmatic dependent of the kernel just before it in the stream.  Only the
// limb loads and the output stores wait for that kernel (every kernel before it has completed when
// this one starts); the digit loads start at once, so that kernel must not write the digits.
cudaError_t launch_limb_gemm_u8(int bn, int ks, const GroupedGemmArgs &args, int num_sms, int *status,
                                cudaStream_t stream, bool pair = false, bool pdl = false);

// The same GEMM with one vector-operand row per vector (b maps {C, NV}): each
// output is the exact signed sum sum_j D[i][j] x_b[j] stored as 32 bits, for
// |x_b[j]| <= 128 (so every 512-deep chunk stays below 2^24 in fp32 and the
// whole sum below 2^31 for fewer than 65793 columns).  bn in {32, 64}, 128-digit
// stages; output zeroed before the launch as above; pdl as above.
cudaError_t launch_limb_gemm_u8_rows(int bn, const GroupedGemmArgs &args, int num_sms, int *status,
                                     cudaStream_t stream, bool pair = false, bool pdl = false);

}  // namespace qpadl
