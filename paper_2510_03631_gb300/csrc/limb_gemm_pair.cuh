// Launch interface of the CTA-pair byte-limb tensor-core GEMM (limb_gemm_pair.cu).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "epilogues.cuh"

namespace qpadl {

// Vector-operand maps of one launch.  Plain mode: m[0] has box 64 x bn/2.
// Planed mode: m[u] has box 64 x (4 - u) bn/8, the rows limb plane u reads.
struct PairBMaps {
    CUtensorMap m[4];
};

cudaError_t prepare_limb_gemm_pair_kernels();

// Rows of the vector-operand box of plane u (planed) or of every stage (plain, u = 0).
__host__ __device__ inline uint32_t pair_b_box_rows(int bn, bool planed, int u) {
    return planed ? static_cast<uint32_t>((4 - u) * bn / 8) : static_cast<uint32_t>(bn / 2);
}

// Tile width (vector-operand rows per pair tile, 128 or 256) for nv vectors of 4 limbs.
int limb_gemm_pair_bn_for(uint32_t nv);

// out[i * ld_m + v * ld_b] = sum_j D[i][j] X[v][j] mod 2^32 (i < M, v < NV, j < K) on CTA
// pairs: a_map covers D16 (box 64 x 128), bm.m[0] the limbs (box 64 x bn/2).
cudaError_t launch_limb_gemm_pair(int bn, const CUtensorMap &a_map, const PairBMaps &bm, uint32_t *out,
                                  uint64_t ld_m, uint64_t ld_b, uint32_t M, uint32_t NV, uint64_t K, int num_sms,
                                  int *status, cudaStream_t stream);

// Client Query / Recover batches on CTA pairs.  plane_chunks = n / 512 selects
// the planed mode (then the vector rows follow launch_secret_limbs_planed with
// qpt = bn / 8, padded to whole tiles, and bm.m[u] has box 64 x (4 - u) bn/8).
cudaError_t launch_limb_gemm_pair_query(int bn, const CUtensorMap &a_map, const PairBMaps &bm,
                                        const QueryNoiseEpi &epi,
                                        uint32_t M, uint32_t NV, uint64_t K, uint32_t plane_chunks, int num_sms,
                                        int *status, cudaStream_t stream);
cudaError_t launch_limb_gemm_pair_recover(int bn, const CUtensorMap &a_map, const PairBMaps &bm,
                                          const RecoverEpi &epi, uint32_t M, uint32_t NV, uint64_t K,
                                          uint32_t plane_chunks, int num_sms, int *status, cudaStream_t stream);

// One centred fp16 row per Z_p vector (Goldberg Response): out[i * ld_m + v * ld_b] =
// (sum_j D[i][j] X[v][j]) mod p in [0, p), on 256-wide pair tiles whose running sums stay in TMEM
// (reduced mod p after every 512-deep chunk); bm.m[0] has box 64 x 128 over the NV rows.
cudaError_t launch_limb_gemm_pair_modp(const CUtensorMap &a_map, const PairBMaps &bm, const ModPEpi &epi, uint32_t M,
                                       uint32_t NV, uint64_t K, int num_sms, int *status, cudaStream_t stream);

}  // namespace qpadl
