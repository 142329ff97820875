// Launch interface of the exact byte-limb tensor-core GEMM (limb_gemm.cu).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "epilogues.cuh"

namespace qpadl {

constexpr int kLimbBoxK = 64;    // fp16 elements per TMA box row (128 bytes, 128-byte swizzle)
constexpr int kLimbBoxM = 128;   // database rows per tile

cudaError_t prepare_limb_gemm_kernels();

// Limb columns per tile (32/64/128/256) for `nv` vectors.
int limb_gemm_bn_for(uint32_t nv);

// out[i * ld_m + v * ld_b] = sum_j D[i][j] X[v][j] mod 2^32, i < M, v < NV,
// j < K; a_map covers D16 (box 64 x 128), b_map the limbs (box 64 x bn).
cudaError_t launch_limb_gemm(int bn, const CUtensorMap &a_map, const CUtensorMap &b_map, uint32_t *out,
                             uint64_t ld_m, uint64_t ld_b, uint32_t M, uint32_t NV, uint64_t K, int num_sms,
                             int *status, cudaStream_t stream);

// The same product with the Query / Recover epilogue (client batches: a_map
// covers the limb planes of A or H, b_map the shifted secret limb rows).
// plane_chunks = n / 512 selects the planed mode (bn >= 64, K = 4n, rows of
// b_map in the planed layout); 0 the plain one.
cudaError_t launch_limb_gemm_query(int bn, const CUtensorMap &a_map, const CUtensorMap &b_map, const QueryNoiseEpi &epi,
                                   uint32_t M, uint32_t NV, uint64_t K, uint32_t plane_chunks, int num_sms,
                                   int *status, cudaStream_t stream);
// Q[b * q_ld + cols[b]] += delta for b < B (the unit-vector term of a batch of Queries).
cudaError_t launch_add_delta(uint32_t *Q, uint64_t q_ld, const uint32_t *cols, uint32_t B, uint32_t delta,
                             cudaStream_t stream);
cudaError_t launch_limb_gemm_recover(int bn, const CUtensorMap &a_map, const CUtensorMap &b_map,
                                     const RecoverEpi &epi, uint32_t M, uint32_t NV, uint64_t K,
                                     uint32_t plane_chunks, int num_sms, int *status, cudaStream_t stream);

// Goldberg Response: out = D * X mod p with one centred fp16 row per vector
// (b_map box 64 x bn rows; bn 32 or 64 keep the running sums in registers,
// 256 keeps them in TMEM, reduced mod p after every chunk), through ModPEpi.
cudaError_t launch_limb_gemm_modp(int bn, const CUtensorMap &a_map, const CUtensorMap &b_map, const ModPEpi &epi,
                                  uint32_t M, uint32_t NV, uint64_t K, int num_sms, int *status, cudaStream_t stream);
// Z_p vectors q -> one centred fp16 row each (q or q - p).  When `zero` is given, the same launch
// zeroes zero_words words there (as launch_vec_limbs does for a dependent uint8-digit GEMM).
cudaError_t launch_centred_rows(const uint32_t *Q, uint32_t B, uint64_t C, uint32_t p, __half *L, uint64_t pitch,
                                int num_sms, cudaStream_t stream, uint32_t *zero = nullptr, uint64_t zero_words = 0);
cudaError_t launch_mod_p(uint32_t *x, uint64_t n, uint32_t p, int num_sms, cudaStream_t stream);
// x[i] = (x[i] as a signed 32-bit integer) mod p, in [0, p).
cudaError_t launch_mod_p_signed(uint32_t *x, uint64_t n, uint32_t p, int num_sms, cudaStream_t stream);

cudaError_t launch_db_to_f16(const uint8_t *D, uint64_t R, uint64_t C, __half *D16, uint64_t pitch, int num_sms,
                             cudaStream_t stream);
// Limbs of NV vectors (vector v at X + v * x_ld) into L (limb k of vector v in row 4 v + k).
// When `zero` is given, the same launch also zeroes zero_words words there (the output block of a
// uint8-digit GEMM launched right after it as its programmatic dependent).
cudaError_t launch_vec_limbs(const uint32_t *X, uint64_t x_ld, uint32_t NV, uint64_t C, __half *L, uint64_t pitch,
                             int num_sms, cudaStream_t stream, uint32_t *zero = nullptr, uint64_t zero_words = 0);
cudaError_t launch_mat_col_limbs(const uint32_t *A, uint64_t C, uint32_t n, __half *L, uint64_t pitch,
                                 cudaStream_t stream);
cudaError_t launch_mat_row_limbs(const uint32_t *X, uint64_t rows, uint32_t n, __half *L, uint64_t pitch, int num_sms,
                                 cudaStream_t stream);
cudaError_t launch_secret_limbs(const uint32_t *S, uint32_t B, uint32_t n, __half *V, uint64_t pitch, int num_sms,
                                cudaStream_t stream);
// Planed layout for tiles of 4 * qpt rows; writes 4 * Bp rows (zeros past B), Bp = roundup(B, qpt)
// unless given (then a multiple of qpt, >= B).
cudaError_t launch_secret_limbs_planed(const uint32_t *S, uint32_t B, uint32_t n, uint32_t qpt, __half *V,
                                       uint64_t pitch, int num_sms, cudaStream_t stream, uint32_t Bp = 0);

}  // namespace qpadl
