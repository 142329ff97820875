// Launch interface of the Chor-style GF(2) Response kernels (chor.cu).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace qpadl {

constexpr uint32_t kChorMaxBatch = 256;   // queries per launch; larger batches run in chunks

cudaError_t prepare_chor_kernels();

// Tile width (words), band height (rows), TMA box width (words) and QT words
// per row that a launch for B queries in scan form `form` (0..3: bit 1 = 8 words
// per thread, bit 0 = predicated XOR) uses; false if B is 0 or > kChorMaxBatch.
bool chor_launch_shape(uint32_t B, int form, uint32_t *tw, uint32_t *rb, uint32_t *box_words, uint32_t *qtw);

// Q (B x qw words) -> QT (r x qtw words): bit j of QT[i][g] = bit i of query 32 g + j.
cudaError_t launch_chor_transpose(const uint32_t *Q, uint64_t qw, uint32_t B, uint64_t r, uint32_t qtw, uint32_t *QT,
                                  int num_sms, cudaStream_t stream);

// out (B x W words, zeroed by the caller) ^= the GF(2) responses; db_map covers
// the database {W, r} words with box {box_words, rb}, qt_map QT {qtw, r} with box {qtw, rb}.
cudaError_t launch_chor_answer(const CUtensorMap &db_map, const CUtensorMap &qt_map, uint64_t r, uint32_t W,
                               uint32_t B, uint32_t qtw, uint32_t *out, int num_sms, int *status,
                               cudaStream_t stream, int form);

// Four-Russians path (large batches): box shape of its database map.
constexpr uint32_t kChorM4TileWords = 64;
constexpr uint32_t kChorM4BandRows = 64;

// Q (B x qw words) -> QS (qw x 256 words): word k of query b at QS[k * 256 + b];
// the buffer must hold roundup(qw, 2) x 256 words (a band reads two query words).
cudaError_t launch_chor_words(const uint32_t *Q, uint64_t qw, uint32_t B, uint64_t r, uint32_t *QS, int num_sms,
                              cudaStream_t stream);

// out (B x W words, zeroed by the caller) ^= the responses of B <= 256 queries;
// db_map covers the database {W, r} words with box {64, 64}.
cudaError_t launch_chor_m4rm(const CUtensorMap &db_map, const uint32_t *QS, uint64_t r, uint32_t W, uint32_t B,
                             uint32_t *out, int num_sms, int *status, cudaStream_t stream);

}  // namespace qpadl
