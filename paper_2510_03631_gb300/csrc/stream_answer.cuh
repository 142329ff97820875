// Launch interface of the streaming Response kernels (stream_answer.cu).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace qpadl {

constexpr int kStreamChunkCols = 256;                       // digits per row per stage (TMA box width)
constexpr int kStreamStages = 3;                            // shared-memory ring depth
constexpr int kStreamConsumerWarps = 16;
constexpr int kStreamThreads = 32 * (1 + kStreamConsumerWarps);   // producer warp + consumers
constexpr int kStreamColGroups = kStreamChunkCols / 16;     // 16 digits (one uint4) per thread
constexpr int kStreamRowLanes = 32 * kStreamConsumerWarps / kStreamColGroups;

// Words of packed query per query: ceil(C / 256) chunks x 256 words.
inline uint64_t stream_pack_words(uint64_t C) {
    return ((C + kStreamChunkCols - 1) / kStreamChunkCols) * kStreamChunkCols;
}

int stream_smem_bytes(int nq);
cudaError_t prepare_stream_kernels();

cudaError_t launch_pack_query(const uint32_t *q, uint64_t q_ld, uint32_t C, uint32_t nq, uint32_t *qpack,
                              uint64_t pack_ld, cudaStream_t stream);

// nq in {1, 2, 4}; ans of query b goes to ans[b * ans_ld + i].
cudaError_t launch_stream_answer(int nq, const CUtensorMap &map, const uint32_t *qpack, uint64_t pack_ld,
                                 uint32_t *ans, uint64_t ans_ld, uint32_t R, uint32_t C, int num_sms, int *status,
                                 cudaStream_t stream);

cudaError_t launch_rowwise_answer(const uint8_t *D, uint64_t R, uint64_t C, const uint32_t *Q, uint64_t q_ld,
                                  uint32_t B, uint32_t *ans, uint64_t ans_ld, int num_sms, cudaStream_t stream);

}  // namespace qpadl
