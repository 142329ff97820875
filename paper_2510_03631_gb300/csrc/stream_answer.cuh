// Launch interface of the streaming Response kernels (stream_answer.cu).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace qpadl {

constexpr int kStreamConsumerWarps = 16;
constexpr int kStreamThreads = 32 * (1 + kStreamConsumerWarps);   // producer warp + consumers
constexpr int kStreamMaxChunk = 4096;

// Words of packed query per query for any supported chunk width.
inline uint64_t stream_pack_words(uint64_t C) {
    return ((C + kStreamMaxChunk - 1) / kStreamMaxChunk) * kStreamMaxChunk;
}

cudaError_t prepare_stream_kernels();
bool stream_config_valid(int nq, int cch);

cudaError_t launch_pack_query(const uint32_t *q, uint64_t q_ld, uint32_t C, uint32_t cch, uint32_t nq,
                              uint32_t *qpack, uint64_t pack_ld, cudaStream_t stream);

// nq in {1, 2, 4}; cch in {512, 1024, 2048, 4096} for nq == 1, 1024 otherwise.
// D must be 16-byte aligned with C % 16 == 0.  Answer b goes to ans[b * ans_ld + i].
// `map` (may be null): 3-D uint8 tensor map over D with dims {256, C/256, R}
// and box {256, cch/256, 8}; used when C % 256 == 0.
cudaError_t launch_stream_answer(int nq, int cch, const CUtensorMap *map, const uint8_t *D, uint32_t R, uint32_t C,
                                 const uint32_t *qpack, uint64_t pack_ld, uint32_t *ans, uint64_t ans_ld,
                                 int num_sms, int *status, cudaStream_t stream);

// One query, raw (no packing pass): the kernel packs the query limbs itself.
// q must be 16-byte aligned.  Answer to ans[i].
cudaError_t launch_stream_answer_raw(int cch, const CUtensorMap *map, const uint8_t *D, uint32_t R, uint32_t C,
                                     const uint32_t *q, uint32_t *ans, int num_sms, int *status,
                                     cudaStream_t stream);

// Two queries, raw: one pass over D answers both (query b at q + b * q_ld,
// answer b at ans + b * ans_ld).  cch in {1024, 2048}; q and q + q_ld must be
// 16-byte aligned (q_ld a multiple of 4).
cudaError_t launch_stream_answer_raw2(int cch, const CUtensorMap *map, const uint8_t *D, uint32_t R, uint32_t C,
                                      const uint32_t *q, uint64_t q_ld, uint32_t *ans, uint64_t ans_ld, int num_sms,
                                      int *status, cudaStream_t stream);

cudaError_t launch_rowwise_answer(const uint8_t *D, uint64_t R, uint64_t C, const uint32_t *Q, uint64_t q_ld,
                                  uint32_t B, uint32_t *ans, uint64_t ans_ld, int num_sms, cudaStream_t stream);

}  // namespace qpadl
