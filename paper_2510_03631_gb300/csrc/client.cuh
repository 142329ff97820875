// Launch interface of the Setup generator and the client-side kernels (client.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qpadl {

cudaError_t prepare_client_kernels();
cudaError_t client_status_take(int *out);
cudaError_t launch_gen_a(uint64_t seed, uint64_t C, uint32_t n, uint32_t *A, int num_sms, cudaStream_t stream);
cudaError_t launch_query(const uint32_t *A, uint64_t C, uint32_t n, const uint32_t *s, const int32_t *e,
                         uint64_t col, uint32_t delta, uint32_t *q, int num_sms, cudaStream_t stream);
cudaError_t launch_query_batch(const uint32_t *A, uint64_t C, uint32_t n, const uint32_t *S, const int32_t *E,
                               const uint32_t *cols, uint32_t B, uint32_t delta, uint32_t *Q, cudaStream_t stream);
cudaError_t launch_recover(const uint32_t *ans, const uint32_t *H, uint64_t R, uint32_t n, const uint32_t *s,
                           uint32_t shift, uint8_t *out, int num_sms, cudaStream_t stream);
cudaError_t launch_recover_batch(const uint32_t *ans, const uint32_t *H, uint64_t R, uint32_t n, const uint32_t *S,
                                 uint32_t B, uint32_t shift, uint8_t *out, cudaStream_t stream);

}  // namespace qpadl
