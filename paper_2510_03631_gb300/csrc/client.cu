// Client-side steps of the LWE-style PIR and the Setup generator.
//
//  Setup    A[j][k] = upper 32 bits of SplitMix64 output number j*n + k from
//           state `seed` (Steele, Lea, Flood, OOPSLA 2014: the state advances
//           by the golden gamma 0x9E3779B97F4A7C15 and each output is the
//           variant-13 finaliser of the state).
//  Query    (Def. 1 Client.Query)      qu = A s + e + Delta * u_col   mod 2^32
//  Recover  (Def. 1 Client.BlockReconst) d = round((ans - H s) / Delta) mod p
//
// Single queries are HBM-bound matrix-vector products: one warp per row of A
// or H; for n in {512, 1024, 2048} each lane keeps its slice of the secret
// in registers and issues all of a row's 16-byte loads (two rows at a time)
// before using them; other n use a shared-memory copy of the secret.
// Batches are u32 GEMMs (Y = X * W^T over Z_{2^32}) on the CUDA cores with
// 8x8 register blocking.
#include <cstdint>
#include <cuda_runtime.h>

#include "client.cuh"
#include "epilogues.cuh"

namespace qpadl {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void gen_a_kernel(uint64_t seed, uint64_t total, uint32_t *__restrict__ A) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride)
        A[e] = static_cast<uint32_t>(splitmix64_at(seed, e) >> 32);
}

// y = X[i] . w for every row i of X (rows x n), then epilogue(i, 0, y).
template <class Epi>
__global__ void matvec_kernel(const uint32_t *__restrict__ X, uint64_t rows, uint32_t n,
                              const uint32_t *__restrict__ w, Epi epi) {
    extern __shared__ uint32_t sw[];
    for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) sw[k] = w[k];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const bool vec = (n % 4u == 0u) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0u);
    for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < rows; i += warps) {
        const uint32_t *xr = X + i * n;
        uint32_t acc = 0;
        if (vec) {
            for (uint32_t k = 4u * lane; k < n; k += 128u) {
                const uint4 a = __ldg(reinterpret_cast<const uint4 *>(xr + k));
                acc += a.x * sw[k] + a.y * sw[k + 1] + a.z * sw[k + 2] + a.w * sw[k + 3];
            }
        } else {
            for (uint32_t k = lane; k < n; k += 32u) acc += xr[k] * sw[k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) epi(i, 0u, acc);
    }
}

// Same product for n = 128 * NK: warp w owns rows [w rows / W, (w+1) rows / W).
template <int NK, class Epi>
__global__ void __launch_bounds__(256) matvec_reg_kernel(const uint32_t *__restrict__ X, uint64_t rows,
                                                         const uint32_t *__restrict__ w, Epi epi) {
    constexpr uint32_t n = 128 * NK;
    const int lane = threadIdx.x & 31;
    uint4 sw[NK];
#pragma unroll
    for (int m = 0; m < NK; ++m) sw[m] = *reinterpret_cast<const uint4 *>(w + 4 * lane + 128 * m);
    const uint64_t W = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t wid = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t r0 = wid * rows / W, r1 = (wid + 1) * rows / W;
    auto dot = [&](const uint4 (&a)[NK]) {
        uint32_t acc = 0;
#pragma unroll
        for (int m = 0; m < NK; ++m) acc += a[m].x * sw[m].x + a[m].y * sw[m].y + a[m].z * sw[m].z + a[m].w * sw[m].w;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        return acc;
    };
    uint64_t i = r0;
    for (; i + 1 < r1; i += 2) {
        const uint4 *x0 = reinterpret_cast<const uint4 *>(X + i * n) + lane;
        const uint4 *x1 = reinterpret_cast<const uint4 *>(X + (i + 1) * n) + lane;
        uint4 a[NK], b[NK];
#pragma unroll
        for (int m = 0; m < NK; ++m) a[m] = __ldg(x0 + 32 * m);
#pragma unroll
        for (int m = 0; m < NK; ++m) b[m] = __ldg(x1 + 32 * m);
        const uint32_t da = dot(a), db = dot(b);
        if (lane == 0) {
            epi(i, 0u, da);
            epi(i + 1, 0u, db);
        }
    }
    if (i < r1) {
        const uint4 *x0 = reinterpret_cast<const uint4 *>(X + i * n) + lane;
        uint4 a[NK];
#pragma unroll
        for (int m = 0; m < NK; ++m) a[m] = __ldg(x0 + 32 * m);
        const uint32_t da = dot(a);
        if (lane == 0) epi(i, 0u, da);
    }
}

template <class Epi>
static cudaError_t launch_matvec(const uint32_t *X, uint64_t rows, uint32_t n, const uint32_t *w, const Epi &epi,
                                 int num_sms, cudaStream_t stream) {
    const bool aligned = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(w)) & 15u) == 0;
    if (aligned && (n == 512 || n == 1024 || n == 2048)) {
        // one resident wave: blocks per SM from the kernel's occupancy
        auto launch = [&](auto kernel) -> cudaError_t {
            int occ = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0);
            if (e != cudaSuccess) return e;
            const uint64_t blocks = (uint64_t)num_sms * (occ > 0 ? occ : 1);
            if (rows < 8 * blocks) return cudaErrorNotReady;   // too few rows: generic kernel
            kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(X, rows, w, epi);
            return cudaGetLastError();
        };
        cudaError_t e = cudaErrorNotReady;
        if (n == 512) e = launch(matvec_reg_kernel<4, Epi>);
        else if (n == 1024) e = launch(matvec_reg_kernel<8, Epi>);
        else e = launch(matvec_reg_kernel<16, Epi>);
        if (e != cudaErrorNotReady) return e;
    }
    const uint64_t want = (rows + 7) / 8;
    const uint64_t cap = (uint64_t)num_sms * 8;
    const int grid = static_cast<int>(want < cap ? (want ? want : 1) : cap);
    matvec_kernel<Epi><<<grid, 256, n * 4u, stream>>>(X, rows, n, w, epi);
    return cudaGetLastError();
}

// Y[i][b] = sum_k X[i][k] * W[b][k]  (mod 2^32), X: M x K, W: N x K, both
// row-major; 128 x 128 output tile per block, 8 x 8 per thread.
constexpr int kGT = 128, kGK = 8;
template <class Epi>
__global__ void __launch_bounds__(256) u32_gemm_nt_kernel(const uint32_t *__restrict__ X, uint64_t M,
                                                          const uint32_t *__restrict__ W, uint32_t N, uint32_t K,
                                                          Epi epi) {
    __shared__ uint32_t xs[kGK][kGT];
    __shared__ uint32_t ws[kGK][kGT];
    const uint64_t i0 = (uint64_t)blockIdx.x * kGT;
    const uint32_t b0 = blockIdx.y * kGT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    uint32_t acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = 0u;
    // loader mapping: 256 threads x 4 elements = one 128 x 8 tile
    const int lr = threadIdx.x / 2;            // tile row 0..127
    const int lk = (threadIdx.x % 2) * 4;      // k offset 0 or 4
    for (uint32_t k0 = 0; k0 < K; k0 += kGK) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t k = k0 + lk + t;
            const uint64_t i = i0 + lr;
            const uint32_t b = b0 + lr;
            xs[lk + t][lr] = (i < M && k < K) ? X[i * K + k] : 0u;
            ws[lk + t][lr] = (b < N && k < K) ? W[(uint64_t)b * K + k] : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            uint32_t xa[8], wb[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) xa[a] = xs[kk][ty + 16 * a];
#pragma unroll
            for (int c = 0; c < 8; ++c) wb[c] = ws[kk][tx + 16 * c];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[a][c] += xa[a] * wb[c];
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const uint64_t i = i0 + ty + 16 * a;
        if (i >= M) continue;
        uint32_t pre_v[8];   // all loads of the row's outputs before any of its stores
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint32_t b = b0 + tx + 16 * c;
            pre_v[c] = b < N ? epi.pre(i, b) : 0u;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint32_t b = b0 + tx + 16 * c;
            if (b < N) epi.put(i, b, acc[a][c], pre_v[c]);
        }
    }
}

// ------------------------------------------------------------------ host side
cudaError_t launch_gen_a(uint64_t seed, uint64_t C, uint32_t n, uint32_t *A, int num_sms, cudaStream_t stream) {
    gen_a_kernel<<<num_sms * 8, 256, 0, stream>>>(seed, C * n, A);
    return cudaGetLastError();
}

cudaError_t launch_query(const uint32_t *A, uint64_t C, uint32_t n, const uint32_t *s, const int32_t *e,
                         uint64_t col, uint32_t delta, uint32_t *q, int num_sms, cudaStream_t stream) {
    const QueryEpi epi{e, 0, nullptr, col, delta, q, 0};
    return launch_matvec(A, C, n, s, epi, num_sms, stream);
}

cudaError_t launch_query_batch(const uint32_t *A, uint64_t C, uint32_t n, const uint32_t *S, const int32_t *E,
                               const uint32_t *cols, uint32_t B, uint32_t delta, uint32_t *Q, cudaStream_t stream) {
    QueryEpi epi{E, C, cols, 0, delta, Q, C};
    dim3 grid(static_cast<unsigned>((C + kGT - 1) / kGT), (B + kGT - 1) / kGT);
    u32_gemm_nt_kernel<QueryEpi><<<grid, 256, 0, stream>>>(A, C, S, B, n, epi);
    return cudaGetLastError();
}

cudaError_t launch_recover(const uint32_t *ans, const uint32_t *H, uint64_t R, uint32_t n, const uint32_t *s,
                           uint32_t shift, uint8_t *out, int num_sms, cudaStream_t stream) {
    const RecoverEpi epi{ans, 0, shift, out, 0};
    return launch_matvec(H, R, n, s, epi, num_sms, stream);
}

cudaError_t launch_recover_batch(const uint32_t *ans, const uint32_t *H, uint64_t R, uint32_t n, const uint32_t *S,
                                 uint32_t B, uint32_t shift, uint8_t *out, cudaStream_t stream) {
    RecoverEpi epi{ans, R, shift, out, R};
    dim3 grid(static_cast<unsigned>((R + kGT - 1) / kGT), (B + kGT - 1) / kGT);
    u32_gemm_nt_kernel<RecoverEpi><<<grid, 256, 0, stream>>>(H, R, S, B, n, epi);
    return cudaGetLastError();
}

cudaError_t prepare_client_kernels() {
    cudaError_t e = cudaFuncSetAttribute(matvec_kernel<QueryEpi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         16384 * 4);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(matvec_kernel<RecoverEpi>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 4);
}

}  // namespace qpadl
