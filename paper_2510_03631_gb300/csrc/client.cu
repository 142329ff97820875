// Client-side steps of the LWE-style PIR and the Setup generator.
//
//  Setup    A[j][k] = upper 32 bits of SplitMix64 output number j*n + k from
//           state `seed` (Steele, Lea, Flood, OOPSLA 2014: the state advances
//           by the golden gamma 0x9E3779B97F4A7C15 and each output is the
//           variant-13 finaliser of the state).
//  Query    (Def. 1 Client.Query)      qu = A s + e + Delta * u_col   mod 2^32
//  Recover  (Def. 1 Client.BlockReconst) d = round((ans - H s) / Delta) mod p
//
// Single queries are HBM-bound matrix-vector products over A or H.  For
// n in {512, 1024, 2048} the rows stream through a shared-memory ring fed by
// bulk copies, each consumer warp takes one row per stage with the secret in
// registers, and the kernel overlaps its start with the end of the kernel
// before it (programmatic dependent launch); other n use one warp per row
// and a shared-memory copy of the secret.
// Batches are u32 GEMMs (Y = X * W^T over Z_{2^32}) on the CUDA cores with
// 8x8 register blocking.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "client.cuh"
#include "epilogues.cuh"
#include "ptx.cuh"

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

// Same product for n = 128 * NK with the rows of X streamed through shared
// memory by bulk copies: CTA b owns the row band [b rows / G, (b+1) rows / G);
// one lane of warp 0 copies it in stages of 8 consecutive rows (one copy per
// stage) into a ring of kStages buffers; consumer warp c takes row c of every
// stage (band rows c, c + 8, c + 16, ...).  Each lane keeps its slice of the
// vector in registers.  A consumer takes its rows in runs of 32: lane t
// gathers the epilogue input of the run's row t when the run begins and
// keeps that row's dot product, so a run ends in one epilogue per lane
// instead of a memory round trip per row.
// Launched with programmatic dependent launch: before griddepcontrol.wait the
// kernel only lets its successor be scheduled and pulls its first stages of X
// into L2 (a hint that moves nothing into the CTA), so it never consumes data
// that the preceding kernel may still be writing.  Every barrier wait is
// bounded; a wait that gives up records kDevTimeout in *status.
constexpr int kMvRows = 8;   // rows per stage = consumer warps
constexpr int kMvThreads = 32 * (1 + kMvRows);
template <int NK>
struct MvCfg {
    static constexpr uint32_t kRowBytes = 512u * NK;
    static constexpr uint32_t kStageBytes = kMvRows * kRowBytes;
    static constexpr int kStages = (196608u / kStageBytes) < 12u ? static_cast<int>(196608u / kStageBytes) : 12;
    static constexpr uint32_t kSmemBytes = kStages * kStageBytes + 2 * kStages * 8 + 16 + 128;   // + alignment slack
};

template <int NK, class Epi>
__global__ void __launch_bounds__(kMvThreads, 1)
    matvec_tma_kernel(const uint32_t *__restrict__ X, uint64_t rows, const uint32_t *__restrict__ w, Epi epi,
                      int *__restrict__ status) {
    using Cfg = MvCfg<NK>;
    constexpr int ST = Cfg::kStages;
    constexpr uint32_t n = 128 * NK;
    extern __shared__ uint8_t mv_smem_raw[];
    uint8_t *buf = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(mv_smem_raw) + 127) & ~uintptr_t(127));
    uint64_t *full = reinterpret_cast<uint64_t *>(buf + ST * Cfg::kStageBytes);
    uint64_t *empty = full + ST;
    volatile int *abort = reinterpret_cast<volatile int *>(empty + ST);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint64_t r0 = (uint64_t)blockIdx.x * rows / gridDim.x;
    const uint64_t r1 = (uint64_t)(blockIdx.x + 1) * rows / gridDim.x;
    const uint32_t nst = static_cast<uint32_t>((r1 - r0 + kMvRows - 1) / kMvRows);
    auto stage_bytes = [&](uint32_t t) {
        const uint64_t g0 = r0 + (uint64_t)t * kMvRows;
        const uint64_t nr = r1 - g0 < (uint64_t)kMvRows ? r1 - g0 : (uint64_t)kMvRows;
        return static_cast<uint32_t>(nr * Cfg::kRowBytes);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kMvRows);
        }
        *abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    if (warp == 0) {
        // ---------------- producer
        if (lane == 0) {
            for (uint32_t t = 0; t < nst && t < (uint32_t)ST; ++t)
                bulk_prefetch_l2(X + (r0 + (uint64_t)t * kMvRows) * n, stage_bytes(t));
            griddep_launch_dependents();
            griddep_wait();
            bool ok = true;
            uint32_t t = 0;
            for (; t < nst; ++t) {
                const uint32_t st = t % ST;
                if (!mbar_wait(&empty[st], ((t / ST) & 1u) ^ 1u, abort)) {
                    ok = false;
                    break;
                }
                const uint32_t bytes = stage_bytes(t);
                mbar_arrive_expect_tx(&full[st], bytes);
                bulk_load(buf + st * Cfg::kStageBytes, X + (r0 + (uint64_t)t * kMvRows) * n, bytes, &full[st]);
            }
            // never leave while copies issued here are still landing
            const uint32_t inflight = t < (uint32_t)ST ? t : (uint32_t)ST;
            for (uint32_t j = t - inflight; j < t; ++j)
                if (!mbar_drain(&full[j % ST], (j / ST) & 1u)) ok = false;
            if (!ok && status) *status = kDevTimeout;
        }
        return;
    }

    // ---------------- consumers
    griddep_wait();
    const int c = warp - 1;
    uint4 sw[NK];
#pragma unroll
    for (int m = 0; m < NK; ++m) sw[m] = *reinterpret_cast<const uint4 *>(w + 4 * lane + 128 * m);
    const uint64_t my0 = r0 + c;   // this warp's rows: my0 + 8 t
    const uint32_t my_n = r1 > my0 ? static_cast<uint32_t>((r1 - my0 + kMvRows - 1) / kMvRows) : 0u;
    uint32_t pv = 0, mine = 0;
    for (uint32_t t = 0; t < nst; ++t) {
        const uint32_t k = t & 31u;
        if (k == 0) {
            if (t && t - 32 + lane < my_n) epi.put(my0 + (uint64_t)kMvRows * (t - 32 + lane), 0u, mine, pv);
            pv = t + lane < my_n ? epi.pre(my0 + (uint64_t)kMvRows * (t + lane), 0u) : 0u;
        }
        const uint32_t st = t % ST;
        if (!mbar_wait(&full[st], (t / ST) & 1u, abort)) {
            if (status) *status = kDevTimeout;
            return;
        }
        const bool have = t < my_n;   // warp-uniform
        uint4 a[NK];
        if (have) {
            const uint4 *src = reinterpret_cast<const uint4 *>(buf + st * Cfg::kStageBytes + c * Cfg::kRowBytes) + lane;
#pragma unroll
            for (int m = 0; m < NK; ++m) a[m] = src[32 * m];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        if (have) {
            uint32_t acc = 0;
#pragma unroll
            for (int m = 0; m < NK; ++m)
                acc += a[m].x * sw[m].x + a[m].y * sw[m].y + a[m].z * sw[m].z + a[m].w * sw[m].w;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == static_cast<int>(k)) mine = acc;
        }
    }
    if (nst) {
        const uint32_t t0 = ((nst - 1) / 32u) * 32u;   // the last run
        if (t0 + lane < my_n) epi.put(my0 + (uint64_t)kMvRows * (t0 + lane), 0u, mine, pv);
    }
}

// Status word of the handle-free client kernels (one per process and
// device; read and cleared by client_status_take).
static __device__ int g_client_status;

template <class Epi>
static cudaError_t set_matvec_attrs() {
    cudaError_t e = cudaFuncSetAttribute(matvec_kernel<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 4);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(matvec_tma_kernel<4, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 MvCfg<4>::kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(matvec_tma_kernel<8, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 MvCfg<8>::kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(matvec_tma_kernel<16, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 MvCfg<16>::kSmemBytes);
    return e;
}

// Once per device, with that device current: kernel attributes and the
// device address of the status word.  Returns nullptr on failure.
static std::mutex g_client_mu;
static int *g_client_status_ptr[64];
static int *client_status_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> g(g_client_mu);
    if (!g_client_status_ptr[dev]) {
        void *p = nullptr;
        if (set_matvec_attrs<QueryEpi>() != cudaSuccess || set_matvec_attrs<RecoverEpi>() != cudaSuccess ||
            cudaGetSymbolAddress(&p, g_client_status) != cudaSuccess)
            return nullptr;
        g_client_status_ptr[dev] = static_cast<int *>(p);
    }
    return g_client_status_ptr[dev];
}

template <int NK, class Epi>
static cudaError_t launch_matvec_tma(const uint32_t *X, uint64_t rows, const uint32_t *w, const Epi &epi,
                                     int num_sms, int *status, cudaStream_t stream) {
    const uint64_t want = (rows + kMvRows - 1) / kMvRows;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(want < (uint64_t)num_sms ? want : (uint64_t)num_sms));
    cfg.blockDim = dim3(kMvThreads);
    cfg.dynamicSmemBytes = MvCfg<NK>::kSmemBytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, matvec_tma_kernel<NK, Epi>, X, rows, w, epi, status);
}

template <class Epi>
static cudaError_t launch_matvec(const uint32_t *X, uint64_t rows, uint32_t n, const uint32_t *w, const Epi &epi,
                                 int num_sms, cudaStream_t stream) {
    const bool aligned = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(w)) & 15u) == 0;
    if (aligned && rows > 0 && (n == 512 || n == 1024 || n == 2048)) {
        int *status = client_status_word();
        if (!status) return cudaErrorUnknown;
        if (n == 512) return launch_matvec_tma<4>(X, rows, w, epi, num_sms, status, stream);
        if (n == 1024) return launch_matvec_tma<8>(X, rows, w, epi, num_sms, status, stream);
        return launch_matvec_tma<16>(X, rows, w, epi, num_sms, status, stream);
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

cudaError_t prepare_client_kernels() { return client_status_word() ? cudaSuccess : cudaErrorUnknown; }

// Waits for the current device, then returns and clears its status word.
cudaError_t client_status_take(int *out) {
    *out = 0;
    int *p = client_status_word();
    if (!p) return cudaErrorUnknown;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out, p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && *out) e = cudaMemset(p, 0, sizeof(int));
    return e;
}

}  // namespace qpadl
