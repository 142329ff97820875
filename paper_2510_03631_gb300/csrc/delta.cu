// Database compression of the spectrum records (Sec. 5.3, "Database
// Compression Techniques"): the DB entries are sorted and each is stored as
// its difference from the entry before it, so close entries take fewer bits
// and every PIR Response scans fewer bytes.
//
// Layout (the reading this library takes): the entries are 32-bit unsigned
// integers x_0 <= x_1 <= ... <= x_{n-1}; block j (one PIR record, i.e. one
// column of the database) holds entries jE .. jE + E - 1, positions past
// n - 1 repeating x_{n-1}.  A block is stored as its first entry in full (4
// little-endian bytes) followed by its E - 1 differences x_{jE+i} -
// x_{jE+i-1} (mod 2^32), each in w little-endian bytes, w the fewest bytes
// that hold every such difference.  The database is then R' = 4 + w (E - 1)
// rows of digits by C = ceil(n / E) columns, row-major, and the usual LWE
// Response, Recover and hint run on it unchanged.  A client that recovers
// block j decodes it on its own by prefix sums.
//
//   delta_width_kernel   largest within-block difference: a warp per block,
//                        a warp max, one atomic max per warp
//   delta_encode_kernel  a CTA per 128 blocks x 64 differences: the entries
//                        staged in shared memory (read run by run), the
//                        database rows written 128 bytes at a time (four
//                        columns per 32-bit store when aligned)
//   delta_decode_kernel  one CTA per recovered block: per-thread runs of
//                        differences, a CTA-wide exclusive scan of the run
//                        totals, then each run's prefix sums
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "qpadl_pir.h"

namespace {

__device__ __forceinline__ uint32_t entry_at(const uint32_t *__restrict__ x, uint64_t n, uint64_t k) {
    return x[k < n ? k : n - 1];
}

// One warp per block (grid-stride over blocks), lanes striding over its differences.
__global__ void delta_width_kernel(const uint32_t *__restrict__ x, uint64_t n, uint64_t E, uint64_t C,
                                   uint32_t *__restrict__ dmax) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    uint32_t m = 0;
    for (uint64_t j = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < C; j += warps)
        for (uint64_t i = 1 + lane; i < E; i += 32) {
            const uint32_t d = entry_at(x, n, j * E + i) - entry_at(x, n, j * E + i - 1);
            m = d > m ? d : m;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t other = __shfl_xor_sync(0xffffffffu, m, o);
        m = other > m ? other : m;
    }
    if (lane == 0 && m) atomicMax(dmax, m);
}

// A CTA writes the rows of kEncCols consecutive blocks (columns) that hold
// differences kEncEntries * blockIdx.y + 1 .. + kEncEntries (and the CTAs with
// blockIdx.y == 0 also the 4 rows of the first entries).  The entries it needs
// are read run by run (consecutive entries of one block are contiguous) into
// shared memory, so both the reads and the row writes are coalesced.
constexpr int kEncCols = 128;     // columns per CTA: each database row segment is 128 bytes
constexpr int kEncEntries = 64;   // differences per block per CTA
constexpr int kEncThreads = 256;

__global__ void __launch_bounds__(kEncThreads) delta_encode_kernel(const uint32_t *__restrict__ x, uint64_t n,
                                                                   uint64_t E, uint32_t w, uint64_t C,
                                                                   uint8_t *__restrict__ db) {
    __shared__ uint32_t ent[kEncCols][kEncEntries + 1];   // entries i0 - 1 .. i0 + kEncEntries - 1
    const uint64_t j0 = (uint64_t)blockIdx.x * kEncCols;
    const uint64_t i0 = 1 + (uint64_t)blockIdx.y * kEncEntries;   // first difference of this CTA
    const uint64_t ncols = C - j0 < (uint64_t)kEncCols ? C - j0 : (uint64_t)kEncCols;
    const uint64_t i1 = i0 + kEncEntries < E ? i0 + kEncEntries : E;   // differences [i0, i1)
    // stage entries (block j0 + c, positions i0 - 1 .. i1 - 1): consecutive threads take
    // consecutive entries of one block's run, and each thread issues its loads independently
    const uint32_t nt = static_cast<uint32_t>(i1 - i0) + 1;
    const uint32_t nload = static_cast<uint32_t>(ncols) * nt;
#pragma unroll 4
    for (uint32_t f = threadIdx.x; f < nload; f += kEncThreads) {
        const uint32_t c = f / nt, t = f - c * nt;
        ent[c][t] = entry_at(x, n, (j0 + c) * E + i0 - 1 + t);
    }
    __syncthreads();
    // rows of this CTA's differences: row 4 + (i - 1) w + b, column j0 + c; threads run over
    // (row, column) with the column fastest
    const uint32_t rows = (nt - 1) * w;   // at most 64 x 4 rows: 32-bit index math below
    const uint64_t row0 = 4 + (i0 - 1) * w;
    // four columns per thread in one 32-bit store when every row segment is 4-byte aligned
    const bool quad = (C % 4 == 0) && (ncols % 4 == 0) && ((reinterpret_cast<uintptr_t>(db) & 3u) == 0);
    if (quad) {
        constexpr uint32_t kQuads = kEncCols / 4;
        for (uint32_t t = threadIdx.x; t < rows * kQuads; t += kEncThreads) {
            const uint32_t r = t / kQuads, c = 4 * (t % kQuads);
            if (c >= ncols) continue;
            const uint32_t di = r / w;   // difference i0 + di
            const uint32_t sh = 8u * (r - di * w);
            uint32_t v = 0;
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k)
                v |= (((ent[c + k][di + 1] - ent[c + k][di]) >> sh) & 255u) << (8u * k);
            *reinterpret_cast<uint32_t *>(db + (row0 + r) * C + j0 + c) = v;
        }
    } else {
        for (uint32_t t = threadIdx.x; t < rows * kEncCols; t += kEncThreads) {
            const uint32_t r = t / kEncCols, c = t % kEncCols;
            if (c >= ncols) continue;
            const uint32_t di = r / w;   // difference i0 + di
            const uint32_t b = r - di * w;
            const uint32_t d = ent[c][di + 1] - ent[c][di];
            db[(row0 + r) * C + j0 + c] = static_cast<uint8_t>(d >> (8u * b));
        }
    }
    if (blockIdx.y == 0) {   // the first entry of each block in full
        for (uint64_t t = threadIdx.x; t < 4 * (uint64_t)kEncCols; t += kEncThreads) {
            const uint64_t r = t / kEncCols, c = t % kEncCols;
            if (c < ncols) db[r * C + j0 + c] = static_cast<uint8_t>(ent[c][0] >> (8u * r));
        }
    }
}

constexpr int kDecodeThreads = 256;

// Block b: digits b * Rp .. (4-byte first entry, then E - 1 differences of w bytes) -> out b * E ..
__global__ void __launch_bounds__(kDecodeThreads) delta_decode_kernel(const uint8_t *__restrict__ digits, uint64_t E,
                                                                      uint32_t w, uint64_t Rp,
                                                                      uint32_t *__restrict__ out) {
    __shared__ uint32_t part[kDecodeThreads];
    const uint8_t *dg = digits + (uint64_t)blockIdx.x * Rp;
    uint32_t *o = out + (uint64_t)blockIdx.x * E;
    const uint64_t nd = E - 1;                                       // differences in the block
    const uint64_t run = (nd + kDecodeThreads - 1) / kDecodeThreads;  // differences per thread
    const uint64_t i0 = (uint64_t)threadIdx.x * run;
    const uint64_t i1 = i0 + run < nd ? i0 + run : nd;
    auto diff = [&](uint64_t i) {   // difference i (0-based) of the block
        const uint8_t *p = dg + 4 + i * w;
        uint32_t d = 0;
        for (uint32_t b = 0; b < w; ++b) d |= static_cast<uint32_t>(p[b]) << (8u * b);
        return d;
    };
    uint32_t sum = 0;
    for (uint64_t i = i0; i < i1; ++i) sum += diff(i);
    part[threadIdx.x] = sum;
    __syncthreads();
    // inclusive scan of the run totals (Hillis-Steele over 256 values)
    for (int off = 1; off < kDecodeThreads; off <<= 1) {
        const uint32_t add = threadIdx.x >= static_cast<unsigned>(off) ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    const uint32_t first = static_cast<uint32_t>(dg[0]) | (static_cast<uint32_t>(dg[1]) << 8) |
                           (static_cast<uint32_t>(dg[2]) << 16) | (static_cast<uint32_t>(dg[3]) << 24);
    uint32_t v = first + (threadIdx.x ? part[threadIdx.x - 1] : 0u);
    if (threadIdx.x == 0) o[0] = first;
    for (uint64_t i = i0; i < i1; ++i) {
        v += diff(i);
        o[i + 1] = v;
    }
}

// The width reduction's result word: one per device, used under g_width_mu for
// the whole (synchronous) call, so the call allocates nothing.
__device__ uint32_t g_width_word;
std::mutex g_width_mu;

int num_sms_current() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    return sms;
}

bool delta_shape_ok(uint64_t n, uint64_t E, uint32_t w) {
    if (n == 0 || E == 0 || w < 1 || w > 4) return false;
    const uint64_t C = (n + E - 1) / E;
    const uint64_t Rp = 4 + (uint64_t)w * (E - 1);
    return C < (1ull << 31) && Rp < (1ull << 31);
}

}  // namespace

extern "C" {

int qpadl_pir_delta_width(const uint32_t *entries_dev, uint64_t n, uint32_t E, uint32_t *w_out,
                          qpadl_stream_t stream) {
    if (!entries_dev || !w_out || !delta_shape_ok(n, E, 4)) return QPADL_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int sms = num_sms_current();
    if (sms <= 0) return QPADL_ECUDA;
    const uint64_t C = (n + E - 1) / E;
    std::lock_guard<std::mutex> guard(g_width_mu);
    uint32_t *dmax = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void **>(&dmax), g_width_word) != cudaSuccess) return QPADL_ECUDA;
    uint32_t h = 0;
    bool ok = cudaMemsetAsync(dmax, 0, sizeof(uint32_t), s) == cudaSuccess;
    if (ok) {
        delta_width_kernel<<<sms * 8, 256, 0, s>>>(entries_dev, n, E, C, dmax);
        ok = cudaGetLastError() == cudaSuccess;
    }
    ok = ok && cudaMemcpyAsync(&h, dmax, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) return QPADL_ECUDA;
    uint32_t w = 1;
    while (w < 4 && h >= (1u << (8u * w))) ++w;
    *w_out = w;
    return QPADL_OK;
}

int qpadl_pir_delta_encode(const uint32_t *entries_dev, uint64_t n, uint32_t E, uint32_t w, uint8_t *db_dev,
                           qpadl_stream_t stream) {
    if (!entries_dev || !db_dev || !delta_shape_ok(n, E, w)) return QPADL_EINVAL;
    const int sms = num_sms_current();
    if (sms <= 0) return QPADL_ECUDA;
    (void)sms;
    const uint64_t C = (n + E - 1) / E;
    const uint64_t ytiles = E > 1 ? (E - 1 + kEncEntries - 1) / kEncEntries : 1;
    if (ytiles > 65535) return QPADL_EINVAL;   // blocks of more than 4 million entries
    const dim3 grid(static_cast<unsigned>((C + kEncCols - 1) / kEncCols), static_cast<unsigned>(ytiles));
    delta_encode_kernel<<<grid, kEncThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(entries_dev, n, E, w, C,
                                                                                          db_dev);
    return cudaGetLastError() == cudaSuccess ? QPADL_OK : QPADL_ECUDA;
}

int qpadl_pir_delta_decode(const uint8_t *digits_dev, uint32_t B, uint32_t E, uint32_t w, uint32_t *entries_dev,
                           qpadl_stream_t stream) {
    if (!digits_dev || !entries_dev || B == 0 || !delta_shape_ok(E, E, w)) return QPADL_EINVAL;
    const uint64_t Rp = 4 + (uint64_t)w * (E - 1);
    delta_decode_kernel<<<B, kDecodeThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(digits_dev, E, w, Rp,
                                                                                          entries_dev);
    return cudaGetLastError() == cudaSuccess ? QPADL_OK : QPADL_ECUDA;
}

}  // extern "C"
