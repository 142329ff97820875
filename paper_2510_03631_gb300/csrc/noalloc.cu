// Allocation-free single-query Response (qpadl_pir_answer_noalloc) and the
// read of its status word (qpadl_pir_noalloc_status).
//
// Some callers cannot call cudaMalloc at the moment they need an answer:
// runtimes whose own memory manager owns all device memory and forbids side
// allocations, and latency-critical serving loops where the implicit
// device-wide synchronisation of cudaMalloc/cudaFree would stall every other
// stream.  This entry point answers one query against a caller-resident
// database with no handle and no allocation of any kind: the packed query
// limbs and the kernels' status word live in one fixed file-scope device
// array (g_noalloc_scratch, 1 MiB + 256 bytes), which every GPU that loads
// the library keeps until the process exits.
//
// The arithmetic is the same streaming Response as qpadl_pir_answer (the
// same pack and streaming kernels, launched with pointers into the fixed
// array instead of a handle's buffers).
//
// Ordering: the streaming kernel is launched with programmatic dependent
// launch and its producer issues its first database loads before it waits
// for its predecessor (a handle's database is immutable while bound).  Here
// the database is the caller's and may have just been written on the same
// stream, so the pack kernel (an ordinary launch, which starts only after
// everything earlier on the stream has finished and never lets its
// successor start early) must stay the streaming kernel's immediate
// predecessor: it is what orders the caller's writes before those loads.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "qpadl_pir.h"
#include "stream_answer.cuh"

namespace {

constexpr uint64_t kMaxCols = QPADL_NOALLOC_MAX_COLS;   // packed limbs: at most kMaxCols words
constexpr uint64_t kScratchWords = kMaxCols + 64;        // + status word (256-byte tail)
constexpr int kChunk = 2048;                             // streaming chunk width used here

static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

std::mutex g_mu;
uint32_t *g_scratch_ptr[64];   // device address of g_noalloc_scratch, per device
int g_num_sms[64];
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;   // resolved at the first set-up

// Once per device, with that device current: resolve the array's device
// address (the host-side name is only a stand-in) and set the kernels'
// shared-memory attributes.
int device_setup(int dev, uint32_t **scratch, int *num_sms) {
    if (dev < 0 || dev >= 64) return QPADL_EINVAL;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            std::fprintf(stderr, "qpadl_pir_answer_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
            return QPADL_ECUDA;
        }
        if (qpadl::prepare_stream_kernels() != cudaSuccess) return QPADL_ECUDA;
        if (!g_encode) {
            void *fp = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fp, 12000, cudaEnableDefault, &q) ==
                    cudaSuccess &&
                q == cudaDriverEntryPointSuccess)
                g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fp);
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QPADL_ECUDA;
        g_num_sms[dev] = sms;
        g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *scratch = g_scratch_ptr[dev];
    *num_sms = g_num_sms[dev];
    return QPADL_OK;
}

bool encode_db_map(CUtensorMap *map, const uint8_t *db, uint64_t R, uint64_t C) {
    if (!g_encode) return false;   // the bulk-copy form is used instead
    cuuint64_t dims[3] = {256, C / 256, R};
    cuuint64_t strides[2] = {256, C};
    cuuint32_t box[3] = {256, kChunk / 256, 8};
    cuuint32_t estr[3] = {1, 1, 1};
    return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(db), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" int qpadl_pir_answer_noalloc(const uint8_t *db_dev, uint64_t rows, uint64_t cols, const uint32_t *q_dev,
                                        uint32_t *ans_dev, qpadl_stream_t stream) {
    if (!db_dev || !q_dev || !ans_dev || rows == 0 || cols == 0 || rows >= (1ull << 31)) return QPADL_EINVAL;
    if (cols > kMaxCols) {
        std::fprintf(stderr,
                     "qpadl_pir_answer_noalloc: %llu columns exceed the fixed scratch limit of %llu "
                     "(QPADL_NOALLOC_MAX_COLS)\n",
                     static_cast<unsigned long long>(cols), static_cast<unsigned long long>(kMaxCols));
        return QPADL_EINVAL;
    }
    int dev = 0, sms = 0;
    uint32_t *scratch = nullptr;
    if (cudaGetDevice(&dev) != cudaSuccess) return QPADL_ECUDA;
    int rc = device_setup(dev, &scratch, &sms);
    if (rc != QPADL_OK) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t R = static_cast<uint32_t>(rows), C = static_cast<uint32_t>(cols);
    const bool bulk_ok = (cols % 16 == 0) && ((reinterpret_cast<uintptr_t>(db_dev) & 15u) == 0);
    if (!bulk_ok) {
        // shapes the bulk-copy kernel cannot take need no scratch at all
        return qpadl::launch_rowwise_answer(db_dev, rows, cols, q_dev, cols, 1, ans_dev, rows, sms, s) ==
                       cudaSuccess
                   ? QPADL_OK
                   : QPADL_ECUDA;
    }
    uint32_t *pack = scratch;
    int *status = reinterpret_cast<int *>(scratch + kMaxCols);
    const uint64_t pack_words = qpadl::stream_pack_words(cols);   // <= kMaxCols for cols <= kMaxCols
    // the packed limbs are fully rewritten by every call; the status word is only ever set (a
    // bounded wait that gave up) and stays set until qpadl_pir_noalloc_status reads it
    CUtensorMap map;
    const bool use_map = (cols % 256 == 0) && encode_db_map(&map, db_dev, rows, cols);
    if (qpadl::launch_pack_query(q_dev, cols, C, kChunk, 1, pack, pack_words, s) != cudaSuccess) return QPADL_ECUDA;
    if (qpadl::launch_stream_answer(1, kChunk, use_map ? &map : nullptr, db_dev, R, C, pack, pack_words, ans_dev,
                                    rows, sms, status, s) != cudaSuccess)
        return QPADL_ECUDA;
    return QPADL_OK;
}

extern "C" int qpadl_pir_noalloc_status(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QPADL_ECUDA;
    if (dev < 0 || dev >= 64) return QPADL_EINVAL;
    uint32_t *scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        scratch = g_scratch_ptr[dev];
    }
    if (!scratch) return QPADL_OK;   // no call has run on this device yet
    int *status = reinterpret_cast<int *>(scratch + kMaxCols);
    if (cudaDeviceSynchronize() != cudaSuccess) return QPADL_ECUDA;
    int word = 0;
    if (cudaMemcpy(&word, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return QPADL_ECUDA;
    if (word == 0) return QPADL_OK;
    if (cudaMemset(status, 0, sizeof(int)) != cudaSuccess) return QPADL_ECUDA;
    return QPADL_ETIMEOUT;
}
