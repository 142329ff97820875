// C-ABI entry points of the LWE-style PIR engine (declared in include/qpadl_pir.h).
//
// This file owns validation, the per-database handle, tensor-map encoding
// and the choice of kernel; the arithmetic lives in stream_answer.cu
// (single/few-query Response), limb_gemm.cu (batched Response and hint) and
// client.cu (Setup's generator, Query, Recover).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "chor.cuh"
#include "client.cuh"
#include "limb_gemm.cuh"
#include "limb_gemm_pair.cuh"
#include "limb_gemm_u8.cuh"
#include "internal.cuh"
#include "qpadl_pir.h"
#include "stream_answer.cuh"

using namespace qpadl;

struct qpadl_db {
    qpadl_params prm;
    const uint8_t *db = nullptr;
    int device = 0;
    int num_sms = 0;
    int *d_status = nullptr;         // device status word (kernels' bounded waits)
    // streaming path
    bool stream_ok = false;          // C % 16 == 0 and D 16-byte aligned
    int stream_chunk = 2048;         // digits per row per stage (QPADL_OPT_STREAM_CHUNK)
    int stream_raw = 0;              // QPADL_OPT_STREAM_RAW
    uint32_t tensor_min_batch = 3;   // QPADL_OPT_TENSOR_MIN_BATCH
    bool stream_maps = false;        // C % 256 == 0: 3-D tensor maps below are valid
    CUtensorMap stream_map[4];       // box {256, cch/256, 8} for cch = 512 << i
    uint32_t *qpack = nullptr;       // packed limbs of up to 4 queries
    uint64_t pack_words = 0;         // per query
    // tensor-core paths
    bool u8_ok = false;              // the u8 GEMM can run (blocked copy built on first use)
    uint8_t *blk = nullptr;          // blocked copy of the digits (128 x 128 tiles)
    uint64_t blk_bytes = 0;
    CUtensorMap u8_map[2];           // over blk: box {128, 128, ks/128, 1} for ks = 128, 256
    uint32_t u8_max_batch = 64;      // QPADL_OPT_U8_MAX_BATCH
    int u8_kstep = 0;                // QPADL_OPT_U8_KSTEP (0 = per tile width default)
    int pair_gemm = 1;               // QPADL_OPT_PAIR_GEMM
    __half *d16 = nullptr;           // digits as fp16, R x pitch
    uint64_t pitch = 0;              // roundup(C, 8)
    CUtensorMap a_map;
    __half *limbs = nullptr;         // limb scratch
    uint64_t limbs_bytes = 0;
    // host-buffer calls
    uint32_t *stage_q = nullptr;
    uint32_t *stage_ans = nullptr;
    uint64_t owned_bytes = 0;
};

// Client context for batched Query / Recover on the tensor cores.
struct qpadl_client {
    qpadl_params prm;
    int device = 0;
    int num_sms = 0;
    uint32_t max_batch = 0;
    uint64_t pitch = 0;              // fp16 elements per limb-plane row: roundup(4n, 8)
    __half *a_planes = nullptr;      // C x pitch: limb planes of A side by side
    __half *h_planes = nullptr;      // R x pitch: limb planes of H (optional)
    __half *v = nullptr;             // 4 max_batch x pitch: shifted secret limbs
    CUtensorMap a_map, h_map;
    int *d_status = nullptr;
    uint64_t owned_bytes = 0;
    bool planed = true;              // skip the zero (plane, shift) blocks when n % 512 == 0
    bool pair = true;                // tiles over pairs of SMs (QPADL_CLIENT_OPT_PAIR_GEMM)
};

// Goldberg-style Z_p database handle: the lattice handle of the same bytes
// (streaming kernel, fp16 operand copy, limb scratch) plus the field.
struct qpadl_goldberg {
    qpadl_db *db = nullptr;
    uint32_t p = 0;
    uint32_t gemm_min_batch = 3;     // batches from this size take a tensor-core GEMM
    uint32_t u8_max_batch = 128;     // ... the uint8-digit one up to this size, the one-limb fp16 one above
};

// Chor-style GF(2) database handle.
struct qpadl_chor {
    uint64_t rows = 0;
    uint32_t words = 0;              // W = bits / 32 per row
    uint64_t qw = 0;                 // query words: ceil(rows / 32)
    const uint32_t *db = nullptr;    // caller-owned, rows x W words
    int device = 0;
    int num_sms = 0;
    uint32_t *qt = nullptr;          // selector scratch: rows x 8 words or ceil(rows/32) x 256 words
    int *d_status = nullptr;
    uint64_t owned_bytes = 0;
    uint32_t m4rm_min_batch = 48;    // batches from this size take the four-Russians kernel
    int scan_form = -1;              // QPADL_CHOR_OPT_SCAN_FORM (-1: by batch size)
};

namespace {

constexpr int kMaxN = 16384;
// Goldberg sums stay exact (|centred sum| < 2^31, unsigned sum < 2^32) below this many columns
constexpr uint64_t kGoldbergMaxCols = 65792;

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return QPADL_OK;
    std::fprintf(stderr, "qpadl: %s: %s\n", what, cudaGetErrorString(e));
    return QPADL_ECUDA;
}

#define QPADL_CU(call)                                        \
    do {                                                      \
        int rc__ = cuda_fail((call), #call);                  \
        if (rc__ != QPADL_OK) return rc__;                    \
    } while (0)

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D map over a row-major matrix: `inner` elements per row (extent),
// `outer` rows, `pitch_bytes` between rows, box of box_inner x box_outer.
bool encode_2d(CUtensorMap *map, CUtensorMapDataType dt, const void *base, uint64_t inner, uint64_t outer,
               uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {pitch_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool prepared[64];
std::mutex prep_mu;

int prepare_device(int dev) {
    std::lock_guard<std::mutex> g(prep_mu);
    if (dev < 0 || dev >= 64) return QPADL_EINVAL;
    if (prepared[dev]) return QPADL_OK;
    QPADL_CU(prepare_stream_kernels());
    QPADL_CU(prepare_limb_gemm_kernels());
    QPADL_CU(prepare_limb_gemm_pair_kernels());
    QPADL_CU(prepare_limb_gemm_u8_kernels());
    QPADL_CU(prepare_client_kernels());
    QPADL_CU(prepare_chor_kernels());
    prepared[dev] = true;
    return QPADL_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int log2_exact(uint32_t p) {
    int l = 0;
    while ((1u << l) < p) ++l;
    return (1u << l) == p ? l : -1;
}

int validate_params(const qpadl_params *prm) {
    if (!prm) return QPADL_EINVAL;
    if (prm->rows == 0 || prm->cols == 0 || prm->n == 0 || prm->n > (uint32_t)kMaxN) return QPADL_EINVAL;
    if (prm->rows >= (1ull << 31) || prm->cols >= (1ull << 31)) return QPADL_EINVAL;
    if (prm->log_q != 32) return QPADL_EINVAL;
    if (prm->p < 2 || prm->p > 256 || log2_exact(prm->p) < 0) return QPADL_EINVAL;
    return QPADL_OK;
}

__global__ void max_digit_kernel(const uint8_t *D, uint64_t total, int *out) {
    uint32_t m = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride)
        m = D[e] > m ? D[e] : m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, static_cast<int>(m));
}

int dev_alloc(qpadl_db *db, void **p, uint64_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return QPADL_ENOMEM;
    }
    db->owned_bytes += bytes;
    return QPADL_OK;
}

void dev_free(qpadl_db *db, void *p, uint64_t bytes) {
    if (p) {
        cudaFree(p);
        db->owned_bytes -= bytes;
    }
}

int ensure_tensor_copy(qpadl_db *db, cudaStream_t stream) {
    if (db->d16) return QPADL_OK;
    const uint64_t R = db->prm.rows, C = db->prm.cols;
    const uint64_t bytes = R * db->pitch * 2;
    int rc = dev_alloc(db, reinterpret_cast<void **>(&db->d16), bytes);
    if (rc != QPADL_OK) return rc;
    QPADL_CU(launch_db_to_f16(db->db, R, C, db->d16, db->pitch, db->num_sms, stream));
    if (!encode_2d(&db->a_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, db->d16, C, R, db->pitch * 2, kLimbBoxK,
                   kLimbBoxM, CU_TENSOR_MAP_SWIZZLE_128B))
        return QPADL_ECUDA;
    return QPADL_OK;
}

int ensure_limbs(qpadl_db *db, uint64_t bytes) {
    if (db->limbs_bytes >= bytes) return QPADL_OK;
    if (db->limbs) {
        // the old scratch may still be read by queued work on any stream
        cudaDeviceSynchronize();
        dev_free(db, db->limbs, db->limbs_bytes);
        db->limbs = nullptr;
        db->limbs_bytes = 0;
    }
    int rc = dev_alloc(db, reinterpret_cast<void **>(&db->limbs), bytes);
    if (rc != QPADL_OK) return rc;
    db->limbs_bytes = bytes;
    return QPADL_OK;
}

int set_device(const qpadl_db *db) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return QPADL_ECUDA;
    if (cur != db->device && cudaSetDevice(db->device) != cudaSuccess) return QPADL_ECUDA;
    return QPADL_OK;
}

// out[i * ld_m + v * ld_b] = D * X[v] for NV vectors given as fp16 limbs at `limbs`
// (4 NV rows of db->pitch elements), on CTA pairs or single SMs (QPADL_OPT_PAIR_GEMM)
int run_limb_gemm_at(qpadl_db *db, const __half *limbs, uint32_t NV, uint32_t *out, uint64_t ld_m, uint64_t ld_b,
                     cudaStream_t stream) {
    if (db->pair_gemm && db->num_sms >= 2) {
        const int bn = limb_gemm_pair_bn_for(NV);
        PairBMaps bm;
        std::memset(&bm, 0, sizeof(bm));
        if (!encode_2d(&bm.m[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, limbs, db->prm.cols, 4ull * NV, db->pitch * 2,
                       kLimbBoxK, pair_b_box_rows(bn, false, 0), CU_TENSOR_MAP_SWIZZLE_128B))
            return QPADL_ECUDA;
        QPADL_CU(launch_limb_gemm_pair(bn, db->a_map, bm, out, ld_m, ld_b, static_cast<uint32_t>(db->prm.rows), NV,
                                       db->prm.cols, db->num_sms, db->d_status, stream));
        return QPADL_OK;
    }
    const int bn = limb_gemm_bn_for(NV);
    CUtensorMap b_map;
    if (!encode_2d(&b_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, limbs, db->prm.cols, 4ull * NV, db->pitch * 2,
                   kLimbBoxK, static_cast<uint32_t>(bn), CU_TENSOR_MAP_SWIZZLE_128B))
        return QPADL_ECUDA;
    QPADL_CU(launch_limb_gemm(bn, db->a_map, b_map, out, ld_m, ld_b, static_cast<uint32_t>(db->prm.rows), NV,
                              db->prm.cols, db->num_sms, db->d_status, stream));
    return QPADL_OK;
}

int run_limb_gemm(qpadl_db *db, uint32_t NV, uint32_t *out, uint64_t ld_m, uint64_t ld_b, cudaStream_t stream) {
    return run_limb_gemm_at(db, db->limbs, NV, out, ld_m, ld_b, stream);
}

int answer_stream_group(qpadl_db *db, const uint32_t *Q, uint32_t nq, uint32_t *ans, cudaStream_t stream) {
    const uint64_t C = db->prm.cols, R = db->prm.rows;
    const int cch = nq == 1 ? db->stream_chunk : 1024;
    QPADL_CU(launch_pack_query(Q, C, static_cast<uint32_t>(C), static_cast<uint32_t>(cch), nq, db->qpack,
                               db->pack_words, stream));
    int mi = 0;
    while ((512 << mi) < cch) ++mi;
    const CUtensorMap *map = db->stream_maps ? &db->stream_map[mi] : nullptr;
    QPADL_CU(launch_stream_answer(static_cast<int>(nq), cch, map, db->db, static_cast<uint32_t>(R),
                                  static_cast<uint32_t>(C), db->qpack, db->pack_words, ans, R, db->num_sms,
                                  db->d_status, stream));
    return QPADL_OK;
}

// Chunk width of the two-query in-kernel-packing form: the handle's single-query width where
// that form has it (1024 or 2048), else 1024.
int raw2_chunk(const qpadl_db *db) { return db->stream_chunk == 2048 ? 2048 : 1024; }

int answer_two_raw(qpadl_db *db, const uint32_t *Q, uint64_t q_ld, uint32_t *ans, uint64_t ans_ld,
                   cudaStream_t stream) {
    const uint64_t C = db->prm.cols, R = db->prm.rows;
    const int cch = raw2_chunk(db);
    int mi = 0;
    while ((512 << mi) < cch) ++mi;
    const CUtensorMap *map = db->stream_maps ? &db->stream_map[mi] : nullptr;
    QPADL_CU(launch_stream_answer_raw2(cch, map, db->db, static_cast<uint32_t>(R), static_cast<uint32_t>(C), Q, q_ld,
                                       ans, ans_ld, db->num_sms, db->d_status, stream));
    return QPADL_OK;
}

int answer_streaming(qpadl_db *db, const uint32_t *Q, uint32_t B, uint32_t *ans, cudaStream_t stream) {
    const uint64_t C = db->prm.cols, R = db->prm.rows;
    if (db->stream_ok && B == 2 && db->stream_raw && aligned16(Q))
        return answer_two_raw(db, Q, C, ans, R, stream);   // both queries in one pass, no scratch
    if (db->stream_ok && B == 1 && db->stream_raw && aligned16(Q)) {
        // one query: the streaming kernel packs its limbs itself (one launch, no scratch)
        int mi = 0;
        while ((512 << mi) < db->stream_chunk) ++mi;
        const CUtensorMap *map = db->stream_maps ? &db->stream_map[mi] : nullptr;
        QPADL_CU(launch_stream_answer_raw(db->stream_chunk, map, db->db, static_cast<uint32_t>(R),
                                          static_cast<uint32_t>(C), Q, ans, db->num_sms, db->d_status, stream));
        return QPADL_OK;
    }
    if (!db->stream_ok) {
        QPADL_CU(launch_rowwise_answer(db->db, R, C, Q, C, B, ans, R, db->num_sms, stream));
        return QPADL_OK;
    }
    uint32_t b = 0;
    while (b < B) {
        const uint32_t left = B - b;
        const uint32_t nq = left >= 4 ? 4 : (left >= 2 ? 2 : 1);
        int rc = answer_stream_group(db, Q + (uint64_t)b * C, nq, ans + (uint64_t)b * R, stream);
        if (rc != QPADL_OK) return rc;
        b += nq;
    }
    return QPADL_OK;
}

// The blocked copy of the digits that the u8 GEMM reads, and its tensor maps.
int ensure_blocked(qpadl_db *db, cudaStream_t stream) {
    if (db->blk) return QPADL_OK;
    const uint64_t R = db->prm.rows, C = db->prm.cols;
    const uint64_t RB = (R + 127) / 128, CB = (C + 127) / 128;
    const uint64_t bytes = RB * CB * 16384;
    int rc = dev_alloc(db, reinterpret_cast<void **>(&db->blk), bytes);
    if (rc != QPADL_OK) return rc;
    db->blk_bytes = bytes;
    QPADL_CU(launch_block_digits(db->db, R, C, db->blk, stream));
    auto fn = encode_fn();
    for (int i = 0; i < 2; ++i) {
        cuuint64_t dims[4] = {128, 128, CB, RB};
        cuuint64_t strides[3] = {128, 16384, CB * 16384};
        cuuint32_t box[4] = {128, 128, static_cast<cuuint32_t>(i + 1), 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        if (!fn || fn(&db->u8_map[i], CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, db->blk, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return QPADL_ECUDA;
    }
    return QPADL_OK;
}

// Batched answer on the u8 GEMM (blocked digits, fp16 made in TMEM): one group of at most
// 4096 queries (the limb scratch), in tiles of up to 128 limb columns.
// out[i * ld_m + v * ld_b] = D * X[v] for B vectors whose fp16 limbs are in db->limbs, on the
// uint8-digit GEMM (the output block must be dense: it is zeroed, split tiles add into it).
// after_prep: the kernel just before this launch in the stream made the limbs and zeroed the
// output block (launch_vec_limbs with `zero`), so the GEMM skips the memset and overlaps that
// kernel as its programmatic dependent.
int run_u8_gemm(qpadl_db *db, uint32_t B, uint32_t *ans, uint64_t ld_m, uint64_t ld_b, cudaStream_t stream,
                bool after_prep = false) {
    const uint64_t R = db->prm.rows, C = db->prm.cols;
    const int bn = std::min(limb_gemm_bn_for(B), 128);
    const int ks = db->u8_kstep ? db->u8_kstep : limb_gemm_u8_default_ks(bn);
    const bool pair = db->pair_gemm && db->num_sms >= 2 && limb_gemm_u8_pair_ok(bn, ks);
    const uint32_t tile_rows = pair ? 2 * kLimbBoxM : kLimbBoxM;
    GroupedGemmArgs args;
    std::memset(&args, 0, sizeof(args));
    args.a[0] = db->u8_map[ks / 128 - 1];
    if (!encode_2d(&args.b[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, db->limbs, C, 4ull * B, db->pitch * 2, kLimbBoxK,
                   static_cast<uint32_t>(pair ? bn / 2 : bn), CU_TENSOR_MAP_SWIZZLE_128B))
        return QPADL_ECUDA;
    GroupDesc &g = args.g[0];
    g.out = ans;
    g.ld_m = ld_m;
    g.ld_b = ld_b;
    g.M = static_cast<uint32_t>(R);
    g.NV = B;
    g.KB = static_cast<uint32_t>((C + ks - 1) / ks);
    g.unit_begin = 0;
    g.n_tiles = (4 * B + bn - 1) / bn;
    args.ngroups = 1;
    args.total_units = static_cast<uint32_t>((R + tile_rows - 1) / tile_rows) * g.n_tiles * g.KB;
    // tiles split between CTAs are accumulated with atomic adds into zeros
    if (!after_prep) QPADL_CU(cudaMemsetAsync(ans, 0, 4ull * B * R, stream));
    QPADL_CU(launch_limb_gemm_u8(bn, ks, args, db->num_sms, db->d_status, stream, pair, after_prep));
    return QPADL_OK;
}

int answer_tensor_u8_chunk(qpadl_db *db, const uint32_t *Q, uint32_t B, uint32_t *ans, cudaStream_t stream) {
    const uint64_t R = db->prm.rows, C = db->prm.cols;
    // one launch makes the limbs and zeroes the answers; the GEMM overlaps its start with it
    QPADL_CU(launch_vec_limbs(Q, C, B, C, db->limbs, db->pitch, db->num_sms, stream, ans, (uint64_t)B * R));
    return run_u8_gemm(db, B, ans, 1, R, stream, true);
}

int answer_tensor_u8(qpadl_db *db, const uint32_t *Q, uint32_t B, uint32_t *ans, cudaStream_t stream) {
    int rc = ensure_blocked(db, stream);
    if (rc != QPADL_OK) return rc;
    constexpr uint32_t kChunk = 4096;
    rc = ensure_limbs(db, 8ull * std::min(B, kChunk) * db->pitch);
    if (rc != QPADL_OK) return rc;
    const uint64_t R = db->prm.rows, C = db->prm.cols;
    for (uint32_t b0 = 0; b0 < B; b0 += kChunk) {
        rc = answer_tensor_u8_chunk(db, Q + (uint64_t)b0 * C, std::min(B - b0, kChunk), ans + (uint64_t)b0 * R,
                                    stream);
        if (rc != QPADL_OK) return rc;
    }
    return QPADL_OK;
}

int answer_tensor(qpadl_db *db, const uint32_t *Q, uint32_t B, uint32_t *ans, cudaStream_t stream) {
    if (db->u8_ok && B <= db->u8_max_batch) return answer_tensor_u8(db, Q, B, ans, stream);
    int rc = ensure_tensor_copy(db, stream);
    if (rc != QPADL_OK) return rc;
    // chunks of at most 4096 queries bound the limb scratch (8 bytes per query per column)
    constexpr uint32_t kChunk = 4096;
    rc = ensure_limbs(db, 8ull * std::min(B, kChunk) * db->pitch);
    if (rc != QPADL_OK) return rc;
    const uint64_t C = db->prm.cols, R = db->prm.rows;
    for (uint32_t b0 = 0; b0 < B; b0 += kChunk) {
        const uint32_t Bc = std::min(B - b0, kChunk);
        QPADL_CU(launch_vec_limbs(Q + (uint64_t)b0 * C, C, Bc, C, db->limbs, db->pitch, db->num_sms, stream));
        rc = run_limb_gemm(db, Bc, ans + (uint64_t)b0 * R, 1, R, stream);
        if (rc != QPADL_OK) return rc;
    }
    return QPADL_OK;
}

}  // namespace

// ------------------------------------------------------------------ internal (serving loop)
namespace qpadl {

uint64_t db_limb_pitch(const qpadl_db *db) { return db->pitch; }
int db_num_sms(const qpadl_db *db) { return db->num_sms; }
int *db_status_word(qpadl_db *db) { return db->d_status; }
int db_prepare_u8(qpadl_db *db, cudaStream_t stream) { return ensure_blocked(db, stream); }
int db_prepare_f16(qpadl_db *db, cudaStream_t stream) { return ensure_tensor_copy(db, stream); }
bool db_pair_gemm(const qpadl_db *db) { return db->pair_gemm && db->num_sms >= 2; }

int db_fill_u8_group(qpadl_db *db, GroupedGemmArgs &args, int g, const __half *limbs, uint32_t NV, uint32_t *out,
                     int bn, int ks, uint32_t unit_begin, uint32_t *units, bool pair) {
    if (!db->blk || g < 0 || g >= kMaxGemmGroups) return QPADL_EINVAL;
    const uint64_t R = db->prm.rows, C = db->prm.cols;
    const uint32_t tile_rows = pair ? 2 * kLimbBoxM : kLimbBoxM;
    args.a[g] = db->u8_map[ks / 128 - 1];
    if (!encode_2d(&args.b[g], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, limbs, C, 4ull * NV, db->pitch * 2, kLimbBoxK,
                   static_cast<uint32_t>(pair ? bn / 2 : bn), CU_TENSOR_MAP_SWIZZLE_128B))
        return QPADL_ECUDA;
    GroupDesc &gd = args.g[g];
    gd.out = out;
    gd.ld_m = 1;
    gd.ld_b = R;
    gd.M = static_cast<uint32_t>(R);
    gd.NV = NV;
    gd.KB = static_cast<uint32_t>((C + ks - 1) / ks);
    gd.unit_begin = unit_begin;
    gd.n_tiles = (4 * NV + bn - 1) / bn;
    *units = static_cast<uint32_t>((R + tile_rows - 1) / tile_rows) * gd.n_tiles * gd.KB;
    return QPADL_OK;
}

int db_answer_f16_ws(qpadl_db *db, const uint32_t *Q, uint32_t B, uint32_t *ans, __half *limbs,
                     cudaStream_t stream) {
    if (!db->d16) return QPADL_EINVAL;
    const uint64_t C = db->prm.cols, R = db->prm.rows;
    QPADL_CU(launch_vec_limbs(Q, C, B, C, limbs, db->pitch, db->num_sms, stream));
    return run_limb_gemm_at(db, limbs, B, ans, 1, R, stream);
}

int db_answer_one_noscratch(qpadl_db *db, const uint32_t *q, uint32_t *ans, cudaStream_t stream) {
    const uint64_t C = db->prm.cols, R = db->prm.rows;
    if (db->stream_ok && aligned16(q)) {
        int mi = 0;
        while ((512 << mi) < db->stream_chunk) ++mi;
        const CUtensorMap *map = db->stream_maps ? &db->stream_map[mi] : nullptr;
        QPADL_CU(launch_stream_answer_raw(db->stream_chunk, map, db->db, static_cast<uint32_t>(R),
                                          static_cast<uint32_t>(C), q, ans, db->num_sms, db->d_status, stream));
        return QPADL_OK;
    }
    QPADL_CU(launch_rowwise_answer(db->db, R, C, q, C, 1, ans, R, db->num_sms, stream));
    return QPADL_OK;
}

int db_answer_two_noscratch(qpadl_db *db, const uint32_t *q, uint64_t q_ld, uint32_t *ans, uint64_t ans_ld,
                            cudaStream_t stream) {
    if (db->stream_ok && aligned16(q) && q_ld % 4 == 0) return answer_two_raw(db, q, q_ld, ans, ans_ld, stream);
    const uint64_t C = db->prm.cols, R = db->prm.rows;
    QPADL_CU(launch_rowwise_answer(db->db, R, C, q, q_ld, 2, ans, ans_ld, db->num_sms, stream));
    return QPADL_OK;
}

}  // namespace qpadl

namespace {

// Mean CUDA-event time of `reps` calls of fn on stream s after one warm-up call; < 0 on failure.
template <class F>
double time_calls(F fn, cudaStream_t s, int reps) {
    if (fn() != QPADL_OK) return -1.0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.0;
    }
    double ms = -1.0;
    bool ok = cudaEventRecord(e0, s) == cudaSuccess;
    for (int i = 0; i < reps && ok; ++i) ok = fn() == QPADL_OK;
    ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float t = 0.f;
    if (ok && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = t / reps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace

extern "C" {

const char *qpadl_strerror(int code) {
    switch (code) {
        case QPADL_OK: return "ok";
        case QPADL_EINVAL: return "invalid argument";
        case QPADL_ENOMEM: return "out of device memory";
        case QPADL_ECUDA: return "CUDA error";
        case QPADL_ETIMEOUT: return "device wait timed out";
        case QPADL_EBUSY: return "busy: admission refused";
        case QPADL_EAGAIN: return "not ready";
        default: return "unknown error";
    }
}

int qpadl_version(void) { return 10000; }

int qpadl_pir_setup(const qpadl_params *prm, const uint8_t *db_dev, qpadl_stream_t stream, qpadl_db **out) {
    if (!out || !db_dev) return QPADL_EINVAL;
    *out = nullptr;
    int rc = validate_params(prm);
    if (rc != QPADL_OK) return rc;
    qpadl_db *db = new (std::nothrow) qpadl_db();
    if (!db) return QPADL_ENOMEM;
    db->prm = *prm;
    db->db = db_dev;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto fail = [&](int code) {
        qpadl_pir_destroy(db);
        return code;
    };
    if (cudaGetDevice(&db->device) != cudaSuccess) return fail(QPADL_ECUDA);
    if (cudaDeviceGetAttribute(&db->num_sms, cudaDevAttrMultiProcessorCount, db->device) != cudaSuccess)
        return fail(QPADL_ECUDA);
    if ((rc = prepare_device(db->device)) != QPADL_OK) return fail(rc);
    if ((rc = dev_alloc(db, reinterpret_cast<void **>(&db->d_status), 16)) != QPADL_OK) return fail(rc);
    if (cudaMemsetAsync(db->d_status, 0, 16, s) != cudaSuccess) return fail(QPADL_ECUDA);
    const uint64_t R = prm->rows, C = prm->cols;
    if (prm->p < 256) {
        max_digit_kernel<<<db->num_sms * 4, 256, 0, s>>>(db_dev, R * C, db->d_status + 1);
        int mx = 0;
        if (cudaGetLastError() != cudaSuccess) return fail(QPADL_ECUDA);
        if (cudaMemcpyAsync(&mx, db->d_status + 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(QPADL_ECUDA);
        if (mx >= static_cast<int>(prm->p)) return fail(QPADL_EINVAL);
    }
    db->stream_ok = (C % 16 == 0) && aligned16(db_dev);
    if (db->stream_ok && C % 256 == 0) {
        db->stream_maps = true;
        for (int i = 0; i < 4; ++i) {
            auto fn = encode_fn();
            cuuint64_t dims[3] = {256, C / 256, R};
            cuuint64_t strides[2] = {256, C};
            cuuint32_t box[3] = {256, static_cast<cuuint32_t>((512u << i) / 256u),
                                 static_cast<cuuint32_t>(16384u / (512u << i))};
            cuuint32_t estr[3] = {1, 1, 1};
            if (!fn || fn(&db->stream_map[i], CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(db_dev), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return fail(QPADL_ECUDA);
        }
    }
    db->pitch = (C + 7) / 8 * 8;
    db->u8_ok = true;
    if (db->stream_ok) {
        db->pack_words = stream_pack_words(C);
        if ((rc = dev_alloc(db, reinterpret_cast<void **>(&db->qpack), 4 * db->pack_words * 4)) != QPADL_OK)
            return fail(rc);
    }
    if ((rc = dev_alloc(db, reinterpret_cast<void **>(&db->stage_q), C * 4)) != QPADL_OK) return fail(rc);
    if ((rc = dev_alloc(db, reinterpret_cast<void **>(&db->stage_ans), R * 4)) != QPADL_OK) return fail(rc);
    if (prm->flags & QPADL_SETUP_TENSOR_COPY) {
        if ((rc = ensure_tensor_copy(db, s)) != QPADL_OK) return fail(rc);
    }
    *out = db;
    return QPADL_OK;
}

int qpadl_pir_destroy(qpadl_db *db) {
    if (!db) return QPADL_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (db->device != cur) cudaSetDevice(db->device);
    cudaDeviceSynchronize();
    dev_free(db, db->d_status, 16);
    dev_free(db, db->qpack, 4 * db->pack_words * 4);
    dev_free(db, db->d16, db->prm.rows * db->pitch * 2);
    dev_free(db, db->blk, db->blk_bytes);
    dev_free(db, db->limbs, db->limbs_bytes);
    dev_free(db, db->stage_q, db->prm.cols * 4);
    dev_free(db, db->stage_ans, db->prm.rows * 4);
    if (cur >= 0 && cur != db->device) cudaSetDevice(cur);
    delete db;
    return QPADL_OK;
}

int qpadl_pir_status(qpadl_db *db) {
    if (!db) return QPADL_EINVAL;
    if (set_device(db) != QPADL_OK) return QPADL_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return QPADL_ECUDA;
    int st = 0;
    if (cudaMemcpy(&st, db->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return QPADL_ECUDA;
    if (st != 0) {
        const int zero = 0;
        cudaMemcpy(db->d_status, &zero, 4, cudaMemcpyHostToDevice);
        return QPADL_ETIMEOUT;
    }
    return QPADL_OK;
}

uint64_t qpadl_pir_device_bytes(const qpadl_db *db) { return db ? db->owned_bytes : 0; }

int qpadl_pir_shape(const qpadl_db *db, uint64_t *rows, uint64_t *cols) {
    if (!db || !rows || !cols) return QPADL_EINVAL;
    *rows = db->prm.rows;
    *cols = db->prm.cols;
    return QPADL_OK;
}

int qpadl_pir_shard_rows(uint64_t rows, uint32_t world, uint32_t rank, uint64_t *r0, uint64_t *r1) {
    if (world == 0 || rank >= world || !r0 || !r1) return QPADL_EINVAL;
    const uint64_t tiles = (rows + kLimbBoxM - 1) / kLimbBoxM;
    const uint64_t t0 = tiles * rank / world, t1 = tiles * (rank + 1ull) / world;
    *r0 = std::min<uint64_t>(rows, t0 * kLimbBoxM);
    *r1 = std::min<uint64_t>(rows, t1 * kLimbBoxM);
    return QPADL_OK;
}

int qpadl_pir_reserve(qpadl_db *db, uint32_t max_batch, qpadl_stream_t stream) {
    if (!db || max_batch == 0) return QPADL_EINVAL;
    if (set_device(db) != QPADL_OK) return QPADL_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (max_batch >= db->tensor_min_batch) {
        if (!(db->u8_ok && max_batch <= db->u8_max_batch)) {
            int rc = ensure_tensor_copy(db, s);
            if (rc != QPADL_OK) return rc;
        }
        if (db->u8_ok && db->u8_max_batch >= db->tensor_min_batch) {
            int rc = ensure_blocked(db, s);
            if (rc != QPADL_OK) return rc;
        }
        // the batched paths work in chunks of at most 4096 queries
        int rc = ensure_limbs(db, 8ull * std::min<uint32_t>(max_batch, 4096u) * db->pitch);
        if (rc != QPADL_OK) return rc;
    }
    QPADL_CU(cudaStreamSynchronize(s));
    return QPADL_OK;
}

int qpadl_pir_gen_a(const qpadl_params *prm, uint32_t *A_dev, qpadl_stream_t stream) {
    int rc = validate_params(prm);
    if (rc != QPADL_OK) return rc;
    if (!A_dev || (reinterpret_cast<uintptr_t>(A_dev) & 3u)) return QPADL_EINVAL;
    int dev = 0, sms = 0;
    QPADL_CU(cudaGetDevice(&dev));
    QPADL_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    QPADL_CU(launch_gen_a(prm->seed, prm->cols, prm->n, A_dev, sms, reinterpret_cast<cudaStream_t>(stream)));
    return QPADL_OK;
}

int qpadl_pir_hint(qpadl_db *db, const uint32_t *A_dev, uint32_t *H_dev, qpadl_stream_t stream) {
    if (!db || !A_dev || !H_dev) return QPADL_EINVAL;
    if (set_device(db) != QPADL_OK) return QPADL_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t n = db->prm.n;
    const bool u8 = db->u8_ok && n <= db->u8_max_batch;   // the lean layout keeps no fp16 copy
    int rc = u8 ? ensure_blocked(db, s) : ensure_tensor_copy(db, s);
    if (rc != QPADL_OK) return rc;
    rc = ensure_limbs(db, 8ull * n * db->pitch);
    if (rc != QPADL_OK) return rc;
    QPADL_CU(launch_mat_col_limbs(A_dev, db->prm.cols, n, db->limbs, db->pitch, s));
    return u8 ? run_u8_gemm(db, n, H_dev, n, 1, s) : run_limb_gemm(db, n, H_dev, n, 1, s);
}

int qpadl_pir_query(const qpadl_params *prm, const uint32_t *A_dev, const uint32_t *s_dev, const int32_t *e_dev,
                    uint64_t col, uint32_t *q_dev, qpadl_stream_t stream) {
    int rc = validate_params(prm);
    if (rc != QPADL_OK) return rc;
    if (!A_dev || !s_dev || !e_dev || !q_dev || col >= prm->cols) return QPADL_EINVAL;
    int dev = 0, sms = 0;
    QPADL_CU(cudaGetDevice(&dev));
    QPADL_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint32_t delta = static_cast<uint32_t>((1ull << 32) / prm->p);
    QPADL_CU(launch_query(A_dev, prm->cols, prm->n, s_dev, e_dev, col, delta, q_dev, sms,
                          reinterpret_cast<cudaStream_t>(stream)));
    return QPADL_OK;
}

int qpadl_pir_client_status(void) {
    int w = 0;
    if (client_status_take(&w) != cudaSuccess) return QPADL_ECUDA;
    return w ? QPADL_ETIMEOUT : QPADL_OK;
}

int qpadl_pir_query_batch(const qpadl_params *prm, const uint32_t *A_dev, const uint32_t *S_dev,
                          const int32_t *E_dev, const uint32_t *cols_dev, uint32_t B, uint32_t *Q_dev,
                          qpadl_stream_t stream) {
    int rc = validate_params(prm);
    if (rc != QPADL_OK) return rc;
    if (!A_dev || !S_dev || !E_dev || !cols_dev || !Q_dev || B == 0) return QPADL_EINVAL;
    const uint32_t delta = static_cast<uint32_t>((1ull << 32) / prm->p);
    QPADL_CU(launch_query_batch(A_dev, prm->cols, prm->n, S_dev, E_dev, cols_dev, B, delta, Q_dev,
                                reinterpret_cast<cudaStream_t>(stream)));
    return QPADL_OK;
}

int qpadl_pir_answer(qpadl_db *db, const uint32_t *q_dev, uint32_t *ans_dev, qpadl_stream_t stream) {
    if (!db || !q_dev || !ans_dev) return QPADL_EINVAL;
    if (set_device(db) != QPADL_OK) return QPADL_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return answer_streaming(db, q_dev, 1, ans_dev, s);
}

int qpadl_pir_answer_batch_path(qpadl_db *db, const uint32_t *Q_dev, uint32_t B, uint32_t *ans_dev, int path,
                                qpadl_stream_t stream) {
    if (!db || !Q_dev || !ans_dev || B == 0 || (path != 0 && path != 1)) return QPADL_EINVAL;
    if (set_device(db) != QPADL_OK) return QPADL_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return path == 0 ? answer_streaming(db, Q_dev, B, ans_dev, s) : answer_tensor(db, Q_dev, B, ans_dev, s);
}

int qpadl_pir_answer_batch(qpadl_db *db, const uint32_t *Q_dev, uint32_t B, uint32_t *ans_dev,
                           qpadl_stream_t stream) {
    if (!db) return QPADL_EINVAL;
    return qpadl_pir_answer_batch_path(db, Q_dev, B, ans_dev, B >= db->tensor_min_batch ? 1 : 0, stream);
}

int qpadl_pir_set_option(qpadl_db *db, int option, int64_t value) {
    if (!db) return QPADL_EINVAL;
    switch (option) {
        case QPADL_OPT_STREAM_CHUNK:
            if (!stream_config_valid(1, static_cast<int>(value))) return QPADL_EINVAL;
            db->stream_chunk = static_cast<int>(value);
            return QPADL_OK;
        case QPADL_OPT_TENSOR_MIN_BATCH:
            if (value < 1 || value > (1ll << 30)) return QPADL_EINVAL;
            db->tensor_min_batch = static_cast<uint32_t>(value);
            return QPADL_OK;
        case QPADL_OPT_STREAM_RAW:
            if (value != 0 && value != 1) return QPADL_EINVAL;
            db->stream_raw = static_cast<int>(value);
            return QPADL_OK;
        case QPADL_OPT_U8_MAX_BATCH:
            if (value < 0 || value > (1ll << 30)) return QPADL_EINVAL;
            db->u8_max_batch = static_cast<uint32_t>(value);
            return QPADL_OK;
        case QPADL_OPT_U8_KSTEP:
            if (value != 0 && value != 128 && value != 256) return QPADL_EINVAL;
            db->u8_kstep = static_cast<int>(value);
            return QPADL_OK;
        case QPADL_OPT_PAIR_GEMM:
            if (value != 0 && value != 1) return QPADL_EINVAL;
            db->pair_gemm = static_cast<int>(value);
            return QPADL_OK;
        default: return QPADL_EINVAL;
    }
}

int qpadl_pir_get_option(const qpadl_db *db, int option, int64_t *value) {
    if (!db || !value) return QPADL_EINVAL;
    switch (option) {
        case QPADL_OPT_STREAM_CHUNK: *value = db->stream_chunk; return QPADL_OK;
        case QPADL_OPT_TENSOR_MIN_BATCH: *value = db->tensor_min_batch; return QPADL_OK;
        case QPADL_OPT_STREAM_RAW: *value = db->stream_raw; return QPADL_OK;
        case QPADL_OPT_U8_MAX_BATCH: *value = db->u8_max_batch; return QPADL_OK;
        case QPADL_OPT_U8_KSTEP: *value = db->u8_kstep; return QPADL_OK;
        case QPADL_OPT_PAIR_GEMM: *value = db->pair_gemm; return QPADL_OK;
        default: return QPADL_EINVAL;
    }
}

int qpadl_pir_autotune(qpadl_db *db, uint32_t max_batch, qpadl_stream_t stream, qpadl_tune_report *report) {
    if (!db || max_batch == 0) return QPADL_EINVAL;
    if (set_device(db) != QPADL_OK) return QPADL_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t R = db->prm.rows, C = db->prm.cols;
    qpadl_tune_report rep;
    std::memset(&rep, 0, sizeof(rep));
    const uint32_t BT = std::min<uint32_t>(std::max<uint32_t>(max_batch, 4u), 16u);
    const uint32_t BQ = max_batch > 32 ? 128u : BT;   // scratch: the GEMM comparison takes 128 queries
    uint32_t *Q = nullptr, *A = nullptr;
    if (cudaMalloc(reinterpret_cast<void **>(&Q), 4ull * C * BQ) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&A), 4ull * R * BQ) != cudaSuccess) {
        cudaGetLastError();
        if (Q) cudaFree(Q);
        return QPADL_ENOMEM;
    }
    auto done = [&](int rc) {
        cudaStreamSynchronize(s);
        cudaFree(Q);
        cudaFree(A);
        if (rc == QPADL_OK && report) *report = rep;
        return rc;
    };
    // synthetic queries (uniform words); the answers are discarded
    if (cuda_fail(launch_gen_a(0x9E3779B97F4A7C15ull, C * BQ, 1, Q, db->num_sms, s), "tune queries") != QPADL_OK)
        return done(QPADL_ECUDA);
    constexpr int kReps = 5;
    // 1. one query: chunk width x in-kernel packing
    const int chunks[3] = {1024, 2048, 4096};
    double best = 1e30;
    int best_chunk = db->stream_chunk, best_raw = db->stream_raw;
    for (int ci = 0; ci < 3; ++ci) {
        for (int raw = 0; raw < 2; ++raw) {
            rep.single_ms[ci][raw] = -1.0;
            if (!db->stream_ok || !stream_config_valid(1, chunks[ci])) continue;
            db->stream_chunk = chunks[ci];
            db->stream_raw = raw;
            const double ms = time_calls([&] { return answer_streaming(db, Q, 1, A, s); }, s, kReps);
            rep.single_ms[ci][raw] = ms;
            if (ms > 0 && ms < best) {
                best = ms;
                best_chunk = chunks[ci];
                best_raw = raw;
            }
        }
    }
    db->stream_chunk = best_chunk;
    db->stream_raw = best_raw;
    // 2. small batches: digit-tile depth of the uint8 GEMM, then the streaming/tensor crossover
    rep.tuned_batch = BT;
    if (max_batch >= 2) {
        if (db->u8_ok && db->u8_max_batch >= BT) {
            const int ks[2] = {128, 256};
            double kbest = 1e30;
            int kpick = db->u8_kstep;
            for (int k = 0; k < 2; ++k) {
                db->u8_kstep = ks[k];
                const double ms = time_calls([&] { return answer_tensor(db, Q, BT, A, s); }, s, kReps);
                rep.u8_kstep_ms[k] = ms;
                if (ms > 0 && ms < kbest) {
                    kbest = ms;
                    kpick = ks[k];
                }
            }
            // the pair form exists only with 128-digit stages: while it is on, a deeper stage would
            // also move every batch onto single-SM tiles, which one probe size cannot weigh (both
            // depths are timed and reported; the depth stays 128)
            db->u8_kstep = (db->pair_gemm && db->num_sms >= 2) ? 128 : kpick;
        }
        uint32_t threshold = db->tensor_min_batch;
        for (uint32_t B = 2; B <= 4; ++B) {
            const double ms_s = time_calls([&] { return answer_streaming(db, Q, B, A, s); }, s, kReps);
            const double ms_t = time_calls([&] { return answer_tensor(db, Q, B, A, s); }, s, kReps);
            rep.stream_ms[B - 2] = ms_s;
            rep.tensor_ms[B - 2] = ms_t;
            if (ms_s > 0 && ms_t > 0 && ms_t < ms_s) {
                threshold = B;
                break;
            }
            threshold = B + 1;
        }
        db->tensor_min_batch = threshold;
    }
    // 3. larger batches: how far the uint8-digit GEMM stays ahead of the fp16-copy GEMM
    rep.u8_vs_f16_ms[0][0] = rep.u8_vs_f16_ms[0][1] = rep.u8_vs_f16_ms[1][0] = rep.u8_vs_f16_ms[1][1] = -1.0;
    if (max_batch > 32 && db->u8_ok) {
        const uint32_t keep = db->u8_max_batch;
        uint32_t pick = 32;
        const uint32_t Bs[2] = {64, 128};
        for (int i = 0; i < 2; ++i) {
            db->u8_max_batch = 1u << 30;
            const double mu = time_calls([&] { return answer_tensor(db, Q, Bs[i], A, s); }, s, kReps);
            db->u8_max_batch = 0;
            const double mf = time_calls([&] { return answer_tensor(db, Q, Bs[i], A, s); }, s, kReps);
            rep.u8_vs_f16_ms[i][0] = mu;
            rep.u8_vs_f16_ms[i][1] = mf;
            if (mu > 0 && mf > 0 && mu <= mf) pick = Bs[i];
        }
        db->u8_max_batch = keep == 64 || keep == 32 || keep == 128 ? pick : keep;
    }
    rep.u8_max_batch = db->u8_max_batch;
    rep.stream_chunk = db->stream_chunk;
    rep.stream_raw = db->stream_raw;
    rep.u8_kstep = db->u8_kstep;
    rep.tensor_min_batch = db->tensor_min_batch;
    return done(QPADL_OK);
}

int qpadl_pir_answer_host(qpadl_db *db, const uint32_t *q_host, uint32_t *ans_host, qpadl_stream_t stream) {
    if (!db || !q_host || !ans_host) return QPADL_EINVAL;
    if (set_device(db) != QPADL_OK) return QPADL_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t C = db->prm.cols, R = db->prm.rows;
    QPADL_CU(cudaMemcpyAsync(db->stage_q, q_host, C * 4, cudaMemcpyHostToDevice, s));
    int rc = answer_streaming(db, db->stage_q, 1, db->stage_ans, s);
    if (rc != QPADL_OK) return rc;
    QPADL_CU(cudaMemcpyAsync(ans_host, db->stage_ans, R * 4, cudaMemcpyDeviceToHost, s));
    QPADL_CU(cudaStreamSynchronize(s));
    return QPADL_OK;
}

int qpadl_pir_recover(const qpadl_params *prm, const uint32_t *ans_dev, const uint32_t *H_dev,
                      const uint32_t *s_dev, uint8_t *out_dev, qpadl_stream_t stream) {
    int rc = validate_params(prm);
    if (rc != QPADL_OK) return rc;
    if (!ans_dev || !H_dev || !s_dev || !out_dev) return QPADL_EINVAL;
    int dev = 0, sms = 0;
    QPADL_CU(cudaGetDevice(&dev));
    QPADL_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint32_t shift = 32u - static_cast<uint32_t>(log2_exact(prm->p));
    QPADL_CU(launch_recover(ans_dev, H_dev, prm->rows, prm->n, s_dev, shift, out_dev, sms,
                            reinterpret_cast<cudaStream_t>(stream)));
    return QPADL_OK;
}

int qpadl_pir_recover_batch(const qpadl_params *prm, const uint32_t *ans_dev, const uint32_t *H_dev,
                            const uint32_t *S_dev, uint32_t B, uint8_t *out_dev, qpadl_stream_t stream) {
    int rc = validate_params(prm);
    if (rc != QPADL_OK) return rc;
    if (!ans_dev || !H_dev || !S_dev || !out_dev || B == 0) return QPADL_EINVAL;
    const uint32_t shift = 32u - static_cast<uint32_t>(log2_exact(prm->p));
    QPADL_CU(launch_recover_batch(ans_dev, H_dev, prm->rows, prm->n, S_dev, B, shift, out_dev,
                                  reinterpret_cast<cudaStream_t>(stream)));
    return QPADL_OK;
}

// ------------------------------------------------------------------ client context

int qpadl_client_destroy(qpadl_client *c) {
    if (!c) return QPADL_OK;
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != c->device) cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->a_planes) cudaFree(c->a_planes);
    if (c->h_planes) cudaFree(c->h_planes);
    if (c->v) cudaFree(c->v);
    if (c->d_status) cudaFree(c->d_status);
    if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
    delete c;
    return QPADL_OK;
}

int qpadl_client_create(const qpadl_params *prm, const uint32_t *A_dev, const uint32_t *H_dev, uint32_t max_batch,
                        qpadl_stream_t stream, qpadl_client **out) {
    if (!out) return QPADL_EINVAL;
    *out = nullptr;
    int rc = validate_params(prm);
    if (rc != QPADL_OK) return rc;
    if (!A_dev || max_batch == 0 || max_batch > 65536) return QPADL_EINVAL;
    qpadl_client *c = new (std::nothrow) qpadl_client();
    if (!c) return QPADL_ENOMEM;
    c->prm = *prm;
    c->max_batch = max_batch;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto fail = [&](int code) {
        qpadl_client_destroy(c);
        return code;
    };
    auto alloc = [&](void **p, uint64_t bytes) {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        c->owned_bytes += bytes;
        return true;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) return fail(QPADL_ECUDA);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return fail(QPADL_ECUDA);
    if ((rc = prepare_device(c->device)) != QPADL_OK) return fail(rc);
    const uint64_t n = prm->n, R = prm->rows, C = prm->cols;
    c->pitch = (4 * n + 7) / 8 * 8;
    if (!alloc(reinterpret_cast<void **>(&c->d_status), 16)) return fail(QPADL_ENOMEM);
    if (!alloc(reinterpret_cast<void **>(&c->a_planes), 2 * C * c->pitch)) return fail(QPADL_ENOMEM);
    if (H_dev && !alloc(reinterpret_cast<void **>(&c->h_planes), 2 * R * c->pitch)) return fail(QPADL_ENOMEM);
    // room for the planed layout: 4 rows per vector, vectors rounded up to 64
    const uint64_t vrows = 4ull * ((max_batch + 63) / 64 * 64);
    if (!alloc(reinterpret_cast<void **>(&c->v), 2ull * vrows * c->pitch)) return fail(QPADL_ENOMEM);
    if (cudaMemsetAsync(c->d_status, 0, 16, s) != cudaSuccess) return fail(QPADL_ECUDA);
    if (cuda_fail(launch_mat_row_limbs(A_dev, C, prm->n, c->a_planes, c->pitch, c->num_sms, s), "A limb planes") !=
        QPADL_OK)
        return fail(QPADL_ECUDA);
    if (!encode_2d(&c->a_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, c->a_planes, 4 * n, C, c->pitch * 2, kLimbBoxK,
                   kLimbBoxM, CU_TENSOR_MAP_SWIZZLE_128B))
        return fail(QPADL_ECUDA);
    if (H_dev) {
        if (cuda_fail(launch_mat_row_limbs(H_dev, R, prm->n, c->h_planes, c->pitch, c->num_sms, s),
                      "H limb planes") != QPADL_OK)
            return fail(QPADL_ECUDA);
        if (!encode_2d(&c->h_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, c->h_planes, 4 * n, R, c->pitch * 2, kLimbBoxK,
                       kLimbBoxM, CU_TENSOR_MAP_SWIZZLE_128B))
            return fail(QPADL_ECUDA);
    }
    *out = c;
    return QPADL_OK;
}

namespace {

int client_set_device(const qpadl_client *c) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return QPADL_ECUDA;
    if (cur != c->device && cudaSetDevice(c->device) != cudaSuccess) return QPADL_ECUDA;
    return QPADL_OK;
}

// Planed mode applies when every 512-deep chunk lies in one limb plane and a
// shift group is at least 16 columns wide.
uint32_t client_plane_chunks(const qpadl_client *c, int bn) {
    return (c->planed && c->prm.n % 512 == 0 && bn >= 64) ? c->prm.n / 512 : 0u;
}

// Shifted secret limbs of Bc secrets into c->v and the tensor map over them.
int client_secret_operand(qpadl_client *c, const uint32_t *S, uint32_t Bc, int bn, uint32_t plane_chunks,
                          CUtensorMap *map, cudaStream_t s) {
    const uint32_t n = c->prm.n;
    uint64_t rows = 4ull * Bc;
    if (plane_chunks) {
        const uint32_t qpt = static_cast<uint32_t>(bn / 4);
        QPADL_CU(launch_secret_limbs_planed(S, Bc, n, qpt, c->v, c->pitch, c->num_sms, s));
        rows = 4ull * ((Bc + qpt - 1) / qpt * qpt);
    } else {
        QPADL_CU(launch_secret_limbs(S, Bc, n, c->v, c->pitch, c->num_sms, s));
    }
    if (!encode_2d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, c->v, 4ull * n, rows, c->pitch * 2, kLimbBoxK,
                   static_cast<uint32_t>(bn), CU_TENSOR_MAP_SWIZZLE_128B))
        return QPADL_ECUDA;
    return QPADL_OK;
}

// Pair-tile form of the secret operand: planed rows with qpt = bn / 8 padded to whole
// pair tiles (bn / 4 secrets), or the plain shifted rows; one map per limb plane.
int client_secret_operand_pair(qpadl_client *c, const uint32_t *S, uint32_t Bc, int bn, uint32_t plane_chunks,
                               PairBMaps *bm, cudaStream_t s) {
    const uint32_t n = c->prm.n;
    std::memset(bm, 0, sizeof(*bm));
    uint64_t rows = 4ull * Bc;
    if (plane_chunks) {
        const uint32_t qpt = static_cast<uint32_t>(bn / 8), per_tile = static_cast<uint32_t>(bn / 4);
        const uint32_t Bp = (Bc + per_tile - 1) / per_tile * per_tile;
        QPADL_CU(launch_secret_limbs_planed(S, Bc, n, qpt, c->v, c->pitch, c->num_sms, s, Bp));
        rows = 4ull * Bp;
    } else {
        QPADL_CU(launch_secret_limbs(S, Bc, n, c->v, c->pitch, c->num_sms, s));
    }
    for (int u = 0; u < (plane_chunks ? 4 : 1); ++u)
        if (!encode_2d(&bm->m[u], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, c->v, 4ull * n, rows, c->pitch * 2, kLimbBoxK,
                       pair_b_box_rows(bn, plane_chunks != 0, u), CU_TENSOR_MAP_SWIZZLE_128B))
            return QPADL_ECUDA;
    return QPADL_OK;
}

// Planed pair tiles need n a multiple of 512 and at least 16 secret rows per shift group.
uint32_t client_pair_plane_chunks(const qpadl_client *c, int bn) {
    return (c->planed && c->prm.n % 512 == 0 && bn >= 128) ? c->prm.n / 512 : 0u;
}

}  // namespace

int qpadl_client_query_batch(qpadl_client *c, const uint32_t *S_dev, const int32_t *E_dev, const uint32_t *cols_dev,
                             uint32_t B, uint32_t *Q_dev, qpadl_stream_t stream) {
    if (!c || !S_dev || !E_dev || !cols_dev || !Q_dev || B == 0) return QPADL_EINVAL;
    if (client_set_device(c) != QPADL_OK) return QPADL_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t C = c->prm.cols, n = c->prm.n;
    const uint32_t delta = static_cast<uint32_t>((1ull << 32) / c->prm.p);
    for (uint32_t b0 = 0; b0 < B; b0 += c->max_batch) {
        const uint32_t Bc = std::min(B - b0, c->max_batch);
        const QueryNoiseEpi epi{E_dev + (uint64_t)b0 * C, C, Q_dev + (uint64_t)b0 * C, C};
        if (c->pair && c->num_sms >= 2) {
            const int bn = limb_gemm_pair_bn_for(Bc);
            const uint32_t pc = client_pair_plane_chunks(c, bn);
            PairBMaps bm;
            int rc = client_secret_operand_pair(c, S_dev + (uint64_t)b0 * n, Bc, bn, pc, &bm, s);
            if (rc != QPADL_OK) return rc;
            QPADL_CU(launch_limb_gemm_pair_query(bn, c->a_map, bm, epi, static_cast<uint32_t>(C), Bc, 4 * n, pc,
                                                 c->num_sms, c->d_status, s));
            QPADL_CU(launch_add_delta(Q_dev + (uint64_t)b0 * C, C, cols_dev + b0, Bc, delta, s));
            continue;
        }
        const int bn = limb_gemm_bn_for(Bc);
        const uint32_t pc = client_plane_chunks(c, bn);
        CUtensorMap v_map;
        int rc = client_secret_operand(c, S_dev + (uint64_t)b0 * n, Bc, bn, pc, &v_map, s);
        if (rc != QPADL_OK) return rc;
        QPADL_CU(launch_limb_gemm_query(bn, c->a_map, v_map, epi, static_cast<uint32_t>(C), Bc, 4 * n, pc,
                                        c->num_sms, c->d_status, s));
        QPADL_CU(launch_add_delta(Q_dev + (uint64_t)b0 * C, C, cols_dev + b0, Bc, delta, s));
    }
    return QPADL_OK;
}

int qpadl_client_recover_batch(qpadl_client *c, const uint32_t *ans_dev, const uint32_t *S_dev, uint32_t B,
                               uint8_t *out_dev, qpadl_stream_t stream) {
    if (!c || !ans_dev || !S_dev || !out_dev || B == 0 || !c->h_planes) return QPADL_EINVAL;
    if (client_set_device(c) != QPADL_OK) return QPADL_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t R = c->prm.rows, n = c->prm.n;
    const uint32_t shift = 32u - static_cast<uint32_t>(log2_exact(c->prm.p));
    for (uint32_t b0 = 0; b0 < B; b0 += c->max_batch) {
        const uint32_t Bc = std::min(B - b0, c->max_batch);
        const RecoverEpi epi{ans_dev + (uint64_t)b0 * R, R, shift, out_dev + (uint64_t)b0 * R, R};
        if (c->pair && c->num_sms >= 2) {
            const int bn = limb_gemm_pair_bn_for(Bc);
            const uint32_t pc = client_pair_plane_chunks(c, bn);
            PairBMaps bm;
            int rc = client_secret_operand_pair(c, S_dev + (uint64_t)b0 * n, Bc, bn, pc, &bm, s);
            if (rc != QPADL_OK) return rc;
            QPADL_CU(launch_limb_gemm_pair_recover(bn, c->h_map, bm, epi, static_cast<uint32_t>(R), Bc, 4 * n, pc,
                                                   c->num_sms, c->d_status, s));
            continue;
        }
        const int bn = limb_gemm_bn_for(Bc);
        const uint32_t pc = client_plane_chunks(c, bn);
        CUtensorMap v_map;
        int rc = client_secret_operand(c, S_dev + (uint64_t)b0 * n, Bc, bn, pc, &v_map, s);
        if (rc != QPADL_OK) return rc;
        QPADL_CU(launch_limb_gemm_recover(bn, c->h_map, v_map, epi, static_cast<uint32_t>(R), Bc, 4 * n, pc,
                                          c->num_sms, c->d_status, s));
    }
    return QPADL_OK;
}

int qpadl_client_status(qpadl_client *c) {
    if (!c) return QPADL_EINVAL;
    if (client_set_device(c) != QPADL_OK) return QPADL_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return QPADL_ECUDA;
    int st = 0;
    if (cudaMemcpy(&st, c->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return QPADL_ECUDA;
    if (st != 0) {
        const int zero = 0;
        cudaMemcpy(c->d_status, &zero, 4, cudaMemcpyHostToDevice);
        return QPADL_ETIMEOUT;
    }
    return QPADL_OK;
}

uint64_t qpadl_client_device_bytes(const qpadl_client *c) { return c ? c->owned_bytes : 0; }

int qpadl_client_set_option(qpadl_client *c, int option, int64_t value) {
    if (!c) return QPADL_EINVAL;
    switch (option) {
        case QPADL_CLIENT_OPT_SKIP_ZERO_BLOCKS:
            if (value != 0 && value != 1) return QPADL_EINVAL;
            c->planed = value != 0;
            return QPADL_OK;
        case QPADL_CLIENT_OPT_PAIR_GEMM:
            if (value != 0 && value != 1) return QPADL_EINVAL;
            c->pair = value != 0;
            return QPADL_OK;
        default: return QPADL_EINVAL;
    }
}

// ------------------------------------------------------------------ Chor-style GF(2) Response

int qpadl_chor_destroy(qpadl_chor *h) {
    if (!h) return QPADL_OK;
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != h->device) cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    if (h->qt) cudaFree(h->qt);
    if (h->d_status) cudaFree(h->d_status);
    if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
    delete h;
    return QPADL_OK;
}

int qpadl_chor_setup(uint64_t rows, uint64_t bits, const uint32_t *db_dev, qpadl_stream_t stream,
                     qpadl_chor **out) {
    if (!out) return QPADL_EINVAL;
    *out = nullptr;
    if (!db_dev || rows == 0 || rows >= (1ull << 31) || bits == 0 || bits % 128 != 0 || bits / 32 >= (1ull << 31) ||
        (reinterpret_cast<uintptr_t>(db_dev) & 15u) != 0)
        return QPADL_EINVAL;
    qpadl_chor *h = new (std::nothrow) qpadl_chor();
    if (!h) return QPADL_ENOMEM;
    h->rows = rows;
    h->words = static_cast<uint32_t>(bits / 32);
    h->qw = (rows + 31) / 32;
    h->db = db_dev;
    auto fail = [&](int code) {
        qpadl_chor_destroy(h);
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(QPADL_ECUDA);
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return fail(QPADL_ECUDA);
    int rc = prepare_device(h->device);
    if (rc != QPADL_OK) return fail(rc);
    const uint64_t qt_bytes = 4ull * std::max<uint64_t>(rows * 8, (h->qw + 1) / 2 * 2 * kChorMaxBatch);
    if (cudaMalloc(reinterpret_cast<void **>(&h->qt), qt_bytes) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&h->d_status), 16) != cudaSuccess) {
        cudaGetLastError();
        return fail(QPADL_ENOMEM);
    }
    h->owned_bytes = qt_bytes + 16;
    if (cudaMemsetAsync(h->d_status, 0, 16, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return fail(QPADL_ECUDA);
    *out = h;
    return QPADL_OK;
}

int qpadl_chor_answer_batch(qpadl_chor *h, const uint32_t *Q_dev, uint32_t B, uint32_t *out_dev,
                            qpadl_stream_t stream) {
    if (!h || !Q_dev || !out_dev || B == 0) return QPADL_EINVAL;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return QPADL_ECUDA;
    if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess) return QPADL_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t W = h->words;
    QPADL_CU(cudaMemsetAsync(out_dev, 0, 4ull * W * B, s));
    for (uint32_t b0 = 0; b0 < B; b0 += kChorMaxBatch) {
        const uint32_t Bc = std::min(B - b0, kChorMaxBatch);
        if (Bc >= h->m4rm_min_batch) {
            QPADL_CU(launch_chor_words(Q_dev + (uint64_t)b0 * h->qw, h->qw, Bc, h->rows, h->qt, h->num_sms, s));
            CUtensorMap db_map;
            if (!encode_2d(&db_map, CU_TENSOR_MAP_DATA_TYPE_UINT32, h->db, W, h->rows, W * 4, kChorM4TileWords,
                           kChorM4BandRows, CU_TENSOR_MAP_SWIZZLE_NONE))
                return QPADL_ECUDA;
            QPADL_CU(launch_chor_m4rm(db_map, h->qt, h->rows, static_cast<uint32_t>(W), Bc,
                                      out_dev + (uint64_t)b0 * W, h->num_sms, h->d_status, s));
            continue;
        }
        uint32_t tw = 0, rb = 0, boxw = 0, qtw = 0;
        // by batch size (measured on the 1 GiB database): the mask form up to 8 queries, the
        // predicated XOR with 4 words per thread up to 16, with 8 words per thread above
        const int form = h->scan_form >= 0 ? h->scan_form : (Bc <= 8 ? 0 : (Bc <= 16 ? 1 : 3));
        if (!chor_launch_shape(Bc, form, &tw, &rb, &boxw, &qtw)) return QPADL_EINVAL;
        QPADL_CU(launch_chor_transpose(Q_dev + (uint64_t)b0 * h->qw, h->qw, Bc, h->rows, qtw, h->qt, h->num_sms, s));
        CUtensorMap db_map, qt_map;
        if (!encode_2d(&db_map, CU_TENSOR_MAP_DATA_TYPE_UINT32, h->db, W, h->rows, W * 4, boxw, rb,
                       CU_TENSOR_MAP_SWIZZLE_NONE) ||
            !encode_2d(&qt_map, CU_TENSOR_MAP_DATA_TYPE_UINT32, h->qt, qtw, h->rows, 4ull * qtw, qtw, rb,
                       CU_TENSOR_MAP_SWIZZLE_NONE))
            return QPADL_ECUDA;
        QPADL_CU(launch_chor_answer(db_map, qt_map, h->rows, static_cast<uint32_t>(W), Bc, qtw,
                                    out_dev + (uint64_t)b0 * W, h->num_sms, h->d_status, s, form));
    }
    return QPADL_OK;
}

int qpadl_chor_set_option(qpadl_chor *h, int option, int64_t value) {
    if (!h) return QPADL_EINVAL;
    switch (option) {
        case QPADL_CHOR_OPT_M4RM_MIN_BATCH:
            if (value < 1 || value > (int64_t)kChorMaxBatch + 1) return QPADL_EINVAL;
            h->m4rm_min_batch = static_cast<uint32_t>(value);
            return QPADL_OK;
        case QPADL_CHOR_OPT_SCAN_FORM:
            if (value < -1 || value > 3) return QPADL_EINVAL;
            h->scan_form = static_cast<int>(value);
            return QPADL_OK;
        default: return QPADL_EINVAL;
    }
}

int qpadl_chor_get_option(qpadl_chor *h, int option, int64_t *value) {
    if (!h || !value) return QPADL_EINVAL;
    switch (option) {
        case QPADL_CHOR_OPT_M4RM_MIN_BATCH: *value = h->m4rm_min_batch; return QPADL_OK;
        case QPADL_CHOR_OPT_SCAN_FORM: *value = h->scan_form; return QPADL_OK;
        default: return QPADL_EINVAL;
    }
}

int qpadl_chor_status(qpadl_chor *h) {
    if (!h) return QPADL_EINVAL;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return QPADL_ECUDA;
    if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess) return QPADL_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return QPADL_ECUDA;
    int st = 0;
    if (cudaMemcpy(&st, h->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return QPADL_ECUDA;
    if (st != 0) {
        const int zero = 0;
        cudaMemcpy(h->d_status, &zero, 4, cudaMemcpyHostToDevice);
        return QPADL_ETIMEOUT;
    }
    return QPADL_OK;
}

// ------------------------------------------------------------------ Goldberg-style Z_p Response

int qpadl_goldberg_destroy(qpadl_goldberg *h) {
    if (!h) return QPADL_OK;
    qpadl_pir_destroy(h->db);
    delete h;
    return QPADL_OK;
}

int qpadl_goldberg_setup(uint64_t rows, uint64_t cols, uint32_t p, const uint8_t *db_dev, qpadl_stream_t stream,
                         qpadl_goldberg **out) {
    if (!out) return QPADL_EINVAL;
    *out = nullptr;
    if (!db_dev || p < 2 || p > 257 || cols == 0 || cols > kGoldbergMaxCols) return QPADL_EINVAL;
    for (uint32_t d = 2; d * d <= p; ++d)
        if (p % d == 0) return QPADL_EINVAL;   // the field needs a prime modulus
    qpadl_goldberg *h = new (std::nothrow) qpadl_goldberg();
    if (!h) return QPADL_ENOMEM;
    h->p = p;
    // the lattice handle of the same bytes; its scheme parameters (n, modulus) are not used here
    qpadl_params prm{rows, cols, 1, 32, 256, 0, 0.0, 1};
    int rc = qpadl_pir_setup(&prm, db_dev, stream, &h->db);
    if (rc != QPADL_OK) {
        delete h;
        return rc;
    }
    if (p < 256) {   // every byte must be a field element
        qpadl_db *db = h->db;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        int mx = 0;
        max_digit_kernel<<<db->num_sms * 4, 256, 0, s>>>(db_dev, rows * cols, db->d_status + 1);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&mx, db->d_status + 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            qpadl_goldberg_destroy(h);
            return QPADL_ECUDA;
        }
        if (mx >= static_cast<int>(p)) {
            qpadl_goldberg_destroy(h);
            return QPADL_EINVAL;
        }
    }
    *out = h;
    return QPADL_OK;
}

int qpadl_goldberg_answer_batch(qpadl_goldberg *h, const uint32_t *Q_dev, uint32_t B, uint32_t *out_dev,
                                qpadl_stream_t stream) {
    if (!h || !Q_dev || !out_dev || B == 0) return QPADL_EINVAL;
    qpadl_db *db = h->db;
    if (set_device(db) != QPADL_OK) return QPADL_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t R = db->prm.rows, C = db->prm.cols;
    if (B < h->gemm_min_batch) {
        // exact integer sums (no wrap below kGoldbergMaxCols columns), then mod p
        int rc = answer_streaming(db, Q_dev, B, out_dev, s);
        if (rc != QPADL_OK) return rc;
        QPADL_CU(launch_mod_p(out_dev, (uint64_t)B * R, h->p, db->num_sms, s));
        return QPADL_OK;
    }
    if (B <= h->u8_max_batch && db->u8_ok) {
        // the uint8-digit GEMM with one centred row per query gives the exact signed sums
        // (below 2^31 in magnitude for at most kGoldbergMaxCols columns), then mod p; above 64
        // queries a row tile takes several 64-wide tiles (one read of the digits, converted once
        // per tile), which beats the fp16 copy's one-limb GEMM up to about 128-192 queries
        int rc = ensure_blocked(db, s);
        if (rc != QPADL_OK) return rc;
        if ((rc = ensure_limbs(db, 2ull * B * db->pitch)) != QPADL_OK) return rc;
        // one launch makes the rows and zeroes the sums; the GEMM overlaps its start with it
        QPADL_CU(launch_centred_rows(Q_dev, B, C, h->p, db->limbs, db->pitch, db->num_sms, s, out_dev,
                                     (uint64_t)B * R));
        const int bn = B <= 32 ? 32 : 64;
        constexpr int ks = 128;
        const bool pair = db->pair_gemm && db->num_sms >= 2;
        const uint32_t tile_rows = pair ? 2 * kLimbBoxM : kLimbBoxM;
        GroupedGemmArgs args;
        std::memset(&args, 0, sizeof(args));
        args.a[0] = db->u8_map[ks / 128 - 1];
        if (!encode_2d(&args.b[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, db->limbs, C, B, db->pitch * 2, kLimbBoxK,
                       static_cast<uint32_t>(pair ? bn / 2 : bn), CU_TENSOR_MAP_SWIZZLE_128B))
            return QPADL_ECUDA;
        GroupDesc &g = args.g[0];
        g.out = out_dev;
        g.ld_m = 1;
        g.ld_b = R;
        g.M = static_cast<uint32_t>(R);
        g.NV = B;
        g.KB = static_cast<uint32_t>((C + ks - 1) / ks);
        g.unit_begin = 0;
        g.n_tiles = (B + bn - 1) / bn;
        args.ngroups = 1;
        args.total_units = static_cast<uint32_t>((R + tile_rows - 1) / tile_rows) * g.n_tiles * g.KB;
        // tiles split between CTAs are accumulated with atomic adds into the zeros
        QPADL_CU(launch_limb_gemm_u8_rows(bn, args, db->num_sms, db->d_status, s, pair, true));
        QPADL_CU(launch_mod_p_signed(out_dev, (uint64_t)B * R, h->p, db->num_sms, s));
        return QPADL_OK;
    }
    int rc = ensure_tensor_copy(db, s);
    if (rc != QPADL_OK) return rc;
    // one centred fp16 row per query, in chunks that the limb scratch holds
    constexpr uint32_t kChunk = 1024;
    if ((rc = ensure_limbs(db, 2ull * std::min(B, kChunk) * db->pitch)) != QPADL_OK) return rc;
    for (uint32_t b0 = 0; b0 < B; b0 += kChunk) {
        const uint32_t Bc = std::min(B - b0, kChunk);
        QPADL_CU(launch_centred_rows(Q_dev + (uint64_t)b0 * C, Bc, C, h->p, db->limbs, db->pitch, db->num_sms, s));
        // up to 64 queries: running sums in registers; more: 256-wide tiles with the sums in TMEM
        const int bn = Bc <= 32 ? 32 : (Bc <= 64 ? 64 : 256);
        const ModPEpi epi{out_dev + (uint64_t)b0 * R, 1, R, static_cast<int32_t>(h->p)};
        if (bn == 256 && db->pair_gemm && db->num_sms >= 2) {
            // 256-row tiles over pairs of SMs, each SM loading half of every vector tile
            PairBMaps bm;
            std::memset(&bm, 0, sizeof(bm));
            if (!encode_2d(&bm.m[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, db->limbs, C, Bc, db->pitch * 2, kLimbBoxK,
                           pair_b_box_rows(256, false, 0), CU_TENSOR_MAP_SWIZZLE_128B))
                return QPADL_ECUDA;
            QPADL_CU(launch_limb_gemm_pair_modp(db->a_map, bm, epi, static_cast<uint32_t>(R), Bc, C, db->num_sms,
                                                db->d_status, s));
            continue;
        }
        CUtensorMap b_map;
        if (!encode_2d(&b_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, db->limbs, C, Bc, db->pitch * 2, kLimbBoxK,
                       static_cast<uint32_t>(bn), CU_TENSOR_MAP_SWIZZLE_128B))
            return QPADL_ECUDA;
        QPADL_CU(launch_limb_gemm_modp(bn, db->a_map, b_map, epi, static_cast<uint32_t>(R), Bc, C, db->num_sms,
                                       db->d_status, s));
    }
    return QPADL_OK;
}

int qpadl_goldberg_set_option(qpadl_goldberg *h, int option, int64_t value) {
    if (!h) return QPADL_EINVAL;
    switch (option) {
        case QPADL_GOLDBERG_OPT_GEMM_MIN_BATCH:
            if (value < 1 || value > (int64_t)UINT32_MAX) return QPADL_EINVAL;
            h->gemm_min_batch = static_cast<uint32_t>(value);
            return QPADL_OK;
        case QPADL_GOLDBERG_OPT_U8_MAX_BATCH:
            if (value < 0 || value > 256) return QPADL_EINVAL;
            h->u8_max_batch = static_cast<uint32_t>(value);
            return QPADL_OK;
        case QPADL_GOLDBERG_OPT_PAIR_GEMM:
            return qpadl_pir_set_option(h->db, QPADL_OPT_PAIR_GEMM, value);
        default: return QPADL_EINVAL;
    }
}

int qpadl_goldberg_status(qpadl_goldberg *h) { return h ? qpadl_pir_status(h->db) : QPADL_EINVAL; }

}  // extern "C"
