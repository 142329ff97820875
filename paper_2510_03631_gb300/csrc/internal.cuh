// Library-internal access to a database handle for the serving loop
// (server.cu): building grouped launches from several handles with
// caller-provided workspace, without touching a handle's own scratch.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "limb_gemm_u8.cuh"
#include "qpadl_pir.h"

namespace qpadl {

// Row pitch (elements) of a limb operand for this database: roundup(C, 8).
uint64_t db_limb_pitch(const qpadl_db *db);
int db_num_sms(const qpadl_db *db);
int *db_status_word(qpadl_db *db);

// Builds the blocked digit copy and its tensor maps if missing (may allocate; call before serving).
int db_prepare_u8(qpadl_db *db, cudaStream_t stream);
// Builds the fp16 operand copy if missing (may allocate; call before serving).
int db_prepare_f16(qpadl_db *db, cudaStream_t stream);

// Fills group slot `g` of a grouped u8 GEMM for NV vectors whose fp16 limbs
// are at `limbs` (4 NV rows of db_limb_pitch elements); answers go to
// out[v * R + i].  `unit_begin` is the group's first unit; returns its unit count.
// pair: the group runs in the pair form of the GEMM (256-row tiles, half-height limb boxes).
int db_fill_u8_group(qpadl_db *db, GroupedGemmArgs &args, int g, const __half *limbs, uint32_t NV, uint32_t *out,
                     int bn, int ks, uint32_t unit_begin, uint32_t *units, bool pair);

// Whether this handle runs its batched GEMMs on CTA pairs (QPADL_OPT_PAIR_GEMM).
bool db_pair_gemm(const qpadl_db *db);

// Batched answer on the fp16 copy with the limbs in caller workspace (8 B pitch bytes).
int db_answer_f16_ws(qpadl_db *db, const uint32_t *Q, uint32_t B, uint32_t *ans, __half *limbs,
                     cudaStream_t stream);

// One query on the streaming kernel without any scratch (query packed in-kernel);
// falls back to the row-wise kernel for shapes the streaming kernel cannot take.
int db_answer_one_noscratch(qpadl_db *db, const uint32_t *q, uint32_t *ans, cudaStream_t stream);

// Two queries (q, q + q_ld) in one pass over the database without any scratch (both packed
// in-kernel); answers to ans and ans + ans_ld.  Falls back to the row-wise kernel likewise.
int db_answer_two_noscratch(qpadl_db *db, const uint32_t *q, uint64_t q_ld, uint32_t *ans, uint64_t ans_ld,
                            cudaStream_t stream);

}  // namespace qpadl
