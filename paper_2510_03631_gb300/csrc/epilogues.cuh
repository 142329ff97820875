// Output epilogues of the client steps and of the limb GEMM.  Each is called
// once per output element with (row of the matrix operand, vector index,
// the mod-2^32 dot product of that row with that vector).  pre() gathers
// what the element needs from memory and put() finishes it, so a caller
// with many elements per thread can issue all their loads before any store
// (a store through one pointer could otherwise alias the next load, which
// serialises every element behind a full memory round trip).  prefetch()
// pulls what the epilogue of one output tile will read into L2 ahead of it
// (rows i0 .. i0+127 of vectors b0 .. b0+nb-1).

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
#pragma once
#include <cstdint>

namespace qpadl {

// kLimbs: limb rows per vector in the GEMM's vector operand (4 byte limbs
// recombined as sum_k 2^{8k} s_k; 1 = each row is its own vector).

// Plain store: out[i * ld_m + b * ld_b] = dot.
struct StoreEpi {
    static constexpr int kLimbs = 4;
    uint32_t *out;
    uint64_t ld_m, ld_b;
    __device__ __forceinline__ void prefetch(uint64_t, uint32_t, uint32_t) const {}
    __device__ __forceinline__ uint32_t pre(uint64_t, uint32_t) const { return 0u; }
    __device__ __forceinline__ void put(uint64_t i, uint32_t b, uint32_t dot, uint32_t) const {
        out[i * ld_m + (uint64_t)b * ld_b] = dot;
    }
    __device__ __forceinline__ void operator()(uint64_t i, uint32_t b, uint32_t dot) const { put(i, b, dot, 0u); }
    // one CTA's part of the element (split tiles; the output starts at zero)
    __device__ __forceinline__ void add(uint64_t i, uint32_t b, uint32_t part) const {
        atomicAdd(out + i * ld_m + (uint64_t)b * ld_b, part);
    }
};

// Query (Def. 1 Client.Query): q_b[j] = (A s_b)[j] + e_b[j] + Delta [j == col_b]  mod 2^32.
struct QueryEpi {
    static constexpr int kLimbs = 4;
    const int32_t *e;        // noise, row b at e + b * e_ld
    uint64_t e_ld;
    const uint32_t *cols;    // target column per vector (device) or nullptr
    uint64_t col;            // target column when cols == nullptr
    uint32_t delta;
    uint32_t *q;             // output, vector b at q + b * q_ld
    uint64_t q_ld;
    __device__ __forceinline__ void prefetch(uint64_t j0, uint32_t b0, uint32_t nb) const {
        for (uint32_t b = b0; b < b0 + nb; ++b)
            for (uint32_t l = 0; l < 4; ++l) prefetch_l2(e + b * e_ld + j0 + 32u * l);   // 128 rows x 4 B
    }
    // e_b[j] + Delta [j == col_b]
    __device__ __forceinline__ uint32_t pre(uint64_t j, uint32_t b) const {
        const uint64_t target = cols ? cols[b] : col;
        return static_cast<uint32_t>(e[b * e_ld + j]) + (j == target ? delta : 0u);
    }
    __device__ __forceinline__ void put(uint64_t j, uint32_t b, uint32_t dot, uint32_t pre_v) const {
        q[b * q_ld + j] = dot + pre_v;
    }
    __device__ __forceinline__ void operator()(uint64_t j, uint32_t b, uint32_t dot) const {
        put(j, b, dot, pre(j, b));
    }
};

// Query without its unit vector: q_b[j] = (A s_b)[j] + e_b[j] mod 2^32.  Delta at the target
// column (one element per vector) is added afterwards by launch_add_delta, so an element's
// epilogue depends on no other load (a compare against a loaded target column would hold up
// every load behind it).
struct QueryNoiseEpi {
    static constexpr int kLimbs = 4;
    const int32_t *e;        // noise, row b at e + b * e_ld
    uint64_t e_ld;
    uint32_t *q;             // output, vector b at q + b * q_ld
    uint64_t q_ld;
    __device__ __forceinline__ void prefetch(uint64_t j0, uint32_t b0, uint32_t nb) const {
        for (uint32_t b = b0; b < b0 + nb; ++b)
            for (uint32_t l = 0; l < 4; ++l) prefetch_l2(e + b * e_ld + j0 + 32u * l);   // 128 rows x 4 B
    }
    __device__ __forceinline__ uint32_t pre(uint64_t j, uint32_t b) const {
        return static_cast<uint32_t>(e[b * e_ld + j]);
    }
    __device__ __forceinline__ void put(uint64_t j, uint32_t b, uint32_t dot, uint32_t pre_v) const {
        q[b * q_ld + j] = dot + pre_v;
    }
    __device__ __forceinline__ void operator()(uint64_t j, uint32_t b, uint32_t dot) const {
        put(j, b, dot, pre(j, b));
    }
};

// Recover (Def. 1 Client.BlockReconst): d_b[i] = round((ans_b[i] - (H s_b)[i]) / Delta) mod p,
// as (x + Delta/2) >> (32 - log2 p) in uint32 arithmetic.
struct RecoverEpi {
    static constexpr int kLimbs = 4;
    const uint32_t *ans;     // answer b at ans + b * ans_ld
    uint64_t ans_ld;
    uint32_t shift;          // 32 - log2 p
    uint8_t *out;            // digits of vector b at out + b * out_ld
    uint64_t out_ld;
    __device__ __forceinline__ void prefetch(uint64_t i0, uint32_t b0, uint32_t nb) const {
        for (uint32_t b = b0; b < b0 + nb; ++b)
            for (uint32_t l = 0; l < 4; ++l) prefetch_l2(ans + b * ans_ld + i0 + 32u * l);
    }
    // ans_b[i]
    __device__ __forceinline__ uint32_t pre(uint64_t i, uint32_t b) const { return ans[b * ans_ld + i]; }
    __device__ __forceinline__ void put(uint64_t i, uint32_t b, uint32_t dot, uint32_t a) const {
        const uint32_t x = a - dot;
        out[b * out_ld + i] = static_cast<uint8_t>((x + (1u << (shift - 1))) >> shift);
    }
    __device__ __forceinline__ void operator()(uint64_t i, uint32_t b, uint32_t dot) const {
        put(i, b, dot, pre(i, b));
    }
};

// Goldberg Response over Z_p (Sec. 5.2, Alg. 4): the vector operand holds
// each query once, centred into [-128, 128], so dot is the exact signed
// integer sum (|sum| < 2^31 for fewer than 65793 columns); out = dot mod p.
struct ModPEpi {
    static constexpr int kLimbs = 1;
    uint32_t *out;
    uint64_t ld_m, ld_b;
    int32_t p;
    __device__ __forceinline__ void prefetch(uint64_t, uint32_t, uint32_t) const {}
    __device__ __forceinline__ uint32_t pre(uint64_t, uint32_t) const { return 0u; }
    __device__ __forceinline__ void put(uint64_t i, uint32_t b, uint32_t dot, uint32_t) const {
        int32_t r = static_cast<int32_t>(dot) % p;
        if (r < 0) r += p;
        out[i * ld_m + (uint64_t)b * ld_b] = static_cast<uint32_t>(r);
    }
    // a residue already in [0, p)
    __device__ __forceinline__ void store(uint64_t i, uint32_t b, uint32_t r) const {
        out[i * ld_m + (uint64_t)b * ld_b] = r;
    }
    __device__ __forceinline__ void operator()(uint64_t i, uint32_t b, uint32_t dot) const { put(i, b, dot, 0u); }
};

}  // namespace qpadl
