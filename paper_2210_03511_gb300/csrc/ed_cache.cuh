// Stored-structure H.x: the arguments of one column segment's pass and what
// the pass kernels (ed_cache.cu: one lane per row, any number of vectors;
// ed_cache_lanes.cu: several lanes per row, one vector) share.
#pragma once

#include "ed_apply_impl.cuh"

namespace ed {

constexpr int NCODE = 256;  // coefficient codes at most (one byte)

// Arguments of one segment's pass of the stored-structure H.x.
struct CachePass {
    const uint8_t* counts;   // [Dpad] entries per row in this segment
    const uint32_t* boff;    // [ns] first entry of each slice, relative to `ent`
    const uint32_t* ent;     // this segment's entries
    const void* x;           // [nvec][D]
    void* y;                 // [nvec][D]
    const void* ctab;        // [256] coefficients of the value kind (R, or T for complex kinds)
    const void* isq;         // [G+1] 1/sqrt(k) of the value kind's real type
    const uint16_t* stab;    // [D] |Stab sigma_i|
    const double* diag;      // [D] Ising part
    int64_t D, ns, xoff;     // xoff: first column of the segment
    int nvec, mode;
    uint32_t off_bits;       // entry = (code << off_bits) | column offset
    uint32_t n_re;           // codes below n_re have real coefficients (complex kinds)
};

// Resident blocks per SM of a pass launch: 32 registers a thread for one
// vector (complex FP64 takes 40 to keep its accumulators out of local memory).
constexpr int pass_blocks(int K, int NV) { return NV == 1 ? (K == 2 ? 6 : 8) : 2; }

// Exclusive prefix sum over the warp.
static __device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, int lane) {
    uint32_t s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += u;
    }
    return s - v;
}

// One vector's pass with `lanes` (2, 4 or 8) consecutive lanes per row
// (p.ctab: the general coefficient table of the kind).
ed_status launch_pass_lanes(const CachePass& p, int K, int lanes, int sms, cudaStream_t s);

}  // namespace ed
