// Device helpers shared by the basis builder and the H.x kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ed_internal.h"

// Helpers are __host__ __device__ so the exact device logic can also run on the
// CPU (table-image self-checks and host-side tests).
#define ED_HD __host__ __device__ __forceinline__

namespace ed {

ED_HD int ctz32(uint32_t v) {
#ifdef __CUDA_ARCH__
    return __ffs((int)v) - 1;
#else
    return __builtin_ctz(v);
#endif
}

template <typename T>
ED_HD T ld_ro(const T* p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// View of the sublattice-coding tables after they were staged into shared
// memory.  CHUNKED selects the SymmetryAction map format: false = one byte
// table of 2^m entries per distinct local map (m <= 8); true = two uint16
// chunk tables (high m-c bits, low c bits) whose images are OR-ed.
template <bool CHUNKED>
struct TabView {
    const uint16_t* rep;      // [n_sub][S]      Rep_X(s)
    const uint32_t* sym_off;  // [n_sub][S+1]    Sym_X(s) ranges
    const uint16_t* sym_ids;  //                 group ids
    const uint32_t* srclid;   // [G][n_sub]      (src block, local map id) for destination block Z
    const void* lmap;         // map tables
    const double2* chi;
    const uint16_t* chi_cls;  // character class id; 0 is the class of the value 1
    const double* sqrtn;      // sqrtn[k] = sqrt(k), k = 0..G
    const double* isqrtn;     // 1/sqrt(k)
    const float2* chif;
    const float* sqrtnf;
    const float* isqrtnf;
    const uint16_t* dl;       // [G][dl_stride] (dest block << 12) | map id, by source block
    const uint8_t* chi_neg;   // [G] real chi(g) < 0
    int n_sub, m, G, c_lo, stride, dl_stride;
};

template <bool CHUNKED>
ED_HD TabView<CHUNKED> tab_view(const uint8_t* base, const DevTables& d) {
    TabView<CHUNKED> v;
    v.rep = (const uint16_t*)(base + d.off_rep);
    v.sym_off = (const uint32_t*)(base + d.off_symoff);
    v.sym_ids = (const uint16_t*)(base + d.off_symids);
    v.srclid = (const uint32_t*)(base + d.off_src);
    v.lmap = (const void*)(base + d.off_sa);
    v.chi = (const double2*)(base + d.off_chi);
    v.chi_cls = (const uint16_t*)(base + d.off_chicls);
    v.sqrtn = (const double*)(base + d.off_sqrt);
    v.isqrtn = v.sqrtn + (d.G + 1);
    v.chif = (const float2*)(base + d.off_chif);
    v.sqrtnf = (const float*)(base + d.off_sqrtf);
    v.isqrtnf = v.sqrtnf + (d.G + 1);
    v.n_sub = d.n_sub;
    v.m = d.m;
    v.G = d.G;
    v.c_lo = d.chunk_lo;
    v.stride = d.lmap_stride;
    v.dl = (const uint16_t*)(base + d.off_dl);
    v.chi_neg = (const uint8_t*)(base + d.off_chineg);
    v.dl_stride = d.dl_stride;
    return v;
}

// Table images up to this size are staged whole into shared memory by the
// basis and representative kernels; larger images (blocks of up to 16 sites)
// are read from global memory, where they stay L2-resident.
constexpr size_t kStageWholeLimit = 200 * 1024;

// Table sections an H.x block may stage into shared memory (the others are
// read from the global image): the packed entries and chi sign bits, the
// character tables of the vector kind, the (source, map) table of the
// generic search, the local block maps, Rep, Sym offsets and lists.
enum : uint32_t { SEC_DL = 1u, SEC_CHI = 2u, SEC_SRC = 4u, SEC_MAPS = 8u, SEC_REP = 16u, SEC_SYM = 32u };

ED_HD uint32_t sec_bytes(const DevTables& d, uint32_t sec, int K) {
    switch (sec) {
        case SEC_DL: return (uint32_t)d.blob_bytes - d.off_dl;  // dl, chi_neg
        case SEC_CHI: {
            uint32_t n = d.off_sqrt - d.off_chicls;  // chi_cls
            if (K == 2) n += (d.off_chicls - d.off_chi) + (d.off_chif - d.off_sqrt);
            if (K == 1 || K == 3) n += (d.off_sqrtf - d.off_chif) + (d.off_dl - d.off_sqrtf);
            return n;
        }
        case SEC_SRC: return d.off_chi - d.off_src;
        case SEC_MAPS: return d.off_src - d.off_sa;
        case SEC_REP: return d.off_symoff - d.off_rep;
        case SEC_SYM: return d.off_sa - d.off_symoff;  // sym_off, sym_ids
    }
    return 0;
}

// Cooperative copy of a table image into shared memory (16-byte chunks).
__device__ __forceinline__ void stage_blob(uint8_t* dst, const uint8_t* src, size_t bytes) {
    const uint4* s4 = (const uint4*)src;
    uint4* d4 = (uint4*)dst;
    const size_t n4 = bytes / 16;
    for (size_t i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = s4[i];
}

// Stage the sections of `mask` into shared memory; the returned view points
// there for them and into the global image for the rest.  Every section
// starts and ends on a 16-byte boundary of the image.
template <bool CHUNKED>
__device__ __forceinline__ TabView<CHUNKED> stage_sections(const DevTables& d, uint8_t* smem, int K, uint32_t mask) {
    TabView<CHUNKED> t = tab_view<CHUNKED>(d.blob, d);
    size_t pos = 0;
    auto put = [&](uint32_t off, uint32_t end) -> const uint8_t* {
        stage_blob(smem + pos, d.blob + off, end - off);
        const uint8_t* p = smem + pos;
        pos += end - off;
        return p;
    };
    if (mask & SEC_DL) {
        const uint8_t* e = put(d.off_dl, (uint32_t)d.blob_bytes);
        t.dl = (const uint16_t*)e;
        t.chi_neg = e + (d.off_chineg - d.off_dl);
    }
    if (mask & SEC_CHI) {
        t.chi_cls = (const uint16_t*)put(d.off_chicls, d.off_sqrt);
        if (K == 2) {
            t.chi = (const double2*)put(d.off_chi, d.off_chicls);
            t.sqrtn = (const double*)put(d.off_sqrt, d.off_chif);
            t.isqrtn = t.sqrtn + (d.G + 1);
        }
        if (K == 1 || K == 3) {
            t.chif = (const float2*)put(d.off_chif, d.off_sqrtf);
            t.sqrtnf = (const float*)put(d.off_sqrtf, d.off_dl);
            t.isqrtnf = t.sqrtnf + (d.G + 1);
        }
    }
    if (mask & SEC_SRC) t.srclid = (const uint32_t*)put(d.off_src, d.off_chi);
    if (mask & SEC_MAPS) t.lmap = (const void*)put(d.off_sa, d.off_src);
    if (mask & SEC_REP) t.rep = (const uint16_t*)put(d.off_rep, d.off_symoff);
    if (mask & SEC_SYM) {
        const uint8_t* b = put(d.off_symoff, d.off_sa);
        t.sym_off = (const uint32_t*)b;
        t.sym_ids = (const uint16_t*)(b + (d.off_symids - d.off_symoff));
    }
    return t;
}

// Whole image in shared memory when it fits kStageWholeLimit, else the
// global image.  All threads of the block must call it (it synchronises).
template <bool CHUNKED>
__device__ __forceinline__ TabView<CHUNKED> stage_whole_or_global(const DevTables& d, uint8_t* smem) {
    const bool staged = d.blob_bytes <= kStageWholeLimit;
    if (staged) stage_blob(smem, d.blob, d.blob_bytes);
    __syncthreads();
    return tab_view<CHUNKED>(staged ? smem : d.blob, d);
}

ED_HD size_t whole_stage_bytes(const DevTables& d) {
    return d.blob_bytes <= kStageWholeLimit ? d.blob_bytes : 0;
}

template <typename W>
ED_HD uint32_t substate(W s, int X, int n_sub, int m) {
    return (uint32_t)((s >> ((n_sub - 1 - X) * m)) & (((W)1 << m) - 1));
}

// SymmetryAction_X(g, s) through the local map `lid` (Eq. symactiondef).
template <bool CHUNKED>
ED_HD uint32_t sym_action(const TabView<CHUNKED>& t, uint32_t lid, uint32_t s) {
    if constexpr (!CHUNKED) {
        return ((const uint8_t*)t.lmap)[lid * t.stride + s];
    } else {
        const uint16_t* tab = (const uint16_t*)t.lmap + lid * t.stride;
        const int hi_n = t.stride - (1 << t.c_lo);
        return (uint32_t)tab[s >> t.c_lo] | (uint32_t)tab[hi_n + (s & ((1u << t.c_lo) - 1))];
    }
}

// Alg. "Sublattice coding algorithm for finding the representative":
// MinRep = min_X Rep_X(sigma_X); for every block Y with Rep_Y = MinRep and
// every g in Sym_Y(sigma_Y), compose g.sigma block by block from the most
// significant destination block (block Z comes from block src(g,Z) through
// SymmetryAction) and keep the smallest.
// Outputs: the representative, one minimising element g_tau, the number of
// minimising elements (the coset Stab(rep) g_tau, so its size is |Stab(rep)|),
// and whether the representative belongs to the sector: the projector of
// the representative is non-zero iff chi is trivial on Stab(rep), i.e. iff chi
// takes one value on the minimising coset.
template <typename W, bool CHUNKED>
ED_HD void find_rep(W s, const TabView<CHUNKED>& t, W& rep, int& gbest, int& nstab, bool& compat) {
    const int n_sub = t.n_sub, m = t.m;
    const int S = 1 << m;
    uint32_t minrep = 0xFFFFFFFFu;
    for (int X = 0; X < n_sub; ++X) {
        const uint32_t r = t.rep[X * S + substate(s, X, n_sub, m)];
        minrep = r < minrep ? r : minrep;
    }
    W best = ~(W)0;
    int gb = 0, ns = 0;
    bool cp = true;
    uint32_t cls = 0;
    for (int Y = 0; Y < n_sub; ++Y) {
        const uint32_t sy = substate(s, Y, n_sub, m);
        if (t.rep[Y * S + sy] != minrep) continue;
        const uint32_t q0 = t.sym_off[Y * (S + 1) + sy], q1 = t.sym_off[Y * (S + 1) + sy + 1];
        for (uint32_t q = q0; q < q1; ++q) {
            const int g = t.sym_ids[q];
            const uint32_t* sl = t.srclid + g * n_sub;
            W img = (W)minrep;
            int cmp = 0;  // sign of (img prefix - best prefix) once decided
            for (int Z = 1; Z < n_sub; ++Z) {
                const uint32_t e = sl[Z];
                img = (img << m) | (W)sym_action<CHUNKED>(t, e >> 8, substate(s, (int)(e & 0xFFu), n_sub, m));
                if (cmp == 0) {
                    const W bp = best >> ((n_sub - 1 - Z) * m);
                    if (img > bp) { cmp = 1; break; }
                    if (img < bp) cmp = -1;
                }
            }
            if (cmp > 0) continue;
            if (img < best) {
                best = img; gb = g; ns = 1; cls = t.chi_cls[g]; cp = true;
            } else if (img == best) {
                ++ns;
                cp = cp && (t.chi_cls[g] == cls);
            }
        }
    }
    rep = best;
    gbest = gb;
    nstab = ns;
    compat = cp;
}

// find_rep for a compile-time number of blocks NS (2..4).  Substates, block
// representatives and the best image so far (block by block) live in
// registers.  Each candidate g reads its packed (source block, map id)
// entries for all destination blocks with one 8-byte load and composes its
// image from the most significant destination block down, stopping at the
// first block that exceeds the best image (most candidates stop after one
// lookup).  Same outputs as find_rep.
template <typename W, bool CHUNKED, int NS>
ED_HD void find_rep_ns(W s, const TabView<CHUNKED>& t, W& rep, int& gbest, int& nstab, bool& compat) {
    static_assert(NS >= 2 && NS <= 4, "specialised for 2..4 blocks");
    const int m = t.m;
    const int S = 1 << m;
    uint32_t sub[NS], r[NS];
    uint32_t minrep = 0xFFFFFFFFu;
#pragma unroll
    for (int X = 0; X < NS; ++X) {
        sub[X] = substate(s, X, NS, m);
        r[X] = t.rep[X * S + sub[X]];
        minrep = r[X] < minrep ? r[X] : minrep;
    }
    uint32_t bestb[NS];
#pragma unroll
    for (int Z = 0; Z < NS; ++Z) bestb[Z] = 0xFFFFFFFFu;
    bestb[0] = minrep;
    bool have = false;
    int gb = 0, ns = 0;
    bool cp = true;
    uint32_t cls = 0;
    // One flat loop over the concatenated Sym_Y lists of all blocks Y with
    // Rep_Y = MinRep: a separate loop per Y would make a warp wait for the
    // longest list of every Y in turn.
    uint32_t ymask = 0;
#pragma unroll
    for (int Y = 0; Y < NS; ++Y) ymask |= (r[Y] == minrep ? 1u : 0u) << Y;
    uint32_t q = 0, q1 = 0;
    while (true) {
        if (q == q1) {
            if (!ymask) break;
            const int Y = ctz32(ymask);
            ymask &= ymask - 1;
            uint32_t sy = sub[0];
#pragma unroll
            for (int k = 1; k < NS; ++k) sy = (Y == k) ? sub[k] : sy;
            q = t.sym_off[Y * (S + 1) + sy];
            q1 = t.sym_off[Y * (S + 1) + sy + 1];
            continue;
        }
        const int g = t.sym_ids[q++];
        const uint2 pk = *(const uint2*)(t.dl + (size_t)g * 4);
        const uint32_t ent[4] = {pk.x & 0xFFFFu, pk.x >> 16, pk.y & 0xFFFFu, pk.y >> 16};
        uint32_t v[NS];
        v[0] = minrep;
        int state = have ? 0 : -1;  // 0: equal so far, -1: smaller, 1: larger
#pragma unroll
        for (int Z = 1; Z < NS; ++Z) {
            if (state == 1) break;
            const uint32_t X = ent[Z] >> 12;
            uint32_t sx = sub[0];
#pragma unroll
            for (int k = 1; k < NS; ++k) sx = (X == (uint32_t)k) ? sub[k] : sx;
            v[Z] = sym_action<CHUNKED>(t, ent[Z] & 0xFFFu, sx);
            if (state == 0) state = v[Z] > bestb[Z] ? 1 : (v[Z] < bestb[Z] ? -1 : 0);
        }
        if (state == 1) continue;
        if (state == -1) {
#pragma unroll
            for (int Z = 1; Z < NS; ++Z) bestb[Z] = v[Z];
            have = true;
            gb = g; ns = 1; cls = t.chi_cls[g]; cp = true;
        } else {
            ++ns;
            cp = cp && (t.chi_cls[g] == cls);
        }
    }
    W best = 0;
#pragma unroll
    for (int Z = 0; Z < NS; ++Z) best = (best << m) | (W)bestb[Z];
    rep = best;
    gbest = gb;
    nstab = ns;
    compat = cp;
}

// Is s its own representative?  Early exit as soon as some g.s < s.
// On success returns |Stab(s)| in nstab and whether chi is 1 on Stab(s).
template <typename W, bool CHUNKED>
ED_HD bool is_rep(W s, const TabView<CHUNKED>& t, int& nstab, bool& compat) {
    const int n_sub = t.n_sub, m = t.m;
    const int S = 1 << m;
    const uint32_t top = substate(s, 0, n_sub, m);
    uint32_t minrep = 0xFFFFFFFFu;
    for (int X = 0; X < n_sub; ++X) {
        const uint32_t r = t.rep[X * S + substate(s, X, n_sub, m)];
        if (r < top) return false;
        minrep = r < minrep ? r : minrep;
    }
    int ns = 0;
    bool cp = true;
    for (int Y = 0; Y < n_sub; ++Y) {
        const uint32_t sy = substate(s, Y, n_sub, m);
        if (t.rep[Y * S + sy] != minrep) continue;
        const uint32_t q0 = t.sym_off[Y * (S + 1) + sy], q1 = t.sym_off[Y * (S + 1) + sy + 1];
        for (uint32_t q = q0; q < q1; ++q) {
            const int g = t.sym_ids[q];
            const uint32_t* sl = t.srclid + g * n_sub;
            int cmp = 0;
            for (int Z = 1; Z < n_sub; ++Z) {
                const uint32_t e = sl[Z];
                const uint32_t v = sym_action<CHUNKED>(t, e >> 8, substate(s, (int)(e & 0xFFu), n_sub, m));
                const uint32_t sz = substate(s, Z, n_sub, m);
                if (v < sz) return false;
                if (v > sz) { cmp = 1; break; }
            }
            if (cmp == 0) {
                ++ns;
                cp = cp && (t.chi_cls[g] == 0);
            }
        }
    }
    nstab = ns;
    compat = cp;
    return true;
}

ED_HD int popc32(uint32_t v) {
#ifdef __CUDA_ARCH__
    return __popc(v);
#else
    return __builtin_popcount(v);
#endif
}

// 8-bit fingerprint of a state (top byte of a Fibonacci hash, so it depends
// on every bit).
template <typename W>
ED_HD uint32_t state_fp(W r) {
    return (uint32_t)(((uint64_t)r * 0x9E3779B97F4A7C15ull) >> 56);
}

// Index of representative r (section "Distributed and hybrid memory
// parallelization": Basis + Limits, then binary search).  Limits is two-level:
// the top sublattice block value v selects a directory entry (base_v, q_v),
// the next q_v bits select a bucket [limits[key].x, limits[key+1].x) of the
// ascending basis.  A bucket of at most 4 states also carries their 8-bit
// fingerprints: r is a compatible representative of this sector, so it is in
// its bucket, and a fingerprint that matches exactly one state of the bucket
// gives its position without reading the basis.  Otherwise (larger bucket, or
// a fingerprint shared within the bucket) binary search; -1 if r is absent.
template <typename W>
ED_HD int64_t find_index(W r, const W* __restrict__ reps, const uint32_t* __restrict__ dir_base,
                         const uint8_t* __restrict__ dir_q, const uint2* __restrict__ limits, int L) {
    const uint32_t top = (uint32_t)(r >> L);
    const int q = dir_q[top];
    const W low = L ? (r & (((W)1 << L) - 1)) : (W)0;
    const uint32_t key = dir_base[top] + (q ? (uint32_t)(low >> (L - q)) : 0u);
    const uint2 e = ld_ro(limits + key);
    uint32_t lo = e.x, hi = ld_ro((const uint32_t*)(limits + key + 1));
    const uint32_t n = hi - lo;
    if (n <= 4u) {
        // bytes of e.y equal to the fingerprint: 0x80 in each zero byte of x
        const uint32_t x = e.y ^ (state_fp(r) * 0x01010101u);
        uint32_t z = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
        z &= n == 4u ? 0xFFFFFFFFu : ((1u << (8u * n)) - 1u);
        if (popc32(z) == 1) return (int64_t)lo + (ctz32(z) >> 3);
    }
    const uint32_t end = hi;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (ld_ro(reps + mid) < r) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && ld_ro(reps + lo) == r) ? (int64_t)lo : -1;
}

}  // namespace ed
