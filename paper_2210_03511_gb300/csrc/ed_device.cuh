// Device helpers shared by the basis builder and the H.x kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ed_internal.h"

namespace ed {

// View of the sublattice-coding tables after they were staged (to shared or
// global memory).  SAT is the element type of SymmetryAction (uint8_t for
// blocks of <= 8 sites, uint16_t otherwise).
template <typename SAT>
struct TabView {
    const uint16_t* rep;
    const uint32_t* sym_off;
    const uint16_t* sym_ids;
    const SAT* sa;
    const uint8_t* src;
    const double2* chi;
    const uint8_t* chi_one;
    const double* sqrtn;     // sqrtn[k] = sqrt(k), k = 0..G
    const double* isqrtn;    // 1/sqrt(k)
    const float2* chif;
    const float* sqrtnf;
    const float* isqrtnf;
    int n_sub, m, G;
};

template <typename SAT>
__device__ __forceinline__ TabView<SAT> tab_view(const uint8_t* base, const DevTables& d) {
    TabView<SAT> v;
    v.rep = (const uint16_t*)(base + d.off_rep);
    v.sym_off = (const uint32_t*)(base + d.off_symoff);
    v.sym_ids = (const uint16_t*)(base + d.off_symids);
    v.sa = (const SAT*)(base + d.off_sa);
    v.src = (const uint8_t*)(base + d.off_src);
    v.chi = (const double2*)(base + d.off_chi);
    v.chi_one = (const uint8_t*)(base + d.off_chione);
    v.sqrtn = (const double*)(base + d.off_sqrt);
    v.isqrtn = v.sqrtn + (d.G + 1);
    v.chif = (const float2*)(base + d.off_chif);
    v.sqrtnf = (const float*)(base + d.off_sqrtf);
    v.isqrtnf = v.sqrtnf + (d.G + 1);
    v.n_sub = d.n_sub;
    v.m = d.m;
    v.G = d.G;
    return v;
}

// Cooperative copy of the table image into shared memory (16-byte chunks).
__device__ __forceinline__ void stage_blob(uint8_t* dst, const uint8_t* src, size_t bytes) {
    const uint4* s4 = (const uint4*)src;
    uint4* d4 = (uint4*)dst;
    const size_t n4 = bytes / 16;
    for (size_t i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = s4[i];
}

template <typename W>
__device__ __forceinline__ uint32_t substate(W s, int X, int n_sub, int m) {
    return (uint32_t)((s >> ((n_sub - 1 - X) * m)) & (((W)1 << m) - 1));
}

// Alg. "Sublattice coding algorithm for finding the representative":
// MinRep = min_X Rep_X(sigma_X); for every block Y with Rep_Y = MinRep and
// every g in Sym_Y(sigma_Y), compose g.sigma block by block from the most
// significant destination block (block Z comes from block src(g,Z) via
// SymmetryAction) and keep the smallest.  Also returns the number of
// minimising elements, which equals |Stab(rep)|, and whether chi is 1 on all
// of them (the representative's projector is non-zero iff chi is trivial on
// the stabilizer).
template <typename W, typename SAT>
__device__ __forceinline__ void find_rep(W s, const TabView<SAT>& t, W& rep, int& gbest, int& nstab, bool& compat) {
    const int n_sub = t.n_sub, m = t.m;
    const int S = 1 << m;
    uint32_t minrep = 0xFFFFFFFFu;
    for (int X = 0; X < n_sub; ++X) {
        uint32_t r = t.rep[X * S + substate(s, X, n_sub, m)];
        minrep = r < minrep ? r : minrep;
    }
    W best = ~(W)0;
    int gb = 0, ns = 0;
    bool cp = true;
    for (int Y = 0; Y < n_sub; ++Y) {
        const uint32_t sy = substate(s, Y, n_sub, m);
        if (t.rep[Y * S + sy] != minrep) continue;
        const uint32_t q0 = t.sym_off[Y * (S + 1) + sy], q1 = t.sym_off[Y * (S + 1) + sy + 1];
        for (uint32_t q = q0; q < q1; ++q) {
            const int g = t.sym_ids[q];
            const uint8_t* srcg = t.src + g * n_sub;
            const SAT* sag = t.sa + (size_t)g * n_sub * S;
            W img = (W)minrep;
            int Z = 1;
            int cmp = 0;  // sign of (img prefix - best prefix) once decided
            for (; Z < n_sub; ++Z) {
                const int X = srcg[Z];
                img = (img << m) | (W)sag[X * S + substate(s, X, n_sub, m)];
                if (cmp == 0) {
                    const W bp = best >> ((n_sub - 1 - Z) * m);
                    if (img > bp) { cmp = 1; break; }
                    if (img < bp) cmp = -1;
                }
            }
            if (cmp > 0) continue;
            if (img < best) {
                best = img; gb = g; ns = 1; cp = t.chi_one[g];
            } else if (img == best) {
                ++ns;
                cp = cp && t.chi_one[g];
            }
        }
    }
    rep = best;
    gbest = gb;
    nstab = ns;
    compat = cp;
}

// Is s its own representative?  Early exit as soon as some g.s < s.
// On success returns |Stab(s)| in nstab and whether chi is trivial on it.
template <typename W, typename SAT>
__device__ __forceinline__ bool is_rep(W s, const TabView<SAT>& t, int& nstab, bool& compat) {
    const int n_sub = t.n_sub, m = t.m;
    const int S = 1 << m;
    const uint32_t top = substate(s, 0, n_sub, m);
    uint32_t minrep = 0xFFFFFFFFu;
    for (int X = 0; X < n_sub; ++X) {
        uint32_t r = t.rep[X * S + substate(s, X, n_sub, m)];
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
            const uint8_t* srcg = t.src + g * n_sub;
            const SAT* sag = t.sa + (size_t)g * n_sub * S;
            int cmp = 0;
            for (int Z = 1; Z < n_sub; ++Z) {
                const int X = srcg[Z];
                const uint32_t v = sag[X * S + substate(s, X, n_sub, m)];
                const uint32_t sz = substate(s, Z, n_sub, m);
                if (v < sz) return false;
                if (v > sz) { cmp = 1; break; }
            }
            if (cmp == 0) {
                ++ns;
                cp = cp && t.chi_one[g];
            }
        }
    }
    nstab = ns;
    compat = cp;
    return true;
}

// Index of representative r (section "Distributed and hybrid memory
// parallelization": Basis + Limits, then binary search).  Limits is two-level:
// the top sublattice block value v selects a directory entry (base_v, q_v),
// the next q_v bits select a bucket [limits[key], limits[key+1]) of the
// ascending basis.  Returns -1 if r is absent.
template <typename W>
__device__ __forceinline__ int64_t find_index(W r, const W* __restrict__ reps, const uint32_t* __restrict__ dir_base,
                                              const uint8_t* __restrict__ dir_q, const uint32_t* __restrict__ limits,
                                              int L) {
    const uint32_t top = (uint32_t)(r >> L);
    const int q = dir_q[top];
    const W low = L ? (r & (((W)1 << L) - 1)) : (W)0;
    const uint32_t key = dir_base[top] + (q ? (uint32_t)(low >> (L - q)) : 0u);
    uint32_t lo = __ldg(limits + key), hi = __ldg(limits + key + 1);
    const uint32_t end = hi;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(reps + mid) < r) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && __ldg(reps + lo) == r) ? (int64_t)lo : -1;
}

}  // namespace ed
