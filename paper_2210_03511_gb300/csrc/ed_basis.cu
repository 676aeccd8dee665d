// Device basis construction (Alg. "Preparation of the distributed and
// symmetrized Hilbert space" on one GPU, with the representative test of
// Alg. "Sublattice coding algorithm for finding the representative").
//
// The candidate space is cut into segments by the value v of the most
// significant sublattice block: a representative's top block equals MinRep,
// so only values with Rep_0(v) = v can start a representative.  Inside a
// segment the remaining L = N - m bits run over all integers with popcount
// n_up - popcount(v) in increasing order, so the concatenation of segments in
// order of v is sorted.  Each thread owns a chunk of CANDS consecutive
// candidates: it unranks the first one (combinatorial number system) and
// steps with the next-same-popcount rule.  A first pass counts kept states per
// chunk, an exclusive scan gives output offsets, a second pass writes them.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "ed_device.cuh"
#include "ed_internal.h"
#include "ed_transfer.h"

namespace ed {

__constant__ uint64_t c_binom[65][65];

static const int CANDS = 128;  // candidates per thread

struct Seg {
    uint32_t v;         // top-block value
    int32_t k;          // ones in the remaining L bits
    uint64_t size;      // C(L, k)
    uint64_t chunk0;    // first chunk index
};

template <typename W>
__device__ __forceinline__ W unrank(uint64_t r, int L, int k) {
    W v = 0;
    for (int b = L - 1; b >= 0 && k > 0; --b) {
        const uint64_t c = c_binom[b][k];
        if (r >= c) {
            v |= (W)1 << b;
            r -= c;
            --k;
        }
    }
    return v;
}

template <typename W>
__device__ __forceinline__ W next_same_popcount(W v) {
    const W c = v & (~v + 1);
    const W r = v + c;
    const int tz = (sizeof(W) == 8) ? (__ffsll((long long)c) - 1) : (__ffs((int)c) - 1);
    return (((r ^ v) >> 2) >> tz) | r;
}

struct EnumArgs {
    DevTables dt;
    const Seg* segs;
    int n_segs;
    uint64_t n_chunks;
    int L;
    uint32_t* counts;          // pass 0 output
    const uint64_t* offsets;   // pass 1 input
    void* reps;                // pass 1 output (W)
    uint16_t* stab;            // pass 1 output
    // SU(N) bases: n_colors colours in col_bits bits per site over col_sites
    // sites; a candidate is kept only if every site holds a colour < n_colors
    // and colour c occurs col_want[c] times (0 sites: spin-1/2, no filter)
    int col_sites, col_bits, n_colors;
    uint64_t col_want[2];      // counts of colours 0..7 and 8..15, one byte each
};

// Every site's colour below n_colors and the colour counts as wanted.
template <typename W>
__device__ __forceinline__ bool colours_ok(W s, const EnumArgs& a) {
    const W mask = ((W)1 << a.col_bits) - 1;
    uint64_t got[2] = {0ull, 0ull};
    for (int k = 0; k < a.col_sites; ++k) {
        const uint32_t c = (uint32_t)((s >> (k * a.col_bits)) & mask);
        if (c >= (uint32_t)a.n_colors) return false;
        got[c >> 3] += 1ull << (8 * (c & 7));
    }
    return got[0] == a.col_want[0] && got[1] == a.col_want[1];
}

template <typename W, bool CHK, int PASS>
__global__ void __launch_bounds__(256) enum_kernel(EnumArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const TabView<CHK> t = stage_whole_or_global<CHK>(a.dt, smem);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.n_chunks; c += stride) {
        // segment of chunk c
        int lo = 0, hi = a.n_segs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.segs[mid].chunk0 <= c) lo = mid;
            else hi = mid - 1;
        }
        const Seg sg = a.segs[lo];
        const uint64_t r0 = (c - sg.chunk0) * CANDS;
        const uint64_t n = min((uint64_t)CANDS, sg.size - r0);
        W suf = unrank<W>(r0, a.L, sg.k);
        const W top = (W)sg.v << a.L;
        uint32_t kept = 0;
        uint64_t out = PASS ? a.offsets[c] : 0;
        for (uint64_t i = 0; i < n; ++i) {
            const W s = top | suf;
            int ns;
            bool cp;
            if ((a.col_sites == 0 || colours_ok<W>(s, a)) && is_rep<W, CHK>(s, t, ns, cp) && cp) {
                if (PASS) {
                    ((W*)a.reps)[out] = s;
                    a.stab[out] = (uint16_t)ns;
                    ++out;
                }
                ++kept;
            }
            if (sg.k > 0 && i + 1 < n) suf = next_same_popcount<W>(suf);
        }
        if (!PASS) a.counts[c] = kept;
    }
}

// ---------------------------------------------------------------- scan (u32 counts -> u64 exclusive offsets)
static const int SCAN_TILE = 4096;

__global__ void scan_tile_sums(const uint32_t* in, uint64_t n, uint64_t* tile_sums) {
    __shared__ uint64_t red[32];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    uint64_t acc = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x)
        if (base + i < n) acc += in[base + i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) tile_sums[blockIdx.x] = acc;
    }
}

// single block: exclusive scan of tile sums in place, total in *total
__global__ void scan_tiles_serial(uint64_t* tile_sums, uint64_t n_tiles, uint64_t* total) {
    __shared__ uint64_t carry;
    __shared__ uint64_t warp_tot[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < n_tiles; base += blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        uint64_t v = i < n_tiles ? tile_sums[i] : 0;
        // inclusive warp scan
        uint64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint64_t w = threadIdx.x < (blockDim.x >> 5) ? warp_tot[threadIdx.x] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (threadIdx.x >= o) w += y;
            }
            warp_tot[threadIdx.x] = w;  // inclusive over warps
        }
        __syncthreads();
        const int wi = threadIdx.x >> 5;
        const uint64_t warp_off = wi ? warp_tot[wi - 1] : 0;
        if (i < n_tiles) tile_sums[i] = carry + warp_off + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_tile_apply(const uint32_t* in, uint64_t n, const uint64_t* tile_off, uint64_t* out) {
    // one block per tile, sequential inside each thread's contiguous piece
    __shared__ uint64_t part[1024];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    const int per = SCAN_TILE / blockDim.x;
    uint64_t acc = 0;
    const uint64_t my0 = base + (uint64_t)threadIdx.x * per;
    for (int i = 0; i < per; ++i)
        if (my0 + i < n) acc += in[my0 + i];
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = tile_off[blockIdx.x];
        for (unsigned j = 0; j < blockDim.x; ++j) {
            const uint64_t t = part[j];
            part[j] = run;
            run += t;
        }
    }
    __syncthreads();
    uint64_t run = part[threadIdx.x];
    for (int i = 0; i < per; ++i)
        if (my0 + i < n) {
            out[my0 + i] = run;
            run += in[my0 + i];
        }
}

// Exclusive scan of n u32 values into u64 offsets (device), total to the host.
ed_status exclusive_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* total, const Alloc& A,
                             cudaStream_t s) {
    const uint64_t n_tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    const size_t bytes = (size_t)(n_tiles + 2) * 8;
    uint64_t* tiles = (uint64_t*)A.get(bytes, s);
    if (!tiles) return fail(ED_ERR_NOMEM, "scan scratch");
    uint64_t* d_total = tiles + n_tiles + 1;
    ed_status st = ED_OK;
    if (n_tiles) {
        scan_tile_sums<<<(unsigned)n_tiles, 256, 0, s>>>(in, n, tiles);
        scan_tiles_serial<<<1, 1024, 0, s>>>(tiles, n_tiles, d_total);
        scan_tile_apply<<<(unsigned)n_tiles, 256, 0, s>>>(in, n, tiles, out);
    } else {
        cudaMemsetAsync(d_total, 0, 8, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(total, d_total, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "exclusive scan");
    A.put(tiles, bytes, s);
    return st;
}

// ---------------------------------------------------------------- Limits
// Two-level Limits: for top-block value v, bucket b = next q_v bits;
// key = base_v + b; limits[key] = first index with state >= (v, b).
template <typename W>
__global__ void limits_kernel(const W* reps, uint64_t D, const uint32_t* seg_base, const uint8_t* seg_q,
                              const uint64_t* v_lo, int S, int L, uint2* limits, uint64_t n_keys) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t key = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; key < n_keys; key += stride) {
        // find v with seg_base[v] <= key < seg_base[v+1]
        int lo = 0, hi = S - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg_base[mid] <= key) lo = mid;
            else hi = mid - 1;
        }
        const int v = lo;
        const uint64_t b = key - seg_base[v];
        const int q = seg_q[v];
        const W target = ((W)v << L) | (W)(q ? (b << (L - q)) : 0);
        // lower_bound inside v's range
        uint64_t a0 = v_lo[v], a1 = v_lo[v + 1];
        while (a0 < a1) {
            const uint64_t mid = (a0 + a1) >> 1;
            if (reps[mid] < target) a0 = mid + 1;
            else a1 = mid;
        }
        limits[key].x = (uint32_t)a0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) limits[n_keys] = make_uint2((uint32_t)D, 0u);
}

// Fingerprints of the first (up to) 4 states of every bucket (after
// limits_kernel has written all bucket starts).
template <typename W>
__global__ void fingerprint_kernel(const W* reps, uint2* limits, uint64_t n_keys) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t key = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; key < n_keys; key += stride) {
        const uint32_t lo = limits[key].x, hi = limits[key + 1].x;
        uint32_t f = 0;
        for (uint32_t p = 0; p < 4 && lo + p < hi; ++p) f |= state_fp(reps[lo + p]) << (8 * p);
        limits[key].y = f;
    }
}

// ---------------------------------------------------------------- representatives of given states
template <typename W, bool CH>
__global__ void __launch_bounds__(256) rep_kernel(DevTables dt, const uint64_t* states, int64_t n, uint64_t* rep,
                                                  int32_t* gout, int32_t* nst, uint8_t* cmp) {
    extern __shared__ __align__(16) uint8_t smem[];
    const TabView<CH> t = stage_whole_or_global<CH>(dt, smem);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        W r;
        int g, ns;
        bool cp;
        find_rep<W, CH>((W)states[i], t, r, g, ns, cp);
        rep[i] = (uint64_t)r;
        gout[i] = g;
        nst[i] = ns;
        cmp[i] = cp ? 1 : 0;
    }
}

template <typename W, bool CH>
static ed_status launch_rep(const ed_basis* b, const uint64_t* st, int64_t n, uint64_t* r, int32_t* g, int32_t* ns,
                            uint8_t* cp, cudaStream_t s) {
    auto k = rep_kernel<W, CH>;
    const size_t smem = whole_stage_bytes(b->dt);
    ED_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
    k<<<grid, 256, smem, s>>>(b->dt, st, n, r, g, ns, cp);
    ED_CUDA(cudaGetLastError());
    return ED_OK;
}

ed_status representatives_device(const ed_basis* b, const uint64_t* st, int64_t n, uint64_t* r, int32_t* g, int32_t* ns,
                                 uint8_t* cp, cudaStream_t s) {
    const bool w8 = b->word == 8, ch = b->dt.chunk_lo > 0;
    if (w8) return ch ? launch_rep<uint64_t, true>(b, st, n, r, g, ns, cp, s) : launch_rep<uint64_t, false>(b, st, n, r, g, ns, cp, s);
    return ch ? launch_rep<uint32_t, true>(b, st, n, r, g, ns, cp, s) : launch_rep<uint32_t, false>(b, st, n, r, g, ns, cp, s);
}

// ---------------------------------------------------------------- restriction to a subgroup's sector
// A state of G's sector transforms with chi under every h of a subgroup H
// (Eq. symmetryadaptedwavefunctiontrafocharacter), so it lies in H's sector.
// Its coefficient on H's normalised projection of sigma (Eq.
// symmetryadaptedwavefunction1d) is sqrt(|H| / |Stab_H(sigma)|) <sigma|psi>, and
// the product-state amplitude is <sigma|psi> = chi(g) sqrt(|Stab_G(r)| / |G|) x_j
// for r = g.sigma the G-representative at index j.  One thread per row of H's
// basis: G's representative search (tables of G), G's index search, one scaled
// copy per vector.
template <int K> struct RVal;
template <> struct RVal<0> { using T = double; };
template <> struct RVal<1> { using T = float; };
template <> struct RVal<2> { using T = double2; };
template <> struct RVal<3> { using T = float2; };

__device__ __forceinline__ double scale_val(double2 c, double x) { return c.x * x; }
__device__ __forceinline__ float scale_val(double2 c, float x) { return (float)(c.x * (double)x); }
__device__ __forceinline__ double2 scale_val(double2 c, double2 x) {
    return make_double2(c.x * x.x - c.y * x.y, c.x * x.y + c.y * x.x);
}
__device__ __forceinline__ float2 scale_val(double2 c, float2 x) {
    return make_float2((float)(c.x * (double)x.x - c.y * (double)x.y), (float)(c.x * (double)x.y + c.y * (double)x.x));
}
template <typename T> __device__ __forceinline__ T zero_val();
template <> __device__ __forceinline__ double zero_val<double>() { return 0.0; }
template <> __device__ __forceinline__ float zero_val<float>() { return 0.f; }
template <> __device__ __forceinline__ double2 zero_val<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 zero_val<float2>() { return make_float2(0.f, 0.f); }

struct RestrictArgs {
    DevTables dt;               // tables of G
    const void* reps_g;         // G's basis
    const uint32_t* dir_base;   // G's Limits directory
    const uint8_t* dir_q;
    const uint2* limits;
    int L;
    int64_t Dg;
    const void* reps_h;         // H's basis and stabiliser orders
    const uint16_t* stab_h;
    int64_t Dh;
    double ratio;               // |H| / |G|
    const void* x;
    void* y;
    int nvec;
    unsigned long long* missing;
};

template <typename W, bool CH, int K>
__global__ void __launch_bounds__(256) restrict_kernel(RestrictArgs a) {
    using T = typename RVal<K>::T;
    extern __shared__ __align__(16) uint8_t smem[];
    const TabView<CH> t = stage_whole_or_global<CH>(a.dt, smem);
    const W* reps_g = (const W*)a.reps_g;
    const W* reps_h = (const W*)a.reps_h;
    const T* x = (const T*)a.x;
    T* y = (T*)a.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.Dh; i += (int64_t)gridDim.x * blockDim.x) {
        W r;
        int g, ns;
        bool cp;
        find_rep<W, CH>(ld_ro(reps_h + i), t, r, g, ns, cp);
        int64_t j = -1;
        double2 c = make_double2(0.0, 0.0);
        if (cp) {
            j = find_index<W>(r, reps_g, a.dir_base, a.dir_q, a.limits, a.L);
            if (j < 0) {
                atomicAdd(a.missing, 1ull);
            } else {
                const double f = sqrt(a.ratio * (double)ns / (double)ld_ro(a.stab_h + i));
                const double2 ch = t.chi[g];
                c = make_double2(ch.x * f, ch.y * f);
            }
        }
        for (int v = 0; v < a.nvec; ++v)
            y[(int64_t)v * a.Dh + i] = j >= 0 ? scale_val(c, ld_ro(x + (int64_t)v * a.Dg + j)) : zero_val<T>();
    }
}

template <typename W, bool CH, int K>
static ed_status launch_restrict(const RestrictArgs& a, cudaStream_t s) {
    auto k = restrict_kernel<W, CH, K>;
    const size_t smem = whole_stage_bytes(a.dt);
    ED_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0;
    ED_CUDA(cudaGetDevice(&dev));
    ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.Dh + 255) / 256, (int64_t)sms * 8));
    k<<<grid, 256, smem, s>>>(a);
    ED_CUDA(cudaGetLastError());
    return ED_OK;
}

template <typename W, bool CH>
static ed_status restrict_dtype(const RestrictArgs& a, ed_dtype dtype, cudaStream_t s) {
    switch (dtype) {
        case ED_F64: return launch_restrict<W, CH, 0>(a, s);
        case ED_F32: return launch_restrict<W, CH, 1>(a, s);
        case ED_C128: return launch_restrict<W, CH, 2>(a, s);
        case ED_C64: return launch_restrict<W, CH, 3>(a, s);
    }
    return fail(ED_ERR_ARG, "bad dtype");
}

// Index in `g` of every element of `h` (same permutation and flip), or an
// error if one is missing or its character differs.
static ed_status subgroup_check(const HostTables& g, const HostTables& h) {
    if (g.N != h.N || g.n_up != h.n_up) return fail(ED_ERR_ARG, "sectors differ in n_sites or n_up");
    const int N = g.N;
    for (int e = 0; e < h.G; ++e) {
        const int32_t* pe = h.perm.data() + (size_t)e * N;
        int found = -1;
        for (int f = 0; f < g.G && found < 0; ++f) {
            if (g.flip[f] != h.flip[e]) continue;
            if (std::equal(pe, pe + N, g.perm.data() + (size_t)f * N)) found = f;
        }
        if (found < 0) return fail(ED_ERR_ARG, "element %d of the target group is not in the source group", e);
        const double dr = g.chi[2 * found] - h.chi[2 * e], di = g.chi[2 * found + 1] - h.chi[2 * e + 1];
        if (dr * dr + di * di > 1e-18)
            return fail(ED_ERR_ARG, "character of element %d differs from the restriction of the source irrep", e);
    }
    return ED_OK;
}

ed_status restrict_vectors(const ed_basis* from, const ed_basis* to, ed_dtype dtype, const void* x, void* y, int nvec,
                           cudaStream_t s) {
    if (!from || !to || !x || !y) return fail(ED_ERR_ARG, "null argument");
    if (nvec < 1 || nvec > 8) return fail(ED_ERR_ARG, "nvec out of range [1,8]");
    if (dtype != ED_F64 && dtype != ED_F32 && dtype != ED_C128 && dtype != ED_C64) return fail(ED_ERR_ARG, "bad dtype");
    ed_status st = subgroup_check(from->ht, to->ht);
    if (st != ED_OK) return st;
    if ((dtype == ED_F64 || dtype == ED_F32) && !from->ht.real_chars)
        return fail(ED_ERR_ARG, "complex characters need a complex dtype");
    if (to->dim == 0) return ED_OK;
    RestrictArgs a{};
    a.dt = from->dt;
    a.reps_g = from->reps.p;
    const uint8_t* dir = (const uint8_t*)from->limits.p;
    a.dir_base = (const uint32_t*)dir;
    a.dir_q = dir + from->dir_q_off();
    a.limits = (const uint2*)(dir + from->dir_lim_off());
    a.L = from->prefix_bits;
    a.Dg = from->dim;
    a.reps_h = to->reps.p;
    a.stab_h = (const uint16_t*)to->stab.p;
    a.Dh = to->dim;
    a.ratio = (double)to->ht.G / (double)from->ht.G;
    a.x = x;
    a.y = y;
    a.nvec = nvec;
    a.missing = (unsigned long long*)to->alloc.get(sizeof(unsigned long long), s);
    if (!a.missing) return fail(ED_ERR_NOMEM, "restriction counter");
    unsigned long long missing = 0;
    cudaError_t e = cudaMemsetAsync(a.missing, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync");
    if (st == ED_OK) {
        const bool w8 = from->word == 8, ch = from->dt.chunk_lo > 0;
        st = w8 ? (ch ? restrict_dtype<uint64_t, true>(a, dtype, s) : restrict_dtype<uint64_t, false>(a, dtype, s))
                : (ch ? restrict_dtype<uint32_t, true>(a, dtype, s) : restrict_dtype<uint32_t, false>(a, dtype, s));
    }
    if (st == ED_OK) {
        e = cudaMemcpyAsync(&missing, a.missing, sizeof(missing), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "restriction");
    }
    to->alloc.put(a.missing, sizeof(unsigned long long), s);
    if (st == ED_OK && missing)
        st = fail(ED_ERR_INDEX_NOT_FOUND, "%llu compatible representatives missing from the source basis", missing);
    return st;
}

// ---------------------------------------------------------------- one-site S^z sums between sectors
// O = sum_i c_i S^z_i is diagonal in the product basis.  When every element
// of the common group G satisfies g O g^-1 = lambda(g) O, O maps the sector
// of chi into the sector of chi' = lambda chi, and for a representative sigma
// of the target <sigma~'|O|psi> = f(sigma) x_j with f(sigma) = sum_i c_i s^z_i(sigma)
// and j the index of sigma in the source basis (the two normalisations
// sqrt(|G| |Stab(sigma)|) cancel; 0 if sigma's projector vanishes in the source).
struct SzArgs {
    const void* reps_from;
    const uint32_t* dir_base;
    const uint8_t* dir_q;
    const uint2* limits;
    int L;
    int64_t Df;
    const void* reps_to;
    int64_t Dt;
    int N;
    const double2* c;           // [N] by bit position (bit N-1-i holds site i)
    double2 c_sum;              // sum_i c_i
    const void* x;
    void* y;
    int nvec;
};

template <typename W, int K>
__global__ void __launch_bounds__(256) sz_kernel(SzArgs a) {
    using T = typename RVal<K>::T;
    __shared__ double2 cb[64];
    for (int b = threadIdx.x; b < 64; b += blockDim.x) cb[b] = b < a.N ? a.c[b] : make_double2(0.0, 0.0);
    __syncthreads();
    const W* reps_f = (const W*)a.reps_from;
    const W* reps_t = (const W*)a.reps_to;
    const T* x = (const T*)a.x;
    T* y = (T*)a.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.Dt; i += (int64_t)gridDim.x * blockDim.x) {
        const W s = ld_ro(reps_t + i);
        int64_t j = find_index<W>(s, reps_f, a.dir_base, a.dir_q, a.limits, a.L);
        // s need not be in the source basis: confirm a fingerprint hit
        if (j >= 0 && ld_ro(reps_f + j) != s) j = -1;
        double2 f = make_double2(-0.5 * a.c_sum.x, -0.5 * a.c_sum.y);
        W rest = s;
        while (rest) {
            const int b = (sizeof(W) == 8) ? __ffsll((long long)rest) - 1 : __ffs((int)(uint32_t)rest) - 1;
            f.x += cb[b].x;
            f.y += cb[b].y;
            rest &= rest - 1;
        }
        for (int v = 0; v < a.nvec; ++v)
            y[(int64_t)v * a.Dt + i] = j >= 0 ? scale_val(f, ld_ro(x + (int64_t)v * a.Df + j)) : zero_val<T>();
    }
}

template <typename W, int K>
static ed_status launch_sz(const SzArgs& a, cudaStream_t s) {
    int dev = 0, sms = 0;
    ED_CUDA(cudaGetDevice(&dev));
    ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.Dt + 255) / 256, (int64_t)sms * 8));
    sz_kernel<W, K><<<grid, 256, 0, s>>>(a);
    ED_CUDA(cudaGetLastError());
    return ED_OK;
}

// lambda(g) with s_g c_{g^-1(j)} = lambda(g) c_j for all sites j (s_g = -1 for a
// spin flip), and chi_to(g) = lambda(g) chi_from(g) for the matching element.
static ed_status sz_check(const HostTables& f, const HostTables& t, const double* c, bool real_kind) {
    if (f.N != t.N || f.n_up != t.n_up || f.G != t.G) return fail(ED_ERR_ARG, "sectors differ in n_sites, n_up or group order");
    const int N = f.N;
    int j0 = 0;
    double cmax = 0.0;
    for (int j = 0; j < N; ++j) {
        const double a = hypot(c[2 * j], c[2 * j + 1]);
        if (a > cmax) { cmax = a; j0 = j; }
        if (real_kind && fabs(c[2 * j + 1]) > 1e-12) return fail(ED_ERR_ARG, "complex coefficients need a complex dtype");
    }
    if (!(cmax > 0.0)) return fail(ED_ERR_ARG, "all coefficients are zero");
    std::vector<int> inv(N);
    for (int e = 0; e < t.G; ++e) {
        const int32_t* p = t.perm.data() + (size_t)e * N;
        for (int i = 0; i < N; ++i) inv[p[i]] = i;
        const double sg = t.flip[e] ? -1.0 : 1.0;
        // lambda = s_g c_{g^-1(j0)} / c_{j0}
        const double ar = sg * c[2 * inv[j0]], ai = sg * c[2 * inv[j0] + 1];
        const double br = c[2 * j0], bi = c[2 * j0 + 1], bb = br * br + bi * bi;
        const double lr = (ar * br + ai * bi) / bb, li = (ai * br - ar * bi) / bb;
        if (fabs(lr * lr + li * li - 1.0) > 1e-9) return fail(ED_ERR_ARG, "element %d does not map the operator onto a multiple of itself", e);
        for (int j = 0; j < N; ++j) {
            const double er = sg * c[2 * inv[j]] - (lr * c[2 * j] - li * c[2 * j + 1]);
            const double ei = sg * c[2 * inv[j] + 1] - (lr * c[2 * j + 1] + li * c[2 * j]);
            if (hypot(er, ei) > 1e-9 * cmax)
                return fail(ED_ERR_ARG, "element %d does not map the operator onto a multiple of itself", e);
        }
        // matching element of the source and its character
        int m = -1;
        for (int g = 0; g < f.G && m < 0; ++g)
            if (f.flip[g] == t.flip[e] && std::equal(p, p + N, f.perm.data() + (size_t)g * N)) m = g;
        if (m < 0) return fail(ED_ERR_ARG, "element %d of the target group is not in the source group", e);
        const double xr = lr * f.chi[2 * m] - li * f.chi[2 * m + 1], xi = lr * f.chi[2 * m + 1] + li * f.chi[2 * m];
        if (hypot(xr - t.chi[2 * e], xi - t.chi[2 * e + 1]) > 1e-9)
            return fail(ED_ERR_ARG, "target characters are not lambda chi for element %d", e);
    }
    return ED_OK;
}

ed_status sz_transfer(const ed_basis* from, const ed_basis* to, const double* c, ed_dtype dtype, const void* x, void* y,
                      int nvec, cudaStream_t s) {
    if (!from || !to || !c || !x || !y) return fail(ED_ERR_ARG, "null argument");
    if (nvec < 1 || nvec > 8) return fail(ED_ERR_ARG, "nvec out of range [1,8]");
    if (dtype != ED_F64 && dtype != ED_F32 && dtype != ED_C128 && dtype != ED_C64) return fail(ED_ERR_ARG, "bad dtype");
    const bool real_kind = dtype == ED_F64 || dtype == ED_F32;
    if (real_kind && (!from->ht.real_chars || !to->ht.real_chars))
        return fail(ED_ERR_ARG, "complex characters need a complex dtype");
    ed_status st = sz_check(from->ht, to->ht, c, real_kind);
    if (st != ED_OK) return st;
    if (to->dim == 0) return ED_OK;
    const int N = from->ht.N;
    std::vector<double2> cb(N);
    double2 csum = make_double2(0.0, 0.0);
    for (int i = 0; i < N; ++i) {
        cb[N - 1 - i] = make_double2(c[2 * i], real_kind ? 0.0 : c[2 * i + 1]);
        csum.x += cb[N - 1 - i].x;
        csum.y += cb[N - 1 - i].y;
    }
    SzArgs a{};
    a.reps_from = from->reps.p;
    const uint8_t* dir = (const uint8_t*)from->limits.p;
    a.dir_base = (const uint32_t*)dir;
    a.dir_q = dir + from->dir_q_off();
    a.limits = (const uint2*)(dir + from->dir_lim_off());
    a.L = from->prefix_bits;
    a.Df = from->dim;
    a.reps_to = to->reps.p;
    a.Dt = to->dim;
    a.N = N;
    a.c_sum = csum;
    a.x = x;
    a.y = y;
    a.nvec = nvec;
    double2* dc = (double2*)to->alloc.get((size_t)N * sizeof(double2), s);
    if (!dc) return fail(ED_ERR_NOMEM, "coefficient table");
    a.c = dc;
    cudaError_t e = cudaMemcpyAsync(dc, cb.data(), (size_t)N * sizeof(double2), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpyAsync");
    if (st == ED_OK) {
        const bool w8 = from->word == 8;
        switch (dtype) {
            case ED_F64: st = w8 ? launch_sz<uint64_t, 0>(a, s) : launch_sz<uint32_t, 0>(a, s); break;
            case ED_F32: st = w8 ? launch_sz<uint64_t, 1>(a, s) : launch_sz<uint32_t, 1>(a, s); break;
            case ED_C128: st = w8 ? launch_sz<uint64_t, 2>(a, s) : launch_sz<uint32_t, 2>(a, s); break;
            case ED_C64: st = w8 ? launch_sz<uint64_t, 3>(a, s) : launch_sz<uint32_t, 3>(a, s); break;
        }
    }
    // the coefficient table is released once the kernel has run
    e = cudaStreamSynchronize(s);
    if (st == ED_OK && e != cudaSuccess) st = cuda_fail(e, "sz transfer");
    to->alloc.put(dc, (size_t)N * sizeof(double2), s);
    return st;
}

// ---------------------------------------------------------------- no-allocation variant
// Some callers cannot allocate device memory themselves: applications whose
// device memory is owned by another runtime's pool (a framework that reserves
// the GPU up front), or loops that must not call cudaMalloc/cudaFree because
// those calls can synchronise the whole device.  For them the table image of
// the representative search lives in this file-scope array instead of a
// per-call allocation.  Every GPU that loads the library holds it until exit.
static constexpr size_t kStaticTableBytes = 224 * 1024;
static __device__ __align__(256) uint8_t g_static_tables[kStaticTableBytes];

// Device address of g_static_tables per device, looked up once per device
// with that device current (the host-side name is only a stand-in).  The
// cache is atomic: host threads making their first call on one device at the
// same time look the address up independently and store the same value.
static uint8_t* static_tables_ptr(int dev, ed_status& st) {
    static std::atomic<uint8_t*> ptrs[256];
    st = ED_OK;
    if (dev < 0 || dev >= 256) {
        st = fail(ED_ERR_ARG, "device ordinal %d out of range", dev);
        return nullptr;
    }
    uint8_t* cur = ptrs[dev].load(std::memory_order_acquire);
    if (!cur) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_tables);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaGetSymbolAddress(g_static_tables)");
            return nullptr;
        }
        cur = (uint8_t*)p;
        ptrs[dev].store(cur, std::memory_order_release);
    }
    return cur;
}

ed_status representatives_static(const ed_sector* sector, const uint64_t* states, int64_t n, uint64_t* rep, int32_t* g,
                                 int32_t* nstab, uint8_t* compat, cudaStream_t s) {
    // First, before any other CUDA call: the table upload below copies from a
    // host buffer that lives only for this call, which a captured graph would
    // read again on every replay, so stream capture is refused.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ED_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(ED_ERR_ARG, "ed_representatives_noalloc must not be called while its stream is being captured");
    if (!sector || n < 0 || (n > 0 && (!states || !rep || !g || !nstab || !compat)))
        return fail(ED_ERR_ARG, "null argument");
    ed_basis tmp;
    ed_status st = build_host_tables(sector, tmp.ht);
    if (st != ED_OK || n == 0) return st;
    std::vector<uint8_t> image;
    make_blob(tmp.ht, tmp.dt, image);
    if (image.size() > kStaticTableBytes)
        return fail(ED_ERR_TABLE_TOO_LARGE, "table image of %zu bytes exceeds the static limit of %zu bytes",
                    image.size(), kStaticTableBytes);
    int dev = 0;
    ED_CUDA(cudaGetDevice(&dev));
    uint8_t* base = static_tables_ptr(dev, st);
    if (!base) return st;
    tmp.word = tmp.ht.N <= 32 ? 4 : 8;
    tmp.dt.blob = base;
    ED_CUDA(cudaMemcpyAsync(base, image.data(), image.size(), cudaMemcpyHostToDevice, s));
    // the kernel masks nothing: callers pass states of n_sites bits
    return representatives_device(&tmp, states, n, rep, g, nstab, compat, s);
}

// ---------------------------------------------------------------- host
void make_blob(const HostTables& t, DevTables& d, std::vector<uint8_t>& h) {
    const int S = 1 << t.m;
    const bool chunked = t.chunk_lo > 0;
    const int stride = chunked ? (1 << (t.m - t.chunk_lo)) + (1 << t.chunk_lo) : S;
    const int eb = chunked ? 2 : 1;
    size_t off = 0;
    auto al = [&](size_t n) {
        off = (off + 15) & ~(size_t)15;
        size_t o = off;
        off += n;
        return (uint32_t)o;
    };
    d.N = t.N; d.G = t.G; d.n_sub = t.n_sub; d.m = t.m; d.sa_bytes = eb;
    d.chunk_lo = t.chunk_lo;
    d.lmap_stride = stride;
    d.off_rep = al((size_t)t.n_sub * S * 2);
    d.off_symoff = al((size_t)t.n_sub * (S + 1) * 4);
    d.off_symids = al(std::max<size_t>(t.sym_ids.size(), 1) * 2);
    d.off_sa = al((size_t)t.n_lmap * stride * eb);
    d.off_src = al((size_t)t.G * t.n_sub * 4);
    d.off_chi = al((size_t)t.G * 16);
    d.off_chicls = al((size_t)t.G * 2);
    d.off_sqrt = al((size_t)2 * (t.G + 1) * 8);
    d.off_chif = al((size_t)t.G * 8);
    d.off_sqrtf = al((size_t)2 * (t.G + 1) * 4);
    d.dl_stride = t.dl_stride;
    d.off_dl = al(std::max<size_t>(t.dl.size(), 1) * 2);
    d.off_chineg = al((size_t)t.G);
    const size_t total = (off + 15) & ~(size_t)15;
    d.blob_bytes = total;
    h.assign(total, 0);
    memcpy(&h[d.off_rep], t.rep.data(), t.rep.size() * 2);
    memcpy(&h[d.off_symoff], t.sym_off.data(), t.sym_off.size() * 4);
    if (!t.sym_ids.empty()) memcpy(&h[d.off_symids], t.sym_ids.data(), t.sym_ids.size() * 2);
    if (!chunked) {
        for (size_t i = 0; i < t.lmap_tab.size(); ++i) h[d.off_sa + i] = (uint8_t)t.lmap_tab[i];
    } else {
        memcpy(&h[d.off_sa], t.lmap_tab.data(), t.lmap_tab.size() * 2);
    }
    memcpy(&h[d.off_src], t.srclid.data(), t.srclid.size() * 4);
    memcpy(&h[d.off_chi], t.chi.data(), (size_t)t.G * 16);
    memcpy(&h[d.off_chicls], t.chi_cls.data(), (size_t)t.G * 2);
    std::vector<double> sq(2 * (size_t)(t.G + 1));
    for (int k = 0; k <= t.G; ++k) {
        sq[k] = sqrt((double)k);
        sq[t.G + 1 + k] = k ? 1.0 / sqrt((double)k) : 0.0;
    }
    memcpy(&h[d.off_sqrt], sq.data(), sq.size() * 8);
    std::vector<float> chif(2 * (size_t)t.G), sqf(sq.size());
    for (size_t i = 0; i < chif.size(); ++i) chif[i] = (float)t.chi[i];
    for (size_t i = 0; i < sq.size(); ++i) sqf[i] = (float)sq[i];
    memcpy(&h[d.off_chif], chif.data(), chif.size() * 4);
    memcpy(&h[d.off_sqrtf], sqf.data(), sqf.size() * 4);
    if (!t.dl.empty()) memcpy(&h[d.off_dl], t.dl.data(), t.dl.size() * 2);
    memcpy(&h[d.off_chineg], t.chi_neg.data(), (size_t)t.G);
}

ed_status upload_tables(ed_basis* b, cudaStream_t s) {
    std::vector<uint8_t> h;
    DevTables& d = b->dt;
    make_blob(b->ht, d, h);
    const size_t total = h.size();
    b->tables.bytes = total;
    b->tables.p = b->alloc.get(total, s);
    if (!b->tables.p) return fail(ED_ERR_NOMEM, "table allocation failed");
    ED_CUDA(cudaMemcpyAsync(b->tables.p, h.data(), total, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaStreamSynchronize(s));
    d.blob = (const uint8_t*)b->tables.p;
    return ED_OK;
}

template <typename W, bool CHK, int PASS>
static ed_status launch_enum(const EnumArgs& a, size_t smem, int sms, cudaStream_t s) {
    auto k = enum_kernel<W, CHK, PASS>;
    ED_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    ED_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));
    if (per_sm < 1) return fail(ED_ERR_TABLE_TOO_LARGE, "lookup tables (%zu bytes) do not fit shared memory", smem);
    uint64_t want = (a.n_chunks + 255) / 256;
    uint64_t grid = std::min<uint64_t>(want, (uint64_t)sms * per_sm * 4);
    if (grid < 1) grid = 1;
    k<<<(unsigned)grid, 256, smem, s>>>(a);
    ED_CUDA(cudaGetLastError());
    return ED_OK;
}

template <typename W, bool CHK>
static ed_status enum_both(ed_basis* b, EnumArgs& a, size_t smem, int sms, cudaStream_t s, int pass) {
    return pass == 0 ? launch_enum<W, CHK, 0>(a, smem, sms, s) : launch_enum<W, CHK, 1>(a, smem, sms, s);
}

static ed_status run_enum(ed_basis* b, EnumArgs& a, int pass, int sms, cudaStream_t s) {
    const size_t smem = whole_stage_bytes(b->dt);
    const bool w8 = b->word == 8, ch = b->dt.chunk_lo > 0;
    if (w8) return ch ? enum_both<uint64_t, true>(b, a, smem, sms, s, pass)
                      : enum_both<uint64_t, false>(b, a, smem, sms, s, pass);
    return ch ? enum_both<uint32_t, true>(b, a, smem, sms, s, pass)
              : enum_both<uint32_t, false>(b, a, smem, sms, s, pass);
}

namespace {
struct Scratch {
    const Alloc* A;
    cudaStream_t s;
    std::vector<std::pair<void*, size_t>> bufs;
    void* get(size_t n) {
        void* p = A->get(n, s);
        if (p) bufs.push_back({p, n});
        return p;
    }
    ~Scratch() {
        cudaStreamSynchronize(s);
        for (auto& b : bufs) A->put(b.first, b.second, s);
    }
};
}  // namespace

ed_status basis_build_device(ed_basis* b, cudaStream_t s) {
    const HostTables& t = b->ht;
    ED_CUDA(cudaGetDevice(&b->device));
    int sms = 0;
    ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->word = t.N <= 32 ? 4 : 8;
    // binomials
    {
        std::vector<uint64_t> C(65 * 65, 0);
        for (int n = 0; n <= 64; ++n) {
            C[n * 65 + 0] = 1;
            for (int k = 1; k <= n; ++k) C[n * 65 + k] = C[(n - 1) * 65 + k - 1] + (k <= n - 1 ? C[(n - 1) * 65 + k] : 0);
        }
        ED_CUDA(cudaMemcpyToSymbol(c_binom, C.data(), C.size() * 8));
    }
    ed_status st = upload_tables(b, s);
    if (st != ED_OK) return st;
    const int m = t.m, L = t.N - m, S = 1 << m;
    std::vector<Seg> segs;
    uint64_t chunks = 0;
    for (int v = 0; v < S; ++v) {
        if (t.rep[v] != v) continue;  // block 0: Rep_0(v) = v is necessary
        const int k = t.n_up - __builtin_popcount((unsigned)v);
        if (k < 0 || k > L) continue;
        uint64_t C = 1;
        for (int i = 0; i < k; ++i) C = C * (uint64_t)(L - i) / (uint64_t)(i + 1);
        Seg sg{(uint32_t)v, k, C, chunks};
        segs.push_back(sg);
        chunks += (C + CANDS - 1) / CANDS;
    }
    if (segs.empty() || chunks == 0) return fail(ED_ERR_EMPTY_SECTOR, "sector has dimension 0");
    Scratch sc{&b->alloc, s, {}};
    Seg* d_segs = (Seg*)sc.get(segs.size() * sizeof(Seg));
    uint32_t* d_counts = (uint32_t*)sc.get(chunks * 4);
    uint64_t* d_offs = (uint64_t*)sc.get(chunks * 8);
    const uint64_t n_tiles = (chunks + SCAN_TILE - 1) / SCAN_TILE;
    uint64_t* d_tiles = (uint64_t*)sc.get(n_tiles * 8 + 8);
    uint64_t* d_total = (uint64_t*)sc.get(8);
    if (!d_segs || !d_counts || !d_offs || !d_tiles || !d_total) return fail(ED_ERR_NOMEM, "enumeration scratch");
    ED_CUDA(cudaMemcpyAsync(d_segs, segs.data(), segs.size() * sizeof(Seg), cudaMemcpyHostToDevice, s));
    EnumArgs a{};
    a.dt = b->dt;
    if (b->sun_d) {
        a.col_sites = b->sun_N;
        a.col_bits = b->sun_b;
        a.n_colors = b->sun_d;
        for (int c = 0; c < b->sun_d; ++c) a.col_want[c >> 3] += (uint64_t)b->sun_counts[c] << (8 * (c & 7));
    }
    a.segs = d_segs;
    a.n_segs = (int)segs.size();
    a.n_chunks = chunks;
    a.L = L;
    a.counts = d_counts;
    st = run_enum(b, a, 0, sms, s);
    if (st != ED_OK) return st;
    scan_tile_sums<<<(unsigned)n_tiles, 256, 0, s>>>(d_counts, chunks, d_tiles);
    scan_tiles_serial<<<1, 1024, 0, s>>>(d_tiles, n_tiles, d_total);
    scan_tile_apply<<<(unsigned)n_tiles, 256, 0, s>>>(d_counts, chunks, d_tiles, d_offs);
    ED_CUDA(cudaGetLastError());
    uint64_t D = 0;
    ED_CUDA(cudaMemcpyAsync(&D, d_total, 8, cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    if (D == 0) return fail(ED_ERR_EMPTY_SECTOR, "sector has dimension 0");
    if (D >= 0xFFFFFFFFull) return fail(ED_ERR_ARG, "dimension %llu exceeds 2^32-1", (unsigned long long)D);
    b->dim = (int64_t)D;
    b->reps.bytes = D * b->word;
    b->reps.p = b->alloc.get(b->reps.bytes, s);
    b->stab.bytes = D * 2;
    b->stab.p = b->alloc.get(b->stab.bytes, s);
    if (!b->reps.p || !b->stab.p) return fail(ED_ERR_NOMEM, "basis allocation (%llu states)", (unsigned long long)D);
    a.offsets = d_offs;
    a.reps = b->reps.p;
    a.stab = (uint16_t*)b->stab.p;
    st = run_enum(b, a, 1, sms, s);
    if (st != ED_OK) return st;
    // per-segment dimensions from the chunk offsets
    std::vector<uint64_t> offs(chunks);
    ED_CUDA(cudaMemcpyAsync(offs.data(), d_offs, chunks * 8, cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    std::vector<uint64_t> v_lo(S + 1, 0);
    {
        // v_lo[v] = first index with top block >= v
        std::vector<uint64_t> start(S, UINT64_MAX);
        for (size_t i = 0; i < segs.size(); ++i) start[segs[i].v] = offs[segs[i].chunk0];
        uint64_t next = D;
        v_lo[S] = D;
        for (int v = S - 1; v >= 0; --v) {
            if (start[v] != UINT64_MAX) next = start[v];
            v_lo[v] = next;
        }
    }
    // two-level Limits: q_v bits for top value v so buckets hold 1-2 states on
    // average (most lookups then resolve by fingerprint without reading the
    // basis; measured faster than ~4 states per bucket on every workload);
    // coarser buckets only if the keys would not fit 32-bit offsets
    std::vector<uint32_t> seg_base(S + 1, 0);
    std::vector<uint8_t> seg_q(S, 0);
    uint64_t keys = 0;
    for (const uint64_t target : {1ull, 2ull, 4ull, 1ull << 20}) {
        keys = 0;
        for (int v = 0; v < S; ++v) {
            const uint64_t Dv = v_lo[v + 1] - v_lo[v];
            int q = 0;
            while (q < L && (Dv >> q) > target) ++q;
            seg_q[v] = (uint8_t)q;
            seg_base[v] = (uint32_t)keys;
            keys += (uint64_t)1 << q;
        }
        if (keys < 0xFFFFFFFFull) break;
    }
    if (keys >= 0xFFFFFFFFull) return fail(ED_ERR_ARG, "basis too large for 32-bit Limits keys");
    seg_base[S] = (uint32_t)keys;
    b->prefix_bits = L;
    // device image of the Limits directory: [S+1] base, [S] q (padded), then limits
    b->limits.bytes = b->dir_lim_off() + (keys + 1) * 8;
    b->limits.p = b->alloc.get(b->limits.bytes, s);
    if (!b->limits.p) return fail(ED_ERR_NOMEM, "limits allocation");
    uint8_t* base = (uint8_t*)b->limits.p;
    ED_CUDA(cudaMemcpyAsync(base, seg_base.data(), (S + 1) * 4, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(base + (S + 1) * 4, seg_q.data(), S, cudaMemcpyHostToDevice, s));
    uint64_t* d_vlo = (uint64_t*)sc.get((S + 1) * 8);
    if (!d_vlo) return fail(ED_ERR_NOMEM, "limits scratch");
    ED_CUDA(cudaMemcpyAsync(d_vlo, v_lo.data(), (S + 1) * 8, cudaMemcpyHostToDevice, s));
    uint2* d_lim = (uint2*)(base + b->dir_lim_off());
    const unsigned g = (unsigned)std::min<uint64_t>((keys + 255) / 256, (uint64_t)sms * 16);
    if (b->word == 8)
        limits_kernel<uint64_t><<<g, 256, 0, s>>>((const uint64_t*)b->reps.p, D, (const uint32_t*)base,
                                                  base + (S + 1) * 4, d_vlo, S, L, d_lim, keys);
    else
        limits_kernel<uint32_t><<<g, 256, 0, s>>>((const uint32_t*)b->reps.p, D, (const uint32_t*)base,
                                                  base + (S + 1) * 4, d_vlo, S, L, d_lim, keys);
    ED_CUDA(cudaGetLastError());
    if (b->word == 8) fingerprint_kernel<uint64_t><<<g, 256, 0, s>>>((const uint64_t*)b->reps.p, d_lim, keys);
    else fingerprint_kernel<uint32_t><<<g, 256, 0, s>>>((const uint32_t*)b->reps.p, d_lim, keys);
    ED_CUDA(cudaGetLastError());
    ED_CUDA(cudaStreamSynchronize(s));
    b->n_keys = keys;
    return ED_OK;
}

}  // namespace ed
