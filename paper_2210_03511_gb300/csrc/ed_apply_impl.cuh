// y = H x in the symmetry-adapted basis (pull form of Alg. "Parallel
// matrix-vector multiply for a non-branching term", summed over all terms as in
// Eq. branchingsum).
//
// Work decomposition.  One thread owns one row sigma_i (a grid-stride loop
// over rows).  It builds the row's activity mask (flip term t acts iff its two
// spins differ) and walks the set bits.  For an acting term the image
// tau = sigma ^ mask is reduced to its representative by sublattice coding
// (tables in shared memory), located by Limits + binary search, and
// contributes
//     conj(h) chi(g_tau) sqrt(|Stab tau~| / |Stab sigma_i|) x_j
// to y_i: H is Hermitian, H_ij = conj(H_ji), and H_ji is the matrix element
// of Eq. matrixelementrepresentatives with the conj(chi) reading.  The thread
// accumulates its row alone and writes y_i once: no atomics, no cross-lane
// reduction (FP64 arithmetic is scarce on this GPU), deterministic.  The
// Ising part is diagonal: sum over pairs of J/4 (1 - 2 act), from popcounts of
// the activity mask per coupling class.
// Templates of the H.x kernels, instantiated per value kind in
// ed_apply_k<K>.cu (one translation unit per kind so they compile in parallel).
#pragma once

#include <algorithm>
#include <type_traits>

#include "ed_device.cuh"
#include "ed_internal.h"

namespace ed {

template <int K> struct Val;
template <> struct Val<0> { using T = double; using R = double; static constexpr bool cplx = false; };
template <> struct Val<1> { using T = float; using R = float; static constexpr bool cplx = false; };
template <> struct Val<2> { using T = double2; using R = double; static constexpr bool cplx = true; };
template <> struct Val<3> { using T = float2; using R = float; static constexpr bool cplx = true; };

constexpr int MAXV = 8;
constexpr int BLOCK = 256;        // threads per block
constexpr int MAXW = 8;           // activity mask words per row (n_flip <= 256)

template <typename W, bool CH, int NS>
__device__ __forceinline__ void rep_of(W tau, const TabView<CH>& t, W& r, int& g, int& nst, bool& cp) {
    if constexpr (NS >= 2 && NS <= 4) find_rep_ns<W, CH, NS>(tau, t, r, g, nst, cp);
    else find_rep<W, CH>(tau, t, r, g, nst, cp);
}

// Resident blocks per SM an H.x instantiation is built for (its register
// budget: 65536 / (256 x blocks) registers a thread).  Measured on the
// workloads: one real vector with 32-bit states runs fastest at 6 (40
// registers, a few spills: square32 3.8 -> 3.4 ms), with 64-bit states at 4
// (fewer registers spill the 64-bit search state: square40 1.77 -> 2.7 s);
// one complex-FP32 vector at 4 (kagome36 294 -> 186 ms); complex FP64 and
// several vectors at 2.
__host__ __device__ constexpr int hx_min_blocks(int wbytes, int nv, int k) {
    return nv != 1 ? 2 : (k < 2 ? (wbytes == 4 ? 6 : 4) : (k == 3 ? 4 : 2));
}

// Shared layout: [staged table sections][flip terms][packed (pa,pb)][jhs
// table][jcls][class masks][Limits directory, when staged].
struct SmemLayout {
    size_t flip, pab, jhs, jcls, cmask, dir, total;
};

__host__ __device__ inline SmemLayout smem_layout(size_t tables, int n_flip, int n_jc, int G, int S, bool dir) {
    SmemLayout l;
    auto up16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
    l.flip = up16(tables);
    l.pab = up16(l.flip + (size_t)n_flip * sizeof(FlipTerm));
    l.jhs = up16(l.pab + (size_t)n_flip * 2);
    l.jcls = up16(l.jhs + (size_t)n_jc * (G + 1) * 8);
    l.cmask = up16(l.jcls + (size_t)n_flip);
    l.dir = up16(l.cmask + (size_t)n_jc * MAXW * 4);
    l.total = dir ? up16(l.dir + (size_t)(S + 1) * 4 + S) : l.dir;
    return l;
}

// What one H.x block keeps in shared memory.  The per-row data (flip terms,
// coefficient table, class masks) always; then, while they fit the share of
// the SM that `blocks` resident blocks leave, in order of accesses per
// flipped image: packed entries and chi signs (every candidate), character
// tables (every gather), the (source, map) table (generic search), the local
// block maps (every composed block), the Limits directory (every gather),
// Rep (every block of every image), Sym offsets and lists.  Host and device
// evaluate the same function, so launch size and kernel layout agree.
struct HxPlan {
    uint32_t mask;
    uint32_t table_bytes;
    bool dir;
    SmemLayout lay;
};

__host__ __device__ inline HxPlan hx_plan(const DevTables& d, int K, bool generic, int blocks, int n_flip,
                                          int n_jc, int S) {
    const size_t per_sm = 228 * 1024, reserved = 1024, max_block = 227 * 1024;
    size_t limit = per_sm / (size_t)(blocks < 1 ? 1 : blocks) - reserved;
    if (limit > max_block) limit = max_block;
    const SmemLayout base = smem_layout(0, n_flip, n_jc, d.G, S, false);
    const size_t dir_bytes = (((size_t)(S + 1) * 4 + S) + 15) & ~(size_t)15;
    size_t used = base.total;
    HxPlan p{0u, 0u, false, base};
    auto take = [&](uint32_t sec) {
        if (sec == SEC_SRC && !generic) return;
        const size_t n = sec_bytes(d, sec, K);
        if (used + n <= limit) {
            p.mask |= sec;
            p.table_bytes += (uint32_t)n;
            used += n;
        }
    };
    take(SEC_DL);
    take(SEC_CHI);
    take(SEC_SRC);
    take(SEC_MAPS);
    if (used + dir_bytes <= limit) {
        p.dir = true;
        used += dir_bytes;
    }
    take(SEC_REP);
    take(SEC_SYM);
    p.lay = smem_layout(p.table_bytes, n_flip, n_jc, d.G, S, p.dir);
    return p;
}

struct Counts {
    unsigned long long gather = 0, skip = 0, miss = 0;
};

// Stage one sector's tables into shared memory and process rows
// first, first + stride, ... < end of that sector.  All threads of the block
// must call it (it synchronises the block).
template <typename W, bool CH, int K, int NV, int NS>
__device__ __forceinline__ void hx_body(const HxArgs& a, uint8_t* smem, int64_t first, int64_t end, int64_t stride,
                                        Counts& cnt) {
    using V = Val<K>;
    using T = typename V::T;
    using R = typename V::R;
    constexpr bool generic = !(NS >= 2 && NS <= 4);
    const HxPlan plan = hx_plan(a.dt, K, generic, a.blocks, a.n_flip, a.n_jc, a.S);
    const SmemLayout lay = plan.lay;
    const TabView<CH> t = stage_sections<CH>(a.dt, smem, K, plan.mask);
    stage_blob(smem + lay.flip, (const uint8_t*)a.flips, (size_t)a.n_flip * sizeof(FlipTerm));
    stage_blob(smem + lay.jhs, (const uint8_t*)a.jhs, (size_t)a.n_jc * (a.dt.G + 1) * 8);
    uint16_t* pab = (uint16_t*)(smem + lay.pab);
    uint8_t* jcls = smem + lay.jcls;
    uint32_t* cmask = (uint32_t*)(smem + lay.cmask);
    for (int i = threadIdx.x; i < a.n_jc * MAXW; i += blockDim.x) cmask[i] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < a.n_flip; i += blockDim.x) {
        const FlipTerm& f = ((const FlipTerm*)(smem + lay.flip))[i];
        pab[i] = (uint16_t)((uint8_t)f.pa | ((uint16_t)(uint8_t)f.pb << 8));
        jcls[i] = a.jcls[i];
        atomicOr(&cmask[a.jcls[i] * MAXW + (i >> 5)], 1u << (i & 31));
    }
    const uint32_t* dir_base = a.dir_base;
    const uint8_t* dir_q = a.dir_q;
    if (plan.dir) {
        uint32_t* db = (uint32_t*)(smem + lay.dir);
        uint8_t* dq = (uint8_t*)(db + a.S + 1);
        for (int i = threadIdx.x; i <= a.S; i += blockDim.x) db[i] = a.dir_base[i];
        for (int i = threadIdx.x; i < a.S; i += blockDim.x) dq[i] = a.dir_q[i];
        dir_base = db;
        dir_q = dq;
    }
    __syncthreads();
    const FlipTerm* flips = (const FlipTerm*)(smem + lay.flip);
    const double* jhs = (const double*)(smem + lay.jhs);
    const W* __restrict__ reps = (const W*)a.reps;
    const T* __restrict__ x = (const T*)a.x;
    T* __restrict__ y = (T*)a.y;
    const int64_t D = a.D;
    const int nvec = NV == 1 ? 1 : a.nvec;
    const int G1 = a.dt.G + 1;
    const int nw = (a.n_flip + 31) >> 5;
    unsigned long long n_gather = 0, n_skip = 0, n_miss = 0;
    for (int64_t row = first; row < end; row += stride) {
        const W s = reps[row];
        const int stab_row = a.stab[row];
        // activity mask: term t acts iff its two spins differ
        uint32_t mask[MAXW];
#pragma unroll
        for (int w = 0; w < MAXW; ++w) mask[w] = 0u;
#pragma unroll
        for (int w = 0; w < MAXW; ++w) {
            if (w < nw) {
                const int tn = min(32, a.n_flip - 32 * w);
                uint32_t mw = 0u;
                for (int b = 0; b < tn; ++b) {
                    const uint32_t e = pab[32 * w + b];
                    mw |= (uint32_t)(((s >> (e & 0xFFu)) ^ (s >> (e >> 8))) & 1) << b;
                }
                mask[w] = mw;
            }
        }
        // Ising part: sum over pairs of J/4 (1 - 2 act) = sum_c jhalf_c (n_c/2 - popc(act & class_c))
        double diag = 0.0;
        for (int c = 0; c < a.n_jc; ++c) {
            int nact = 0, ntot = 0;
#pragma unroll
            for (int w = 0; w < MAXW; ++w) {
                if (w < nw) {
                    const uint32_t cm = cmask[c * MAXW + w];
                    nact += __popc(mask[w] & cm);
                    ntot += __popc(cm);
                }
            }
            diag += jhs[c * G1 + 1] * (0.5 * (double)ntot - (double)nact);
        }
        R accr[NV], acci[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { accr[v] = 0; acci[v] = 0; }
#pragma unroll
        for (int w = 0; w < MAXW; ++w) {
            if (w >= nw) continue;
            uint32_t mw = mask[w];
            while (mw) {
                const int tt = 32 * w + ctz32(mw);
                mw &= mw - 1u;
                const uint32_t e = pab[tt];
                const W tau = s ^ (((W)1 << (e & 0xFFu)) | ((W)1 << (e >> 8)));
                W rp;
                int g, nst;
                bool cp;
                rep_of<W, CH, NS>(tau, t, rp, g, nst, cp);
                if (!cp) {
                    ++n_skip;
                    continue;
                }
                const int64_t jx = find_index<W>(rp, reps, dir_base, dir_q, a.limits, a.L);
                if (jx < 0) {
                    ++n_miss;
                    continue;
                }
                ++n_gather;
                if constexpr (!V::cplx) {
                    // jhalf * sqrt(n) from the table; real chi(g) = +-1 enters as a sign bit
                    R c;
                    if constexpr (K == 0) {
                        const double cd = jhs[jcls[tt] * G1 + nst];
                        c = __longlong_as_double(__double_as_longlong(cd) ^ ((long long)t.chi_neg[g] << 63));
                    } else {
                        c = (R)flips[tt].jhalf * t.chif[g].x * t.sqrtnf[nst];
                    }
#pragma unroll
                    for (int v = 0; v < NV; ++v)
                        if (v < nvec) accr[v] += c * x[(int64_t)v * D + jx];
                } else {
                    const FlipTerm ft = flips[tt];
                    // h = jhalf + i sum_t k_t s^z_c (spin a down ? +1 : -1)
                    double him = 0.0;
                    if (ft.pc0 >= 0) him += ft.k0 * (((s >> ft.pc0) & 1) ? 0.5 : -0.5);
                    if (ft.pc1 >= 0) him += ft.k1 * (((s >> ft.pc1) & 1) ? 0.5 : -0.5);
                    if ((s >> ft.pa) & 1) him = -him;
                    R cr, ci;
                    if constexpr (K == 2) {
                        const double2 ch = t.chi[g];
                        const double sq = t.sqrtn[nst];
                        // conj(h) chi = (jh - i him)(chr + i chi)
                        cr = (ft.jhalf * ch.x + him * ch.y) * sq;
                        ci = (ft.jhalf * ch.y - him * ch.x) * sq;
                    } else {
                        const float2 ch = t.chif[g];
                        const float sq = t.sqrtnf[nst];
                        const float jh = (float)ft.jhalf, hm = (float)him;
                        cr = (jh * ch.x + hm * ch.y) * sq;
                        ci = (jh * ch.y - hm * ch.x) * sq;
                    }
#pragma unroll
                    for (int v = 0; v < NV; ++v)
                        if (v < nvec) {
                            const T xj = x[(int64_t)v * D + jx];
                            accr[v] += cr * xj.x - ci * xj.y;
                            acci[v] += cr * xj.y + ci * xj.x;
                        }
                }
            }
        }
        // y_i = acc_i / sqrt(|Stab sigma_i|) + diag_i x_i
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v < nvec) {
                const int64_t o = (int64_t)v * D + row;
                if constexpr (!V::cplx) {
                    const R inv = (K == 0) ? (R)t.isqrtn[stab_row] : (R)t.isqrtnf[stab_row];
                    y[o] = accr[v] * inv + (R)diag * x[o];
                } else {
                    const R inv = (K == 2) ? (R)t.isqrtn[stab_row] : (R)t.isqrtnf[stab_row];
                    const T xi = x[o];
                    T out;
                    out.x = accr[v] * inv + (R)diag * xi.x;
                    out.y = acci[v] * inv + (R)diag * xi.y;
                    y[o] = out;
                }
            }
        }
    }
    cnt.gather += n_gather;
    cnt.skip += n_skip;
    cnt.miss += n_miss;
    __syncthreads();  // shared memory is restaged by the next call
}

__device__ __forceinline__ void flush_counts(Counts c, unsigned long long* counters) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c.gather += __shfl_xor_sync(0xffffffffu, c.gather, o);
        c.skip += __shfl_xor_sync(0xffffffffu, c.skip, o);
        c.miss += __shfl_xor_sync(0xffffffffu, c.miss, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (c.gather) atomicAdd(counters + 0, c.gather);
        if (c.skip) atomicAdd(counters + 1, c.skip);
        if (c.miss) atomicAdd(counters + 2, c.miss);
    }
}

template <typename W, bool CH, int K, int NV, int NS>
__global__ void __launch_bounds__(BLOCK, hx_min_blocks(sizeof(W), NV, K)) hx_kernel(HxArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    Counts c;
    hx_body<W, CH, K, NV, NS>(a, smem, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, a.D,
                              (int64_t)gridDim.x * blockDim.x, c);
    flush_counts(c, a.counters);
}

// All sectors of a batch in one launch.  Rows of all sectors form one index
// space (sector s owns [row_off[s], row_off[s+1])); block b takes the
// contiguous range [b*chunk, (b+1)*chunk) and, for every sector that range
// meets, stages that sector's tables and processes its rows in a
// block-stride loop.  Vectors are concatenated: sector s's block of nvec
// vectors starts at element nvec*row_off[s] of x and y.
template <typename W, bool CH, int K, int NV, int NS>
__global__ void __launch_bounds__(BLOCK, hx_min_blocks(sizeof(W), NV, K))
    hx_batch_kernel(const HxArgs* __restrict__ desc, const int64_t* __restrict__ row_off, int n_sec, int64_t chunk,
                    const void* x, void* y, int nvec, const int* __restrict__ x_step, int64_t x_step_elems,
                    unsigned long long* counters, int blocks, const int* __restrict__ active) {
    using T = typename Val<K>::T;
    // optional device-side block index: x advances by x_step_elems per step
    // (lets one captured launch serve every step of a block Lanczos run)
    if (x_step) x = (const T*)x + (int64_t)(*x_step) * x_step_elems;
    extern __shared__ __align__(16) uint8_t smem[];
    const int64_t total = row_off[n_sec];
    const int64_t g0 = (int64_t)blockIdx.x * chunk;
    const int64_t g1 = min(total, g0 + chunk);
    Counts c;
    if (g0 < g1) {
        // first sector meeting [g0, g1)
        int lo = 0, hi = n_sec - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_off[mid] <= g0) lo = mid;
            else hi = mid - 1;
        }
        for (int sct = lo; sct < n_sec && row_off[sct] < g1; ++sct) {
            if (active && !active[sct]) continue;  // uniform over the block
            HxArgs a = desc[sct];
            a.nvec = nvec;
            a.blocks = blocks;
            const int64_t off = row_off[sct];
            a.x = (const T*)x + (int64_t)a.nvec * off;
            a.y = (T*)y + (int64_t)a.nvec * off;
            const int64_t b = max(g0, off) - off, e = min(g1, row_off[sct + 1]) - off;
            hx_body<W, CH, K, NV, NS>(a, smem, b + threadIdx.x, e, (int64_t)blockDim.x, c);
        }
    }
    flush_counts(c, counters);
}


// Resident blocks per SM of one instantiation at `smem` bytes (cached per
// instantiation for the last size asked).
template <typename KernelT>
static ed_status occupancy(KernelT k, size_t smem, int& cfg_smem, int& cfg_per_sm, int& cfg_sms) {
    if ((int)smem != cfg_smem) {
        ED_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, sms = 0, per_sm = 0;
        ED_CUDA(cudaGetDevice(&dev));
        ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        ED_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BLOCK, smem));
        if (per_sm < 1) return fail(ED_ERR_TABLE_TOO_LARGE, "H.x shared memory (%zu bytes) exceeds the device limit", smem);
        cfg_smem = (int)smem;
        cfg_per_sm = per_sm;
        cfg_sms = sms;
    }
    return ED_OK;
}

template <typename W, bool CH, int K, int NV, int NS>
static ed_status launch(const HxArgs& a, size_t smem, cudaStream_t s) {
    auto k = hx_kernel<W, CH, K, NV, NS>;
    static int cfg_smem = -1, cfg_per_sm = 0, cfg_sms = 0;  // per instantiation
    const ed_status st = occupancy(k, smem, cfg_smem, cfg_per_sm, cfg_sms);
    if (st != ED_OK) return st;
    const int per_sm = std::min(cfg_per_sm, std::max(1, a.blocks));
    int64_t grid = std::min<int64_t>((int64_t)cfg_sms * per_sm, (a.D + BLOCK - 1) / BLOCK);
    if (grid < 1) grid = 1;
    k<<<(unsigned)grid, BLOCK, smem, s>>>(a);
    ED_CUDA(cudaGetLastError());
    return ED_OK;
}

template <typename W, bool CH, int K, int NV>
static ed_status launch_ns(const HxArgs& a, size_t smem, int n_sub, bool ns_ok, cudaStream_t s) {
    if (ns_ok) {
        if (n_sub == 2) return launch<W, CH, K, NV, 2>(a, smem, s);
        if (n_sub == 3) return launch<W, CH, K, NV, 3>(a, smem, s);
        if (n_sub == 4) return launch<W, CH, K, NV, 4>(a, smem, s);
    }
    return launch<W, CH, K, NV, 0>(a, smem, s);
}

template <typename W, bool CH, int K>
static ed_status launch_nv(const HxArgs& a, size_t smem, int n_sub, bool ns_ok, cudaStream_t s) {
    return a.nvec == 1 ? launch_ns<W, CH, K, 1>(a, smem, n_sub, ns_ok, s)
                       : launch_ns<W, CH, K, MAXV>(a, smem, n_sub, ns_ok, s);
}

template <typename W, bool CH, int K, int NV, int NS>
static ed_status launch_batch(const BatchLaunch& L, cudaStream_t s) {
    auto k = hx_batch_kernel<W, CH, K, NV, NS>;
    static int cfg_smem = -1, cfg_per_sm = 0, cfg_sms = 0;  // per instantiation
    const ed_status st = occupancy(k, L.smem, cfg_smem, cfg_per_sm, cfg_sms);
    if (st != ED_OK) return st;
    const int per_sm = std::min(cfg_per_sm, std::max(1, L.blocks));
    const int64_t grid = std::max<int64_t>(1, (int64_t)cfg_sms * per_sm * std::max(1, L.waves));
    const int64_t chunk = std::max<int64_t>(1, (L.total_rows + grid - 1) / grid);
    const int64_t nblk = (L.total_rows + chunk - 1) / chunk;
    k<<<(unsigned)nblk, BLOCK, L.smem, s>>>(L.desc, L.row_off, L.n_sec, chunk, L.x, L.y, L.nvec, L.x_step,
                                               L.x_step_elems, L.counters, L.blocks, L.active);
    ED_CUDA(cudaGetLastError());
    return ED_OK;
}

template <typename W, bool CH, int K>
static ed_status batch_nv(const BatchLaunch& L, cudaStream_t s) {
    auto ns = [&](auto nvtag) -> ed_status {
        constexpr int NV = decltype(nvtag)::value;
        if (L.ns_ok) {
            if (L.n_sub == 2) return launch_batch<W, CH, K, NV, 2>(L, s);
            if (L.n_sub == 3) return launch_batch<W, CH, K, NV, 3>(L, s);
            if (L.n_sub == 4) return launch_batch<W, CH, K, NV, 4>(L, s);
        }
        return launch_batch<W, CH, K, NV, 0>(L, s);
    };
    return L.nvec == 1 ? ns(std::integral_constant<int, 1>{}) : ns(std::integral_constant<int, MAXV>{});
}

// entry points of one value kind (defined by ed_apply_kind.cuh per TU)
template <int K>
ed_status apply_launch_kind(const HxArgs& a, size_t smem, int n_sub, bool ns_ok, bool w8, bool chunked, cudaStream_t s) {
    if (w8) return chunked ? launch_nv<uint64_t, true, K>(a, smem, n_sub, ns_ok, s)
                           : launch_nv<uint64_t, false, K>(a, smem, n_sub, ns_ok, s);
    return chunked ? launch_nv<uint32_t, true, K>(a, smem, n_sub, ns_ok, s)
                   : launch_nv<uint32_t, false, K>(a, smem, n_sub, ns_ok, s);
}

template <int K>
ed_status apply_batch_kind(const BatchLaunch& L, cudaStream_t s) {
    if (L.w8) return L.chunked ? batch_nv<uint64_t, true, K>(L, s) : batch_nv<uint64_t, false, K>(L, s);
    return L.chunked ? batch_nv<uint32_t, true, K>(L, s) : batch_nv<uint32_t, false, K>(L, s);
}

}  // namespace ed
