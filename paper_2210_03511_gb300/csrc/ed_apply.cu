// y = H x in the symmetry-adapted basis (pull form of Alg. "Parallel
// matrix-vector multiply for a non-branching term", summed over all terms as in
// Eq. branchingsum).
//
// Work decomposition.  A warp takes a batch of R consecutive rows.  For every
// (row, flip term) pair it tests whether the term acts (the two spins differ)
// with one ballot per 32 terms, and compacts the acting pairs into a per-warp
// list in shared memory, ordered by row.  The list is then processed 32 items
// per round, one item per lane, so no lane idles on a term that does not act
// and rows of different length share rounds.  For an item, the image
// tau = sigma ^ mask is reduced to its representative by sublattice coding
// (tables in shared memory), located by Limits + binary search, and
// contributes
//     conj(h) chi(g_tau) sqrt(|Stab tau~| / |Stab sigma_i|) x_j
// to y_i: H is Hermitian, H_ij = conj(H_ji), and H_ji is the matrix element
// of Eq. matrixelementrepresentatives with the conj(chi) reading.  Each row's
// sum is formed by warp reductions over the lanes holding its items, in a
// fixed order, and y_i is written once by the lane that owns row i: no
// atomics, deterministic.  The Ising part is diagonal; it is counted with
// ballots over the bonds of each coupling class.
#include <algorithm>

#include "ed_device.cuh"
#include "ed_internal.h"

namespace ed {

struct HxArgs {
    DevTables dt;
    const void* reps;
    const uint16_t* stab;
    const uint32_t* dir_base;
    const uint8_t* dir_q;
    const uint32_t* limits;
    int L, S;
    const FlipTerm* flips;
    int n_flip;
    const int8_t* diag_pos;       // [2*n_diag_bonds] bit positions, bonds sorted by class
    const DiagClass* diag_cls;
    int n_diag_cls, n_diag_bonds;
    const double* jhs;            // [n_jc][G+1] jhalf_c * sqrt(n) for real kinds (class c of each term)
    const uint8_t* jcls;          // [n_flip] class of each flip term
    int n_jc;
    const void* x;
    void* y;
    int nvec;
    int64_t D;
    unsigned long long* counters;  // [0] gathers, [1] incompatible images, [2] missing representatives
};

// value kinds: 0 = f64, 1 = f32, 2 = c128, 3 = c64
template <int K> struct Val;
template <> struct Val<0> { using T = double; using R = double; static constexpr bool cplx = false; };
template <> struct Val<1> { using T = float; using R = float; static constexpr bool cplx = false; };
template <> struct Val<2> { using T = double2; using R = double; static constexpr bool cplx = true; };
template <> struct Val<3> { using T = float2; using R = float; static constexpr bool cplx = true; };

constexpr int MAXV = 8;
constexpr int ROWS = 4;           // rows per warp batch
constexpr int BLOCK = 256;        // threads per block
constexpr int WARPS = BLOCK / 32;

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename W>
__device__ __forceinline__ W shfl_w(W v, int src) {
    if constexpr (sizeof(W) == 8) {
        const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)v, src);
        const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(v >> 32), src);
        return ((W)hi << 32) | (W)lo;
    } else {
        return __shfl_sync(0xffffffffu, v, src);
    }
}

template <typename W, bool CH, int NS>
__device__ __forceinline__ void rep_of(W tau, const TabView<CH>& t, W& r, int& g, int& nst, bool& cp) {
    if constexpr (NS >= 2 && NS <= 4) find_rep_ns<W, CH, NS>(tau, t, r, g, nst, cp);
    else find_rep<W, CH>(tau, t, r, g, nst, cp);
}

// Shared layout: [table blob][flip terms][jhs table][jcls][diag positions]
// [Limits directory][per-warp item lists].
struct SmemLayout {
    size_t flip, jhs, jcls, diag, dir, items, total;
    int item_cap;
};

__host__ __device__ inline SmemLayout smem_layout(size_t blob, int n_flip, int n_jc, int G, int n_diag_bonds, int S) {
    SmemLayout l;
    auto up16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
    l.flip = up16(blob);
    l.jhs = up16(l.flip + (size_t)n_flip * sizeof(FlipTerm));
    l.jcls = up16(l.jhs + (size_t)n_jc * (G + 1) * 8);
    l.diag = up16(l.jcls + (size_t)n_flip);
    l.dir = up16(l.diag + 2 * (size_t)n_diag_bonds);
    l.items = up16(l.dir + (size_t)(S + 1) * 4 + S);
    l.item_cap = ROWS * n_flip;
    l.total = up16(l.items + (size_t)WARPS * l.item_cap * 2);
    return l;
}

template <typename W, bool CH, int K, int NV, int NS>
__global__ void __launch_bounds__(BLOCK) hx_kernel(HxArgs a) {
    using V = Val<K>;
    using T = typename V::T;
    using R = typename V::R;
    extern __shared__ __align__(16) uint8_t smem[];
    const SmemLayout lay = smem_layout(a.dt.blob_bytes, a.n_flip, a.n_jc, a.dt.G, a.n_diag_bonds, a.S);
    stage_blob(smem, a.dt.blob, a.dt.blob_bytes);
    stage_blob(smem + lay.flip, (const uint8_t*)a.flips, (size_t)a.n_flip * sizeof(FlipTerm));
    if (!V::cplx) stage_blob(smem + lay.jhs, (const uint8_t*)a.jhs, (size_t)a.n_jc * (a.dt.G + 1) * 8);
    for (int i = threadIdx.x; i < a.n_flip; i += blockDim.x) smem[lay.jcls + i] = a.jcls[i];
    for (int i = threadIdx.x; i < 2 * a.n_diag_bonds; i += blockDim.x) ((int8_t*)(smem + lay.diag))[i] = a.diag_pos[i];
    uint32_t* dir_base = (uint32_t*)(smem + lay.dir);
    uint8_t* dir_q = (uint8_t*)(dir_base + a.S + 1);
    for (int i = threadIdx.x; i <= a.S; i += blockDim.x) dir_base[i] = a.dir_base[i];
    for (int i = threadIdx.x; i < a.S; i += blockDim.x) dir_q[i] = a.dir_q[i];
    __syncthreads();
    const TabView<CH> t = tab_view<CH>(smem, a.dt);
    const FlipTerm* flips = (const FlipTerm*)(smem + lay.flip);
    const double* jhs = (const double*)(smem + lay.jhs);
    const uint8_t* jcls = smem + lay.jcls;
    const int8_t* dpos = (const int8_t*)(smem + lay.diag);
    const int warp_in_block = threadIdx.x >> 5;
    uint16_t* items = (uint16_t*)(smem + lay.items) + (size_t)warp_in_block * lay.item_cap;
    const W* __restrict__ reps = (const W*)a.reps;
    const T* __restrict__ x = (const T*)a.x;
    T* __restrict__ y = (T*)a.y;
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t D = a.D;
    const int nvec = NV == 1 ? 1 : a.nvec;
    const int G1 = a.dt.G + 1;
    const int64_t n_batches = (D + ROWS - 1) / ROWS;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long n_gather = 0, n_skip = 0, n_miss = 0;

    for (int64_t batch = warp_global; batch < n_batches; batch += n_warps) {
        const int64_t r0 = batch * ROWS;
        const int nrows = (int)min((int64_t)ROWS, D - r0);
        // lane r < nrows owns row r0 + r
        W s_own = 0;
        int stab_own = 1;
        if (lane < nrows) {
            s_own = reps[r0 + lane];
            stab_own = a.stab[r0 + lane];
        }
        // ---- diagonal (Ising) part and the compacted list of acting flip terms
        double diag_own = 0.0;
        int n_items = 0;
        for (int r = 0; r < nrows; ++r) {
            const W s = shfl_w<W>(s_own, r);
            double dg = 0.0;
            for (int c = 0; c < a.n_diag_cls; ++c) {
                const DiagClass dc = a.diag_cls[c];
                int anti = 0;
                for (int b0 = dc.first; b0 < dc.first + dc.count; b0 += 32) {
                    const int b = b0 + lane;
                    const bool ap = b < dc.first + dc.count &&
                                    (((s >> dpos[2 * b]) ^ (s >> dpos[2 * b + 1])) & 1);
                    anti += __popc(__ballot_sync(0xffffffffu, ap));
                }
                dg += 0.25 * dc.J * (double)(dc.count - 2 * anti);
            }
            if (lane == r) diag_own = dg;
            for (int t0 = 0; t0 < a.n_flip; t0 += 32) {
                const int tt = t0 + lane;
                bool act = false;
                if (tt < a.n_flip) {
                    const FlipTerm& ft = flips[tt];
                    act = (((s >> ft.pa) ^ (s >> ft.pb)) & 1) != 0;
                }
                const uint32_t m = __ballot_sync(0xffffffffu, act);
                if (act) items[n_items + __popc(m & lt_mask)] = (uint16_t)((r << 8) | tt);
                n_items += __popc(m);
            }
        }
        __syncwarp();
        R accr[NV], acci[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { accr[v] = 0; acci[v] = 0; }
        // ---- rounds of 32 items
        for (int base = 0; base < n_items; base += 32) {
            const int j = base + lane;
            const bool active = j < n_items;
            const uint32_t item = active ? items[j] : 0u;
            const int row = (int)(item >> 8);
            const int tt = (int)(item & 0xFFu);
            const W s = shfl_w<W>(s_own, row);
            R vr[NV], vi[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) { vr[v] = 0; vi[v] = 0; }
            if (active) {
                const FlipTerm ft = flips[tt];
                const W tau = s ^ (((W)1 << ft.pa) | ((W)1 << ft.pb));
                W rp;
                int g, nst;
                bool cp;
                rep_of<W, CH, NS>(tau, t, rp, g, nst, cp);
                if (!cp) {
                    ++n_skip;
                } else {
                    const int64_t jx = find_index<W>(rp, reps, dir_base, dir_q, a.limits, a.L);
                    if (jx < 0) {
                        ++n_miss;
                    } else {
                        ++n_gather;
                        if constexpr (!V::cplx) {
                            // jhalf * sqrt(n) from the table; real chi(g) = +-1 enters as a sign bit
                            R c;
                            if constexpr (K == 0) {
                                const double cd = jhs[jcls[tt] * G1 + nst];
                                c = __longlong_as_double(__double_as_longlong(cd) ^ ((long long)t.chi_neg[g] << 63));
                            } else {
                                c = (R)ft.jhalf * t.chif[g].x * t.sqrtnf[nst];
                            }
#pragma unroll
                            for (int v = 0; v < NV; ++v)
                                if (v < nvec) vr[v] = c * x[(int64_t)v * D + jx];
                        } else {
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
                                    vr[v] = cr * xj.x - ci * xj.y;
                                    vi[v] = cr * xj.y + ci * xj.x;
                                }
                        }
                    }
                }
            }
            // rows present in this round are contiguous: [first, last]
            const int r_first = __shfl_sync(0xffffffffu, row, 0);
            const int last_lane = min(31, n_items - 1 - base);
            const int r_last = __shfl_sync(0xffffffffu, row, last_lane);
            for (int rr = r_first; rr <= r_last; ++rr) {
                const bool mine = active && row == rr;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (v < nvec) {
                        const R sr = warp_sum<R>(mine ? vr[v] : (R)0);
                        if (lane == rr) accr[v] += sr;
                        if constexpr (V::cplx) {
                            const R si = warp_sum<R>(mine ? vi[v] : (R)0);
                            if (lane == rr) acci[v] += si;
                        }
                    }
                }
            }
        }
        __syncwarp();
        // ---- y_i = acc_i / sqrt(|Stab sigma_i|) + diag_i x_i
        if (lane < nrows) {
            const int64_t row_g = r0 + lane;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (v < nvec) {
                    const int64_t o = (int64_t)v * D + row_g;
                    if constexpr (!V::cplx) {
                        const R inv = (K == 0) ? (R)t.isqrtn[stab_own] : (R)t.isqrtnf[stab_own];
                        y[o] = accr[v] * inv + (R)diag_own * x[o];
                    } else {
                        const R inv = (K == 2) ? (R)t.isqrtn[stab_own] : (R)t.isqrtnf[stab_own];
                        const T xi = x[o];
                        T out;
                        out.x = accr[v] * inv + (R)diag_own * xi.x;
                        out.y = acci[v] * inv + (R)diag_own * xi.y;
                        y[o] = out;
                    }
                }
            }
        }
    }
    n_gather = warp_sum<unsigned long long>(n_gather);
    n_skip = warp_sum<unsigned long long>(n_skip);
    n_miss = warp_sum<unsigned long long>(n_miss);
    if (lane == 0) {
        if (n_gather) atomicAdd(a.counters + 0, n_gather);
        if (n_skip) atomicAdd(a.counters + 1, n_skip);
        if (n_miss) atomicAdd(a.counters + 2, n_miss);
    }
}

static SmemLayout layout_for(const ed_hamiltonian* h) {
    const ed_basis* b = h->basis;
    return smem_layout(b->dt.blob_bytes, h->n_flip, h->n_jc, b->dt.G, h->n_diag_bonds, 1 << b->ht.m);
}

size_t apply_smem_bytes(const ed_hamiltonian* h, ed_dtype) { return layout_for(h).total; }

template <typename W, bool CH, int K, int NV, int NS>
static ed_status launch(const HxArgs& a, size_t smem, cudaStream_t s) {
    auto k = hx_kernel<W, CH, K, NV, NS>;
    static int cfg_smem = -1, cfg_grid = 0;  // per instantiation
    if ((int)smem != cfg_smem) {
        ED_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, sms = 0, per_sm = 0;
        ED_CUDA(cudaGetDevice(&dev));
        ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        ED_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BLOCK, smem));
        if (per_sm < 1) return fail(ED_ERR_TABLE_TOO_LARGE, "H.x shared memory (%zu bytes) exceeds the device limit", smem);
        cfg_smem = (int)smem;
        cfg_grid = sms * per_sm;
    }
    const int64_t batches = (a.D + ROWS - 1) / ROWS;
    int64_t grid = std::min<int64_t>(cfg_grid, (batches + WARPS - 1) / WARPS);
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

template <typename W, bool CH>
static ed_status dispatch_k(const HxArgs& a, size_t smem, ed_dtype dt, int n_sub, bool ns_ok, cudaStream_t s) {
    switch (dt) {
        case ED_F64: return launch_nv<W, CH, 0>(a, smem, n_sub, ns_ok, s);
        case ED_F32: return launch_nv<W, CH, 1>(a, smem, n_sub, ns_ok, s);
        case ED_C128: return launch_nv<W, CH, 2>(a, smem, n_sub, ns_ok, s);
        case ED_C64: return launch_nv<W, CH, 3>(a, smem, n_sub, ns_ok, s);
    }
    return fail(ED_ERR_ARG, "bad dtype");
}

ed_status apply_launch(const ed_hamiltonian* h, ed_dtype dt, const void* x, void* y, int nvec, cudaStream_t s) {
    const ed_basis* b = h->basis;
    if (h->n_flip > 256) return fail(ED_ERR_ARG, "more than 256 flip terms are not supported");
    HxArgs a{};
    a.dt = b->dt;
    a.reps = b->reps.p;
    a.stab = (const uint16_t*)b->stab.p;
    const uint8_t* dir = (const uint8_t*)b->limits.p;
    a.dir_base = (const uint32_t*)dir;
    a.dir_q = dir + b->dir_q_off();
    a.limits = (const uint32_t*)(dir + b->dir_lim_off());
    a.L = b->prefix_bits;
    a.S = 1 << b->ht.m;
    a.flips = (const FlipTerm*)h->d_flips.p;
    a.n_flip = h->n_flip;
    a.diag_pos = (const int8_t*)h->d_diag_pos.p;
    a.diag_cls = (const DiagClass*)h->d_diag_cls.p;
    a.n_diag_cls = h->n_diag_cls;
    a.n_diag_bonds = h->n_diag_bonds;
    a.jhs = (const double*)h->d_jhs.p;
    a.jcls = (const uint8_t*)h->d_jcls.p;
    a.n_jc = h->n_jc;
    a.x = x;
    a.y = y;
    a.nvec = nvec;
    a.D = b->dim;
    a.counters = (unsigned long long*)h->d_counters.p;
    ED_CUDA(cudaMemsetAsync(h->d_counters.p, 0, 24, s));
    const size_t smem = layout_for(h).total;
    const bool w8 = b->word == 8, ch = b->dt.chunk_lo > 0;
    const bool ns_ok = b->dt.dl_stride == 4;
    const int n_sub = b->ht.n_sub;
    if (w8) return ch ? dispatch_k<uint64_t, true>(a, smem, dt, n_sub, ns_ok, s)
                      : dispatch_k<uint64_t, false>(a, smem, dt, n_sub, ns_ok, s);
    return ch ? dispatch_k<uint32_t, true>(a, smem, dt, n_sub, ns_ok, s)
              : dispatch_k<uint32_t, false>(a, smem, dt, n_sub, ns_ok, s);
}

}  // namespace ed
