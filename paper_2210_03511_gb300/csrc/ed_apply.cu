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
constexpr int BLOCK = 256;        // threads per block
constexpr int MAXW = 8;           // activity mask words per row (n_flip <= 256)

template <typename W, bool CH, int NS>
__device__ __forceinline__ void rep_of(W tau, const TabView<CH>& t, W& r, int& g, int& nst, bool& cp) {
    if constexpr (NS >= 2 && NS <= 4) find_rep_ns<W, CH, NS>(tau, t, r, g, nst, cp);
    else find_rep<W, CH>(tau, t, r, g, nst, cp);
}

// Shared layout: [table blob][flip terms][packed (pa,pb)][jhs table][jcls]
// [class masks][Limits directory].
struct SmemLayout {
    size_t flip, pab, jhs, jcls, cmask, dir, total;
};

__host__ __device__ inline SmemLayout smem_layout(size_t blob, int n_flip, int n_jc, int G, int S) {
    SmemLayout l;
    auto up16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
    l.flip = up16(blob);
    l.pab = up16(l.flip + (size_t)n_flip * sizeof(FlipTerm));
    l.jhs = up16(l.pab + (size_t)n_flip * 2);
    l.jcls = up16(l.jhs + (size_t)n_jc * (G + 1) * 8);
    l.cmask = up16(l.jcls + (size_t)n_flip);
    l.dir = up16(l.cmask + (size_t)n_jc * MAXW * 4);
    l.total = up16(l.dir + (size_t)(S + 1) * 4 + S);
    return l;
}

template <typename W, bool CH, int K, int NV, int NS>
__global__ void __launch_bounds__(BLOCK, (NV == 1 && K < 2) ? 4 : 2) hx_kernel(HxArgs a) {
    using V = Val<K>;
    using T = typename V::T;
    using R = typename V::R;
    extern __shared__ __align__(16) uint8_t smem[];
    const SmemLayout lay = smem_layout(a.dt.blob_bytes, a.n_flip, a.n_jc, a.dt.G, a.S);
    stage_blob(smem, a.dt.blob, a.dt.blob_bytes);
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
    uint32_t* dir_base = (uint32_t*)(smem + lay.dir);
    uint8_t* dir_q = (uint8_t*)(dir_base + a.S + 1);
    for (int i = threadIdx.x; i <= a.S; i += blockDim.x) dir_base[i] = a.dir_base[i];
    for (int i = threadIdx.x; i < a.S; i += blockDim.x) dir_q[i] = a.dir_q[i];
    __syncthreads();
    const TabView<CH> t = tab_view<CH>(smem, a.dt);
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
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < D; row += stride) {
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
    // counters: one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_gather += __shfl_xor_sync(0xffffffffu, n_gather, o);
        n_skip += __shfl_xor_sync(0xffffffffu, n_skip, o);
        n_miss += __shfl_xor_sync(0xffffffffu, n_miss, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n_gather) atomicAdd(a.counters + 0, n_gather);
        if (n_skip) atomicAdd(a.counters + 1, n_skip);
        if (n_miss) atomicAdd(a.counters + 2, n_miss);
    }
}

static SmemLayout layout_for(const ed_hamiltonian* h) {
    const ed_basis* b = h->basis;
    return smem_layout(b->dt.blob_bytes, h->n_flip, h->n_jc, b->dt.G, 1 << b->ht.m);
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
    int64_t grid = std::min<int64_t>(cfg_grid, (a.D + BLOCK - 1) / BLOCK);
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
