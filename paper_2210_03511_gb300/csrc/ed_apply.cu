// y = H x in the symmetry-adapted basis (pull form of Alg. "Parallel
// matrix-vector multiply for a non-branching term", summed over all terms as in
// Eq. branchingsum).
//
// One warp owns one row sigma_i at a time, so y_i is written once and no
// atomics are needed.  The Ising part is diagonal and computed from bond
// parities grouped by coupling.  Lanes take the off-diagonal flip terms: for a
// site pair with opposite spins the image tau = sigma ^ mask is reduced to its
// representative by sublattice coding (tables in shared memory), located by
// Limits + binary search, and contributes
//     conj(h) chi(g_tau) sqrt(|Stab tau~| / |Stab sigma_i|) x_j
// because H is Hermitian: H_ij = conj(H_ji) and H_ji is the matrix element of
// Eq. matrixelementrepresentatives with the conj(chi) reading.
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
    const int8_t* diag_pos;
    const DiagClass* diag_cls;
    int n_diag_cls, n_diag_bonds;
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

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename W, bool CH, int K, int NV>
__global__ void __launch_bounds__(1024, 1) hx_kernel(HxArgs a) {
    using V = Val<K>;
    using T = typename V::T;
    using R = typename V::R;
    extern __shared__ __align__(16) uint8_t smem[];
    // shared layout: [table blob][flip terms][diag positions][Limits directory]
    const size_t flip_off = a.dt.blob_bytes;
    const size_t diag_off = flip_off + (size_t)a.n_flip * sizeof(FlipTerm);
    const size_t dir_off = (diag_off + 2 * (size_t)a.n_diag_bonds + 15) & ~(size_t)15;
    stage_blob(smem, a.dt.blob, a.dt.blob_bytes);
    stage_blob(smem + flip_off, (const uint8_t*)a.flips, (size_t)a.n_flip * sizeof(FlipTerm));
    for (int i = threadIdx.x; i < 2 * a.n_diag_bonds; i += blockDim.x) ((int8_t*)(smem + diag_off))[i] = a.diag_pos[i];
    uint32_t* dir_base = (uint32_t*)(smem + dir_off);
    uint8_t* dir_q = (uint8_t*)(dir_base + a.S + 1);
    for (int i = threadIdx.x; i <= a.S; i += blockDim.x) dir_base[i] = a.dir_base[i];
    for (int i = threadIdx.x; i < a.S; i += blockDim.x) dir_q[i] = a.dir_q[i];
    __syncthreads();
    const TabView<CH> t = tab_view<CH>(smem, a.dt);
    const FlipTerm* flips = (const FlipTerm*)(smem + flip_off);
    const int8_t* dpos = (const int8_t*)(smem + diag_off);
    const W* __restrict__ reps = (const W*)a.reps;
    const T* __restrict__ x = (const T*)a.x;
    T* __restrict__ y = (T*)a.y;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long n_gather = 0, n_skip = 0, n_miss = 0;
    const int nvec = NV == 1 ? 1 : a.nvec;
    const int64_t D = a.D;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < D; row += nwarps) {
        const W s = reps[row];
        // Ising part: sum_c J_c/4 (n_c - 2 * antiparallel_c)
        double diag = 0.0;
        for (int c = 0; c < a.n_diag_cls; ++c) {
            const DiagClass dc = a.diag_cls[c];
            int anti = 0;
            for (int b = dc.first + lane; b < dc.first + dc.count; b += 32)
                anti += (int)(((s >> dpos[2 * b]) ^ (s >> dpos[2 * b + 1])) & 1);
            anti = __reduce_add_sync(0xffffffffu, anti);
            diag += 0.25 * dc.J * (double)(dc.count - 2 * anti);
        }
        R accr[NV], acci[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { accr[v] = 0; acci[v] = 0; }
        for (int f = lane; f < a.n_flip; f += 32) {
            const FlipTerm ft = flips[f];
            const int ba = (int)((s >> ft.pa) & 1), bb = (int)((s >> ft.pb) & 1);
            if (ba == bb) continue;
            const W tau = s ^ (((W)1 << ft.pa) | ((W)1 << ft.pb));
            W r;
            int g, nst;
            bool cp;
            find_rep<W, CH>(tau, t, r, g, nst, cp);
            if (!cp) { ++n_skip; continue; }
            const int64_t j = find_index<W>(r, reps, dir_base, dir_q, a.limits, a.L);
            if (j < 0) { ++n_miss; continue; }
            ++n_gather;
            if constexpr (!V::cplx) {
                R c;
                if constexpr (K == 0) c = (R)ft.jhalf * t.chi[g].x * t.sqrtn[nst];
                else c = (R)ft.jhalf * t.chif[g].x * t.sqrtnf[nst];
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    if (v < nvec) accr[v] += c * x[(int64_t)v * D + j];
            } else {
                // h = jhalf + i * sum_t k_t s^z_c (a down ? +1 : -1)
                double him = 0.0;
                if (ft.pc0 >= 0) him += ft.k0 * (((s >> ft.pc0) & 1) ? 0.5 : -0.5);
                if (ft.pc1 >= 0) him += ft.k1 * (((s >> ft.pc1) & 1) ? 0.5 : -0.5);
                if (ba) him = -him;
                R cr, ci;
                if constexpr (K == 2) {
                    const double2 ch = t.chi[g];
                    const double sq = t.sqrtn[nst];
                    // conj(h) * chi = (jh - i him)(chr + i chi)
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
                        const T xj = x[(int64_t)v * D + j];
                        accr[v] += cr * xj.x - ci * xj.y;
                        acci[v] += cr * xj.y + ci * xj.x;
                    }
            }
        }
        const int ni = a.stab[row];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v < nvec) {
                const R sr = warp_sum<R>(accr[v]);
                R si = 0;
                if constexpr (V::cplx) si = warp_sum<R>(acci[v]);
                if (lane == 0) {
                    const int64_t o = (int64_t)v * D + row;
                    if constexpr (!V::cplx) {
                        const R inv = (K == 0) ? (R)t.isqrtn[ni] : (R)t.isqrtnf[ni];
                        y[o] = sr * inv + (R)diag * x[o];
                    } else {
                        const R inv = (K == 2) ? (R)t.isqrtn[ni] : (R)t.isqrtnf[ni];
                        const T xi = x[o];
                        T out;
                        out.x = sr * inv + (R)diag * xi.x;
                        out.y = si * inv + (R)diag * xi.y;
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

static size_t smem_bytes(const ed_hamiltonian* h) {
    const ed_basis* b = h->basis;
    const size_t flip_off = b->dt.blob_bytes;
    const size_t diag_off = flip_off + (size_t)h->n_flip * sizeof(FlipTerm);
    const size_t dir_off = (diag_off + 2 * (size_t)h->n_diag_bonds + 15) & ~(size_t)15;
    const size_t S = (size_t)1 << b->ht.m;
    return dir_off + (S + 1) * 4 + S;
}

size_t apply_smem_bytes(const ed_hamiltonian* h, ed_dtype) { return smem_bytes(h); }

template <typename W, bool CH, int K, int NV>
static ed_status launch(const HxArgs& a, size_t smem, cudaStream_t s) {
    auto k = hx_kernel<W, CH, K, NV>;
    // per instantiation: block size with the most resident warps, and the grid
    static int cfg_smem = -1, cfg_block = 0, cfg_grid = 0;
    if ((int)smem != cfg_smem) {
        ED_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, sms = 0;
        ED_CUDA(cudaGetDevice(&dev));
        ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int best_warps = 0, best_block = 0, best_per_sm = 0;
        for (int bs : {256, 512, 1024}) {
            int per_sm = 0;
            ED_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, bs, smem));
            if (per_sm * bs / 32 > best_warps) { best_warps = per_sm * bs / 32; best_block = bs; best_per_sm = per_sm; }
        }
        if (best_warps == 0)
            return fail(ED_ERR_TABLE_TOO_LARGE, "H.x shared memory (%zu bytes) exceeds the device limit", smem);
        cfg_smem = (int)smem;
        cfg_block = best_block;
        cfg_grid = sms * best_per_sm;
    }
    const int64_t warps_per_block = cfg_block / 32;
    int64_t grid = std::min<int64_t>(cfg_grid, (a.D + warps_per_block - 1) / warps_per_block);
    if (grid < 1) grid = 1;
    k<<<(unsigned)grid, cfg_block, smem, s>>>(a);
    ED_CUDA(cudaGetLastError());
    return ED_OK;
}

template <typename W, bool CH, int K>
static ed_status launch_nv(const HxArgs& a, size_t smem, cudaStream_t s) {
    return a.nvec == 1 ? launch<W, CH, K, 1>(a, smem, s) : launch<W, CH, K, MAXV>(a, smem, s);
}

template <typename W, bool CH>
static ed_status dispatch_k(const HxArgs& a, size_t smem, ed_dtype dt, cudaStream_t s) {
    switch (dt) {
        case ED_F64: return launch_nv<W, CH, 0>(a, smem, s);
        case ED_F32: return launch_nv<W, CH, 1>(a, smem, s);
        case ED_C128: return launch_nv<W, CH, 2>(a, smem, s);
        case ED_C64: return launch_nv<W, CH, 3>(a, smem, s);
    }
    return fail(ED_ERR_ARG, "bad dtype");
}

ed_status apply_launch(const ed_hamiltonian* h, ed_dtype dt, const void* x, void* y, int nvec, cudaStream_t s) {
    const ed_basis* b = h->basis;
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
    a.x = x;
    a.y = y;
    a.nvec = nvec;
    a.D = b->dim;
    a.counters = (unsigned long long*)h->d_counters.p;
    ED_CUDA(cudaMemsetAsync(h->d_counters.p, 0, 24, s));
    const size_t smem = smem_bytes(h);
    const bool w8 = b->word == 8, ch = b->dt.chunk_lo > 0;
    if (w8) return ch ? dispatch_k<uint64_t, true>(a, smem, dt, s) : dispatch_k<uint64_t, false>(a, smem, dt, s);
    return ch ? dispatch_k<uint32_t, true>(a, smem, dt, s) : dispatch_k<uint32_t, false>(a, smem, dt, s);
}

}  // namespace ed
