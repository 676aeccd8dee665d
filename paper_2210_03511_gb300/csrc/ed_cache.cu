// Stored structure of H for repeated H.x (the Lanczos loop applies one H
// tens to hundreds of times).
//
// The matrix-free kernel (ed_apply_impl.cuh) repeats, for every gather, the
// representative search of Alg. "Sublattice coding algorithm for finding the
// representative" and the Limits + binary search of section "Distributed and
// hybrid memory parallelization".  On sectors whose basis exceeds L2 both the
// Limits entry and x_j are random DRAM accesses.  Here both searches run
// once: two passes of the same per-row walk record, for every row i and
// every gather of the pull form y_i = sum_j conj(H_ji) x_j, the column j and
// a one-byte code of its coefficient conj(h) chi(g_tau) sqrt(|Stab tau~|)
// (the row factor 1/sqrt(|Stab sigma_i|) and the Ising diagonal are kept per
// row).  H.x then streams this structure and gathers x.
//
// Column segments.  x is cut into segments of 2^seg_bits elements (chosen so
// one segment of the vector type fits comfortably in L2); the entries of each
// row are stored per segment, and H.x runs one pass per segment, so every
// pass gathers from an L2-resident slice of x instead of from all of HBM.
// Layout (rows in slices of 32, one warp per slice):
//   counts[b][row]  (u8)  entries of row `row` in segment b
//   boff[b][slice]  (u32) first entry of the slice's segment-b entries, relative
//                         to the segment's base bbase[b]; inside, the rows of
//                         the slice follow each other
//   ent[...]        (u32) (code << off_bits) | (j - b 2^seg_bits), in flip order
//                         (off_bits = 32 - the bits the occurring codes need)
//   diag[row]       (f64) Ising part of row `row`
// The coefficient of code c is ctab[c] (built once per Hamiltonian from the
// codes that occur: distinct (h, chi(g), |Stab tau~|) combinations).
#include <math.h>

#include <algorithm>
#include <vector>

#include "ed_cache.cuh"

namespace ed {

namespace {

constexpr int CMAXNB = 128;   // column segments at most

struct CacheBuild {
    HxArgs a;                      // basis and terms (x, y unused)
    int seg_bits, nb, off_bits;    // entry = (code << off_bits) | column offset
    int64_t ns, Dpad;              // slices of 32 rows, 32 * ns
    uint8_t* counts;               // [nb][Dpad]
    const uint32_t* boff;          // [nb][ns]            (pass 1)
    const uint64_t* bbase;         // [nb]                (pass 1)
    uint32_t* ent;                 //                     (pass 1)
    double* diag;                  // [D]                 (pass 0)
    const uint16_t* hmap;          // [n_flip][8] h-value id by the spins at (a, c0, c1)
    const uint16_t* chi_id;        // [G] id of the exact value chi(g)
    uint32_t n_chi, Gp1;           // code key = (h id * n_chi + chi id) * (G+1) + |Stab tau~|
    uint64_t dmask;                // bits of one site's state: 1 (spin-1/2) or 2^b - 1 (SU(N) colours)
    double diag_off;               // Ising part per pair class: jhs(1) (diag_off n_pairs - n_acting): 1/2 spin, 1 SU(N)
    uint32_t* seen;                // bit set of keys that occur  (pass 0)
    const uint8_t* code;           // key -> code               (pass 1)
    unsigned long long* counters;  // [0] entries, [1] incompatible images, [2] missing, [3] overflow
};

// One pass of the structure build over all rows, one warp per slice of 32
// rows (the per-slice offsets of pass 1 need the whole warp).  The row walk
// (activity mask, representative, index search) is that of hx_body.
template <typename W, bool CH, int NS, int PASS>
__global__ void __launch_bounds__(BLOCK, hx_min_blocks(sizeof(W), 1, 0)) cache_build_kernel(CacheBuild c) {
    extern __shared__ __align__(16) uint8_t smem[];
    const HxArgs& a = c.a;
    constexpr bool generic = !(NS >= 2 && NS <= 4);
    const HxPlan plan = hx_plan(a.dt, 0, generic, a.blocks, a.n_flip, a.n_jc, a.S);
    const SmemLayout lay = plan.lay;
    const TabView<CH> t = stage_sections<CH>(a.dt, smem, 0, plan.mask);
    stage_blob(smem + lay.flip, (const uint8_t*)a.flips, (size_t)a.n_flip * sizeof(FlipTerm));
    stage_blob(smem + lay.jhs, (const uint8_t*)a.jhs, (size_t)a.n_jc * (a.dt.G + 1) * 8);
    uint16_t* pab = (uint16_t*)(smem + lay.pab);
    uint32_t* cmask = (uint32_t*)(smem + lay.cmask);
    for (int i = threadIdx.x; i < a.n_jc * MAXW; i += blockDim.x) cmask[i] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < a.n_flip; i += blockDim.x) {
        const FlipTerm& f = ((const FlipTerm*)(smem + lay.flip))[i];
        pab[i] = (uint16_t)((uint8_t)f.pa | ((uint16_t)(uint8_t)f.pb << 8));
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
    const int64_t D = a.D;
    const int G1 = a.dt.G + 1;
    const int nw = (a.n_flip + 31) >> 5;
    const int lane = threadIdx.x & 31;
    const uint64_t segmask = ((uint64_t)1 << c.seg_bits) - 1;
    unsigned long long n_gather = 0, n_skip = 0, n_miss = 0, n_over = 0;
    uint8_t cnt[CMAXNB];
    uint16_t cur[CMAXNB], lim[CMAXNB];
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t sl = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sl < c.ns; sl += warps) {
        const int64_t row = sl * 32 + lane;
        const bool live = row < D;
        if (PASS == 0) {
            for (int b = 0; b < c.nb; ++b) cnt[b] = 0;
        } else {
            for (int b = 0; b < c.nb; ++b) {
                const uint32_t my = c.counts[(int64_t)b * c.Dpad + row];
                const uint32_t st = warp_excl_scan(my, lane);
                cur[b] = (uint16_t)st;
                lim[b] = (uint16_t)(st + my);
            }
        }
        if (live) {
            const W s = reps[row];
            uint32_t mask[MAXW];
#pragma unroll
            for (int w = 0; w < MAXW; ++w) mask[w] = 0u;
#pragma unroll
            for (int w = 0; w < MAXW; ++w) {
                if (w < nw) {
                    const int tn = min(32, a.n_flip - 32 * w);
                    uint32_t mw = 0u;
                    for (int bb = 0; bb < tn; ++bb) {
                        // a term acts iff the two sites' states differ (spins, or packed colours)
                        const uint32_t e = pab[32 * w + bb];
                        mw |= (uint32_t)((((s >> (e & 0xFFu)) ^ (s >> (e >> 8))) & (W)c.dmask) != 0) << bb;
                    }
                    mask[w] = mw;
                }
            }
            if (PASS == 0) {
                // Ising part, as in hx_body
                double diag = 0.0;
                for (int cc = 0; cc < a.n_jc; ++cc) {
                    int nact = 0, ntot = 0;
#pragma unroll
                    for (int w = 0; w < MAXW; ++w) {
                        if (w < nw) {
                            const uint32_t cm = cmask[cc * MAXW + w];
                            nact += __popc(mask[w] & cm);
                            ntot += __popc(cm);
                        }
                    }
                    diag += jhs[cc * G1 + 1] * (c.diag_off * (double)ntot - (double)nact);
                }
                c.diag[row] = diag;
            }
#pragma unroll
            for (int w = 0; w < MAXW; ++w) {
                if (w >= nw) continue;
                uint32_t mw = mask[w];
                while (mw) {
                    const int tt = 32 * w + ctz32(mw);
                    mw &= mw - 1u;
                    const uint32_t e = pab[tt];
                    // exchange the two sites' states: flip both spins, or swap two packed colours
                    const W dd = ((s >> (e & 0xFFu)) ^ (s >> (e >> 8))) & (W)c.dmask;
                    const W tau = s ^ ((dd << (e & 0xFFu)) | (dd << (e >> 8)));
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
                    const FlipTerm& ft = flips[tt];
                    uint32_t hb = (uint32_t)((s >> ft.pa) & 1);
                    if (ft.pc0 >= 0) hb |= (uint32_t)((s >> ft.pc0) & 1) << 1;
                    if (ft.pc1 >= 0) hb |= (uint32_t)((s >> ft.pc1) & 1) << 2;
                    const uint32_t key = ((uint32_t)__ldg(c.hmap + tt * 8 + hb) * c.n_chi + __ldg(c.chi_id + g)) * c.Gp1 +
                                         (uint32_t)nst;
                    const int b = (int)((uint64_t)jx >> c.seg_bits);
                    if (PASS == 0) {
                        ++cnt[b];
                        const uint32_t bit = 1u << (key & 31);
                        if (!(c.seen[key >> 5] & bit)) atomicOr(&c.seen[key >> 5], bit);
                    } else {
                        if (cur[b] < lim[b]) {
                            const uint32_t word =
                                ((uint32_t)__ldg(c.code + key) << c.off_bits) | (uint32_t)((uint64_t)jx & segmask);
                            c.ent[c.bbase[b] + c.boff[(int64_t)b * c.ns + sl] + cur[b]] = word;
                            ++cur[b];
                        } else {
                            ++n_over;
                        }
                    }
                }
            }
        }
        if (PASS == 0)
            for (int b = 0; b < c.nb; ++b) c.counts[(int64_t)b * c.Dpad + row] = live ? cnt[b] : (uint8_t)0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_gather += __shfl_xor_sync(0xffffffffu, n_gather, o);
        n_skip += __shfl_xor_sync(0xffffffffu, n_skip, o);
        n_miss += __shfl_xor_sync(0xffffffffu, n_miss, o);
        n_over += __shfl_xor_sync(0xffffffffu, n_over, o);
    }
    if (lane == 0) {
        if (n_gather) atomicAdd(c.counters + 0, n_gather);
        if (n_skip) atomicAdd(c.counters + 1, n_skip);
        if (n_miss) atomicAdd(c.counters + 2, n_miss);
        if (n_over) atomicAdd(c.counters + 3, n_over);
    }
}

// Sum of each slice's counts per segment: tot[b][sl].
__global__ void slice_totals(const uint8_t* counts, int64_t ns, int nb, uint32_t* tot) {
    const int64_t n = ns * nb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / ns, sl = i % ns;
        const uint4* p = (const uint4*)(counts + b * ns * 32 + sl * 32);  // 32 bytes, 16-aligned
        uint32_t acc = 0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint4 v = p[q];
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                acc += (w[k] & 0xFFu) + ((w[k] >> 8) & 0xFFu) + ((w[k] >> 16) & 0xFFu) + (w[k] >> 24);
        }
        tot[i] = acc;
    }
}

// boff[b][sl] = abs[b][sl] - abs[b][0]; bbase[b] = abs[b][0].
__global__ void slice_offsets(const uint64_t* abs_off, int64_t ns, int nb, uint32_t* boff, uint64_t* bbase) {
    const int64_t n = ns * nb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / ns;
        boff[i] = (uint32_t)(abs_off[i] - abs_off[b * ns]);
        if (i == b * ns) bbase[b] = abs_off[i];
    }
}

// One segment's pass of y = H x from the stored structure: one warp per
// slice of 32 rows, one lane per row.  With tens of segments a row has only a
// few entries per segment, so a pass is bound by the latency of each slice's
// dependent loads (count -> offset -> entry -> x_j); the loop therefore loads
// the next slice's count and offset, and this row's partial sum of earlier
// segments, before it walks the current entries, two at a time.  (Walking
// several slices side by side cost registers and occupancy and was slower.)
// A row's sum continues from that partial sum (no separate add per row and
// segment: FP64 arithmetic is scarce on this GPU).  In mode 0 every row sums
// its entries in the matrix-free kernel's order with the same coefficients,
// so for real vector types the result is bit-identical to it.
// AX (complex kinds): every code's coefficient is real or purely imaginary
// (real characters: Heisenberg terms real, chirality terms imaginary), so one
// entry costs two real multiply-adds instead of four.  The real codes come
// first (codes below p.n_re), so the choice is an integer compare; the table
// holds (c, c) for a real c and (-c, c) for i c, and the imaginary case takes
// x_j's parts swapped.
// PREV: modes 2 and 3 (a partial sum from earlier segments exists), a
// compile-time flag so that the one-segment pass carries no such register.
template <int K, int NV, bool AX, bool PREV>
__global__ void __launch_bounds__(BLOCK, pass_blocks(K, NV)) cache_pass_kernel(CachePass p) {
    using V = Val<K>;
    using T = typename V::T;
    using R = typename V::R;
    using CT = typename std::conditional<V::cplx, T, R>::type;
    __shared__ CT ctab[NCODE];
    for (int i = threadIdx.x; i < NCODE; i += blockDim.x) ctab[i] = ((const CT*)p.ctab)[i];
    __syncthreads();
    const T* __restrict__ x = (const T*)p.x;
    T* __restrict__ y = (T*)p.y;
    const R* __restrict__ isq = (const R*)p.isq;
    const int lane = threadIdx.x & 31;
    const int nvec = NV == 1 ? 1 : p.nvec;
    const int64_t D = p.D;
    const uint32_t ob = p.off_bits, om = (1u << ob) - 1u, n_re = p.n_re;
    const int mode = p.mode;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int64_t sl = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    uint32_t my_n = 0, bo_n = 0;
    if (sl < p.ns) {
        my_n = __ldg(p.counts + sl * 32 + lane);
        bo_n = __ldg(p.boff + sl);
    }
    for (; sl < p.ns; sl += warps) {
        const uint32_t my = my_n, bo = bo_n;
        const int64_t nx = sl + warps;
        if (nx < p.ns) {
            my_n = __ldg(p.counts + nx * 32 + lane);
            bo_n = __ldg(p.boff + nx);
        }
        const int64_t row = sl * 32 + lane;
        const bool live = row < D;
        // earlier segments' partial sum of this row (modes 2 and 3), loaded ahead of the walk
        T prev[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if constexpr (V::cplx) prev[v] = T{0, 0};
            else prev[v] = 0;
            if (PREV && v < nvec && live) prev[v] = y[(int64_t)v * D + row];
        }
        const uint32_t st = warp_excl_scan(my, lane);
        const uint32_t* __restrict__ pe = p.ent + bo + st;
        R accr[NV], acci[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if constexpr (V::cplx) { accr[v] = prev[v].x; acci[v] = prev[v].y; }
            else { accr[v] = prev[v]; acci[v] = 0; }
        }
        auto add = [&](uint32_t w) {
            const int64_t j = p.xoff + (int64_t)(w & om);
            const CT cf = ctab[w >> ob];
#pragma unroll
            for (int v = 0; v < NV; ++v)
                if (v < nvec) {
                    if constexpr (!V::cplx) {
                        accr[v] += cf * x[(int64_t)v * D + j];
                    } else if constexpr (AX) {
                        const T xj = x[(int64_t)v * D + j];
                        const bool im = (w >> ob) >= n_re;
                        accr[v] += cf.x * (im ? xj.y : xj.x);
                        acci[v] += cf.y * (im ? xj.x : xj.y);
                    } else {
                        const T xj = x[(int64_t)v * D + j];
                        accr[v] += cf.x * xj.x - cf.y * xj.y;
                        acci[v] += cf.x * xj.y + cf.y * xj.x;
                    }
                }
        };
        uint32_t k = 0;
        for (; k + 1 < my; k += 2) {
            const uint32_t w0 = __ldg(pe + k), w1 = __ldg(pe + k + 1);
            add(w0);
            add(w1);
        }
        if (k < my) add(__ldg(pe + k));
        if (!live) continue;
        R inv = 0, dg = 0;
        if (mode == 0 || mode == 3) {
            inv = isq[__ldg(p.stab + row)];
            dg = (R)__ldg(p.diag + row);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v >= nvec) continue;
            const int64_t o = (int64_t)v * D + row;
            if constexpr (!V::cplx) {
                if (mode == 0 || mode == 3) y[o] = accr[v] * inv + dg * x[o];
                else y[o] = accr[v];
            } else {
                T out;
                if (mode == 0 || mode == 3) {
                    const T xi = x[o];
                    out.x = accr[v] * inv + dg * xi.x;
                    out.y = acci[v] * inv + dg * xi.y;
                } else {
                    out.x = accr[v];
                    out.y = acci[v];
                }
                y[o] = out;
            }
        }
    }
}

// All sectors of a batch from their stored structures (one segment each),
// in one launch: warp w takes slice w of the concatenated slice list, finds
// its sector from the slices' first indices, and processes it as the mode-0
// pass of cache_pass_kernel (same sums, same order).  Vectors are those of a
// batch: sector s's nvec columns start at element nvec * row_off[s].  x may
// advance by x_step_elems per device-side step (block Lanczos graphs);
// sectors with active[s] == 0 are skipped.
template <int K, int NV>
__global__ void __launch_bounds__(BLOCK, NV == 1 ? 8 : 2)
    cache_batch_kernel(const CacheSector* __restrict__ sec, int n_sec, int64_t n_slices,
                       const int64_t* __restrict__ row_off, const void* xv, void* yv, int nvec,
                       const int* __restrict__ x_step, int64_t x_step_elems, const int* __restrict__ active) {
    using V = Val<K>;
    using T = typename V::T;
    using R = typename V::R;
    using CT = typename std::conditional<V::cplx, T, R>::type;
    const T* __restrict__ xb = (const T*)xv;
    if (x_step) xb += (int64_t)(*x_step) * x_step_elems;
    T* __restrict__ yb = (T*)yv;
    const int lane = threadIdx.x & 31;
    const int nv = NV == 1 ? 1 : nvec;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t gs = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gs < n_slices; gs += warps) {
        int lo = 0, hi = n_sec - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sec[mid].slice0 <= gs) lo = mid;
            else hi = mid - 1;
        }
        if (active && !active[lo]) continue;  // uniform over the warp
        const CacheSector& c = sec[lo];
        const int64_t ls = gs - c.slice0, row = ls * 32 + lane, D = c.D;
        const T* __restrict__ x = xb + (int64_t)nv * row_off[lo];
        T* __restrict__ y = yb + (int64_t)nv * row_off[lo];
        const CT* __restrict__ ctab;
        const R* __restrict__ isq;
        if constexpr (K == 0) ctab = (const CT*)(c.ctab + NCODE * 16);
        else if constexpr (K == 1) ctab = (const CT*)(c.ctab + NCODE * 32);
        else if constexpr (K == 2) ctab = (const CT*)c.ctab;
        else ctab = (const CT*)(c.ctab + NCODE * 24);
        if constexpr (K == 0 || K == 2) isq = (const R*)c.sq + c.G1;
        else isq = (const R*)c.sqf + c.G1;
        const uint32_t ob = c.off_bits, om = (1u << ob) - 1u;
        const uint32_t my = __ldg(c.counts + row);
        const uint32_t st = warp_excl_scan(my, lane);
        const uint32_t* __restrict__ pe = c.ent + __ldg(c.boff + ls) + st;
        R accr[NV], acci[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { accr[v] = 0; acci[v] = 0; }
        for (uint32_t k = 0; k < my; ++k) {
            const uint32_t w = __ldg(pe + k);
            const int64_t j = (int64_t)(w & om);
            const CT cf = __ldg(ctab + (w >> ob));
#pragma unroll
            for (int v = 0; v < NV; ++v)
                if (v < nv) {
                    if constexpr (!V::cplx) {
                        accr[v] += cf * x[(int64_t)v * D + j];
                    } else {
                        const T xj = x[(int64_t)v * D + j];
                        accr[v] += cf.x * xj.x - cf.y * xj.y;
                        acci[v] += cf.x * xj.y + cf.y * xj.x;
                    }
                }
        }
        if (row >= D) continue;
        const R inv = isq[__ldg(c.stab + row)];
        const R dg = (R)__ldg(c.diag + row);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v >= nv) continue;
            const int64_t o = (int64_t)v * D + row;
            if constexpr (!V::cplx) {
                y[o] = accr[v] * inv + dg * x[o];
            } else {
                const T xi = x[o];
                T out;
                out.x = accr[v] * inv + dg * xi.x;
                out.y = acci[v] * inv + dg * xi.y;
                y[o] = out;
            }
        }
    }
}

template <typename W, bool CH, int NS, int PASS>
static ed_status launch_build(const CacheBuild& c, size_t smem, cudaStream_t s) {
    auto k = cache_build_kernel<W, CH, NS, PASS>;
    static int cfg_smem = -1, cfg_per_sm = 0, cfg_sms = 0;
    const ed_status st = occupancy(k, smem, cfg_smem, cfg_per_sm, cfg_sms);
    if (st != ED_OK) return st;
    const int per_sm = std::min(cfg_per_sm, std::max(1, c.a.blocks));
    const int64_t warps_needed = c.ns;
    int64_t grid = std::min<int64_t>((int64_t)cfg_sms * per_sm, (warps_needed + (BLOCK / 32) - 1) / (BLOCK / 32));
    if (grid < 1) grid = 1;
    k<<<(unsigned)grid, BLOCK, smem, s>>>(c);
    ED_CUDA(cudaGetLastError());
    return ED_OK;
}

template <int PASS>
static ed_status build_dispatch(const CacheBuild& c, size_t smem, int n_sub, bool ns_ok, bool w8, bool ch,
                                cudaStream_t s) {
    auto go = [&](auto wtag, auto chtag) -> ed_status {
        using W = decltype(wtag);
        constexpr bool CH = decltype(chtag)::value;
        if (ns_ok) {
            if (n_sub == 2) return launch_build<W, CH, 2, PASS>(c, smem, s);
            if (n_sub == 3) return launch_build<W, CH, 3, PASS>(c, smem, s);
            if (n_sub == 4) return launch_build<W, CH, 4, PASS>(c, smem, s);
        }
        return launch_build<W, CH, 0, PASS>(c, smem, s);
    };
    if (w8) return ch ? go(uint64_t{}, std::true_type{}) : go(uint64_t{}, std::false_type{});
    return ch ? go(uint32_t{}, std::true_type{}) : go(uint32_t{}, std::false_type{});
}

template <int K, bool AX = false>
static ed_status launch_pass(const CachePass& p, int nvec, int sms, cudaStream_t s) {
    const int64_t blocks_needed = (p.ns + (BLOCK / 32) - 1) / (BLOCK / 32);
    const int per_sm = pass_blocks(K, nvec == 1 ? 1 : MAXV);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks_needed, (int64_t)sms * per_sm));
    if (p.mode >= 2) {
        if (nvec == 1) cache_pass_kernel<K, 1, AX, true><<<grid, BLOCK, 0, s>>>(p);
        else cache_pass_kernel<K, MAXV, AX, true><<<grid, BLOCK, 0, s>>>(p);
    } else {
        if (nvec == 1) cache_pass_kernel<K, 1, AX, false><<<grid, BLOCK, 0, s>>>(p);
        else cache_pass_kernel<K, MAXV, AX, false><<<grid, BLOCK, 0, s>>>(p);
    }
    ED_CUDA(cudaGetLastError());
    return ED_OK;
}

// Freed together with the structure.
struct BuildScratch {
    const Alloc* A;
    cudaStream_t s;
    std::vector<std::pair<void*, size_t>> bufs;
    void* get(size_t n) {
        void* p = A->get(n, s);
        if (p) bufs.push_back({p, n});
        return p;
    }
    ~BuildScratch() {
        cudaStreamSynchronize(s);
        for (auto& b : bufs) A->put(b.first, b.second, s);
    }
};

}  // namespace

bool cache_sector_desc(const ed_hamiltonian* h, CacheSector& d) {
    const HCache& c = h->cache;
    if (!c.valid || c.nb != 1) return false;
    const ed_basis* b = h->basis;
    d.counts = (const uint8_t*)c.counts.p;
    d.boff = (const uint32_t*)c.boff.p;
    d.ent = (const uint32_t*)c.ent.p;
    d.diag = (const double*)c.diag.p;
    d.stab = (const uint16_t*)b->stab.p;
    d.ctab = (const uint8_t*)c.ctab.p;
    d.sq = b->dt.blob + b->dt.off_sqrt;
    d.sqf = b->dt.blob + b->dt.off_sqrtf;
    d.D = b->dim;
    d.ns = c.ns;
    d.slice0 = 0;
    d.G1 = b->ht.G + 1;
    d.off_bits = (uint32_t)c.off_bits;
    return true;
}

ed_status cache_batch_launch(const BatchLaunch& L, cudaStream_t s) {
    int dev = 0, sms = 0;
    ED_CUDA(cudaGetDevice(&dev));
    ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t blocks_needed = (L.stored_slices + (BLOCK / 32) - 1) / (BLOCK / 32);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks_needed, (int64_t)sms * 8));
    auto go = [&](auto ktag) -> ed_status {
        constexpr int K = decltype(ktag)::value;
        if (L.nvec == 1)
            cache_batch_kernel<K, 1><<<grid, BLOCK, 0, s>>>(L.stored, L.n_sec, L.stored_slices, L.row_off, L.x, L.y,
                                                            L.nvec, L.x_step, L.x_step_elems, L.active);
        else
            cache_batch_kernel<K, MAXV><<<grid, BLOCK, 0, s>>>(L.stored, L.n_sec, L.stored_slices, L.row_off, L.x,
                                                               L.y, L.nvec, L.x_step, L.x_step_elems, L.active);
        ED_CUDA(cudaGetLastError());
        return ED_OK;
    };
    switch (L.dtype) {
        case ED_F64: return go(std::integral_constant<int, 0>{});
        case ED_F32: return go(std::integral_constant<int, 1>{});
        case ED_C128: return go(std::integral_constant<int, 2>{});
        case ED_C64: return go(std::integral_constant<int, 3>{});
    }
    return fail(ED_ERR_ARG, "bad dtype");
}

void cache_free(ed_hamiltonian* h) {
    HCache& c = h->cache;
    const Alloc& A = h->basis->alloc;
    A.put(c.counts.p, c.counts.bytes, 0);
    A.put(c.boff.p, c.boff.bytes, 0);
    A.put(c.ent.p, c.ent.bytes, 0);
    A.put(c.diag.p, c.diag.bytes, 0);
    A.put(c.ctab.p, c.ctab.bytes, 0);
    A.put(c.ctr.p, c.ctr.bytes, 0);
    c = HCache{};
}

// Default column segment: 128 MB of the vector type, at most 2^24 elements.
static int default_seg_bits(ed_dtype dtype) {
    const int sx = dtype == ED_F32 ? 4 : dtype == ED_C128 ? 16 : 8;
    const uint64_t elems = (uint64_t)(128u << 20) / (uint64_t)sx;
    int bits = 0;
    while (((uint64_t)2 << bits) <= elems) ++bits;
    return std::min(bits, 24);
}

ed_status cache_build(ed_hamiltonian* h, ed_dtype dtype, int seg_log2, size_t max_bytes, cudaStream_t s) {
    const ed_basis* b = h->basis;
    const HostTables& t = b->ht;
    if (h->cache.valid) cache_free(h);
    if (h->n_flip > 255) return fail(ED_ERR_ARG, "the stored structure needs at most 255 flip terms (%d)", h->n_flip);
    const int64_t D = b->dim;
    int bits = seg_log2 ? seg_log2 : default_seg_bits(dtype);
    if (bits < 5 || bits > 28) return fail(ED_ERR_ARG, "segment bits %d out of range [5,28]", bits);
    const int nb = (int)(((uint64_t)D + ((uint64_t)1 << bits) - 1) >> bits);
    if (nb > CMAXNB) return fail(ED_ERR_ARG, "%d column segments exceed %d; use larger segments", nb, CMAXNB);
    const int64_t ns = (D + 31) / 32, Dpad = ns * 32;
    // code keys: distinct values of h (by flip term and the spins at a, c0, c1) and of chi(g)
    std::vector<std::pair<double, double>> hval;
    std::vector<uint16_t> hmap((size_t)std::max(h->n_flip, 1) * 8);
    for (int f = 0; f < h->n_flip; ++f) {
        const FlipTerm& ft = h->flips[f];
        for (int hb = 0; hb < 8; ++hb) {
            double him = 0.0;
            if (ft.pc0 >= 0) him += ft.k0 * ((hb & 2) ? 0.5 : -0.5);
            if (ft.pc1 >= 0) him += ft.k1 * ((hb & 4) ? 0.5 : -0.5);
            if (hb & 1) him = -him;
            const std::pair<double, double> v{ft.jhalf, him};
            size_t id = std::find(hval.begin(), hval.end(), v) - hval.begin();
            if (id == hval.size()) hval.push_back(v);
            hmap[(size_t)f * 8 + hb] = (uint16_t)id;
        }
    }
    std::vector<std::pair<double, double>> cval;
    std::vector<uint16_t> chi_id(t.G);
    for (int g = 0; g < t.G; ++g) {
        const std::pair<double, double> v{t.chi[2 * g], t.chi[2 * g + 1]};
        size_t id = std::find(cval.begin(), cval.end(), v) - cval.begin();
        if (id == cval.size()) cval.push_back(v);
        chi_id[g] = (uint16_t)id;
    }
    const uint64_t n_keys = (uint64_t)hval.size() * cval.size() * (uint64_t)(t.G + 1);
    if (n_keys > ((uint64_t)1 << 26))
        return fail(ED_ERR_TABLE_TOO_LARGE, "coefficient key space of %llu too large", (unsigned long long)n_keys);
    const Alloc& A = b->alloc;
    BuildScratch sc{&A, s, {}};
    HCache c;
    c.seg_bits = bits;
    c.nb = nb;
    c.ns = ns;
    c.counts.bytes = (size_t)nb * Dpad;
    c.counts.p = A.get(c.counts.bytes, s);
    c.diag.bytes = (size_t)D * 8;
    c.diag.p = A.get(c.diag.bytes, s);
    auto give_up = [&](ed_status st) {
        h->cache = c;
        cache_free(h);
        return st;
    };
    const size_t seen_bytes = ((n_keys + 31) / 32) * 4;
    uint16_t* d_hmap = (uint16_t*)sc.get(hmap.size() * 2);
    uint16_t* d_chi = (uint16_t*)sc.get((size_t)t.G * 2);
    uint32_t* d_seen = (uint32_t*)sc.get(seen_bytes);
    uint8_t* d_code = (uint8_t*)sc.get((size_t)n_keys);
    unsigned long long* d_cnt = (unsigned long long*)sc.get(64);
    if (!c.counts.p || !c.diag.p || !d_hmap || !d_chi || !d_seen || !d_code || !d_cnt)
        return give_up(fail(ED_ERR_NOMEM, "structure build: allocation failed"));
    ED_CUDA(cudaMemcpyAsync(d_hmap, hmap.data(), hmap.size() * 2, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(d_chi, chi_id.data(), (size_t)t.G * 2, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemsetAsync(d_seen, 0, seen_bytes, s));
    ED_CUDA(cudaMemsetAsync(d_cnt, 0, 64, s));
    CacheBuild cb{};
    cb.a = make_args(h);
    cb.seg_bits = bits;
    cb.nb = nb;
    cb.ns = ns;
    cb.Dpad = Dpad;
    cb.counts = (uint8_t*)c.counts.p;
    cb.diag = (double*)c.diag.p;
    cb.hmap = d_hmap;
    cb.chi_id = d_chi;
    cb.n_chi = (uint32_t)cval.size();
    cb.Gp1 = (uint32_t)(t.G + 1);
    cb.dmask = h->sun ? (((uint64_t)1 << b->sun_b) - 1) : 1ull;
    cb.diag_off = h->sun ? 1.0 : 0.5;
    cb.seen = d_seen;
    cb.code = d_code;
    cb.counters = d_cnt;
    const bool w8 = b->word == 8, ch = b->dt.chunk_lo > 0, ns_ok = b->dt.dl_stride == 4;
    const int n_sub = t.n_sub;
    const bool generic = !(ns_ok && n_sub >= 2 && n_sub <= 4);
    cb.a.blocks = hx_min_blocks(b->word, 1, 0);
    const size_t smem = hx_plan(b->dt, 0, generic, cb.a.blocks, h->n_flip, h->n_jc, 1 << t.m).lay.total;
    ed_status st = build_dispatch<0>(cb, smem, n_sub, ns_ok, w8, ch, s);
    if (st != ED_OK) return give_up(st);
    unsigned long long cnt0[4];
    ED_CUDA(cudaMemcpyAsync(cnt0, d_cnt, 32, cudaMemcpyDeviceToHost, s));
    std::vector<uint32_t> seen(seen_bytes / 4);
    ED_CUDA(cudaMemcpyAsync(seen.data(), d_seen, seen_bytes, cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    if (cnt0[2]) return give_up(fail(ED_ERR_INDEX_NOT_FOUND, "%llu representatives missing from the basis", cnt0[2]));
    // codes of the occurring keys, in key order, and their coefficients per value kind
    std::vector<uint8_t> code((size_t)n_keys, 0);
    std::vector<double> c_d(NCODE, 0.0);
    std::vector<float> c_f(NCODE, 0.f);
    std::vector<double> c_d2(2 * NCODE, 0.0);
    std::vector<float> c_f2(2 * NCODE, 0.f);
    int n_code = 0;
    for (uint64_t key = 0; key < n_keys; ++key) {
        if (!((seen[key >> 5] >> (key & 31)) & 1u)) continue;
        if (n_code >= NCODE)
            return give_up(fail(ED_ERR_TABLE_TOO_LARGE, "more than %d distinct coefficients", NCODE));
        const int nst = (int)(key % (uint64_t)(t.G + 1));
        const uint64_t hc = key / (uint64_t)(t.G + 1);
        const int ci = (int)(hc % cval.size()), hi = (int)(hc / cval.size());
        const double jh = hval[hi].first, him = hval[hi].second;
        const double chr = cval[ci].first, chim = cval[ci].second;
        // the matrix-free kernel's coefficient of this gather, per value kind:
        // real FP64: jhalf sqrt(n) with the sign of chi; real FP32: (jhalf chi) sqrt(n) in float
        double vd = jh * sqrt((double)nst);
        if (chr < 0.0) vd = -vd;
        c_d[n_code] = vd;
        const float sqf = (float)sqrt((double)nst);
        c_f[n_code] = (float)jh * (float)chr * sqf;
        // complex: conj(h) chi sqrt(n) with h = jhalf + i him
        const double sq = sqrt((double)nst);
        c_d2[2 * n_code] = (jh * chr + him * chim) * sq;
        c_d2[2 * n_code + 1] = (jh * chim - him * chr) * sq;
        const float jf = (float)jh, hf = (float)him, cxf = (float)chr, cyf = (float)chim;
        c_f2[2 * n_code] = (jf * cxf + hf * cyf) * sqf;
        c_f2[2 * n_code + 1] = (jf * cyf - hf * cxf) * sqf;
        code[key] = (uint8_t)n_code;
        ++n_code;
    }
    c.n_code = n_code;
    // real coefficients first (complex kinds: codes below n_re), then the others
    {
        std::vector<int> order, to(n_code);
        for (int k = 0; k < n_code; ++k)
            if (c_d2[2 * k + 1] == 0.0) order.push_back(k);
        c.n_re = (int)order.size();
        for (int k = 0; k < n_code; ++k)
            if (c_d2[2 * k + 1] != 0.0) order.push_back(k);
        for (int k = 0; k < n_code; ++k) to[order[k]] = k;
        auto permute = [&](auto& v, int w) {
            auto u = v;
            for (int k = 0; k < n_code; ++k)
                for (int e = 0; e < w; ++e) v[(size_t)to[k] * w + e] = u[(size_t)k * w + e];
        };
        permute(c_d, 1);
        permute(c_f, 1);
        permute(c_d2, 2);
        permute(c_f2, 2);
        if (n_code > 0)
            for (auto& cd : code) cd = (uint8_t)to[cd];  // keys that do not occur keep a valid code
    }
    // axis-aligned tables: (c, c) for a real c, (-c, c) for i c
    std::vector<double> a_d2(2 * NCODE, 0.0);
    std::vector<float> a_f2(2 * NCODE, 0.f);
    c.axis_d = c.axis_f = true;
    for (int k = 0; k < n_code; ++k) {
        const bool re = k < c.n_re;
        c.axis_d = c.axis_d && (re || c_d2[2 * k] == 0.0);
        c.axis_f = c.axis_f && (re ? c_f2[2 * k + 1] == 0.f : c_f2[2 * k] == 0.f);
        const double vd = re ? c_d2[2 * k] : c_d2[2 * k + 1];
        const float vf = re ? c_f2[2 * k] : c_f2[2 * k + 1];
        a_d2[2 * k] = re ? vd : -vd;
        a_d2[2 * k + 1] = vd;
        a_f2[2 * k] = re ? vf : -vf;
        a_f2[2 * k + 1] = vf;
    }
    int code_bits = 1;
    while ((1 << code_bits) < n_code) ++code_bits;
    c.off_bits = 32 - code_bits;
    if (bits > c.off_bits)
        return give_up(fail(ED_ERR_TABLE_TOO_LARGE, "%d coefficient codes leave %d bits of column offset, fewer than "
                            "the %d segment bits", n_code, c.off_bits, bits));
    cb.off_bits = c.off_bits;
    c.ctab.bytes = (size_t)NCODE * (16 + 8 + 8 + 4 + 16 + 8);
    c.ctab.p = A.get(c.ctab.bytes, s);
    if (!c.ctab.p) return give_up(fail(ED_ERR_NOMEM, "coefficient table"));
    uint8_t* ct = (uint8_t*)c.ctab.p;
    ED_CUDA(cudaMemcpyAsync(ct, c_d2.data(), NCODE * 16, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(ct + NCODE * 16, c_d.data(), NCODE * 8, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(ct + NCODE * 24, c_f2.data(), NCODE * 8, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(ct + NCODE * 32, c_f.data(), NCODE * 4, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(ct + NCODE * 36, a_d2.data(), NCODE * 16, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(ct + NCODE * 52, a_f2.data(), NCODE * 8, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(d_code, code.data(), (size_t)n_keys, cudaMemcpyHostToDevice, s));
    // per-slice offsets of every segment
    uint32_t* d_tot = (uint32_t*)sc.get((size_t)nb * ns * 4);
    uint64_t* d_abs = (uint64_t*)sc.get((size_t)nb * ns * 8);
    uint64_t* d_bbase = (uint64_t*)sc.get((size_t)nb * 8);
    c.boff.bytes = (size_t)nb * ns * 4;
    c.boff.p = A.get(c.boff.bytes, s);
    if (!d_tot || !d_abs || !d_bbase || !c.boff.p) return give_up(fail(ED_ERR_NOMEM, "structure offsets"));
    int dev = 0, sms = 0;
    ED_CUDA(cudaGetDevice(&dev));
    ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)nb * ns + 255) / 256, (int64_t)sms * 16));
    slice_totals<<<g, 256, 0, s>>>((const uint8_t*)c.counts.p, ns, nb, d_tot);
    ED_CUDA(cudaGetLastError());
    uint64_t total = 0;
    st = exclusive_scan_u32(d_tot, (uint64_t)nb * ns, d_abs, &total, A, s);
    if (st != ED_OK) return give_up(st);
    if (total != cnt0[0])
        return give_up(fail(ED_ERR_INDEX_NOT_FOUND, "structure count mismatch (%llu vs %llu)",
                            (unsigned long long)total, cnt0[0]));
    slice_offsets<<<g, 256, 0, s>>>(d_abs, ns, nb, (uint32_t*)c.boff.p, d_bbase);
    ED_CUDA(cudaGetLastError());
    c.bbase.resize(nb + 1);
    ED_CUDA(cudaMemcpyAsync(c.bbase.data(), d_bbase, (size_t)nb * 8, cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    c.bbase[nb] = total;
    for (int k = 0; k < nb; ++k)
        if (c.bbase[k + 1] - c.bbase[k] >= 0xFFFFFFFFull)
            return give_up(fail(ED_ERR_ARG, "segment %d holds 2^32 or more entries; use smaller segments", k));
    c.n_ent = total;
    c.n_skip = cnt0[1];
    const size_t need = c.counts.bytes + c.diag.bytes + c.boff.bytes + c.ctab.bytes + (size_t)total * 4 + 16;
    if (need > max_bytes)
        return give_up(fail(ED_ERR_NOMEM, "the stored structure needs %zu bytes, more than the limit of %zu", need,
                            max_bytes));
    c.ent.bytes = (size_t)total * 4 + 16;
    c.ent.p = A.get(c.ent.bytes, s);
    if (!c.ent.p) return give_up(fail(ED_ERR_NOMEM, "structure entries (%zu bytes)", c.ent.bytes));
    ED_CUDA(cudaMemsetAsync(d_cnt, 0, 64, s));
    cb.boff = (const uint32_t*)c.boff.p;
    cb.bbase = d_bbase;
    cb.ent = (uint32_t*)c.ent.p;
    st = build_dispatch<1>(cb, smem, n_sub, ns_ok, w8, ch, s);
    if (st != ED_OK) return give_up(st);
    unsigned long long cnt1[4];
    ED_CUDA(cudaMemcpyAsync(cnt1, d_cnt, 32, cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    if (cnt1[0] != cnt0[0] || cnt1[3] != 0 || cnt1[2] != 0)
        return give_up(fail(ED_ERR_INDEX_NOT_FOUND, "structure fill mismatch (%llu entries, %llu overflow)", cnt1[0],
                            cnt1[3]));
    c.ctr.bytes = 32;
    c.ctr.p = A.get(32, s);
    if (!c.ctr.p) return give_up(fail(ED_ERR_NOMEM, "structure counters"));
    const unsigned long long ctr[4] = {cnt1[0], cnt0[1], 0ull, 0ull};
    ED_CUDA(cudaMemcpyAsync(c.ctr.p, ctr, 32, cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaStreamSynchronize(s));
    c.sms = sms;
    c.bytes = need;
    c.valid = true;
    h->cache = c;
    return ED_OK;
}

ed_status cache_apply(const ed_hamiltonian* h, ed_dtype dt, const void* x, void* y, int nvec, cudaStream_t s) {
    const HCache& c = h->cache;
    const ed_basis* b = h->basis;
    // counters of ed_apply_counters: the structure's entries and skipped images
    ED_CUDA(cudaMemcpyAsync(h->d_counters.p, c.ctr.p, 24, cudaMemcpyDeviceToDevice, s));
    CachePass p{};
    p.x = x;
    p.y = y;
    p.stab = (const uint16_t*)b->stab.p;
    p.diag = (const double*)c.diag.p;
    p.D = b->dim;
    p.ns = c.ns;
    p.nvec = nvec;
    const uint8_t* ct = (const uint8_t*)c.ctab.p;
    const uint8_t* sq = b->dt.blob + b->dt.off_sqrt;    // sqrt(k), then 1/sqrt(k), k = 0..G (double)
    const uint8_t* sqf = b->dt.blob + b->dt.off_sqrtf;  // the same in float
    const int G1 = b->ht.G + 1;
    const bool lanes = nvec == 1 && c.lanes > 1;  // several lanes per row: the general tables
    const bool ax_d = c.axis_d && !lanes, ax_f = c.axis_f && !lanes;
    switch (dt) {
        case ED_F64: p.ctab = ct + NCODE * 16; p.isq = sq + (size_t)G1 * 8; break;
        case ED_F32: p.ctab = ct + NCODE * 32; p.isq = sqf + (size_t)G1 * 4; break;
        case ED_C128: p.ctab = ax_d ? ct + NCODE * 36 : ct; p.isq = sq + (size_t)G1 * 8; break;
        case ED_C64: p.ctab = ax_f ? ct + NCODE * 52 : ct + NCODE * 24; p.isq = sqf + (size_t)G1 * 4; break;
        default: return fail(ED_ERR_ARG, "bad dtype");
    }
    for (int k = 0; k < c.nb; ++k) {
        p.counts = (const uint8_t*)c.counts.p + (size_t)k * c.ns * 32;
        p.boff = (const uint32_t*)c.boff.p + (size_t)k * c.ns;
        p.ent = (const uint32_t*)c.ent.p + c.bbase[k];
        p.xoff = (int64_t)k << c.seg_bits;
        p.mode = c.nb == 1 ? 0 : (k == 0 ? 1 : (k == c.nb - 1 ? 3 : 2));
        p.off_bits = (uint32_t)c.off_bits;
        p.n_re = (uint32_t)c.n_re;
        ed_status st = ED_OK;
        if (lanes) {
            st = launch_pass_lanes(p, dt == ED_F64 ? 0 : dt == ED_F32 ? 1 : dt == ED_C128 ? 2 : 3, c.lanes, c.sms, s);
        } else {
            switch (dt) {
                case ED_F64: st = launch_pass<0>(p, nvec, c.sms, s); break;
                case ED_F32: st = launch_pass<1>(p, nvec, c.sms, s); break;
                case ED_C128: st = ax_d ? launch_pass<2, true>(p, nvec, c.sms, s) : launch_pass<2>(p, nvec, c.sms, s); break;
                case ED_C64: st = ax_f ? launch_pass<3, true>(p, nvec, c.sms, s) : launch_pass<3>(p, nvec, c.sms, s); break;
            }
        }
        if (st != ED_OK) return st;
    }
    return ED_OK;
}

}  // namespace ed

extern "C" ed_status ed_hamiltonian_store(ed_hamiltonian* h, ed_dtype dtype, int32_t seg_log2, size_t max_bytes,
                                          ed_stream stream, size_t* bytes) {
    using namespace ed;
    if (!h) return fail(ED_ERR_ARG, "null argument");
    if ((int)dtype < 0 || (int)dtype > 3) return fail(ED_ERR_ARG, "bad dtype");
    if (seg_log2 != 0 && (seg_log2 < 5 || seg_log2 > 28)) return fail(ED_ERR_ARG, "seg_log2 out of range");
    cudaSetDevice(h->basis->device);
    const ed_status st = cache_build(h, dtype, seg_log2, max_bytes, (cudaStream_t)stream);
    if (bytes) *bytes = st == ED_OK ? h->cache.bytes : 0;
    return st;
}

extern "C" ed_status ed_hamiltonian_store_info(const ed_hamiltonian* h, int64_t* entries, int32_t* segments,
                                               int32_t* codes, size_t* bytes) {
    using namespace ed;
    if (!h) return fail(ED_ERR_ARG, "null argument");
    const HCache& c = h->cache;
    if (entries) *entries = c.valid ? (int64_t)c.n_ent : 0;
    if (segments) *segments = c.valid ? c.nb : 0;
    if (codes) *codes = c.valid ? c.n_code : 0;
    if (bytes) *bytes = c.valid ? c.bytes : 0;
    return ED_OK;
}

extern "C" void ed_hamiltonian_store_free(ed_hamiltonian* h) {
    if (!h) return;
    cudaSetDevice(h->basis->device);
    ed::cache_free(h);
}

// Segment-size autotuner: a segment of x must stay in L2 while its pass
// gathers from it, but every pass also reads each row's count and updates its
// partial sum, so fewer, larger segments pay where rows are many (the 40-site
// square sector prefers 128 MB of FP64) and smaller ones where the gathers
// dominate (the 36-site kagome sector, complex FP32, prefers 64 MB).
extern "C" ed_status ed_hamiltonian_store_set_lanes(ed_hamiltonian* h, int32_t lanes_per_row) {
    using namespace ed;
    if (!h) return fail(ED_ERR_ARG, "null argument");
    if (!h->cache.valid) return fail(ED_ERR_ARG, "no stored structure");
    if (lanes_per_row != 1 && lanes_per_row != 2 && lanes_per_row != 4 && lanes_per_row != 8)
        return fail(ED_ERR_ARG, "lanes per row must be 1, 2, 4 or 8");
    h->cache.lanes = lanes_per_row;
    return ED_OK;
}

extern "C" ed_status ed_hamiltonian_store_schedule(const ed_hamiltonian* h, int32_t* seg_log2,
                                                   int32_t* lanes_per_row) {
    using namespace ed;
    if (!h) return fail(ED_ERR_ARG, "null argument");
    const bool v = h->cache.valid;
    if (seg_log2) *seg_log2 = v ? h->cache.seg_bits : 0;
    if (lanes_per_row) *lanes_per_row = v ? h->cache.lanes : 0;
    return ED_OK;
}

extern "C" ed_status ed_hamiltonian_store_autotune(ed_hamiltonian* h, ed_dtype dtype, size_t max_bytes,
                                                   ed_stream stream, int32_t* seg_log2, size_t* bytes) {
    using namespace ed;
    if (!h) return fail(ED_ERR_ARG, "null argument");
    if ((int)dtype < 0 || (int)dtype > 3) return fail(ED_ERR_ARG, "bad dtype");
    if ((dtype == ED_F64 || dtype == ED_F32) && !h->is_real)
        return fail(ED_ERR_ARG, "complex Hamiltonian or characters need a complex dtype");
    cudaSetDevice(h->basis->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t D = h->basis->dim;
    const int b0 = default_seg_bits(dtype);
    std::vector<int> cands;
    for (int b = b0 - 1; b <= b0 + 1; ++b)
        if (b >= 5 && b <= 26 && (((uint64_t)D + ((uint64_t)1 << b) - 1) >> b) <= (uint64_t)CMAXNB) cands.push_back(b);
    if (cands.empty()) cands.push_back(b0);
    const size_t sx = dtype == ED_F32 ? 4 : dtype == ED_C128 ? 16 : 8;
    const Alloc& A = h->basis->alloc;
    BuildScratch sc{&A, s, {}};
    void* x = sc.get((size_t)D * sx);
    void* y = sc.get((size_t)D * sx);
    if (!x || !y) return fail(ED_ERR_NOMEM, "autotune vectors");
    ED_CUDA(cudaMemsetAsync(x, 0, (size_t)D * sx, s));
    cudaEvent_t e0, e1;
    ED_CUDA(cudaEventCreate(&e0));
    ED_CUDA(cudaEventCreate(&e1));
    struct EFree {
        cudaEvent_t a, b;
        ~EFree() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } ef{e0, e1};
    float best = 1e30f;
    int best_b = 0, best_l = 1;
    ed_status last = ED_OK;
    for (int b : cands) {
        last = cache_build(h, dtype, b, max_bytes, s);
        if (last == ED_ERR_NOMEM || last == ED_ERR_TABLE_TOO_LARGE || (last == ED_ERR_ARG && b != b0)) continue;
        if (last != ED_OK) return last;
        for (int l = 1; l <= 8; l *= 2) {
            h->cache.lanes = l;
            ed_status st = cache_apply(h, dtype, x, y, 1, s);  // warm-up
            if (st != ED_OK) return st;
            ED_CUDA(cudaEventRecord(e0, s));
            for (int r = 0; r < 2 && st == ED_OK; ++r) st = cache_apply(h, dtype, x, y, 1, s);
            if (st != ED_OK) return st;
            ED_CUDA(cudaEventRecord(e1, s));
            ED_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            ED_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_b = b;
                best_l = l;
            }
        }
    }
    if (!best_b) {
        if (bytes) *bytes = 0;
        return last != ED_OK ? last : fail(ED_ERR_NOMEM, "no segment size fits the limit");
    }
    if (!h->cache.valid || h->cache.seg_bits != best_b) {
        const ed_status st = cache_build(h, dtype, best_b, max_bytes, s);
        if (st != ED_OK) return st;
    }
    h->cache.lanes = best_l;
    if (seg_log2) *seg_log2 = best_b;
    if (bytes) *bytes = h->cache.bytes;
    return ED_OK;
}
