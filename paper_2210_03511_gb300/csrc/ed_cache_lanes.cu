// Stored-structure H.x pass with several lanes per row (one vector).
//
// The one-lane-per-row pass (ed_cache.cu) walks each row's elements of the
// segment serially, so a warp runs as long as its longest row and reads the
// entries of 32 rows in every load.  Here groups of L consecutive lanes share
// a row: element k of the row goes to lane k mod L of its group (consecutive
// lanes read consecutive entries), and a butterfly of L - 1 warp shuffles
// combines the lanes' sums.  A warp still owns one slice of 32 rows and takes
// them in L rounds of 32 / L rows; the row counts and offsets of the slice
// come from one coalesced load and a warp prefix sum, as in the one-lane
// pass, and lane i ends with row i's sum, so the writes of y stay coalesced.
// The sums are the same elements combined in a different order (per lane
// k = s, s + L, ..., then the butterfly, then the earlier segments' partial
// sum), so results agree with the one-lane pass up to rounding.  Which of the
// schedules is faster depends on the row lengths per segment and the vector
// type (the butterfly adds L log2 L additions per row in the vector's
// arithmetic); ed_hamiltonian_store_autotune picks by timing.
#include "ed_cache.cuh"

namespace ed {

namespace {

// Resident blocks per SM: the round loop needs a few more registers than the
// one-lane pass (40 a thread; 48 for complex FP64).
constexpr int lanes_blocks(int K) { return K == 2 ? 5 : 6; }

template <int K, int L>
__global__ void __launch_bounds__(BLOCK, lanes_blocks(K)) cache_pass_lanes(CachePass p) {
    using V = Val<K>;
    using T = typename V::T;
    using R = typename V::R;
    using CT = typename std::conditional<V::cplx, T, R>::type;
    constexpr int NG = 32 / L;  // rows per round
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ CT ctab[NCODE];
    for (int i = threadIdx.x; i < NCODE; i += blockDim.x) ctab[i] = ((const CT*)p.ctab)[i];
    __syncthreads();
    const T* __restrict__ x = (const T*)p.x;
    T* __restrict__ y = (T*)p.y;
    const R* __restrict__ isq = (const R*)p.isq;
    const int lane = threadIdx.x & 31, sub = lane % L, grp = lane / L;
    const int64_t D = p.D;
    const uint32_t ob = p.off_bits, om = (1u << ob) - 1u;
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
        T prev;
        if constexpr (V::cplx) prev = T{0, 0};
        else prev = 0;
        if (mode >= 2 && live) prev = y[row];
        const uint32_t st = warp_excl_scan(my, lane);
        const uint32_t* __restrict__ pe = p.ent + bo;
        R ownr = 0, owni = 0;
#pragma unroll 1
        for (int r = 0; r < L; ++r) {
            const int q = r * NG + grp;  // the row this group takes in round r
            const uint32_t nq = __shfl_sync(FULL, my, q);
            const uint32_t* __restrict__ pq = pe + __shfl_sync(FULL, st, q);
            R ar = 0, ai = 0;
            for (uint32_t k = sub; k < nq; k += L) {
                const uint32_t w = __ldg(pq + k);
                const int64_t j = p.xoff + (int64_t)(w & om);
                const CT cf = ctab[w >> ob];
                if constexpr (!V::cplx) {
                    ar += cf * x[j];
                } else {
                    const T xj = x[j];
                    ar += cf.x * xj.x - cf.y * xj.y;
                    ai += cf.x * xj.y + cf.y * xj.x;
                }
            }
#pragma unroll
            for (int o = L / 2; o > 0; o >>= 1) {
                ar += __shfl_xor_sync(FULL, ar, o);
                if constexpr (V::cplx) ai += __shfl_xor_sync(FULL, ai, o);
            }
            // lane i's row is taken in round i / NG by group i % NG
            const int src = (lane % NG) * L;
            const R vr = __shfl_sync(FULL, ar, src);
            R vi = 0;
            if constexpr (V::cplx) vi = __shfl_sync(FULL, ai, src);
            if (lane / NG == r) {
                ownr = vr;
                owni = vi;
            }
        }
        if (!live) continue;
        R sr, si = 0;
        if constexpr (V::cplx) {
            sr = prev.x + ownr;
            si = prev.y + owni;
        } else {
            sr = prev + ownr;
        }
        if (mode == 0 || mode == 3) {
            const R inv = isq[__ldg(p.stab + row)];
            const R dg = (R)__ldg(p.diag + row);
            if constexpr (V::cplx) {
                const T xi = x[row];
                T out;
                out.x = sr * inv + dg * xi.x;
                out.y = si * inv + dg * xi.y;
                y[row] = out;
            } else {
                y[row] = sr * inv + dg * x[row];
            }
        } else {
            if constexpr (V::cplx) y[row] = T{sr, si};
            else y[row] = sr;
        }
    }
}

template <int K, int L>
ed_status launch(const CachePass& p, int sms, cudaStream_t s) {
    const int64_t blocks_needed = (p.ns + (BLOCK / 32) - 1) / (BLOCK / 32);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks_needed, (int64_t)sms * lanes_blocks(K)));
    cache_pass_lanes<K, L><<<grid, BLOCK, 0, s>>>(p);
    ED_CUDA(cudaGetLastError());
    return ED_OK;
}

template <int K>
ed_status launch_k(const CachePass& p, int lanes, int sms, cudaStream_t s) {
    switch (lanes) {
        case 2: return launch<K, 2>(p, sms, s);
        case 4: return launch<K, 4>(p, sms, s);
        case 8: return launch<K, 8>(p, sms, s);
    }
    return fail(ED_ERR_ARG, "lanes per row must be 2, 4 or 8");
}

}  // namespace

ed_status launch_pass_lanes(const CachePass& p, int K, int lanes, int sms, cudaStream_t s) {
    switch (K) {
        case 0: return launch_k<0>(p, lanes, sms, s);
        case 1: return launch_k<1>(p, lanes, sms, s);
        case 2: return launch_k<2>(p, lanes, sms, s);
        case 3: return launch_k<3>(p, lanes, sms, s);
    }
    return fail(ED_ERR_ARG, "bad value kind");
}

}  // namespace ed
