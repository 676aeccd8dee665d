// Batches of sectors: one H.x launch over all sectors, and block Lanczos
// (several right-hand sides per sector) for all sectors at once.
//
// Vector layout of a batch: sectors are concatenated in order; sector s owns
// rows [row_off[s], row_off[s+1]) and its block of b vectors starts at
// element b*row_off[s], column-major (column c at b*row_off[s] + c*D_s).
//
// Block Lanczos (the block form of the Lanczos recursion, Eqs.
// lanczosrecursionabbrev and tmatrix with b x b blocks): for block k,
// W = H V_k; classical Gram-Schmidt twice against every stored block V_j
// (j <= k), which also yields the diagonal block A_k = V_k^H H V_k; then
// W = V_{k+1} B_k by Cholesky QR applied twice.  All inner products accumulate
// in FP64 over fixed row tiles and are reduced in a fixed order.  Every kernel
// of a step takes the block index from device memory, so the whole step is
// captured once as a CUDA graph and replayed; the host only reads the small
// blocks A_k, B_k and solves the banded T-matrix for eigenvalues by bisection
// on Sturm (inertia) counts of its banded LDL^H factorisation.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <thread>
#include <type_traits>
#include <vector>

#include "ed_internal.h"

struct ed_batch {
    std::vector<const ed_hamiltonian*> hs;
    std::vector<int64_t> row_off;          // host [n+1]
    ed::DevBuf d_desc, d_row_off, d_counters, d_tiles;
    int n = 0;
    int64_t total = 0;
    size_t smem[4][2] = {};   // per dtype, for one / several vectors
    int blocks[4][2] = {};    // resident blocks per SM, same index
    bool w8 = false, chunked = false, ns_ok = false, all_real = true;
    bool has_sun = false;                  // SU(N) sectors: applied through stored structures only
    int n_sub = 0;
    int waves[4][2] = {{1, 1}, {1, 1}, {1, 1}, {1, 1}};  // [dtype][nvec>1]: tuned grid waves
    std::vector<int64_t> tiles;            // row tiles: (sector, begin, end) triples
    int n_tiles = 0;
    const ed::Alloc* alloc = nullptr;
    // descriptors of the sectors' stored structures, when every sector has
    // one (one column segment each): H.x of the batch then streams them
    mutable std::vector<ed::CacheSector> stored_h;
    mutable ed::DevBuf d_stored;
    mutable int64_t stored_slices = 0;
};

namespace ed {

static const int TILE = 4096;  // rows per reduction tile
static const int MAXB = 8;

// Vector kinds of block Lanczos: T is the stored element, A the complex type
// of the elementwise arithmetic (FP32 for FP32 vectors, so that the block
// Gram-Schmidt runs on the FP32 pipes; sums across tiles and the b x b
// matrices stay FP64).
template <int K> struct BV;
template <> struct BV<0> { using T = double; using A = double2; static constexpr bool cplx = false, single = false; };
template <> struct BV<1> { using T = float; using A = float2; static constexpr bool cplx = false, single = true; };
template <> struct BV<2> { using T = double2; using A = double2; static constexpr bool cplx = true, single = false; };
template <> struct BV<3> { using T = float2; using A = float2; static constexpr bool cplx = true, single = true; };

__device__ __forceinline__ double2 c_ld(const double& v) { return make_double2(v, 0.0); }
__device__ __forceinline__ double2 c_ld(const double2& v) { return v; }
__device__ __forceinline__ float2 c_ld(const float& v) { return make_float2(v, 0.f); }
__device__ __forceinline__ float2 c_ld(const float2& v) { return v; }
__device__ __forceinline__ void c_st(double& d, double2 v) { d = v.x; }
__device__ __forceinline__ void c_st(double2& d, double2 v) { d = v; }
__device__ __forceinline__ void c_st(float& d, float2 v) { d = v.x; }
__device__ __forceinline__ void c_st(float2& d, float2 v) { d = v; }
__device__ __forceinline__ void c_st(float& d, double2 v) { d = (float)v.x; }
__device__ __forceinline__ void c_st(float2& d, double2 v) { d = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 c_conjmul(double2 a, double2 b) {  // conj(a) b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 c_conjmul(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ int sector_of(const int64_t* row_off, int n, int64_t r) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint64_t bmix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double bunif(uint64_t seed, uint64_t stream, uint64_t state) {
    const uint64_t key = bmix(seed * 256ull + stream);
    return ((double)(bmix(state ^ key) >> 11) + 0.5) * (1.0 / 9007199254740992.0);  // (0,1)
}

// Start block: Gaussian entries (Box-Muller on keyed SplitMix64 uniforms of
// the state integer, one stream pair per column and component).
template <int K>
__global__ void bl_init(typename BV<K>::T* X, const HxArgs* desc, const int64_t* row_off, int n, int b, uint64_t seed,
                        int word) {
    const int64_t total = row_off[n];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
        const int s = sector_of(row_off, n, r);
        const int64_t i = r - row_off[s];
        const int64_t D = row_off[s + 1] - row_off[s];
        const uint64_t st = word == 8 ? ((const uint64_t*)desc[s].reps)[i] : ((const uint32_t*)desc[s].reps)[i];
        for (int c = 0; c < b; ++c) {
            const double u1 = bunif(seed, 4 * c, st), u2 = bunif(seed, 4 * c + 1, st);
            const double rr = sqrt(-2.0 * log(u1));
            double2 z = make_double2(rr * cos(6.283185307179586 * u2), 0.0);
            if (BV<K>::cplx) {
                const double u3 = bunif(seed, 4 * c + 2, st), u4 = bunif(seed, 4 * c + 3, st);
                z.y = sqrt(-2.0 * log(u3)) * cos(6.283185307179586 * u4);
            }
            c_st(X[b * row_off[s] + (int64_t)c * D + i], z);
        }
    }
}

// partial[j][tile][a][c] = sum over tile rows of conj(X_j[a][i]) Y[c][i],
// X_j = X + j*xs (j = 0..*jmax, or 0 when jmax is null).  One block per
// (tile, j); thread t handles pair (a, c) = (t / b % b, t % b) for rows
// i = t / b^2 + m * (256 / b^2).
// With local != 0 only the last two blocks take part (j = *jmax - 1 + blockIdx.y):
// the plain three-term recursion.  Tiles of sectors with active[s] == 0 are skipped.
template <int K>
__global__ void __launch_bounds__(256) bl_gram(const typename BV<K>::T* X, int64_t xs, const int* jmax,
                                               const typename BV<K>::T* Y, const int64_t* tiles,
                                               const int64_t* row_off, int b, double2* partial, int n_tiles,
                                               int local, const int* active) {
    const int j = local ? *jmax - 1 + (int)blockIdx.y : (int)blockIdx.y;
    if (j < 0 || (jmax ? j > *jmax : j > 0)) return;
    const int tile = blockIdx.x;
    const int s = (int)tiles[3 * tile];
    if (!active[s]) return;  // a converged sector: its coefficients are not used
    const int64_t i0 = tiles[3 * tile + 1], i1 = tiles[3 * tile + 2];
    const int64_t D = row_off[s + 1] - row_off[s];
    const int64_t base = (int64_t)b * row_off[s];
    const int bb = b * b;
    const int lanes = 256 / bb;
    const int t = threadIdx.x;
    __shared__ double2 red[256];
    using A = typename BV<K>::A;
    A acc{0, 0};
    if (t < lanes * bb) {
        const int a = (t / b) % b, c = t % b, l = t / bb;
        const typename BV<K>::T* xa = X + (int64_t)j * xs + base + (int64_t)a * D;
        const typename BV<K>::T* yc = Y + base + (int64_t)c * D;
        for (int64_t i = i0 + l; i < i1; i += lanes) {
            const A p = c_conjmul(c_ld(xa[i]), c_ld(yc[i]));
            acc.x += p.x;
            acc.y += p.y;
        }
    }
    red[t] = to_d2(acc);  // FP64 from here on
    __syncthreads();
    if (t < bb) {
        double2 sum = make_double2(0.0, 0.0);
        for (int l = 0; l < lanes; ++l) {
            sum.x += red[l * bb + t].x;
            sum.y += red[l * bb + t].y;
        }
        partial[((int64_t)j * n_tiles + tile) * bb + t] = sum;
    }
}

// C[s][j][a][c] = sum over the tiles of sector s (fixed order); Cf (if not
// null) receives the same values in FP32 for the FP32 update
__global__ void bl_reduce(const double2* partial, const int* tile_first, int n, int b, int n_tiles, const int* jmax,
                          int jcap, double2* C, int local, float2* Cf = nullptr) {
    const int s = blockIdx.x;
    const int bb = b * b;
    const int jm = jmax ? *jmax : 0;
    const int j0 = local ? max(0, jm - 1) : 0;
    for (int e = threadIdx.x; e < (jm + 1 - j0) * bb; e += blockDim.x) {
        const int j = j0 + e / bb, ac = e % bb;
        double2 sum = make_double2(0.0, 0.0);
        for (int tl = tile_first[s]; tl < tile_first[s + 1]; ++tl) {
            const double2 v = partial[((int64_t)j * n_tiles + tl) * bb + ac];
            sum.x += v.x;
            sum.y += v.y;
        }
        C[((int64_t)s * jcap + j) * bb + ac] = sum;
        if (Cf) Cf[((int64_t)s * jcap + j) * bb + ac] = make_float2((float)sum.x, (float)sum.y);
    }
}

// W[c][i] -= sum_{j <= jmax} sum_a X_j[a][i] C[s][j][a][c]
// B: the block size at compile time (1, 2, 4, 8; the per-row accumulators
// then live in registers), or 0 for any b <= MAXB.
template <int K, int B = 0>
__global__ void bl_update(typename BV<K>::T* W, const typename BV<K>::T* X, int64_t xs, const int* jmax,
                          const double2* C, int jcap, const int64_t* row_off, int n, int b_run, int local,
                          const int* active, const float2* Cf = nullptr) {
    using A = typename BV<K>::A;
    const int b = B ? B : b_run;
    const int64_t total = row_off[n];
    const int jm = *jmax;
    const int j0 = local ? max(0, jm - 1) : 0;
    const int bb = b * b;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
        const int s = sector_of(row_off, n, r);
        if (!active[s]) continue;
        const int64_t i = r - row_off[s];
        const int64_t D = row_off[s + 1] - row_off[s];
        const int64_t base = (int64_t)b * row_off[s];
        A w[B ? B : MAXB];
#pragma unroll
        for (int c = 0; c < (B ? B : MAXB); ++c)
            if (c < b) w[c] = c_ld(W[base + (int64_t)c * D + i]);
        for (int j = j0; j <= jm; ++j) {
            const int64_t cj = ((int64_t)s * jcap + j) * bb;
#pragma unroll
            for (int a = 0; a < (B ? B : MAXB); ++a) {
                if (a >= b) break;
                const A x = c_ld(X[(int64_t)j * xs + base + (int64_t)a * D + i]);
#pragma unroll
                for (int c = 0; c < (B ? B : MAXB); ++c) {
                    if (c >= b) break;
                    A cv;
                    if constexpr (BV<K>::single) cv = Cf[cj + a * b + c];
                    else cv = C[cj + a * b + c];
                    const A p = c_mul(x, cv);
                    w[c].x -= p.x;
                    w[c].y -= p.y;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < (B ? B : MAXB); ++c)
            if (c < b) c_st(W[base + (int64_t)c * D + i], w[c]);
    }
}

// Per sector: G = R^H R (Cholesky, G from the W^H W gram), store R^{-1} and
// accumulate Bacc = R * Bacc (Bacc starts as the identity).  A column whose
// pivot collapses is dropped (R^{-1} column zero).
__global__ void bl_chol(const double2* G, int jcap, int n, int b, double2* Rinv, double2* Bacc, int first_pass,
                        const int* active, float2* Rinvf = nullptr) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n || !active[s]) return;
    const int bb = b * b;
    const double2* g = G + (int64_t)s * jcap * bb;  // j = 0 slot
    double2 R[MAXB][MAXB], Ri[MAXB][MAXB];
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) { R[r][c] = make_double2(0, 0); Ri[r][c] = make_double2(0, 0); }
    double scale = 0.0;
    for (int a = 0; a < b; ++a) scale = fmax(scale, g[a * b + a].x);
    for (int c = 0; c < b; ++c) {
        // R[r][c] for r < c, then R[c][c]
        for (int r = 0; r < c; ++r) {
            // G[r][c] = sum_{k<=r} conj(R[k][r]) R[k][c]
            double2 v = g[r * b + c];
            for (int k = 0; k < r; ++k) {
                const double2 p = c_conjmul(R[k][r], R[k][c]);
                v.x -= p.x;
                v.y -= p.y;
            }
            const double d = R[r][r].x;
            R[r][c] = d > 0 ? make_double2(v.x / d, v.y / d) : make_double2(0, 0);
        }
        double v = g[c * b + c].x;
        for (int k = 0; k < c; ++k) v -= R[k][c].x * R[k][c].x + R[k][c].y * R[k][c].y;
        R[c][c] = make_double2(v > 1e-28 * scale ? sqrt(v) : 0.0, 0.0);
    }
    // inverse of the upper-triangular R (zero rows/columns for dropped pivots)
    for (int c = 0; c < b; ++c) {
        if (R[c][c].x <= 0) continue;
        Ri[c][c] = make_double2(1.0 / R[c][c].x, 0.0);
        for (int r = c - 1; r >= 0; --r) {
            if (R[r][r].x <= 0) continue;
            double2 v = make_double2(0, 0);
            for (int k = r + 1; k <= c; ++k) {
                const double2 p = c_mul(R[r][k], Ri[k][c]);
                v.x += p.x;
                v.y += p.y;
            }
            Ri[r][c] = make_double2(-v.x / R[r][r].x, -v.y / R[r][r].x);
        }
    }
    double2* ri = Rinv + (int64_t)s * bb;
    double2* ba = Bacc + (int64_t)s * bb;
    double2 Bn[MAXB][MAXB];
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) {
            ri[r * b + c] = Ri[r][c];
            if (Rinvf) Rinvf[(int64_t)s * bb + r * b + c] = make_float2((float)Ri[r][c].x, (float)Ri[r][c].y);
            double2 v = make_double2(0, 0);
            for (int k = 0; k < b; ++k) {
                const double2 prev = first_pass ? make_double2(k == c ? 1.0 : 0.0, 0.0) : ba[k * b + c];
                const double2 p = c_mul(R[r][k], prev);
                v.x += p.x;
                v.y += p.y;
            }
            Bn[r][c] = v;
        }
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) ba[r * b + c] = Bn[r][c];
}

// Out[c][i] = sum_a W[a][i] Rinv[s][a][c]; Out may be W + (*kout)*os (device index) or W itself
template <int K, int B = 0>
__global__ void bl_scale(const typename BV<K>::T* W, typename BV<K>::T* Out, int64_t os, const int* kout, int kadd,
                         const double2* Rinv, const int64_t* row_off, int n, int b_run, const int* active,
                         const float2* Rinvf = nullptr) {
    using A = typename BV<K>::A;
    const int b = B ? B : b_run;
    const int64_t total = row_off[n];
    typename BV<K>::T* out = Out + (kout ? (int64_t)(*kout + kadd) * os : 0);
    const int bb = b * b;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
        const int s = sector_of(row_off, n, r);
        if (!active[s]) continue;
        const int64_t i = r - row_off[s];
        const int64_t D = row_off[s + 1] - row_off[s];
        const int64_t base = (int64_t)b * row_off[s];
        A w[B ? B : MAXB];
#pragma unroll
        for (int a = 0; a < (B ? B : MAXB); ++a)
            if (a < b) w[a] = c_ld(W[base + (int64_t)a * D + i]);
#pragma unroll
        for (int c = 0; c < (B ? B : MAXB); ++c) {
            if (c >= b) break;
            A v{0, 0};
#pragma unroll
            for (int a = 0; a < (B ? B : MAXB); ++a) {
                if (a >= b) break;
                A rv;
                if constexpr (BV<K>::single) rv = Rinvf[(int64_t)s * bb + a * b + c];
                else rv = Rinv[(int64_t)s * bb + a * b + c];
                const A p = c_mul(w[a], rv);
                v.x += p.x;
                v.y += p.y;
            }
            c_st(out[base + (int64_t)c * D + i], v);
        }
    }
}

// Save A_k (= the j = k block of the first and second reorthogonalisation
// coefficients, summed) and B_k (Bacc) into the per-step arrays; advance k.
__global__ void bl_save(const double2* C1, const double2* C2, const double2* Bacc, int jcap, int n, int b, int* k,
                        double2* Ahist, double2* Bhist, int kcap, const int* active) {
    const int kk = *k;
    const int bb = b * b;
    for (int e = threadIdx.x; e < n * bb; e += blockDim.x) {
        const int s = e / bb, ac = e % bb;
        if (!active[s]) continue;
        const double2 a1 = C1[((int64_t)s * jcap + kk) * bb + ac], a2 = C2[((int64_t)s * jcap + kk) * bb + ac];
        Ahist[((int64_t)s * kcap + kk) * bb + ac] = make_double2(a1.x + a2.x, a1.y + a2.y);
        Bhist[((int64_t)s * kcap + kk) * bb + ac] = Bacc[(int64_t)s * bb + ac];
    }
    __syncthreads();
    if (threadIdx.x == 0) *k = kk + 1;
}

__global__ void bl_set_int(int* p, int v) { *p = v; }

// Refinement of FP32 block Lanczos: Ritz vectors in FP64,
// Y[e][i] = sum over j < its[s] and a < b of V_j[a][i] Z[s][e][j b + a]
// (sector s's ne columns start at ne * row_off[s], column e at + e D).
template <int KV, int KO>
__global__ void bl_combine(typename BV<KO>::T* Y, int ne, const typename BV<KV>::T* V, int64_t bs, const double2* Z,
                           int zcap, const int* its, const int64_t* row_off, int n, int b) {
    const int64_t total = row_off[n];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
        const int s = sector_of(row_off, n, r);
        const int64_t i = r - row_off[s];
        const int64_t D = row_off[s + 1] - row_off[s];
        const int64_t base = (int64_t)b * row_off[s];
        double2 acc[MAXB];
        for (int e = 0; e < ne; ++e) acc[e] = make_double2(0, 0);
        const int it = its[s];
        for (int j = 0; j < it; ++j)
            for (int a = 0; a < b; ++a) {
                const double2 x = to_d2(c_ld(V[(int64_t)j * bs + base + (int64_t)a * D + i]));
                for (int e = 0; e < ne; ++e) {
                    const double2 p = c_mul(x, Z[((int64_t)s * ne + e) * zcap + j * b + a]);
                    acc[e].x += p.x;
                    acc[e].y += p.y;
                }
            }
        const int64_t yb = (int64_t)ne * row_off[s];
        for (int e = 0; e < ne; ++e) c_st(Y[yb + (int64_t)e * D + i], acc[e]);
    }
}

// Y[.][i] <- Y[.][i] C[s] and HY[.][i] <- HY[.][i] C[s] (C[s]: ne x ne, [a][e]),
// in place row by row (the Ritz vectors of the Rayleigh-Ritz step)
template <int KO>
__global__ void bl_rotate(typename BV<KO>::T* Y, typename BV<KO>::T* HY, const double2* C, int ne,
                          const int64_t* row_off, int n) {
    const int64_t total = row_off[n];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
        const int s = sector_of(row_off, n, r);
        const int64_t i = r - row_off[s];
        const int64_t D = row_off[s + 1] - row_off[s];
        const int64_t yb = (int64_t)ne * row_off[s];
        const double2* Cs = C + (int64_t)s * ne * ne;
        for (int w = 0; w < 2; ++w) {
            typename BV<KO>::T* X = w == 0 ? Y : HY;
            double2 in[MAXB], out[MAXB];
            for (int a = 0; a < ne; ++a) in[a] = c_ld(X[yb + (int64_t)a * D + i]);
            for (int e = 0; e < ne; ++e) {
                out[e] = make_double2(0, 0);
                for (int a = 0; a < ne; ++a) {
                    const double2 p = c_mul(in[a], Cs[a * ne + e]);
                    out[e].x += p.x;
                    out[e].y += p.y;
                }
            }
            for (int e = 0; e < ne; ++e) c_st(X[yb + (int64_t)e * D + i], out[e]);
        }
    }
}

// R[e][i] = HY[e][i] - E[s][e] Y[e][i], in place on HY (FP64 kinds)
template <int KO>
__global__ void bl_resid(typename BV<KO>::T* HY, const typename BV<KO>::T* Y, const double* E, int ne,
                         const int64_t* row_off, int n) {
    const int64_t total = row_off[n];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
        const int s = sector_of(row_off, n, r);
        const int64_t i = r - row_off[s];
        const int64_t D = row_off[s + 1] - row_off[s];
        const int64_t yb = (int64_t)ne * row_off[s];
        for (int e = 0; e < ne; ++e) {
            const int64_t o = yb + (int64_t)e * D + i;
            const double2 h = c_ld(HY[o]), y = c_ld(Y[o]);
            const double en = E[s * ne + e];
            c_st(HY[o], make_double2(h.x - en * y.x, h.y - en * y.y));
        }
    }
}

// ------------------------------------------------------------------ host: banded eigenvalues
using cd = std::complex<double>;

// Hermitian band matrix in band storage: L[i*(bw+1) + k] = T[i][i-k], k = 0..bw.
struct Band {
    int n = 0, bw = 0;
    std::vector<cd> L;
    cd& at(int i, int k) { return L[(size_t)i * (bw + 1) + k]; }
    cd get(int i, int k) const { return L[(size_t)i * (bw + 1) + k]; }
};

// number of eigenvalues of T below x: negative pivots of the banded LDL^H of T - x I
static int band_count(const Band& T, double x) {
    const int n = T.n, bw = T.bw;
    std::vector<cd> L((size_t)n * (bw + 1), cd(0));  // L[i][i-k] at i*(bw+1)+k
    std::vector<double> d(n, 0.0);
    int neg = 0;
    for (int j = 0; j < n; ++j) {
        double dj = T.get(j, 0).real() - x;
        for (int k = std::max(0, j - bw); k < j; ++k) dj -= std::norm(L[(size_t)j * (bw + 1) + (j - k)]) * d[k];
        if (dj == 0.0) dj = 1e-300;
        d[j] = dj;
        if (dj < 0) ++neg;
        for (int i = j + 1; i <= std::min(n - 1, j + bw); ++i) {
            cd v = T.get(i, i - j);
            for (int k = std::max(0, i - bw); k < j; ++k)
                v -= L[(size_t)i * (bw + 1) + (i - k)] * std::conj(L[(size_t)j * (bw + 1) + (j - k)]) * d[k];
            L[(size_t)i * (bw + 1) + (i - j)] = v / dj;
        }
    }
    return neg;
}

// lowest m eigenvalues by bisection on the inertia
static std::vector<double> band_lowest(const Band& T, int m) {
    const int n = T.n, bw = T.bw;
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
        double r = 0;
        for (int k = 1; k <= bw && k <= i; ++k) r += std::abs(T.get(i, k));
        for (int k = 1; k <= bw && i + k < n; ++k) r += std::abs(T.get(i + k, k));
        lo = std::min(lo, T.get(i, 0).real() - r);
        hi = std::max(hi, T.get(i, 0).real() + r);
    }
    std::vector<double> out;
    for (int e = 0; e < std::min(m, n); ++e) {
        double a = lo, b2 = hi;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (a + b2);
            if (mid <= a || mid >= b2) break;
            if (band_count(T, mid) > e) b2 = mid;
            else a = mid;
        }
        out.push_back(0.5 * (a + b2));
    }
    return out;
}

// max row sum of |T| (a bound on its spectral radius)
static double band_norm(const Band& T) {
    double tn = 0.0;
    for (int i = 0; i < T.n; ++i) {
        double r = 0.0;
        for (int k = 0; k <= T.bw && k <= i; ++k) r += std::abs(T.get(i, k));
        for (int k = 1; k <= T.bw && i + k < T.n; ++k) r += std::abs(T.get(i + k, k));
        tn = std::max(tn, r);
    }
    return tn;
}

// Eigenvector of the Hermitian band matrix T for its eigenvalue lam, by
// inverse iteration: (T - lam I) z_new = z, solved by Gaussian elimination
// with partial pivoting inside the band (row interchanges make the upper
// bandwidth 2 bw; the multipliers of step k stay in column k, as the solve
// applies interchange k before elimination k).  Three iterations from a
// fixed start; each iterate is orthogonalised against `prev` (vectors of
// lower eigenvalues of the same T, which matters for close pairs).
static std::vector<cd> band_vector(const Band& T, double lam, const std::vector<std::vector<cd>>& prev) {
    const int n = T.n, bw = T.bw, w = 3 * bw + 1;  // row i holds columns i - bw .. i + 2 bw
    double tn = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        for (int k = 0; k <= bw && k <= i; ++k) r += std::abs(T.get(i, k));
        for (int k = 1; k <= bw && i + k < n; ++k) r += std::abs(T.get(i + k, k));
        tn = std::max(tn, r);
    }
    const double tiny = 1e-14 * std::max(tn, 1e-300);
    std::vector<cd> M((size_t)n * w, cd(0));
    auto at = [&](int i, int j) -> cd& { return M[(size_t)i * w + (j - i + bw)]; };
    for (int i = 0; i < n; ++i)
        for (int j = std::max(0, i - bw); j <= std::min(n - 1, i + bw); ++j)
            at(i, j) = (i >= j ? T.get(i, i - j) : std::conj(T.get(j, j - i))) - (i == j ? cd(lam) : cd(0));
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i <= std::min(n - 1, k + bw); ++i)
            if (std::abs(at(i, k)) > std::abs(at(p, k))) p = i;
        piv[k] = p;
        const int jend = std::min(n - 1, k + 2 * bw);
        if (p != k)
            for (int j = k; j <= jend; ++j) std::swap(at(k, j), at(p, j));
        if (std::abs(at(k, k)) < tiny) at(k, k) = cd(tiny);
        for (int i = k + 1; i <= std::min(n - 1, k + bw); ++i) {
            const cd f = at(i, k) / at(k, k);
            at(i, k) = f;
            for (int j = k + 1; j <= jend; ++j) at(i, j) -= f * at(k, j);
        }
    }
    std::vector<cd> z(n);
    for (int i = 0; i < n; ++i) z[i] = cd(1.0 + 0.5 * std::sin(1.0 + 0.77 * i), 0.25 * std::cos(0.3 + 1.3 * i));
    for (int iter = 0; iter < 3; ++iter) {
        for (int k = 0; k < n; ++k) {
            std::swap(z[k], z[piv[k]]);
            for (int i = k + 1; i <= std::min(n - 1, k + bw); ++i) z[i] -= at(i, k) * z[k];
        }
        for (int i = n - 1; i >= 0; --i) {
            cd v = z[i];
            for (int j = i + 1; j <= std::min(n - 1, i + 2 * bw); ++j) v -= at(i, j) * z[j];
            z[i] = v / at(i, i);
        }
        for (const auto& q : prev) {
            cd d = 0;
            for (int i = 0; i < n; ++i) d += std::conj(q[i]) * z[i];
            for (int i = 0; i < n; ++i) z[i] -= d * q[i];
        }
        double nr = 0.0;
        for (int i = 0; i < n; ++i) nr += std::norm(z[i]);
        nr = std::sqrt(nr);
        if (!(nr > 0.0)) break;
        for (int i = 0; i < n; ++i) z[i] /= nr;
    }
    return z;
}

// Rayleigh-Ritz on an ne-dimensional subspace spanned by the columns of Y:
// M = Y^H H Y and G = Y^H Y (row-major ne x ne).  With G = L L^H (Cholesky)
// the pencil (M, G) becomes the Hermitian A = L^-1 M L^-H; its eigenpairs
// (A v = E v; bisection and inverse iteration on A as a band of width ne - 1)
// give C = L^-H V, so that Y C is orthonormal and (Y C)^H H (Y C) = diag(E).
// False if G is not positive definite.
static bool small_ritz(int ne, const std::vector<cd>& M, const std::vector<cd>& G, std::vector<double>& E,
                       std::vector<cd>& C) {
    std::vector<cd> L((size_t)ne * ne, cd(0));
    for (int j = 0; j < ne; ++j) {
        double d = G[(size_t)j * ne + j].real();
        for (int k = 0; k < j; ++k) d -= std::norm(L[(size_t)j * ne + k]);
        if (!(d > 0.0)) return false;
        L[(size_t)j * ne + j] = std::sqrt(d);
        for (int i = j + 1; i < ne; ++i) {
            cd v = G[(size_t)i * ne + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * ne + k] * std::conj(L[(size_t)j * ne + k]);
            L[(size_t)i * ne + j] = v / L[(size_t)j * ne + j];
        }
    }
    auto fwd = [&](std::vector<cd>& x) {  // x <- L^-1 x
        for (int i = 0; i < ne; ++i) {
            cd v = x[i];
            for (int k = 0; k < i; ++k) v -= L[(size_t)i * ne + k] * x[k];
            x[i] = v / L[(size_t)i * ne + i];
        }
    };
    // X = L^-1 M (column by column), A = (L^-1 X^H)^H
    std::vector<cd> X((size_t)ne * ne), A((size_t)ne * ne), col(ne);
    for (int c = 0; c < ne; ++c) {
        for (int i = 0; i < ne; ++i) col[i] = M[(size_t)i * ne + c];
        fwd(col);
        for (int i = 0; i < ne; ++i) X[(size_t)i * ne + c] = col[i];
    }
    for (int c = 0; c < ne; ++c) {
        for (int i = 0; i < ne; ++i) col[i] = std::conj(X[(size_t)c * ne + i]);  // column c of X^H
        fwd(col);
        for (int i = 0; i < ne; ++i) A[(size_t)c * ne + i] = std::conj(col[i]);
    }
    Band T;
    T.n = ne;
    T.bw = ne - 1;
    T.L.assign((size_t)ne * ne, cd(0));
    for (int i = 0; i < ne; ++i)
        for (int k = 0; k <= i; ++k)
            T.at(i, k) = 0.5 * (A[(size_t)i * ne + (i - k)] + std::conj(A[(size_t)(i - k) * ne + i]));
    E = band_lowest(T, ne);
    if ((int)E.size() != ne) return false;
    std::vector<std::vector<cd>> vs;
    C.assign((size_t)ne * ne, cd(0));
    for (int e = 0; e < ne; ++e) {
        std::vector<cd> v = band_vector(T, E[e], vs);
        // c = L^-H v: back substitution with the upper-triangular L^H
        std::vector<cd> c = v;
        for (int i = ne - 1; i >= 0; --i) {
            cd w = c[i];
            for (int k = i + 1; k < ne; ++k) w -= std::conj(L[(size_t)k * ne + i]) * c[k];
            c[i] = w / std::conj(L[(size_t)i * ne + i]);
        }
        for (int a = 0; a < ne; ++a) C[(size_t)a * ne + e] = c[a];
        vs.push_back(std::move(v));
    }
    return true;
}

// ------------------------------------------------------------------ batch construction and apply
static ed_status batch_init(ed_batch* B, const ed_hamiltonian* const* hs, int n) {
    if (!hs || n < 1) return fail(ED_ERR_ARG, "empty batch");
    B->hs.assign(hs, hs + n);
    B->n = n;
    const ed_basis* b0 = hs[0]->basis;
    B->alloc = &b0->alloc;
    B->w8 = b0->word == 8;
    B->chunked = b0->dt.chunk_lo > 0;
    B->n_sub = b0->ht.n_sub;
    B->ns_ok = true;
    B->row_off.assign(n + 1, 0);
    std::vector<HxArgs> desc(n);
    B->all_real = true;
    for (int s = 0; s < n; ++s) {
        const ed_hamiltonian* h = hs[s];
        if (!h) return fail(ED_ERR_ARG, "null Hamiltonian %d", s);
        const ed_basis* b = h->basis;
        if ((b->word == 8) != B->w8 || (b->dt.chunk_lo > 0) != B->chunked || b->ht.n_sub != B->n_sub ||
            b->ht.m != b0->ht.m)
            return fail(ED_ERR_ARG, "sector %d has a different state word or block structure", s);
        if (h->n_flip > 256) return fail(ED_ERR_ARG, "more than 256 flip terms");
        B->ns_ok = B->ns_ok && b->dt.dl_stride == 4;
        B->all_real = B->all_real && h->is_real;
        B->has_sun = B->has_sun || h->sun;
        desc[s] = make_args(h);
        B->row_off[s + 1] = B->row_off[s] + b->dim;
    }
    // every sector's tables must fit the batch's staging plan: the fewest
    // resident blocks any sector needs
    for (int k = 0; k < 4; ++k)
        for (int v = 0; v < 2; ++v) {
            int bl = 4;
            for (int s = 0; s < n; ++s) bl = std::min(bl, hx_default_blocks(hs[s], (ed_dtype)k, B->ns_ok, v ? 8 : 1));
            B->blocks[k][v] = bl;
            for (int s = 0; s < n; ++s)
                B->smem[k][v] = std::max(B->smem[k][v], hx_smem_bytes(hs[s], (ed_dtype)k, B->ns_ok, v ? 8 : 1, bl));
        }
    B->total = B->row_off[n];
    // reduction tiles: (sector, begin, end), TILE rows, never crossing sectors
    B->tiles.clear();
    for (int s = 0; s < n; ++s)
        for (int64_t i = 0; i < B->row_off[s + 1] - B->row_off[s]; i += TILE)
            B->tiles.insert(B->tiles.end(),
                            {(int64_t)s, i, std::min<int64_t>(i + TILE, B->row_off[s + 1] - B->row_off[s])});
    B->n_tiles = (int)(B->tiles.size() / 3);
    const Alloc& A = *B->alloc;
    auto up = [&](DevBuf& d, const void* src, size_t bytes) -> bool {
        d.bytes = bytes ? bytes : 16;
        d.p = A.get(d.bytes, 0);
        return d.p && (!bytes || cudaMemcpy(d.p, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess);
    };
    if (!up(B->d_desc, desc.data(), desc.size() * sizeof(HxArgs)) ||
        !up(B->d_row_off, B->row_off.data(), B->row_off.size() * 8) ||
        !up(B->d_tiles, B->tiles.data(), B->tiles.size() * 8))
        return fail(ED_ERR_NOMEM, "batch descriptors");
    B->d_counters.bytes = 32;
    B->d_counters.p = A.get(32, 0);
    if (!B->d_counters.p) return fail(ED_ERR_NOMEM, "batch counters");
    ED_CUDA(cudaMemset(B->d_counters.p, 0, 32));
    return ED_OK;
}

static int dkind(ed_dtype d) { return d == ED_F64 ? 0 : d == ED_F32 ? 1 : d == ED_C128 ? 2 : 3; }

// The stored-structure descriptors of the batch's sectors (uploaded when
// they change), or null when some sector has no one-segment structure.
static const CacheSector* stored_descs(const ed_batch* B, ed_status& st) {
    st = ED_OK;
    std::vector<CacheSector> d(B->n);
    int64_t slices = 0;
    for (int s = 0; s < B->n; ++s) {
        if (!cache_sector_desc(B->hs[s], d[s])) return nullptr;
        d[s].slice0 = slices;
        slices += d[s].ns;
    }
    const bool same = B->stored_h.size() == d.size() &&
                      memcmp(B->stored_h.data(), d.data(), d.size() * sizeof(CacheSector)) == 0;
    if (!same) {
        if (!B->d_stored.p) {
            B->d_stored.bytes = d.size() * sizeof(CacheSector);
            B->d_stored.p = B->alloc->get(B->d_stored.bytes, 0);
            if (!B->d_stored.p) {
                st = fail(ED_ERR_NOMEM, "batch descriptors");
                return nullptr;
            }
        }
        if (cudaMemcpy(B->d_stored.p, d.data(), d.size() * sizeof(CacheSector), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            st = fail(ED_ERR_CUDA, "descriptor upload");
            return nullptr;
        }
        B->stored_h = d;
        B->stored_slices = slices;
    }
    return (const CacheSector*)B->d_stored.p;
}

static BatchLaunch make_launch(const ed_batch* B, ed_dtype dt, const void* x, void* y, int nvec) {
    BatchLaunch L{};
    L.desc = (const HxArgs*)B->d_desc.p;
    L.row_off = (const int64_t*)B->d_row_off.p;
    L.n_sec = B->n;
    L.total_rows = B->total;
    L.smem = B->smem[(int)dt][nvec > 1 ? 1 : 0];
    L.blocks = B->blocks[(int)dt][nvec > 1 ? 1 : 0];
    L.w8 = B->w8;
    L.chunked = B->chunked;
    L.ns_ok = B->ns_ok;
    L.n_sub = B->n_sub;
    L.dtype = dt;
    L.nvec = nvec;
    L.x = x;
    L.y = y;
    L.counters = (unsigned long long*)B->d_counters.p;
    L.waves = B->waves[dkind(dt)][nvec > 1 ? 1 : 0];
    ed_status st;
    L.stored = stored_descs(B, st);
    L.stored_slices = B->stored_slices;
    return L;
}

}  // namespace ed

using namespace ed;

extern "C" {

ed_status ed_batch_create(const ed_hamiltonian* const* h, int32_t n, ed_batch** out) {
    if (!out) return fail(ED_ERR_ARG, "out is null");
    *out = nullptr;
    ed_batch* B = new ed_batch();
    ed_status st = batch_init(B, h, n);
    if (st != ED_OK) {
        ed_batch_free(B);
        return st;
    }
    *out = B;
    return ED_OK;
}

ed_status ed_batch_rows(const ed_batch* B, int64_t* row_off) {
    if (!B || !row_off) return fail(ED_ERR_ARG, "null argument");
    for (int s = 0; s <= B->n; ++s) row_off[s] = B->row_off[s];
    return ED_OK;
}

ed_status ed_apply_batch(const ed_batch* B, ed_dtype dtype, const void* x, void* y, int32_t nvec, ed_stream stream) {
    if (!B || !x || !y) return fail(ED_ERR_ARG, "null argument");
    if (nvec < 1 || nvec > 8) return fail(ED_ERR_ARG, "nvec out of range [1,8]");
    if ((dtype == ED_F64 || dtype == ED_F32) && !B->all_real)
        return fail(ED_ERR_ARG, "a complex sector needs a complex dtype");
    BatchLaunch L = make_launch(B, dtype, x, y, nvec);
    if (B->has_sun && !L.stored) return fail(ED_ERR_ARG, "a batch with SU(N) sectors needs every sector's stored structure");
    ED_CUDA(cudaMemsetAsync(B->d_counters.p, 0, 24, (cudaStream_t)stream));
    return apply_batch_launch(L, (cudaStream_t)stream);
}

ed_status ed_batch_autotune(ed_batch* B, ed_dtype dtype, const void* x, void* y, int32_t nvec, ed_stream stream,
                            int32_t* waves_out) {
    if (!B || !x || !y) return fail(ED_ERR_ARG, "null argument");
    if (nvec < 1 || nvec > 8) return fail(ED_ERR_ARG, "nvec out of range [1,8]");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    ED_CUDA(cudaEventCreate(&e0));
    ED_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_w = 1;
    for (int w : {1, 2, 4, 8, 16}) {
        BatchLaunch L = make_launch(B, dtype, x, y, nvec);
        L.waves = w;
        ed_status st = apply_batch_launch(L, s);  // warm-up
        if (st != ED_OK) return st;
        ED_CUDA(cudaEventRecord(e0, s));
        for (int r = 0; r < 3; ++r) {
            st = apply_batch_launch(L, s);
            if (st != ED_OK) return st;
        }
        ED_CUDA(cudaEventRecord(e1, s));
        ED_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        ED_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; best_w = w; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->waves[dkind(dtype)][nvec > 1 ? 1 : 0] = best_w;
    if (waves_out) *waves_out = best_w;
    return ED_OK;
}

void ed_batch_free(ed_batch* B) {
    if (!B) return;
    if (B->alloc) {
        B->alloc->put(B->d_desc.p, B->d_desc.bytes, 0);
        B->alloc->put(B->d_row_off.p, B->d_row_off.bytes, 0);
        B->alloc->put(B->d_tiles.p, B->d_tiles.bytes, 0);
        B->alloc->put(B->d_counters.p, B->d_counters.bytes, 0);
        B->alloc->put(B->d_stored.p, B->d_stored.bytes, 0);
    }
    delete B;
}

}  // extern "C"

namespace ed {

// start (optional): DEVICE start blocks of the vector kind (b columns per
// sector, the batch layout) instead of Gaussian ones; only (optional): the
// sectors that iterate (others keep their slots untouched); conv (optional):
// per sector whether it converged.
template <int K>
static ed_status block_lanczos(const ed_batch* B, const ed_block_lanczos_opts* o, double* evals,
                               ed_block_lanczos_report* rep, cudaStream_t user_stream, const void* start = nullptr,
                               const std::vector<int>* only = nullptr, std::vector<char>* conv = nullptr) {
    using T = typename BV<K>::T;
    auto t0 = std::chrono::steady_clock::now();
    const int n = B->n, b = o->block, kcap = o->max_iter + 1, nt = B->n_tiles;
    const int local = o->reorth ? 0 : 1;
    const int64_t tot = B->total;
    const int64_t bs = (int64_t)b * tot;  // elements per block vector
    const Alloc& A = *B->alloc;
    std::vector<std::pair<void*, size_t>> bufs;
    auto get = [&](size_t bytes) {
        void* p = A.get(bytes, 0);
        if (p) bufs.push_back({p, bytes});
        return p;
    };
    struct Free {
        std::vector<std::pair<void*, size_t>>& v;
        const Alloc& A;
        ~Free() {
            cudaDeviceSynchronize();
            for (auto& p : v) A.put(p.first, p.second, 0);
        }
    } freer{bufs, A};
    const int bb = b * b;
    T* V = (T*)get((size_t)kcap * bs * sizeof(T));
    T* W = (T*)get((size_t)bs * sizeof(T));
    double2* part = (double2*)get((size_t)kcap * nt * bb * sizeof(double2));
    double2* C1 = (double2*)get((size_t)n * kcap * bb * sizeof(double2));
    double2* C2 = (double2*)get((size_t)n * kcap * bb * sizeof(double2));
    double2* G = (double2*)get((size_t)n * kcap * bb * sizeof(double2));
    double2* Rinv = (double2*)get((size_t)n * bb * sizeof(double2));
    double2* Bacc = (double2*)get((size_t)n * bb * sizeof(double2));
    double2* Ahist = (double2*)get((size_t)n * kcap * bb * sizeof(double2));
    double2* Bhist = (double2*)get((size_t)n * kcap * bb * sizeof(double2));
    int* dk = (int*)get(16);
    int* tile_first = (int*)get((size_t)(n + 1) * 4);
    int* active = (int*)get((size_t)n * 4);  // 1 while a sector iterates; converged sectors drop out
    if (!V || !W || !part || !C1 || !C2 || !G || !Rinv || !Bacc || !Ahist || !Bhist || !dk || !tile_first || !active)
        return fail(ED_ERR_NOMEM, "block Lanczos workspace");
    // FP32 vectors: FP32 copies of the coefficients for the elementwise updates
    constexpr bool single = BV<K>::single;
    float2* C1f = nullptr;
    float2* C2f = nullptr;
    float2* Rinvf = nullptr;
    if (single) {
        C1f = (float2*)get((size_t)n * kcap * bb * sizeof(float2));
        C2f = (float2*)get((size_t)n * kcap * bb * sizeof(float2));
        Rinvf = (float2*)get((size_t)n * bb * sizeof(float2));
        if (!C1f || !C2f || !Rinvf) return fail(ED_ERR_NOMEM, "block Lanczos workspace");
    }
    std::vector<int> act_h(n, 1);
    if (only) act_h = *only;
    const int n_run = (int)std::count(act_h.begin(), act_h.end(), 1);
    ED_CUDA(cudaMemcpy(active, act_h.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
    {
        std::vector<int> tf(n + 1, 0);
        for (int t = 0, s = 0; s <= n; ++s) {
            while (t < nt && B->tiles[3 * t] < s) ++t;
            tf[s] = t;
        }
        tf[n] = nt;
        ED_CUDA(cudaMemcpy(tile_first, tf.data(), (n + 1) * 4, cudaMemcpyHostToDevice));
    }
    cudaStream_t s;
    ED_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct SFree {
        cudaStream_t s;
        ~SFree() { cudaStreamDestroy(s); }
    } sfree{s};
    (void)user_stream;
    int sms = 0, dev = 0;
    ED_CUDA(cudaGetDevice(&dev));
    ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned g = (unsigned)std::min<int64_t>((tot + 255) / 256, (int64_t)sms * 8);
    const int64_t* ro = (const int64_t*)B->d_row_off.p;
    const int64_t* tiles = (const int64_t*)B->d_tiles.p;
    const HxArgs* desc = (const HxArgs*)B->d_desc.p;
    // the elementwise block kernels specialised for the block size
    auto with_b = [&](auto f) {
        switch (b) {
            case 1: f(std::integral_constant<int, 1>{}); break;
            case 2: f(std::integral_constant<int, 2>{}); break;
            case 4: f(std::integral_constant<int, 4>{}); break;
            case 8: f(std::integral_constant<int, 8>{}); break;
            default: f(std::integral_constant<int, 0>{}); break;
        }
    };
    // start block V_0 = orth(X), via CholQR2 on the Gaussian block
    if (start) ED_CUDA(cudaMemcpyAsync(W, start, (size_t)bs * sizeof(T), cudaMemcpyDeviceToDevice, s));
    else bl_init<K><<<g, 256, 0, s>>>(W, desc, ro, n, b, o->seed, B->w8 ? 8 : 4);
    auto cholqr = [&](T* src, T* dst, int64_t dst_os, const int* kout, int kadd) {
        for (int pass = 0; pass < 2; ++pass) {
            bl_gram<K><<<dim3(nt, 1), 256, 0, s>>>(src, 0, nullptr, src, tiles, ro, b, part, nt, 0, active);
            bl_reduce<<<n, 128, 0, s>>>(part, tile_first, n, b, nt, nullptr, kcap, G, 0);
            bl_chol<<<(n + 63) / 64, 64, 0, s>>>(G, kcap, n, b, Rinv, Bacc, pass == 0, active, Rinvf);
            with_b([&](auto bt) {
                bl_scale<K, decltype(bt)::value><<<g, 256, 0, s>>>(src, pass == 0 ? src : dst, dst_os,
                                                                   pass == 0 ? nullptr : kout, kadd, Rinv, ro, n, b,
                                                                   active, Rinvf);
            });
        }
    };
    bl_set_int<<<1, 1, 0, s>>>(dk, 0);
    cholqr(W, V, bs, dk, 0);  // V_0
    ED_CUDA(cudaGetLastError());
    // one step, all sectors
    BatchLaunch L = make_launch(B, o->dtype, V, W, b);
    if (B->has_sun && !L.stored) return fail(ED_ERR_ARG, "a batch with SU(N) sectors needs every sector's stored structure");
    L.active = active;
    L.x_step = dk;
    L.x_step_elems = bs;
    auto step = [&]() -> ed_status {
        ed_status st = apply_batch_launch(L, s);  // W = H V_k
        if (st != ED_OK) return st;
        // Classical Gram-Schmidt against the stored blocks, then a second pass
        // against the last two: W = H V_k has large components only along
        // V_k and V_{k-1} (the block three-term relation); the first pass
        // leaves errors of order eps |H| there and far smaller ones along
        // older blocks, so repeating only the local part restores
        // orthogonality at half the FP64 cost of two full passes.
        for (int pass = 0; pass < 2; ++pass) {
            double2* Cp = pass == 0 ? C1 : C2;
            float2* Cpf = pass == 0 ? C1f : C2f;
            const int win = (local || pass == 1) ? 1 : 0;
            bl_gram<K><<<dim3(nt, win ? 2 : kcap), 256, 0, s>>>(V, bs, dk, W, tiles, ro, b, part, nt, win, active);
            bl_reduce<<<n, 128, 0, s>>>(part, tile_first, n, b, nt, dk, kcap, Cp, win, Cpf);
            with_b([&](auto bt) {
                bl_update<K, decltype(bt)::value><<<g, 256, 0, s>>>(W, V, bs, dk, Cp, kcap, ro, n, b, win, active, Cpf);
            });
        }
        cholqr(W, V, bs, dk, 1);  // V_{k+1} = W R^-1, B_k accumulated in Bacc
        bl_save<<<1, 256, 0, s>>>(C1, C2, Bacc, kcap, n, b, dk, Ahist, Bhist, kcap, active);
        return ED_OK;
    };
    // load every kernel of the step once outside any capture; the values this
    // writes (W, C1, the step-0 history) are recomputed by the first step
    {
        ed_status st = apply_batch_launch(L, s);
        if (st != ED_OK) return st;
        ED_CUDA(cudaMemsetAsync(C1, 0, (size_t)n * kcap * bb * sizeof(double2), s));
        if (single) ED_CUDA(cudaMemsetAsync(C1f, 0, (size_t)n * kcap * bb * sizeof(float2), s));
        with_b([&](auto bt) {
            bl_update<K, decltype(bt)::value><<<g, 256, 0, s>>>(W, V, bs, dk, C1, kcap, ro, n, b, local, active, C1f);
        });
        bl_save<<<1, 256, 0, s>>>(C1, C2, Bacc, kcap, n, b, dk, Ahist, Bhist, kcap, active);
        bl_set_int<<<1, 1, 0, s>>>(dk, 0);
        ED_CUDA(cudaGetLastError());
        ED_CUDA(cudaStreamSynchronize(s));
    }
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    if (o->use_graph) {
        ED_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        ed_status st = step();
        cudaGraph_t gr = nullptr;
        cudaError_t ce = cudaStreamEndCapture(s, &gr);
        if (st != ED_OK) return st;
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        graph = gr;
        ED_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
    }
    struct GFree {
        cudaGraphExec_t e;
        cudaGraph_t g;
        ~GFree() {
            if (e) cudaGraphExecDestroy(e);
            if (g) cudaGraphDestroy(g);
        }
    } gfree{gexec, graph};
    const int n_eig = o->n_eig;
    std::vector<std::vector<double>> prev(n, std::vector<double>(n_eig, 1e300)), cur = prev;
    std::vector<int> steady(n, 0);
    std::vector<double2> Ah((size_t)n * kcap * bb), Bh((size_t)n * kcap * bb);
    int iters = 0, conv_all = 0;
    double t_steps = 0;
    const int every = std::max(1, o->check_every);
    std::vector<int> its_last(n, 0);  // Krylov blocks of each sector's last check
    // Sector sct's T over its first `it` blocks (it*b square): diagonal blocks
    // A_j (Hermitian part), block (j+1, j) = B_j, in band storage.  Columns of
    // V_{j+1} that collapsed in the Cholesky QR (zero diagonal of B_j, a sector
    // smaller than the Krylov space) are left out; pos maps the full index
    // j b + a to T's row (-1 when left out).  Returns T's size.
    auto build_T = [&](int sct, int it, Band& T, std::vector<int>& pos) -> int {
        const int ntf = it * b;
        std::vector<char> valid(ntf, 1);
        double tn = 0.0;
        for (int j = 0; j < it; ++j) {
            const double2* Aj = &Ah[((size_t)sct * kcap + j) * bb];
            for (int r = 0; r < b; ++r) tn = std::max(tn, std::abs(cd(Aj[r * b + r].x, Aj[r * b + r].y)));
        }
        for (int j = 0; j + 1 < it; ++j) {
            const double2* Bj = &Bh[((size_t)sct * kcap + j) * bb];
            for (int r = 0; r < b; ++r)
                if (!(Bj[r * b + r].x > 1e-12 * std::max(tn, 1e-300))) valid[(j + 1) * b + r] = 0;
        }
        pos.assign(ntf, -1);
        int nk2 = 0;
        for (int q = 0; q < ntf; ++q)
            if (valid[q]) pos[q] = nk2++;
        T.n = nk2;
        T.bw = 2 * b - 1;
        T.L.assign((size_t)nk2 * (T.bw + 1), cd(0));
        auto put = [&](int r, int c, cd v) {  // lower-triangle entry (r >= c) of the full index space
            if (pos[r] < 0 || pos[c] < 0) return;
            T.at(pos[r], pos[r] - pos[c]) = v;
        };
        for (int j = 0; j < it; ++j) {
            const double2* Aj = &Ah[((size_t)sct * kcap + j) * bb];
            for (int r = 0; r < b; ++r)
                for (int c = 0; c <= r; ++c)
                    put(j * b + r, j * b + c,
                        0.5 * (cd(Aj[r * b + c].x, Aj[r * b + c].y) + std::conj(cd(Aj[c * b + r].x, Aj[c * b + r].y))));
            if (j + 1 < it) {
                const double2* Bj = &Bh[((size_t)sct * kcap + j) * bb];
                for (int r = 0; r < b; ++r)
                    for (int c = 0; c < b; ++c) put((j + 1) * b + r, j * b + c, cd(Bj[r * b + c].x, Bj[r * b + c].y));
            }
        }
        return nk2;
    };
    for (int k = 0; k + 1 < kcap; ++k) {
        auto ts = std::chrono::steady_clock::now();
        if (gexec) ED_CUDA(cudaGraphLaunch(gexec, s));
        else {
            ed_status st = step();
            if (st != ED_OK) return st;
        }
        ED_CUDA(cudaStreamSynchronize(s));
        t_steps += std::chrono::duration<double>(std::chrono::steady_clock::now() - ts).count();
        iters = k + 1;
        const bool last = k + 2 >= kcap;
        if ((k + 1) % every && !last) continue;
        ED_CUDA(cudaMemcpy(Ah.data(), Ahist, Ah.size() * sizeof(double2), cudaMemcpyDeviceToHost));
        ED_CUDA(cudaMemcpy(Bh.data(), Bhist, Bh.size() * sizeof(double2), cudaMemcpyDeviceToHost));
        const int nt2 = iters * b;
        auto check_sector = [&](int sct) {
            if (!act_h[sct]) return;  // converged earlier: its values stay
            its_last[sct] = iters;
            Band T;
            std::vector<int> pos;
            const int nk2 = build_T(sct, iters, T, pos);
            // FP32 vectors: eigenvalue changes below the FP32 noise of T count as steady
            const double floor32 = single ? 8.0 * 5.960464477539063e-08 * band_norm(T) : 0.0;
            // converged: every wanted value changed by at most tol/10 (relative)
            // since the last check, on two checks in a row, and its Ritz pair
            // has a small residual bound r (eigenvalue error at most
            // min(r, r^2/gap)), as in ed_lanczos; FP32 vectors stop at their
            // noise floor instead (the refinement below certifies the values)
            std::vector<double> lam, last;
            bool ok;
            if (b == 1) {
                std::vector<double> a1(nk2), b1(nk2, 0.0);
                for (int i = 0; i < nk2; ++i) a1[i] = T.get(i, 0).real();
                for (int i = 0; i + 1 < nk2; ++i) b1[i] = std::abs(T.get(i + 1, 1));
                tridiag_lowest(a1, b1, nk2, n_eig + 1, local != 0, 2.220446049250313e-16, lam, &last);
                const double2 bl = Bh[((size_t)sct * kcap + iters - 1) * bb];
                const double bh = nk2 < nt2 ? 0.0 : std::abs(cd(bl.x, bl.y));  // a collapsed column: invariant
                ok = (int)lam.size() >= n_eig;
                for (int e = 0; e < n_eig && ok; ++e) {
                    const double sc = std::max(1.0, fabs(lam[e]));
                    double gap = 1e300;
                    for (int q = 0; q < (int)lam.size(); ++q)
                        if (q != e) gap = std::min(gap, fabs(lam[q] - lam[e]));
                    const double rb = bh * fabs(last[e]);
                    if (!(rb <= std::max(o->tol * sc, floor32) || rb * rb <= o->tol * sc * gap)) ok = false;
                }
                if ((int)lam.size() > n_eig) lam.resize(n_eig);
            } else {
                // blocks: the wanted values first; only when all of them are
                // steady, the Ritz vector z of each (inverse iteration on T)
                // gives the residual |H y - lam y| = |B_last z_last| of y = V z
                // (z_last: the components in the last block), and only when
                // that alone does not settle it, b further values of T give
                // the gap (the host's band solves cost more than a step)
                lam = band_lowest(T, n_eig);
                ok = (int)lam.size() == n_eig;
                for (int e = 0; e < n_eig && ok; ++e) {
                    const double sc = std::max(1.0, fabs(lam[e]));
                    if (fabs(lam[e] - prev[sct][e]) > std::max(0.1 * o->tol * sc, floor32)) ok = false;
                }
                const double2* Bl = &Bh[((size_t)sct * kcap + iters - 1) * bb];
                std::vector<std::vector<cd>> zs;
                std::vector<double> more;  // n_eig + b lowest values, when a gap is needed
                for (int e = 0; e < n_eig && ok; ++e) {
                    std::vector<cd> z = band_vector(T, lam[e], zs);
                    double rb = 0.0;
                    for (int r = 0; r < b; ++r) {
                        cd v = 0;
                        for (int c = 0; c < b; ++c) {
                            const int q = pos[(iters - 1) * b + c];
                            if (q >= 0) v += cd(Bl[r * b + c].x, Bl[r * b + c].y) * z[q];
                        }
                        rb += std::norm(v);
                    }
                    rb = std::sqrt(rb);
                    zs.push_back(std::move(z));
                    const double sc = std::max(1.0, fabs(lam[e]));
                    if (rb <= std::max(o->tol * sc, floor32)) continue;
                    if (rb * rb > o->tol * sc * 2.0 * band_norm(T)) {  // no gap of T is that wide
                        ok = false;
                        continue;
                    }
                    if (more.empty()) more = band_lowest(T, n_eig + b);
                    const double same = std::max(10.0 * rb, 1e-6 * sc);  // copies of the same level
                    double gap = 1e300;
                    for (double q : more)
                        if (fabs(q - lam[e]) > same) gap = std::min(gap, fabs(q - lam[e]));
                    if (!(rb * rb <= o->tol * sc * gap)) ok = false;
                }
            }
            for (int e = 0; e < (int)lam.size(); ++e) {
                cur[sct][e] = lam[e];
                const double sc = std::max(1.0, fabs(lam[e]));
                if (fabs(lam[e] - prev[sct][e]) > std::max(0.1 * o->tol * sc, floor32)) ok = false;
            }
            steady[sct] = ok ? steady[sct] + 1 : 0;
            prev[sct] = cur[sct];
        };
        {
            // sectors are independent: spread them over the host's cores
            const int nth = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
            std::vector<std::thread> pool;
            for (int t = 1; t < nth; ++t)
                pool.emplace_back([&, t]() {
                    for (int sct = t; sct < n; sct += nth) check_sector(sct);
                });
            for (int sct = 0; sct < n; sct += nth) check_sector(sct);
            for (auto& th : pool) th.join();
        }
        int nconv = 0;
        bool changed = false;
        for (int sct = 0; sct < n; ++sct)
            if (steady[sct] >= 2 && (!only || (*only)[sct])) {
                ++nconv;
                if (act_h[sct]) {
                    act_h[sct] = 0;  // converged: later steps skip its rows
                    changed = true;
                }
            }
        if (changed && nconv < n_run) ED_CUDA(cudaMemcpy(active, act_h.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
        conv_all = nconv;
        if (nconv == n_run || last) break;
    }
    std::vector<char> okv(n, 0);  // per sector: converged
    for (int sct = 0; sct < n; ++sct) okv[sct] = steady[sct] >= 2 && (!only || (*only)[sct]);
    if constexpr (single) {
        // Refinement (as ed_lanczos's mixed path): per sector the Ritz vectors
        // of its n_eig lowest values in FP64 from the FP32 blocks, one FP64 H.x
        // of all of them in one batched launch, then Rayleigh-Ritz on their
        // span (a block run holds degenerate copies, which one quotient per
        // vector could not resolve) giving values E and vectors y with
        // residuals r = |Hy - E y| / |y|.  A sector counts as converged when
        // each value has r <= tol |E| or r^2 / gap <= tol |E| (the
        // Rayleigh-quotient error is at most r^2 / gap), gap = the distance
        // from E to the nearest FP32 Ritz value of another level, less r.
        constexpr int KO = BV<K>::cplx ? 2 : 0;
        using TO = typename BV<KO>::T;
        const int ne = n_eig, zcap = kcap * b;
        std::vector<double2> Zh((size_t)n * ne * zcap, make_double2(0, 0));
        std::vector<std::vector<double>> raw(n);
        auto ritz = [&](int sct) {
            Band T;
            std::vector<int> pos;
            const int it = std::max(1, its_last[sct]);
            build_T(sct, it, T, pos);
            raw[sct] = band_lowest(T, ne + b + 1);  // far enough to see copies of a degenerate level
            std::vector<std::vector<cd>> zs;
            for (int e = 0; e < ne && e < (int)raw[sct].size(); ++e) {
                std::vector<cd> z = band_vector(T, raw[sct][e], zs);
                for (int q = 0; q < it * b; ++q)
                    if (pos[q] >= 0) Zh[((size_t)sct * ne + e) * zcap + q] = make_double2(z[pos[q]].real(), z[pos[q]].imag());
                zs.push_back(std::move(z));
            }
        };
        {
            const int nth = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
            std::vector<std::thread> pool;
            for (int t = 1; t < nth; ++t)
                pool.emplace_back([&, t]() {
                    for (int sct = t; sct < n; sct += nth) ritz(sct);
                });
            for (int sct = 0; sct < n; sct += nth) ritz(sct);
            for (auto& th : pool) th.join();
        }
        for (int sct = 0; sct < n; ++sct) its_last[sct] = std::max(1, its_last[sct]);
        double2* Zd = (double2*)get(Zh.size() * sizeof(double2));
        int* its_d = (int*)get((size_t)n * 4);
        int* act_all = (int*)get((size_t)n * 4);
        TO* Y = (TO*)get((size_t)ne * tot * sizeof(TO));
        TO* HY = (TO*)get((size_t)ne * tot * sizeof(TO));
        double2* part2 = (double2*)get((size_t)nt * ne * ne * sizeof(double2));
        double2* Cq = (double2*)get((size_t)n * ne * ne * sizeof(double2));
        double* Ed = (double*)get((size_t)n * ne * sizeof(double));
        if (!Zd || !its_d || !act_all || !Y || !HY || !part2 || !Cq || !Ed)
            return fail(ED_ERR_NOMEM, "block Lanczos refinement workspace");
        const std::vector<int> ones(n, 1);
        ED_CUDA(cudaMemcpyAsync(Zd, Zh.data(), Zh.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
        ED_CUDA(cudaMemcpyAsync(its_d, its_last.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
        ED_CUDA(cudaMemcpyAsync(act_all, ones.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
        bl_combine<K, KO><<<g, 256, 0, s>>>(Y, ne, V, bs, Zd, zcap, its_d, ro, n, b);
        ED_CUDA(cudaGetLastError());
        BatchLaunch L2 = make_launch(B, KO == 0 ? ED_F64 : ED_C128, Y, HY, ne);
        L2.active = act_all;
        {
            const ed_status st = apply_batch_launch(L2, s);
            if (st != ED_OK) return st;
        }
        // per sector and column pair: sum_i conj(X_a[i]) Z_c[i]
        auto sums = [&](const TO* X, const TO* Z, std::vector<double2>& out) -> ed_status {
            bl_gram<KO><<<dim3(nt, 1), 256, 0, s>>>(X, 0, nullptr, Z, tiles, ro, ne, part2, nt, 0, act_all);
            bl_reduce<<<n, 128, 0, s>>>(part2, tile_first, n, ne, nt, nullptr, 1, Cq, 0);
            ED_CUDA(cudaGetLastError());
            out.resize((size_t)n * ne * ne);
            ED_CUDA(cudaMemcpyAsync(out.data(), Cq, out.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
            ED_CUDA(cudaStreamSynchronize(s));
            return ED_OK;
        };
        std::vector<double2> yhy, yy, rr;
        ed_status st = sums(Y, HY, yhy);
        if (st == ED_OK) st = sums(Y, Y, yy);
        if (st != ED_OK) return st;
        // Rayleigh-Ritz per sector on the span of its refined vectors
        std::vector<double> E((size_t)n * ne, 0.0);
        std::vector<double2> Ch((size_t)n * ne * ne, make_double2(0, 0));
        std::vector<char> rr_ok(n, 1);
        for (int sct = 0; sct < n; ++sct) {
            std::vector<cd> Mh((size_t)ne * ne), Gh((size_t)ne * ne), Cs;
            for (size_t q = 0; q < (size_t)ne * ne; ++q) {
                const double2 m = yhy[(size_t)sct * ne * ne + q], gq = yy[(size_t)sct * ne * ne + q];
                Mh[q] = cd(m.x, m.y);
                Gh[q] = cd(gq.x, gq.y);
            }
            std::vector<double> Es;
            if (small_ritz(ne, Mh, Gh, Es, Cs)) {
                for (int e = 0; e < ne; ++e) E[(size_t)sct * ne + e] = Es[e];
                for (size_t q = 0; q < (size_t)ne * ne; ++q)
                    Ch[(size_t)sct * ne * ne + q] = make_double2(Cs[q].real(), Cs[q].imag());
            } else {  // a degenerate subspace: keep the vectors, report unrefined values
                rr_ok[sct] = 0;
                for (int e = 0; e < ne; ++e) {
                    E[(size_t)sct * ne + e] = cur[sct][e];
                    Ch[((size_t)sct * ne + e) * ne + e] = make_double2(1, 0);
                }
            }
        }
        double2* Cd = (double2*)get(Ch.size() * sizeof(double2));
        if (!Cd) return fail(ED_ERR_NOMEM, "block Lanczos refinement workspace");
        ED_CUDA(cudaMemcpyAsync(Cd, Ch.data(), Ch.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
        bl_rotate<KO><<<g, 256, 0, s>>>(Y, HY, Cd, ne, ro, n);
        ED_CUDA(cudaMemcpyAsync(Ed, E.data(), E.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        bl_resid<KO><<<g, 256, 0, s>>>(HY, Y, Ed, ne, ro, n);
        ED_CUDA(cudaGetLastError());
        st = sums(HY, HY, rr);
        if (st == ED_OK) st = sums(Y, Y, yy);
        if (st != ED_OK) return st;
        auto dg = [&](const std::vector<double2>& v, int sct, int e) { return v[((size_t)sct * ne + e) * ne + e].x; };
        int certified = 0;
        std::vector<int> polish(n, 0);
        for (int sct = 0; sct < n; ++sct) {
            if (only && !(*only)[sct]) continue;
            bool ok = rr_ok[sct] != 0;
            for (int e = 0; e < ne; ++e) {
                const double en = E[(size_t)sct * ne + e], nrm = dg(yy, sct, e);
                const double r = nrm > 0 ? std::sqrt(std::max(dg(rr, sct, e) / nrm, 0.0)) : 1e300;
                const double sc = std::max(1.0, fabs(en));
                // gap: distance to the nearest other level of T (values within
                // max(10 r, 1e-6 |E|) of E count as copies of E's own level)
                const double same = std::max(10.0 * r, 1e-6 * sc);
                double gap = 1e300;
                for (double q : raw[sct])
                    if (fabs(q - en) > same) gap = std::min(gap, fabs(q - en));
                gap = std::max(gap - r, 1e-300);
                if (!(r <= o->tol * sc || r * r <= o->tol * sc * gap)) ok = false;
                cur[sct][e] = en;
            }
            if (ok) ++certified;
            else polish[sct] = 1;
        }
        // Sectors whose values the FP32 Ritz vectors cannot certify (a close
        // next level) continue in FP64: block Lanczos with their refined
        // vectors as the start block (one vector per value), only these
        // sectors iterating; from such a start it converges in a few steps.
        if (std::count(polish.begin(), polish.end(), 1) > 0) {
            ed_block_lanczos_opts o2 = *o;
            o2.dtype = KO == 0 ? ED_F64 : ED_C128;
            o2.block = ne;
            o2.reorth = 1;
            o2.max_iter = std::min(o->max_iter, 60);
            std::vector<double> ev2((size_t)n * ne, 0.0);
            std::vector<char> ok2;
            const ed_status st2 = block_lanczos<KO>(B, &o2, ev2.data(), nullptr, user_stream, Y, &polish, &ok2);
            if (st2 != ED_OK && st2 != ED_ERR_NOT_CONVERGED) return st2;
            for (int sct = 0; sct < n; ++sct)
                if (polish[sct] && ok2[sct]) {
                    for (int e = 0; e < ne; ++e) cur[sct][e] = ev2[(size_t)sct * ne + e];
                    ++certified;
                    polish[sct] = 0;
                }
        }
        conv_all = certified;
        for (int sct = 0; sct < n; ++sct) okv[sct] = (!only || (*only)[sct]) && !polish[sct];
    }
    for (int sct = 0; sct < n; ++sct)
        for (int e = 0; e < n_eig; ++e) evals[(size_t)sct * n_eig + e] = cur[sct][e];
    if (rep) {
        rep->iters = iters;
        rep->converged_sectors = conv_all;
        rep->krylov_dim = iters * b;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        rep->step_seconds = t_steps;
        rep->used_graph = gexec ? 1 : 0;
    }
    if (conv) *conv = okv;
    return conv_all == n_run ? ED_OK : fail(ED_ERR_NOT_CONVERGED, "%d of %d sectors converged", conv_all, n_run);
}

}  // namespace ed

extern "C" ed_status ed_band_eigs(const double* band, int32_t n, int32_t bw, int32_t k, double* evals, double* evecs,
                                  int32_t* n_found) {
    if (!band || !evals || n < 1 || bw < 0 || k < 1) return fail(ED_ERR_ARG, "bad argument");
    if (bw > n - 1) bw = n - 1;
    Band T;
    T.n = n;
    T.bw = bw;
    T.L.assign((size_t)n * (bw + 1), cd(0));
    for (int i = 0; i < n; ++i)
        for (int q = 0; q <= bw && q <= i; ++q) {
            const double* v = band + 2 * ((size_t)i * (bw + 1) + q);
            T.at(i, q) = q == 0 ? cd(v[0], 0.0) : cd(v[0], v[1]);  // the diagonal of a Hermitian T is real
        }
    const std::vector<double> lam = band_lowest(T, k);
    std::vector<std::vector<cd>> zs;
    for (size_t e = 0; e < lam.size(); ++e) {
        evals[e] = lam[e];
        if (evecs) {
            std::vector<cd> z = band_vector(T, lam[e], zs);
            for (int i = 0; i < n; ++i) {
                evecs[2 * ((size_t)e * n + i)] = z[i].real();
                evecs[2 * ((size_t)e * n + i) + 1] = z[i].imag();
            }
            zs.push_back(std::move(z));
        }
    }
    if (n_found) *n_found = (int32_t)lam.size();
    return ED_OK;
}

extern "C" ed_status ed_lanczos_batch(const ed_batch* B, const ed_block_lanczos_opts* o, double* evals,
                                      ed_block_lanczos_report* rep, ed_stream stream) {
    if (!B || !o || !evals) return fail(ED_ERR_ARG, "null argument");
    if (o->block < 1 || o->block > 8) return fail(ED_ERR_ARG, "block size out of range [1,8]");
    if (o->n_eig < 1 || o->n_eig > 64) return fail(ED_ERR_ARG, "n_eig out of range");
    if (o->max_iter < 2 || o->max_iter > 400) return fail(ED_ERR_ARG, "max_iter out of range [2,400]");
    // blocks of several vectors keep full reorthogonalisation: without it, the
    // copies of converged values cannot be told from genuine multiplicities
    if (!o->reorth && o->block != 1) return fail(ED_ERR_ARG, "the plain recursion needs block = 1");
    if (o->dtype == ED_F64 || o->dtype == ED_F32) {
        if (!B->all_real) return fail(ED_ERR_ARG, "a complex sector needs a complex dtype");
    }
    if (o->dtype == ED_F32 || o->dtype == ED_C64) {
        // FP32 vectors: the Ritz vectors for the FP64 refinement come from the stored blocks
        if (!o->reorth) return fail(ED_ERR_ARG, "FP32 vectors need full reorthogonalisation");
        if (o->n_eig > 8) return fail(ED_ERR_ARG, "FP32 vectors: n_eig at most 8");
    }
    switch (o->dtype) {
        case ED_F64: return block_lanczos<0>(B, o, evals, rep, (cudaStream_t)stream);
        case ED_F32: return block_lanczos<1>(B, o, evals, rep, (cudaStream_t)stream);
        case ED_C128: return block_lanczos<2>(B, o, evals, rep, (cudaStream_t)stream);
        case ED_C64: return block_lanczos<3>(B, o, evals, rep, (cudaStream_t)stream);
    }
    return fail(ED_ERR_ARG, "bad dtype");
}
