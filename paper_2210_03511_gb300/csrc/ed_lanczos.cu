// Lanczos eigensolver on the device (Eqs. lanczosrecursionabbrev, tmatrix;
// Algs. "Real-symmetric Lanczos step" and "Complex-Hermitian Lanczos step").
//
// Per step: w = H v_n; alpha_n = Re<v_n|w>; w -= alpha_n v_n + beta_n v_{n-1};
// optionally full reorthogonalisation against all stored v (classical
// Gram-Schmidt, then once more against v_{n-1}, v_n); beta_{n+1} = ||w||;
// v_{n+1} = w / beta_{n+1}.
// Vectors are stored in the caller's dtype; every inner product accumulates
// in FP64 with a fixed reduction tree (deterministic).  alpha and beta stay on
// the device for the vector updates and are copied to the host for the
// T-matrix, whose lowest eigenpairs are found in FP64 by Sturm bisection and
// inverse iteration.
#include <math.h>
#include <string.h>

#include <sys/mman.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "ed_internal.h"

namespace ed {

template <int K> struct LV;
template <> struct LV<0> { using T = double; static constexpr bool cplx = false; };
template <> struct LV<1> { using T = float; static constexpr bool cplx = false; };
template <> struct LV<2> { using T = double2; static constexpr bool cplx = true; };
template <> struct LV<3> { using T = float2; static constexpr bool cplx = true; };

__device__ __forceinline__ double2 ld2(const double& v) { return make_double2(v, 0.0); }
__device__ __forceinline__ double2 ld2(const float& v) { return make_double2((double)v, 0.0); }
__device__ __forceinline__ double2 ld2(const double2& v) { return v; }
__device__ __forceinline__ double2 ld2(const float2& v) { return make_double2((double)v.x, (double)v.y); }
__device__ __forceinline__ void st2(double& d, double2 v) { d = v.x; }
__device__ __forceinline__ void st2(float& d, double2 v) { d = (float)v.x; }
__device__ __forceinline__ void st2(double2& d, double2 v) { d = v; }
__device__ __forceinline__ void st2(float2& d, double2 v) { d = make_float2((float)v.x, (float)v.y); }

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) keyed by the state integer.
__device__ __forceinline__ uint64_t smix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double keyed_u(uint64_t seed, int stream, uint64_t state) {
    const uint64_t key = smix(seed * 256ull + (uint64_t)stream);
    return (double)(smix(state ^ key) >> 11) * (1.0 / 9007199254740992.0);
}

template <typename W, int K>
__global__ void init_random(typename LV<K>::T* v, const W* reps, int64_t n, uint64_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t st = (uint64_t)reps[i];
        double2 z = make_double2(2.0 * keyed_u(seed, 0, st) - 1.0, LV<K>::cplx ? 2.0 * keyed_u(seed, 1, st) - 1.0 : 0.0);
        st2(v[i], z);
    }
}

__device__ __forceinline__ double2 block_sum2(double2 v) {
    __shared__ double2 red[32];
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : make_double2(0, 0);
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, o);
            v.y += __shfl_down_sync(0xffffffffu, v.y, o);
        }
    }
    return v;  // valid in thread 0
}

// partial[blockIdx.y * gridDim.x + blockIdx.x] = sum_i conj(A_k[i]) b[i] over this block's slice
template <int K>
__global__ void multi_dot(const typename LV<K>::T* A, int64_t ld, const typename LV<K>::T* b, int64_t n,
                          double2* partial) {
    const typename LV<K>::T* a = A + (int64_t)blockIdx.y * ld;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(n, i0 + per);
    double2 acc = make_double2(0, 0);
    if constexpr (!LV<K>::cplx) {
        // real vectors: one FP64 FMA per element (FP64 throughput is scarce on this GPU)
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc.x += (double)a[i] * (double)b[i];
    } else {
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const double2 x = ld2(a[i]), y = ld2(b[i]);
            acc.x += x.x * y.x + x.y * y.y;
            acc.y += x.x * y.y - x.y * y.x;
        }
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// Reorthogonalisation coefficients for FP32 vectors: each thread forms
// partial sums of 16 consecutive products in FP32 and adds them to its FP64
// accumulator (GB300 has little FP64 throughput).  The coefficients then
// carry a relative error ~16 eps_32 of sum |x_i y_i|, far below what
// keeping the Lanczos vectors orthogonal to working precision needs; the
// Lanczos coefficients alpha and beta keep full FP64 accumulation.
template <int K>
__global__ void multi_dot_f32(const typename LV<K>::T* A, int64_t ld, const typename LV<K>::T* b, int64_t n,
                              double2* partial) {
    static_assert(K == 1 || K == 3, "FP32 vectors only");
    const typename LV<K>::T* a = A + (int64_t)blockIdx.y * ld;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(n, i0 + per);
    double2 acc = make_double2(0, 0);
    float cx = 0.f, cy = 0.f;
    int cnt = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        if constexpr (K == 1) {
            cx = fmaf(a[i], b[i], cx);
        } else {
            const float2 x = a[i], y = b[i];
            cx = fmaf(x.x, y.x, fmaf(x.y, y.y, cx));
            cy = fmaf(x.x, y.y, fmaf(-x.y, y.x, cy));
        }
        if (++cnt == 16) {
            acc.x += (double)cx;
            acc.y += (double)cy;
            cx = cy = 0.f;
            cnt = 0;
        }
    }
    acc.x += (double)cx;
    acc.y += (double)cy;
    acc = block_sum2(acc);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// w -= sum_k c_k A_k in FP32 arithmetic for FP32 vectors (the coefficients
// of a reorthogonalisation are small, so the FP32 update adds no error above
// the rounding of w itself)
template <int K>
__global__ void multi_axpy_f32(typename LV<K>::T* w, const typename LV<K>::T* A, int64_t ld, int nk, const double2* c,
                               int64_t n) {
    static_assert(K == 1 || K == 3, "FP32 vectors only");
    __shared__ float2 cf[2048];  // nk <= max_iter + 1 <= 2001 (ed_lanczos checks max_iter)
    for (int k = threadIdx.x; k < nk; k += blockDim.x) cf[k] = make_float2((float)c[k].x, (float)c[k].y);
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (K == 1) {
            float x = w[i];
            for (int k = 0; k < nk; ++k) x = fmaf(-cf[k].x, A[(int64_t)k * ld + i], x);
            w[i] = x;
        } else {
            float2 x = w[i];
            for (int k = 0; k < nk; ++k) {
                const float2 a = A[(int64_t)k * ld + i];
                x.x -= cf[k].x * a.x - cf[k].y * a.y;
                x.y -= cf[k].x * a.y + cf[k].y * a.x;
            }
            w[i] = x;
        }
    }
}

// out[k] = sum over nb partials (fixed order)
__global__ void reduce_partials(const double2* partial, int nb, int nk, double2* out) {
    for (int k = blockIdx.x; k < nk; k += gridDim.x) {
        double2 acc = make_double2(0, 0);
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            acc.x += partial[(int64_t)k * nb + i].x;
            acc.y += partial[(int64_t)k * nb + i].y;
        }
        acc = block_sum2(acc);
        if (threadIdx.x == 0) out[k] = acc;
    }
}

// w -= alpha v + beta vprev  (alpha = Re sc[0], beta = sc[1].x; vprev may be null)
template <int K>
__global__ void lanczos_axpy(typename LV<K>::T* w, const typename LV<K>::T* v, const typename LV<K>::T* vp, int64_t n,
                             const double2* alpha, const double* beta) {
    const double a = alpha->x;
    const double bt = vp ? *beta : 0.0;
    if constexpr (!LV<K>::cplx) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            double x = (double)w[i] - a * (double)v[i];
            if (vp) x -= bt * (double)vp[i];
            w[i] = (typename LV<K>::T)x;
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            double2 x = ld2(w[i]);
            const double2 y = ld2(v[i]);
            x.x -= a * y.x;
            x.y -= a * y.y;
            if (vp) {
                const double2 z = ld2(vp[i]);
                x.x -= bt * z.x;
                x.y -= bt * z.y;
            }
            st2(w[i], x);
        }
    }
}

// w -= sum_k c_k A_k  (classical Gram-Schmidt update)
template <int K>
__global__ void multi_axpy(typename LV<K>::T* w, const typename LV<K>::T* A, int64_t ld, int nk, const double2* c,
                           int64_t n) {
    if constexpr (!LV<K>::cplx) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            double x = (double)w[i];
            for (int k = 0; k < nk; ++k) x -= c[k].x * (double)A[(int64_t)k * ld + i];
            w[i] = (typename LV<K>::T)x;
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            double2 x = ld2(w[i]);
            for (int k = 0; k < nk; ++k) {
                const double2 a = ld2(A[(int64_t)k * ld + i]);
                const double2 ck = c[k];
                x.x -= ck.x * a.x - ck.y * a.y;
                x.y -= ck.x * a.y + ck.y * a.x;
            }
            st2(w[i], x);
        }
    }
}

// out = sum_k s_k A_k with real coefficients s (FP64 accumulation, output type O)
template <int K, typename O>
__global__ void combine(O* out, const typename LV<K>::T* A, int64_t ld, int nk, const double* s, int64_t n) {
    if constexpr (!LV<K>::cplx) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            double x = 0.0;
            for (int k = 0; k < nk; ++k) x += s[k] * (double)A[(int64_t)k * ld + i];
            st2(out[i], make_double2(x, 0.0));
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            double2 x = make_double2(0, 0);
            for (int k = 0; k < nk; ++k) {
                const double2 a = ld2(A[(int64_t)k * ld + i]);
                x.x += s[k] * a.x;
                x.y += s[k] * a.y;
            }
            st2(out[i], x);
        }
    }
}

// out = sum_k c_k A_k with complex coefficients c (FP64 accumulation)
template <int K>
__global__ void combine_c(typename LV<K>::T* out, const typename LV<K>::T* A, int64_t ld, int nk, const double2* c,
                          int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 x = make_double2(0, 0);
        for (int k = 0; k < nk; ++k) {
            const double2 a = ld2(A[(int64_t)k * ld + i]);
            x.x += c[k].x * a.x - c[k].y * a.y;
            x.y += c[k].x * a.y + c[k].y * a.x;
        }
        st2(out[i], x);
    }
}

// out_k += c[k] v for k < nk (out_k = out + k*ldo): the second pass of the
// plain recursion builds Ritz vectors one Lanczos vector at a time
template <int K, typename O>
__global__ void accumulate(O* out, int64_t ldo, int nk, const double* c, const typename LV<K>::T* v, int64_t n) {
    if constexpr (!LV<K>::cplx) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const double a = (double)v[i];
            for (int k = 0; k < nk; ++k) {
                const double x = ld2(out[(int64_t)k * ldo + i]).x + c[k] * a;
                st2(out[(int64_t)k * ldo + i], make_double2(x, 0.0));
            }
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const double2 a = ld2(v[i]);
            for (int k = 0; k < nk; ++k) {
                double2 x = ld2(out[(int64_t)k * ldo + i]);
                x.x += c[k] * a.x;
                x.y += c[k] * a.y;
                st2(out[(int64_t)k * ldo + i], x);
            }
        }
    }
}

// dst = src * (1/norm), norm = sqrt(Re nrm2->x) unless given as beta
template <int K>
__global__ void scale_by(typename LV<K>::T* dst, const typename LV<K>::T* src, int64_t n, const double* beta) {
    const double inv = 1.0 / *beta;
    if constexpr (!LV<K>::cplx) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            dst[i] = (typename LV<K>::T)((double)src[i] * inv);
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            double2 x = ld2(src[i]);
            x.x *= inv;
            x.y *= inv;
            st2(dst[i], x);
        }
    }
}

__global__ void sqrt_re(const double2* in, double* out) { *out = sqrt(in->x); }

// Fused Lanczos step kernels.  Each ends with a grid-wide sum: every block
// writes its partial, and the block that finishes last (one atomic counter,
// no waiting) adds all partials in index order with a fixed tree, so the
// result does not depend on which block was last.  The counter is reset by
// that block for the next launch.
__device__ __forceinline__ bool last_block_done(unsigned int* counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    return last;
}

__device__ __forceinline__ double2 sum_partials(const double2* partial, int nb) {
    double2 acc = make_double2(0, 0);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const double2 v = __ldcg(partial + i);  // L2: written by other blocks of this launch
        acc.x += v.x;
        acc.y += v.y;
    }
    return block_sum2(acc);  // valid in thread 0
}

// *out = sum_i conj(a_i) b_i (alpha of a Lanczos step: a = v_n, b = w = H v_n)
template <int K>
__global__ void dot_step(const typename LV<K>::T* a, const typename LV<K>::T* b, int64_t n, double2* partial,
                         unsigned int* counter, double2* out) {
    double2 acc = make_double2(0, 0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (!LV<K>::cplx) {
            acc.x += (double)a[i] * (double)b[i];
        } else {
            const double2 x = ld2(a[i]), y = ld2(b[i]);
            acc.x += x.x * y.x + x.y * y.y;
            acc.y += x.x * y.y - x.y * y.x;
        }
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
    if (last_block_done(counter)) {
        const double2 t = sum_partials(partial, gridDim.x);
        if (threadIdx.x == 0) {
            *out = t;
            *counter = 0u;
        }
    }
}

// w -= alpha v + beta_prev vprev (the arithmetic of lanczos_axpy, so that the
// second pass of the plain recursion regenerates the vectors bit for bit),
// then beta_next = |w| of the stored (rounded) w.
template <int K>
__global__ void axpy_norm_step(typename LV<K>::T* w, const typename LV<K>::T* v, const typename LV<K>::T* vp,
                               int64_t n, const double2* alpha, const double* beta_prev, double2* partial,
                               unsigned int* counter, double* beta_next) {
    const double a = alpha->x;
    const double bt = vp ? *beta_prev : 0.0;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (!LV<K>::cplx) {
            double x = (double)w[i] - a * (double)v[i];
            if (vp) x -= bt * (double)vp[i];
            const typename LV<K>::T xr = (typename LV<K>::T)x;
            w[i] = xr;
            acc += (double)xr * (double)xr;
        } else {
            double2 x = ld2(w[i]);
            const double2 y = ld2(v[i]);
            x.x -= a * y.x;
            x.y -= a * y.y;
            if (vp) {
                const double2 z = ld2(vp[i]);
                x.x -= bt * z.x;
                x.y -= bt * z.y;
            }
            st2(w[i], x);
            const double2 xr = ld2(w[i]);
            acc += xr.x * xr.x + xr.y * xr.y;
        }
    }
    const double2 bs = block_sum2(make_double2(acc, 0.0));
    if (threadIdx.x == 0) partial[blockIdx.x] = bs;
    if (last_block_done(counter)) {
        const double2 t = sum_partials(partial, gridDim.x);
        if (threadIdx.x == 0) {
            *beta_next = sqrt(t.x);
            *counter = 0u;
        }
    }
}

// *beta_next = sqrt(sum of the nb partial squared norms) (the reorthogonalised
// step's |w|, from multi_dot partials)
__global__ void norm_from_partials(const double2* partial, int nb, double* beta_next) {
    const double2 t = sum_partials(partial, nb);
    if (threadIdx.x == 0) *beta_next = sqrt(t.x);
}

// r = Hy - E y ; FP64 vectors of kind K (0 or 2)
template <int K>
__global__ void residual(typename LV<K>::T* r, const typename LV<K>::T* hy, const typename LV<K>::T* y, int64_t n,
                         double E) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 a = ld2(hy[i]);
        const double2 b = ld2(y[i]);
        a.x -= E * b.x;
        a.y -= E * b.y;
        st2(r[i], a);
    }
}

// ---------------------------------------------------------------- host tridiagonal eigensolver
// Number of eigenvalues of T (diag a, off-diag b) smaller than x (Sturm count
// from the pivots of the LDL^T factorisation of T - x).
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, int n, double x) {
    int cnt = 0;
    double q = a[0] - x;
    const double tiny = 1e-300;
    if (q < 0) ++cnt;
    for (int i = 1; i < n; ++i) {
        if (q == 0.0) q = tiny;
        q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

static double kth_eig(const std::vector<double>& a, const std::vector<double>& b, int n, int k) {
    double lo = a[0], hi = a[0];
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < n - 1 ? fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(a, b, n, mid) > k) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Solve (T - lam) z = rhs by Gaussian elimination with partial pivoting on the
// tridiagonal band (one extra superdiagonal appears from row swaps).
static void tri_solve(const std::vector<double>& a, const std::vector<double>& b, int n, double lam,
                      std::vector<double>& z) {
    std::vector<double> dl(n), d(n), du(n), du2(n, 0.0);
    for (int i = 0; i < n; ++i) {
        d[i] = a[i] - lam;
        dl[i] = i < n - 1 ? b[i] : 0.0;
        du[i] = i < n - 1 ? b[i] : 0.0;
    }
    const double tiny = 1e-300 + 1e-15 * (fabs(lam) + 1.0) * 1e-3;
    for (int i = 0; i < n - 1; ++i) {
        if (fabs(d[i]) >= fabs(dl[i])) {
            if (d[i] == 0.0) d[i] = tiny;
            const double f = dl[i] / d[i];
            d[i + 1] -= f * du[i];
            z[i + 1] -= f * z[i];
            dl[i] = 0.0;
        } else {
            // swap rows i and i+1
            const double f = d[i] / dl[i];
            d[i] = dl[i];
            const double t = d[i + 1];
            d[i + 1] = du[i] - f * t;
            if (i < n - 2) {
                du2[i] = du[i + 1];
                du[i + 1] = -f * du2[i];
            }
            du[i] = t;
            std::swap(z[i], z[i + 1]);
            z[i + 1] -= f * z[i];
            dl[i] = 0.0;
        }
    }
    if (d[n - 1] == 0.0) d[n - 1] = tiny;
    z[n - 1] /= d[n - 1];
    if (n > 1) z[n - 2] = (z[n - 2] - du[n - 2] * z[n - 1]) / d[n - 2];
    for (int i = n - 3; i >= 0; --i) z[i] = (z[i] - du[i] * z[i + 1] - du2[i] * z[i + 2]) / d[i];
}

// Lowest k eigenpairs of the n x n T-matrix.
static void tri_eig(const std::vector<double>& a, const std::vector<double>& b, int n, int k, std::vector<double>& lam,
                    std::vector<std::vector<double>>& vec) {
    k = std::min(k, n);
    lam.assign(k, 0.0);
    vec.assign(k, std::vector<double>(n, 0.0));
    for (int j = 0; j < k; ++j) {
        lam[j] = kth_eig(a, b, n, j);
        std::vector<double>& z = vec[j];
        for (int i = 0; i < n; ++i) z[i] = 1.0 + 0.01 * ((i * 7919 + 13 * j) % 101);
        for (int it = 0; it < 3; ++it) {
            tri_solve(a, b, n, lam[j], z);
            // keep orthogonal to earlier vectors of (near-)equal eigenvalues
            for (int p = 0; p < j; ++p) {
                if (fabs(lam[p] - lam[j]) > 1e-10 * (1.0 + fabs(lam[j]))) continue;
                double dp = 0;
                for (int i = 0; i < n; ++i) dp += z[i] * vec[p][i];
                for (int i = 0; i < n; ++i) z[i] -= dp * vec[p][i];
            }
            double nr = 0;
            for (int i = 0; i < n; ++i) nr += z[i] * z[i];
            nr = sqrt(nr);
            if (nr == 0.0) break;
            for (int i = 0; i < n; ++i) z[i] /= nr;
        }
    }
}

// Lowest k eigenpairs of T after removing the spurious copies that the plain
// recursion (no reorthogonalisation) produces once Lanczos vectors lose
// orthogonality (Cullum and Willoughby, "Lanczos Algorithms for Large
// Symmetric Eigenvalue Computations", 1985).  Ritz values within `cluster` of
// each other are copies of one eigenvalue and count once; a value without
// copies that is also an eigenvalue of T^ (T without its first row and
// column, within `cw`) is spurious and dropped.  Each kept value gets a
// T-eigenvector by inverse iteration (for a multiple value: a vector of the
// near-invariant subspace of its copies).
static void tri_eig_filtered(const std::vector<double>& a, const std::vector<double>& b, int n, int k,
                             double cluster, double cw, std::vector<double>& lam,
                             std::vector<std::vector<double>>& vec) {
    lam.clear();
    std::vector<double> ah(a.begin() + 1, a.begin() + n), bh;
    if (n > 2) bh.assign(b.begin() + 1, b.begin() + n - 1);
    bh.resize(std::max(0, n - 1), 0.0);
    int m = std::min(n, 3 * k + 6);
    while (true) {
        std::vector<double> th(m);
        for (int j = 0; j < m; ++j) th[j] = kth_eig(a, b, n, j);
        lam.clear();
        int j = 0;
        while (j < m && (int)lam.size() < k) {
            int e = j + 1;
            while (e < m && th[e] - th[e - 1] <= cluster) ++e;
            // a cluster reaching the end of the computed values may continue
            if (e == m && m < n) break;
            bool keep = e - j >= 2;
            if (!keep) {
                keep = true;
                if (n > 1) {
                    const int c = sturm_count(ah, bh, n - 1, th[j] + cw) - sturm_count(ah, bh, n - 1, th[j] - cw);
                    keep = c == 0;
                }
            }
            if (keep) lam.push_back(th[j]);
            j = e;
        }
        if ((int)lam.size() >= k || m >= n) break;
        m = std::min(n, 2 * m);
    }
    vec.assign(lam.size(), std::vector<double>(n, 0.0));
    for (size_t q = 0; q < lam.size(); ++q) {
        std::vector<double>& z = vec[q];
        for (int i = 0; i < n; ++i) z[i] = 1.0 + 0.01 * ((i * 7919 + 13 * (int)q) % 101);
        for (int it = 0; it < 3; ++it) {
            tri_solve(a, b, n, lam[q], z);
            double nr = 0;
            for (int i = 0; i < n; ++i) nr += z[i] * z[i];
            nr = sqrt(nr);
            if (nr == 0.0) break;
            for (int i = 0; i < n; ++i) z[i] /= nr;
        }
    }
}

// Lowest k eigenvalues of the tridiagonal T (diagonal a, off-diagonal b),
// optionally with the spurious-value filter (eps_v: unit roundoff of the
// Lanczos vectors); shared with the batched solver and ed_tridiag_eigs.
// With `last`, also the last component of each eigenvector (times the next
// beta, the residual norm of the Ritz pair).
void tridiag_lowest(const std::vector<double>& a, const std::vector<double>& b, int n, int k, bool filter,
                    double eps_v, std::vector<double>& lam, std::vector<double>* last) {
    std::vector<std::vector<double>> vec;
    if (!filter) {
        tri_eig(a, b, n, k, lam, vec);
    } else {
        double tn = 0.0;
        for (int i = 0; i < n; ++i)
            tn = std::max(tn, fabs(a[i]) + (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < n ? fabs(b[i]) : 0.0));
        tri_eig_filtered(a, b, n, k, 100.0 * eps_v * tn, 1e3 * 2.220446049250313e-16 * tn, lam, vec);
    }
    if (last) {
        last->assign(lam.size(), 0.0);
        for (size_t p = 0; p < lam.size() && p < vec.size(); ++p)
            if (n > 0 && (int)vec[p].size() >= n) (*last)[p] = vec[p][n - 1];
    }
}

// ---------------------------------------------------------------- driver
template <int K>
struct Lz {
    using T = typename LV<K>::T;
    const ed_hamiltonian* h;
    const ed_basis* b;
    cudaStream_t s;
    int64_t D;
    int sms;
    int nb;  // reduction blocks per vector
    std::vector<std::pair<void*, size_t>> bufs;
    ~Lz() {
        cudaStreamSynchronize(s);
        for (auto& p : bufs) b->alloc.put(p.first, p.second, s);
    }
    void* get(size_t n) {
        void* p = b->alloc.get(n, s);
        if (p) bufs.push_back({p, n});
        return p;
    }
    unsigned grid() const { return (unsigned)std::min<int64_t>((D + 255) / 256, (int64_t)sms * 8); }
};

static int dtype_kind(ed_dtype d) { return d == ED_F64 ? 0 : d == ED_F32 ? 1 : d == ED_C128 ? 2 : 3; }
template <int K>
static ed_dtype dtype_of() {
    return K == 0 ? ED_F64 : K == 1 ? ED_F32 : K == 2 ? ED_C128 : ED_C64;
}

// dst[i] = src[i] for n 4-byte words; dst may be pageable host memory (read
// by the device over NVLink-C2C), so the copy is asynchronous to the host,
// unlike cudaMemcpyAsync into pageable memory.
__global__ void copy_words(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, int64_t n) {
    // 16-byte moves only when both vectors are 16-byte aligned (a Lanczos vector of an
    // odd dimension in FP32 starts at 8 bytes past a 16-byte boundary)
    const bool al16 = ((((uintptr_t)dst) | ((uintptr_t)src)) & 15u) == 0;
    const int64_t n4 = al16 ? n / 4 : 0;
    uint4* d4 = (uint4*)dst;
    const uint4* s4 = (const uint4*)src;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        d4[i] = s4[i];
    for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Lanczos vectors of the plain recursion kept in host (system) memory, for
// devices that read pageable host memory (NVLink-C2C): one reserved virtual
// range for max_iter + 1 vectors, each vector's pages touched by host threads
// while the GPU works, then filled by a copy kernel on a second stream.  The Ritz vectors are combined from there by the device.
struct HostKrylov {
    void* base = nullptr;
    size_t reserved = 0, vec_bytes = 0;
    cudaStream_t copy = nullptr;
    cudaEvent_t made[4] = {}, copied[4] = {};  // by vector index mod 4
    // First touch of the host pages runs on a thread of its own, a few
    // vectors ahead of the copies, so that the page faults overlap the GPU's
    // steps instead of stalling the loop that enqueues them.
    static constexpr int AHEAD = 3;
    int n_vec = 0;
    std::thread toucher;
    std::mutex mu;
    std::condition_variable cv;
    int want = 0, touched = 0;
    bool stop = false;
    ~HostKrylov() {
        {
            std::lock_guard<std::mutex> l(mu);
            stop = true;
        }
        cv.notify_all();
        if (toucher.joinable()) toucher.join();
        if (copy) {
            cudaStreamSynchronize(copy);
            cudaStreamDestroy(copy);
        }
        for (int i = 0; i < 4; ++i) {
            if (made[i]) cudaEventDestroy(made[i]);
            if (copied[i]) cudaEventDestroy(copied[i]);
        }
        if (base) munmap(base, reserved);
    }
    uint8_t* vec(int k) const { return (uint8_t*)base + (size_t)k * vec_bytes; }
    void start(int n) {
        n_vec = n;
        madvise(base, reserved, MADV_HUGEPAGE);  // a hint: fewer faults where the kernel allows it
        toucher = std::thread([this]() {
            for (int k = 0; k < n_vec; ++k) {
                {
                    std::unique_lock<std::mutex> l(mu);
                    cv.wait(l, [&]() { return stop || want > k; });
                    if (stop) return;
                }
                touch(k);
                {
                    std::lock_guard<std::mutex> l(mu);
                    touched = k + 1;
                }
                cv.notify_all();
            }
        });
    }
    // vector k's pages are resident (and the next AHEAD are being touched)
    void ensure(int k) {
        std::unique_lock<std::mutex> l(mu);
        want = std::max(want, std::min(n_vec, k + 1 + AHEAD));
        cv.notify_all();
        cv.wait(l, [&]() { return touched > k; });
    }
    // queue the copy of device vector k (made on stream s) to host slot k
    cudaError_t save(int k, const void* dev, size_t bytes, cudaStream_t s) {
        ensure(k);
        cudaError_t e = cudaEventRecord(made[k & 3], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(copy, made[k & 3], 0);
        if (e == cudaSuccess) {
            copy_words<<<512, 256, 0, copy>>>((uint32_t*)vec(k), (const uint32_t*)dev, (int64_t)(bytes / 4));
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(copied[k & 3], copy);
        return e;
    }
    // first-touch the pages of vector k (parallel; the copy kernel then writes resident pages)
    void touch(int k) const {
        const int nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        const size_t per = (vec_bytes + nth - 1) / nth;
        std::vector<std::thread> th;
        for (int t = 0; t < nth; ++t)
            th.emplace_back([=]() {
                const size_t a = (size_t)t * per, b = std::min(vec_bytes, a + per);
                if (a < b) memset(vec(k) + a, 0, b - a);
            });
        for (auto& x : th) x.join();
    }
};

template <int K>
static ed_status run(const ed_hamiltonian* h, const ed_lanczos_opts* o, double* evals, void* evecs,
                     ed_lanczos_report* rep, cudaStream_t s, const void* start = nullptr) {
    using T = typename LV<K>::T;
    auto t0 = std::chrono::steady_clock::now();
    Lz<K> z;
    z.h = h;
    z.b = h->basis;
    z.s = s;
    z.D = h->basis->dim;
    ED_CUDA(cudaDeviceGetAttribute(&z.sms, cudaDevAttrMultiProcessorCount, h->basis->device));
    const int64_t D = z.D;
    z.nb = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (D + 4095) / 4096));
    const int max_it = (int)std::min<int64_t>(o->max_iter, D);
    const int n_eig = std::min<int>(o->n_eig, (int)D);
    // plain recursion whose Ritz vectors are needed: keep its vectors on the
    // device (host_vectors = 2) or in host memory (1), else a second pass
    const bool need_vectors = !o->reorth && (evecs || ((K == 1 || K == 3) && o->refine > 0));
    const bool keep_dev = need_vectors && o->host_vectors == 2;
    const bool all_slots = o->reorth || keep_dev;
    const int nstore = all_slots ? max_it + 1 : 3;
    T* V = (T*)z.get((size_t)nstore * D * sizeof(T));
    T* w = (T*)z.get((size_t)D * sizeof(T));
    // partials: (max_it + 2) vectors' worth for the Gram-Schmidt dots, and two
    // grids' worth (<= 1024 blocks each) for the fused step kernels
    const size_t n_part = std::max<size_t>((size_t)(max_it + 2) * z.nb, 2048);
    double2* partial = (double2*)z.get(n_part * sizeof(double2));
    double2* coef = (double2*)z.get((size_t)(max_it + 2) * sizeof(double2));
    double* beta_d = (double*)z.get(2 * sizeof(double));
    if (!V || !w || !partial || !coef || !beta_d) return fail(ED_ERR_NOMEM, "Lanczos workspace");
    const unsigned g = z.grid();
    auto vec = [&](int k) -> T* { return V + (int64_t)(all_slots ? k : (k % 3)) * D; };
    auto dot = [&](const T* A, int nk, const T* bv, double2* out) {
        multi_dot<K><<<dim3(z.nb, nk), 256, 0, s>>>(A, D, bv, D, partial);
        reduce_partials<<<std::min(nk, 1024), 256, 0, s>>>(partial, z.nb, nk, out);
    };
    // v_1: keyed random (or the caller's start vector), normalised
    if (start) ED_CUDA(cudaMemcpyAsync(vec(0), start, (size_t)D * sizeof(T), cudaMemcpyDeviceToDevice, s));
    else if (h->basis->word == 8) init_random<uint64_t, K><<<g, 256, 0, s>>>(vec(0), (const uint64_t*)h->basis->reps.p, D, o->seed);
    else init_random<uint32_t, K><<<g, 256, 0, s>>>(vec(0), (const uint32_t*)h->basis->reps.p, D, o->seed);
    dot(vec(0), 1, vec(0), coef);
    sqrt_re<<<1, 1, 0, s>>>(coef, beta_d);
    scale_by<K><<<g, 256, 0, s>>>(vec(0), vec(0), D, beta_d);
    ED_CUDA(cudaGetLastError());
    // Lanczos vectors in host memory (plain recursion whose Ritz vectors are needed)
    HostKrylov hk;
    {
        int pageable = 0;
        if (o->host_vectors == 1 && need_vectors)
            ED_CUDA(cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, h->basis->device));
        if (pageable) {
            hk.vec_bytes = (((size_t)D * sizeof(T)) + 4095) & ~(size_t)4095;
            hk.reserved = hk.vec_bytes * (size_t)(max_it + 1);
            void* p = mmap(nullptr, hk.reserved, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS | MAP_NORESERVE,
                           -1, 0);
            if (p == MAP_FAILED) return fail(ED_ERR_NOMEM, "host range for %d Lanczos vectors", max_it + 1);
            hk.base = p;
            hk.start(max_it + 1);
            ED_CUDA(cudaStreamCreateWithFlags(&hk.copy, cudaStreamNonBlocking));
            for (int i = 0; i < 4; ++i) {
                ED_CUDA(cudaEventCreateWithFlags(&hk.made[i], cudaEventDisableTiming));
                ED_CUDA(cudaEventCreateWithFlags(&hk.copied[i], cudaEventDisableTiming));
            }
            ED_CUDA(hk.save(0, vec(0), (size_t)D * sizeof(T), s));
        }
    }
    std::vector<double> al, be;  // al[n] = alpha_n, be[n] = beta_{n+1}
    std::vector<double> prev(n_eig, 0.0), lam;
    std::vector<std::vector<double>> svec;
    int n_apply = 0, iters = 0;
    bool conv = false;
    const int every = std::max(1, o->check_every);
    // FP32 vectors resolve eigenvalues to ~1e-7 relative: their phase runs at
    // a tolerance of at least 1e-6 and `tol` is the target of the refinement.
    const double tol = (K == 1 || K == 3) ? std::max(o->tol, 1e-6) : o->tol;
    // unit roundoff of the vectors: copies of one eigenvalue agree to ~eps_v |T|
    const double eps_v = (K == 1 || K == 3) ? 1.1920928955078125e-07 : 2.220446049250313e-16;
    ed_dtype vdt = o->dtype;
    // Mixed precision with refinement: the FP32 phase runs on until every
    // wanted Ritz pair's residual bound r allows a Rayleigh quotient in FP64
    // to meet the final tolerance (its error is at most r^2/gap), or until r
    // reaches the FP32 noise floor ~2 eps_32 |T| (the rounding of the FP32
    // Lanczos vectors alone leaves a residual of that size).
    const bool rq_refine = (K == 1 || K == 3) && o->refine > 0;
    std::vector<double> lam_full, rb_full;  // last check: n_eig + 1 Ritz values, residual bounds
    // Device history of the recursion: al_dev[n] = (alpha_n, 0), be_dev[n] =
    // beta_{n+1} = |w_n|; copied to pinned host memory step by step.  The
    // host reads step n's coefficients only after step n+1 has been queued,
    // so the GPU never waits for the T-matrix check (one step of look-ahead;
    // a step queued past convergence is discarded).
    double2* al_dev = (double2*)z.get((size_t)(max_it + 1) * sizeof(double2));
    double* be_dev = (double*)z.get((size_t)(max_it + 1) * sizeof(double));
    unsigned int* ctr = (unsigned int*)z.get(2 * sizeof(unsigned int));
    if (!al_dev || !be_dev || !ctr) return fail(ED_ERR_NOMEM, "Lanczos workspace");
    ED_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned int), s));
    struct PinnedHist {
        double* p = nullptr;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        ~PinnedHist() {
            if (p) cudaFreeHost(p);
            for (auto e : ev)
                if (e) cudaEventDestroy(e);
        }
    } ph;
    ED_CUDA(cudaHostAlloc((void**)&ph.p, (size_t)(max_it + 1) * 3 * sizeof(double), cudaHostAllocDefault));
    ED_CUDA(cudaEventCreateWithFlags(&ph.ev[0], cudaEventDisableTiming));
    ED_CUDA(cudaEventCreateWithFlags(&ph.ev[1], cudaEventDisableTiming));
    const unsigned gs = (unsigned)std::max<int64_t>(1, std::min<int64_t>((D + 255) / 256, 1024));
    auto enqueue = [&](int n) -> ed_status {
        ed_status st = apply_launch(h, vdt, vec(n), w, 1, s);
        if (st != ED_OK) return st;
        ++n_apply;
        const T* vp = n > 0 ? vec(n - 1) : nullptr;
        const double* bprev = n > 0 ? be_dev + n - 1 : be_dev;
        if (!o->reorth) {
            dot_step<K><<<gs, 256, 0, s>>>(vec(n), w, D, partial, ctr, al_dev + n);
            axpy_norm_step<K><<<gs, 256, 0, s>>>(w, vec(n), vp, D, al_dev + n, bprev, partial + gs, ctr + 1,
                                                 be_dev + n);
        } else {
            dot_step<K><<<gs, 256, 0, s>>>(vec(n), w, D, partial, ctr, al_dev + n);
            lanczos_axpy<K><<<g, 256, 0, s>>>(w, vec(n), vp, D, al_dev + n, bprev);
            // classical Gram-Schmidt against all stored vectors, then again
            // against the last two (v_{n-1}, v_n), where the three-term step
            // leaves the largest rounding components
            for (int pass = 0; pass < 2; ++pass) {
                const int j0 = pass == 0 ? 0 : std::max(0, n - 1);
                const int nj = n + 1 - j0;
                const T* Vj = V + (int64_t)j0 * D;
                if constexpr (K == 1 || K == 3) {
                    multi_dot_f32<K><<<dim3(z.nb, nj), 256, 0, s>>>(Vj, D, w, D, partial);
                    reduce_partials<<<std::min(nj, 1024), 256, 0, s>>>(partial, z.nb, nj, coef);
                    multi_axpy_f32<K><<<g, 256, 0, s>>>(w, Vj, D, nj, coef, D);
                } else {
                    dot(Vj, nj, w, coef);
                    multi_axpy<K><<<g, 256, 0, s>>>(w, Vj, D, nj, coef, D);
                }
            }
            multi_dot<K><<<dim3(z.nb, 1), 256, 0, s>>>(w, D, w, D, partial);
            norm_from_partials<<<1, 256, 0, s>>>(partial, z.nb, be_dev + n);
        }
        // v_{n+1} = w / beta_{n+1} (unused when the recursion stops at n); in
        // the plain recursion its slot held v_{n-2}, whose host copy must be done
        if (hk.base && n >= 2) ED_CUDA(cudaStreamWaitEvent(s, hk.copied[(n - 2) & 3], 0));
        scale_by<K><<<g, 256, 0, s>>>(vec(n + 1), w, D, be_dev + n);
        if (hk.base) ED_CUDA(hk.save(n + 1, vec(n + 1), (size_t)D * sizeof(T), s));
        ED_CUDA(cudaMemcpyAsync(ph.p + 3 * n, al_dev + n, sizeof(double2), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaMemcpyAsync(ph.p + 3 * n + 2, be_dev + n, sizeof(double), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaEventRecord(ph.ev[n & 1], s));
        return ED_OK;
    };
    {
        ed_status st = enqueue(0);
        if (st != ED_OK) return st;
    }
    for (int n = 0; n < max_it; ++n) {
        // queue step n+1 before waiting for step n (the extra slot of the
        // reorthogonalised basis: nstore = max_it + 1)
        if (n + 1 < max_it) {
            ed_status st = enqueue(n + 1);
            if (st != ED_OK) return st;
        }
        ED_CUDA(cudaEventSynchronize(ph.ev[n & 1]));
        const double ahx = ph.p[3 * n], bh = ph.p[3 * n + 2];
        // step n+1's event (same slot) may only be re-recorded after this read:
        // enqueue(n+2) happens in the next iteration, after it
        al.push_back(ahx);
        be.push_back(bh);
        iters = n + 1;
        const double tnorm = fabs(ahx) + bh + 1e-300;
        const bool breakdown = bh < 1e-13 * tnorm;
        const bool last = breakdown || n + 1 == max_it;
        if ((n + 1) % every == 0 || last) {
            double tn = 0.0;
            for (int i = 0; i < iters; ++i)
                tn = std::max(tn, fabs(al[i]) + (i > 0 ? be[i - 1] : 0.0) + (i + 1 < iters ? be[i] : 0.0));
            if (o->reorth) {
                tri_eig(al, be, iters, n_eig + 1, lam, svec);
            } else {
                tri_eig_filtered(al, be, iters, n_eig + 1, 100.0 * eps_v * tn, 1e3 * 2.220446049250313e-16 * tn, lam,
                                 svec);
            }
            lam_full = lam;
            rb_full.assign(lam.size(), 0.0);
            for (size_t p = 0; p < lam.size(); ++p) rb_full[p] = bh * fabs(svec[p][iters - 1]);
            // converged: for each wanted Ritz value, a small change since the
            // last check and a small residual bound r = beta |s_last| (the
            // eigenvalue error is at most min(r, r^2/gap)); with eigenvectors
            // requested also r <= sqrt(tol).  At least n_eig + 3 steps.
            bool ok = (int)lam.size() >= n_eig && iters >= n_eig + 3;
            for (int k = 0; k < n_eig && k < (int)lam.size() && ok; ++k) {
                const double sc = std::max(1.0, fabs(lam[k]));
                const double rb = bh * fabs(svec[k][iters - 1]);
                double gap = 1e300;
                for (int p = 0; p < (int)lam.size(); ++p)
                    if (p != k) gap = std::min(gap, fabs(lam[p] - lam[k]));
                const bool steady = fabs(lam[k] - prev[k]) <= 0.1 * tol * sc;
                const bool small_res = rq_refine ? (rb * rb <= 0.25 * o->tol * sc * gap || rb <= 2.0 * eps_v * tn)
                                                 : (rb <= tol * sc || rb * rb <= tol * sc * gap);
                const bool vec_ok = !evecs || rb <= sqrt(tol) * sc;
                if (!(steady && small_res && vec_ok)) ok = false;
            }
            if (breakdown) ok = true;
            for (int k = 0; k < n_eig && k < (int)lam.size(); ++k) prev[k] = lam[k];
            if (ok) conv = true;
            if ((int)lam.size() > n_eig) {
                lam.resize(n_eig);
                svec.resize(n_eig);
            }
        }
        if (conv || last) break;
    }
    // drain the queued look-ahead step before the workspace is reused
    ED_CUDA(cudaStreamSynchronize(s));
    n_apply = iters;
    ED_CUDA(cudaGetLastError());
    const int nk = (int)lam.size();
    ed_lanczos_report r{};
    r.iters = iters;
    r.converged = conv ? 1 : 0;
    for (int k = nk; k < o->n_eig; ++k) evals[k] = NAN;
    for (int k = 0; k < nk && k < 8; ++k) {
        r.ritz[k] = lam[k];
        r.resid_bound[k] = be[iters - 1] * fabs(svec[k][iters - 1]);
        evals[k] = lam[k];
    }
    // Ritz vectors: from the stored Lanczos vectors, or (plain recursion) by
    // a second pass that regenerates v_1, v_2, ... from the same start with
    // the recorded alpha, beta (the reductions are deterministic, so the
    // vectors repeat bit for bit) and accumulates sum_j s_j v_j.
    const bool mixed = (K == 1 || K == 3);
    const bool want_refine = mixed && o->refine > 0 && nk > 0;
    constexpr int K64 = LV<K>::cplx ? 2 : 0;
    using T64 = typename LV<K64>::T;
    T64* y64 = nullptr;
    std::vector<double> ssum(iters, 0.0);
    for (int k = 0; k < nk; ++k)
        for (int i = 0; i < iters; ++i) ssum[i] += svec[k][i];
    // FP64 Ritz vectors of the refinement: slots 0..nk-1 one per wanted pair,
    // slot nk their sum (the start of the fallback polish)
    const int ny = want_refine ? nk + 1 : 0;
    if (want_refine) {
        y64 = (T64*)z.get((size_t)ny * D * sizeof(T64));
        if (!y64) return fail(ED_ERR_NOMEM, "refinement workspace");
    }
    const T* Vsrc = V;          // stored Lanczos vectors to combine (reorthogonalised run)
    int64_t Vld = D;
    if (hk.base) {              // the plain recursion's vectors kept in host memory
        ED_CUDA(cudaStreamSynchronize(hk.copy));
        Vsrc = (const T*)hk.base;
        Vld = (int64_t)(hk.vec_bytes / sizeof(T));
    }
    const bool stored_vectors = all_slots || hk.base;
    if (!stored_vectors && nk > 0 && (evecs || want_refine)) {
        const int nacc = evecs ? nk : 0;
        const int ncol = nacc + ny;
        std::vector<double2> alh(iters);
        for (int j = 0; j < iters; ++j) alh[j] = make_double2(al[j], 0.0);
        std::vector<double> sc((size_t)iters * std::max(ncol, 1));
        for (int j = 0; j < iters; ++j) {
            for (int k = 0; k < nacc; ++k) sc[(size_t)j * ncol + k] = svec[k][j];
            for (int k = 0; k < ny - 1; ++k) sc[(size_t)j * ncol + nacc + k] = svec[k][j];
            if (ny) sc[(size_t)j * ncol + nacc + ny - 1] = ssum[j];
        }
        double2* al_d = (double2*)z.get((size_t)iters * sizeof(double2));
        double* be_d = (double*)z.get((size_t)iters * sizeof(double));
        double* sc_d = (double*)z.get(sc.size() * sizeof(double));
        if (!al_d || !be_d || !sc_d) return fail(ED_ERR_NOMEM, "second-pass workspace");
        ED_CUDA(cudaMemcpyAsync(al_d, alh.data(), (size_t)iters * sizeof(double2), cudaMemcpyHostToDevice, s));
        ED_CUDA(cudaMemcpyAsync(be_d, be.data(), (size_t)iters * sizeof(double), cudaMemcpyHostToDevice, s));
        ED_CUDA(cudaMemcpyAsync(sc_d, sc.data(), sc.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        if (evecs) ED_CUDA(cudaMemsetAsync(evecs, 0, (size_t)nk * D * sizeof(T), s));
        if (y64) ED_CUDA(cudaMemsetAsync(y64, 0, (size_t)ny * D * sizeof(T64), s));
        // v_1 exactly as in the first pass
        if (start) ED_CUDA(cudaMemcpyAsync(vec(0), start, (size_t)D * sizeof(T), cudaMemcpyDeviceToDevice, s));
        else if (h->basis->word == 8)
            init_random<uint64_t, K><<<g, 256, 0, s>>>(vec(0), (const uint64_t*)h->basis->reps.p, D, o->seed);
        else init_random<uint32_t, K><<<g, 256, 0, s>>>(vec(0), (const uint32_t*)h->basis->reps.p, D, o->seed);
        dot(vec(0), 1, vec(0), coef);
        sqrt_re<<<1, 1, 0, s>>>(coef, beta_d);
        scale_by<K><<<g, 256, 0, s>>>(vec(0), vec(0), D, beta_d);
        for (int j = 0; j < iters; ++j) {
            const double* cj = sc_d + (size_t)j * ncol;
            if (nacc) accumulate<K, T><<<g, 256, 0, s>>>((T*)evecs, D, nacc, cj, vec(j), D);
            if (y64) accumulate<K, T64><<<g, 256, 0, s>>>(y64, D, ny, cj + nacc, vec(j), D);
            if (j + 1 == iters) break;
            ed_status st = apply_launch(h, vdt, vec(j), w, 1, s);
            if (st != ED_OK) return st;
            ++n_apply;
            lanczos_axpy<K><<<g, 256, 0, s>>>(w, vec(j), j > 0 ? vec(j - 1) : nullptr, D, al_d + j,
                                              j > 0 ? be_d + j - 1 : be_d);
            scale_by<K><<<g, 256, 0, s>>>(vec(j + 1), w, D, be_d + j);
        }
        ED_CUDA(cudaGetLastError());
        // the Lanczos vectors are not orthogonal: normalise each Ritz vector
        for (int k = 0; k < nacc; ++k) {
            T* ek = (T*)evecs + (int64_t)k * D;
            dot(ek, 1, ek, coef);
            sqrt_re<<<1, 1, 0, s>>>(coef, beta_d);
            scale_by<K><<<g, 256, 0, s>>>(ek, ek, D, beta_d);
        }
        ED_CUDA(cudaStreamSynchronize(s));
    }
    if (stored_vectors && evecs) {
        double* sd = (double*)z.get((size_t)iters * sizeof(double));
        if (!sd) return fail(ED_ERR_NOMEM, "Ritz workspace");
        for (int k = 0; k < nk; ++k) {
            ED_CUDA(cudaMemcpyAsync(sd, svec[k].data(), (size_t)iters * 8, cudaMemcpyHostToDevice, s));
            combine<K, T><<<g, 256, 0, s>>>((T*)evecs + (int64_t)k * D, Vsrc, Vld, iters, sd, D);
            ED_CUDA(cudaStreamSynchronize(s));
        }
        if (!o->reorth) {  // without reorthogonalisation the Lanczos vectors are not orthogonal: normalise
            for (int k = 0; k < nk; ++k) {
                T* ek = (T*)evecs + (int64_t)k * D;
                dot(ek, 1, ek, coef);
                sqrt_re<<<1, 1, 0, s>>>(coef, beta_d);
                scale_by<K><<<g, 256, 0, s>>>(ek, ek, D, beta_d);
            }
            ED_CUDA(cudaStreamSynchronize(s));
        }
    }
    // Mixed precision refinement (Rayleigh-quotient argument, Eq. rayleighcoeff):
    // the FP32 Ritz vectors promoted to FP64, one FP64 H.x for all of them,
    // E_k = <y_k|H y_k> / <y_k|y_k> and r_k = |H y_k - E_k y_k| / |y_k|.  E_k is
    // within r_k^2 / gap_k of an eigenvalue, gap_k bounded below by the other
    // Ritz values less their residual bounds; when that meets the tolerance
    // for every k the refinement is done, else an FP64 Lanczos polish starts
    // from the sum of the Ritz vectors (its Krylov space already overlaps the
    // wanted eigenvectors and converges in a few steps).
    if constexpr (K == 1 || K == 3) {
        if (want_refine) {
            double* sd = nullptr;
            if (stored_vectors) {
                sd = (double*)z.get((size_t)iters * sizeof(double));
                if (!sd) return fail(ED_ERR_NOMEM, "refinement workspace");
                for (int k = 0; k <= nk; ++k) {
                    if (k == nk && nk == 1) {  // the sum of one Ritz vector is that vector
                        ED_CUDA(cudaMemcpyAsync(y64 + D, y64, (size_t)D * sizeof(T64), cudaMemcpyDeviceToDevice, s));
                        break;
                    }
                    const std::vector<double>& cvec = k < nk ? svec[k] : ssum;
                    ED_CUDA(cudaMemcpyAsync(sd, cvec.data(), (size_t)iters * 8, cudaMemcpyHostToDevice, s));
                    combine<K, T64><<<g, 256, 0, s>>>(y64 + (int64_t)k * D, Vsrc, Vld, iters, sd, D);
                    ED_CUDA(cudaStreamSynchronize(s));
                }
            }
            const ed_dtype d64 = K64 == 2 ? ED_C128 : ED_F64;
            bool rq_ok = false;
            std::vector<double> Ek(nk), rk(nk);
            if (rq_refine && nk <= 8) {
                T64* w64 = (T64*)z.get((size_t)nk * D * sizeof(T64));
                double2* part64 = (double2*)z.get((size_t)z.nb * sizeof(double2));
                double2* res64 = (double2*)z.get((size_t)3 * nk * sizeof(double2));
                if (!w64 || !part64 || !res64) return fail(ED_ERR_NOMEM, "refinement workspace");
                auto dot64 = [&](const T64* a, const T64* b2, double2* out) {
                    multi_dot<K64><<<dim3(z.nb, 1), 256, 0, s>>>(a, D, b2, D, part64);
                    reduce_partials<<<1, 256, 0, s>>>(part64, z.nb, 1, out);
                };
                ed_status st = apply_launch(h, d64, y64, w64, nk, s);
                if (st != ED_OK) return st;
                n_apply += nk;
                std::vector<double2> hres(2 * (size_t)nk);
                for (int k = 0; k < nk; ++k) {
                    dot64(y64 + (int64_t)k * D, y64 + (int64_t)k * D, res64 + 2 * k);
                    dot64(y64 + (int64_t)k * D, w64 + (int64_t)k * D, res64 + 2 * k + 1);
                }
                ED_CUDA(cudaMemcpyAsync(hres.data(), res64, hres.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
                ED_CUDA(cudaStreamSynchronize(s));
                for (int k = 0; k < nk; ++k) {
                    Ek[k] = hres[2 * k + 1].x / hres[2 * k].x;
                    residual<K64><<<g, 256, 0, s>>>(w64 + (int64_t)k * D, w64 + (int64_t)k * D, y64 + (int64_t)k * D,
                                                    D, Ek[k]);
                    dot64(w64 + (int64_t)k * D, w64 + (int64_t)k * D, res64 + 2 * nk + k);
                }
                std::vector<double2> rres(nk);
                ED_CUDA(cudaMemcpyAsync(rres.data(), res64 + 2 * nk, nk * sizeof(double2), cudaMemcpyDeviceToHost, s));
                ED_CUDA(cudaStreamSynchronize(s));
                rq_ok = true;
                for (int k = 0; k < nk; ++k) {
                    rk[k] = sqrt(std::max(0.0, rres[k].x / hres[2 * k].x));
                    double gap = 1e300;
                    for (size_t p = 0; p < lam_full.size(); ++p)
                        if ((int)p != k) gap = std::min(gap, fabs(lam_full[p] - Ek[k]) - rb_full[p]);
                    const double sc = std::max(1.0, fabs(Ek[k]));
                    if (!(gap > 0.0) || rk[k] * rk[k] > o->tol * sc * gap) rq_ok = false;
                }
            }
            // the FP64 refinement certifies the result: its outcome decides
            // convergence (the FP32 phase may stop at max_iter or at the
            // dimension of a small sector without meeting its own criterion)
            if (rq_ok) {
                for (int k = 0; k < nk; ++k) {
                    r.refined[k] = Ek[k];
                    r.refined_resid[k] = rk[k];
                    evals[k] = Ek[k];
                }
                conv = nk >= std::min(o->n_eig, (int)D);
            } else {
                ed_lanczos_opts o2 = *o;
                o2.dtype = d64;
                o2.reorth = 0;  // a few steps from a close start: the plain recursion, no stored FP64 vectors
                o2.max_iter = std::max(o->refine, o->n_eig + 2);
                o2.refine = 0;
                o2.check_every = 1;
                double ev2[8];
                ed_lanczos_report r2{};
                ed_status st2 = run<K64>(h, &o2, ev2, nullptr, &r2, s, y64 + (int64_t)nk * D);
                if (st2 != ED_OK && st2 != ED_ERR_NOT_CONVERGED) return st2;
                n_apply += r2.n_apply;
                const int n2 = std::min(nk, o->n_eig);
                for (int k = 0; k < n2; ++k) {
                    r.refined[k] = r2.ritz[k];
                    r.refined_resid[k] = r2.resid_bound[k];
                    evals[k] = r2.ritz[k];
                }
                conv = r2.converged != 0;
            }
        }
    }
    (void)mixed;
    ED_CUDA(cudaStreamSynchronize(s));
    r.n_apply = n_apply;
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = r;
    return conv ? ED_OK : fail(ED_ERR_NOT_CONVERGED, "Lanczos did not converge in %d steps", iters);
}

ed_status lanczos_run(const ed_hamiltonian* h, const ed_lanczos_opts* o, double* evals, void* evecs,
                      ed_lanczos_report* rep, cudaStream_t s) {
    switch (dtype_kind(o->dtype)) {
        case 0: return run<0>(h, o, evals, evecs, rep, s);
        case 1: return run<1>(h, o, evals, evecs, rep, s);
        case 2: return run<2>(h, o, evals, evecs, rep, s);
        default: return run<3>(h, o, evals, evecs, rep, s);
    }
}

template <int K>
static ed_status expectation_kind(const ed_hamiltonian* h, const void* x, int nvec, cudaStream_t s, double* out) {
    using T = typename LV<K>::T;
    Lz<K> z;
    z.h = h;
    z.b = h->basis;
    z.s = s;
    z.D = h->basis->dim;
    ED_CUDA(cudaDeviceGetAttribute(&z.sms, cudaDevAttrMultiProcessorCount, h->basis->device));
    const int64_t D = z.D;
    z.nb = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (D + 4095) / 4096));
    T* y = (T*)z.get((size_t)nvec * D * sizeof(T));
    double2* partial = (double2*)z.get((size_t)z.nb * sizeof(double2));
    double2* res = (double2*)z.get((size_t)2 * nvec * sizeof(double2));
    if (!y || !partial || !res) return fail(ED_ERR_NOMEM, "expectation workspace");
    const ed_status st = apply_launch(h, dtype_of<K>(), x, y, nvec, s);
    if (st != ED_OK) return st;
    const T* xv = (const T*)x;
    for (int v = 0; v < nvec; ++v) {
        multi_dot<K><<<dim3(z.nb, 1), 256, 0, s>>>(xv + (int64_t)v * D, D, y + (int64_t)v * D, D, partial);
        reduce_partials<<<1, 256, 0, s>>>(partial, z.nb, 1, res + 2 * v);
        multi_dot<K><<<dim3(z.nb, 1), 256, 0, s>>>(xv + (int64_t)v * D, D, xv + (int64_t)v * D, D, partial);
        reduce_partials<<<1, 256, 0, s>>>(partial, z.nb, 1, res + 2 * v + 1);
    }
    ED_CUDA(cudaGetLastError());
    std::vector<double2> hres(2 * (size_t)nvec);
    ED_CUDA(cudaMemcpyAsync(hres.data(), res, hres.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    for (int v = 0; v < nvec; ++v) {
        out[3 * v] = hres[2 * v].x;
        out[3 * v + 1] = hres[2 * v].y;
        out[3 * v + 2] = hres[2 * v + 1].x;
    }
    return ED_OK;
}

// All eigenpairs of a small dense real symmetric matrix (cyclic Jacobi
// rotations, Golub & Van Loan sec. 8.5): A (n x n, row-major) is overwritten,
// lam[k] and column k of Q (Q[i*n + k]) are the k-th eigenpair.
static void jacobi_eig(std::vector<double>& A, int n, std::vector<double>& lam, std::vector<double>& Q) {
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {  // Q <- Q J
                    const double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
                    Q[(size_t)k * n + p] = c * qkp - sn * qkq;
                    Q[(size_t)k * n + q] = sn * qkp + c * qkq;
                }
            }
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
}

// psi <- exp(-i H dt) psi by one Krylov step: m Lanczos vectors from psi
// (full reorthogonalisation), T = V^H H V tridiagonal, and
// psi_new = |psi| V exp(-i T dt) e_1.  err = |psi| beta_m |[exp(-i T dt) e_1]_m|,
// the usual a-posteriori estimate of the step's error.
template <int K>
static ed_status evolve_kind(const ed_hamiltonian* h, void* psi, double dt, int m, cudaStream_t s, double* err,
                             int* m_used) {
    using T = typename LV<K>::T;
    Lz<K> z;
    z.h = h;
    z.b = h->basis;
    z.s = s;
    z.D = h->basis->dim;
    ED_CUDA(cudaDeviceGetAttribute(&z.sms, cudaDevAttrMultiProcessorCount, h->basis->device));
    const int64_t D = z.D;
    m = (int)std::min<int64_t>(m, D);
    z.nb = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (D + 4095) / 4096));
    T* V = (T*)z.get((size_t)(m + 1) * D * sizeof(T));
    T* w = (T*)z.get((size_t)D * sizeof(T));
    double2* partial = (double2*)z.get((size_t)(m + 2) * z.nb * sizeof(double2));
    double2* coef = (double2*)z.get((size_t)(m + 2) * sizeof(double2));
    double* beta_d = (double*)z.get(2 * sizeof(double));
    double2* alpha_d = (double2*)z.get(sizeof(double2));
    if (!V || !w || !partial || !coef || !beta_d || !alpha_d) return fail(ED_ERR_NOMEM, "time-evolution workspace");
    const unsigned g = z.grid();
    auto dot = [&](const T* A, int nk, const T* bv, double2* out) {
        multi_dot<K><<<dim3(z.nb, nk), 256, 0, s>>>(A, D, bv, D, partial);
        reduce_partials<<<std::min(nk, 1024), 256, 0, s>>>(partial, z.nb, nk, out);
    };
    // v_0 = psi / |psi|
    ED_CUDA(cudaMemcpyAsync(V, psi, (size_t)D * sizeof(T), cudaMemcpyDeviceToDevice, s));
    dot(V, 1, V, coef);
    sqrt_re<<<1, 1, 0, s>>>(coef, beta_d);
    double nrm = 0.0;
    ED_CUDA(cudaMemcpyAsync(&nrm, beta_d, sizeof(double), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    if (!(nrm > 0.0)) return fail(ED_ERR_ARG, "psi is zero");
    scale_by<K><<<g, 256, 0, s>>>(V, V, D, beta_d);
    std::vector<double> al, be;
    int mm = 0;
    for (int n = 0; n < m; ++n) {
        T* vn = V + (int64_t)n * D;
        ed_status st = apply_launch(h, K == 2 ? ED_C128 : ED_C64, vn, w, 1, s);
        if (st != ED_OK) return st;
        dot(vn, 1, w, alpha_d);
        lanczos_axpy<K><<<g, 256, 0, s>>>(w, vn, n > 0 ? vn - D : nullptr, D, alpha_d, beta_d);
        for (int pass = 0; pass < 2; ++pass) {
            const int j0 = pass == 0 ? 0 : std::max(0, n - 1);
            const int nj = n + 1 - j0;
            dot(V + (int64_t)j0 * D, nj, w, coef);
            multi_axpy<K><<<g, 256, 0, s>>>(w, V + (int64_t)j0 * D, D, nj, coef, D);
        }
        dot(w, 1, w, coef + m + 1);
        sqrt_re<<<1, 1, 0, s>>>(coef + m + 1, beta_d);
        double2 ah;
        double bh;
        ED_CUDA(cudaMemcpyAsync(&ah, alpha_d, sizeof(double2), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaMemcpyAsync(&bh, beta_d, sizeof(double), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaStreamSynchronize(s));
        al.push_back(ah.x);
        be.push_back(bh);
        mm = n + 1;
        // an invariant subspace: the step is exact in it
        if (bh < 1e-14 * (fabs(ah.x) + 1.0)) break;
        scale_by<K><<<g, 256, 0, s>>>(V + (int64_t)(n + 1) * D, w, D, beta_d);
    }
    ED_CUDA(cudaGetLastError());
    // exp(-i T dt) e_1 from the eigenpairs of T
    std::vector<double> Td((size_t)mm * mm, 0.0), lam, Q;
    for (int i = 0; i < mm; ++i) {
        Td[(size_t)i * mm + i] = al[i];
        if (i + 1 < mm) Td[(size_t)i * mm + i + 1] = Td[(size_t)(i + 1) * mm + i] = be[i];
    }
    jacobi_eig(Td, mm, lam, Q);
    std::vector<double2> c(mm);
    for (int j = 0; j < mm; ++j) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k < mm; ++k) {
            const double q = Q[(size_t)j * mm + k] * Q[(size_t)0 * mm + k];
            re += q * cos(lam[k] * dt);
            im -= q * sin(lam[k] * dt);
        }
        c[j] = make_double2(nrm * re, nrm * im);
    }
    if (err) *err = be[mm - 1] * sqrt(c[mm - 1].x * c[mm - 1].x + c[mm - 1].y * c[mm - 1].y);
    if (m_used) *m_used = mm;
    double2* c_d = (double2*)z.get((size_t)mm * sizeof(double2));
    if (!c_d) return fail(ED_ERR_NOMEM, "time-evolution workspace");
    ED_CUDA(cudaMemcpyAsync(c_d, c.data(), (size_t)mm * sizeof(double2), cudaMemcpyHostToDevice, s));
    combine_c<K><<<g, 256, 0, s>>>((T*)psi, V, D, mm, c_d, D);
    ED_CUDA(cudaGetLastError());
    ED_CUDA(cudaStreamSynchronize(s));
    return ED_OK;
}

// The Lanczos recursion (Eqs. lanczosrecursion, tmatrix) from a given vector
// x: v_0 = x/|x|, alpha_n = <v_n|H v_n>, beta_n = |w_n| with
// w_n = H v_n - alpha_n v_n - beta_{n-1} v_{n-1}, v_{n+1} = w_n / beta_n.  With
// reorth the m+1 vectors are kept and w_n is orthogonalised against all of them
// (classical Gram-Schmidt, then again against the last two); without, three
// vectors live at a time (the continued-fraction expansion needs only T).
template <int K>
static ed_status tridiag_kind(const ed_hamiltonian* h, ed_dtype dt, const void* x, int m, bool reorth, cudaStream_t s,
                              double* alpha, double* beta, double* norm2, int* m_used) {
    using T = typename LV<K>::T;
    Lz<K> z;
    z.h = h;
    z.b = h->basis;
    z.s = s;
    z.D = h->basis->dim;
    ED_CUDA(cudaDeviceGetAttribute(&z.sms, cudaDevAttrMultiProcessorCount, h->basis->device));
    const int64_t D = z.D;
    if (reorth) m = (int)std::min<int64_t>(m, D);
    const int slots = reorth ? m + 1 : 2;
    z.nb = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (D + 4095) / 4096));
    T* V = (T*)z.get((size_t)slots * D * sizeof(T));
    T* w = (T*)z.get((size_t)D * sizeof(T));
    double2* partial = (double2*)z.get((size_t)(slots + 2) * z.nb * sizeof(double2));
    double2* coef = (double2*)z.get((size_t)(slots + 2) * sizeof(double2));
    double* beta_d = (double*)z.get(2 * sizeof(double));
    double2* alpha_d = (double2*)z.get(sizeof(double2));
    if (!V || !w || !partial || !coef || !beta_d || !alpha_d) return fail(ED_ERR_NOMEM, "Lanczos workspace");
    const unsigned g = z.grid();
    auto dot = [&](const T* A, int nk, const T* bv, double2* out) {
        multi_dot<K><<<dim3(z.nb, nk), 256, 0, s>>>(A, D, bv, D, partial);
        reduce_partials<<<std::min(nk, 1024), 256, 0, s>>>(partial, z.nb, nk, out);
    };
    auto slot = [&](int n) { return V + (int64_t)(reorth ? n : (n & 1)) * D; };
    ED_CUDA(cudaMemcpyAsync(V, x, (size_t)D * sizeof(T), cudaMemcpyDeviceToDevice, s));
    dot(V, 1, V, coef);
    double2 n2;
    ED_CUDA(cudaMemcpyAsync(&n2, coef, sizeof(double2), cudaMemcpyDeviceToHost, s));
    sqrt_re<<<1, 1, 0, s>>>(coef, beta_d);
    ED_CUDA(cudaStreamSynchronize(s));
    if (!(n2.x > 0.0)) return fail(ED_ERR_ARG, "the start vector is zero");
    if (norm2) *norm2 = n2.x;
    scale_by<K><<<g, 256, 0, s>>>(V, V, D, beta_d);
    int mm = 0;
    for (int n = 0; n < m; ++n) {
        T* vn = slot(n);
        ed_status st = apply_launch(h, dt, vn, w, 1, s);
        if (st != ED_OK) return st;
        dot(vn, 1, w, alpha_d);
        lanczos_axpy<K><<<g, 256, 0, s>>>(w, vn, n > 0 ? slot(n - 1) : nullptr, D, alpha_d, beta_d);
        if (reorth) {
            for (int pass = 0; pass < 2; ++pass) {
                const int j0 = pass == 0 ? 0 : std::max(0, n - 1);
                const int nj = n + 1 - j0;
                dot(V + (int64_t)j0 * D, nj, w, coef);
                multi_axpy<K><<<g, 256, 0, s>>>(w, V + (int64_t)j0 * D, D, nj, coef, D);
            }
        }
        dot(w, 1, w, coef + slots + 1);
        sqrt_re<<<1, 1, 0, s>>>(coef + slots + 1, beta_d);
        double2 ah;
        double bh;
        ED_CUDA(cudaMemcpyAsync(&ah, alpha_d, sizeof(double2), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaMemcpyAsync(&bh, beta_d, sizeof(double), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaStreamSynchronize(s));
        alpha[n] = ah.x;
        beta[n] = bh;
        mm = n + 1;
        // an invariant subspace: T is complete
        if (bh < 1e-14 * (fabs(ah.x) + 1.0)) break;
        if (n + 1 < m) scale_by<K><<<g, 256, 0, s>>>(slot(n + 1), w, D, beta_d);
    }
    ED_CUDA(cudaGetLastError());
    ED_CUDA(cudaStreamSynchronize(s));
    if (m_used) *m_used = mm;
    return ED_OK;
}

}  // namespace ed

extern "C" ed_status ed_lanczos_tridiag(const ed_hamiltonian* h, ed_dtype dtype, const void* x, int32_t m,
                                        int32_t reorth, ed_stream stream, double* alpha, double* beta, double* norm2,
                                        int32_t* m_used) {
    using namespace ed;
    if (!h || !x || !alpha || !beta) return fail(ED_ERR_ARG, "null argument");
    if (m < 1 || m > 100000) return fail(ED_ERR_ARG, "number of steps out of range [1,100000]");
    // the Gram-Schmidt dot products run one grid row per stored vector
    if (reorth && m > 65534) return fail(ED_ERR_ARG, "reorthogonalisation needs m <= 65534");
    if ((dtype == ED_F64 || dtype == ED_F32) && !h->is_real)
        return fail(ED_ERR_ARG, "complex Hamiltonian or characters need a complex dtype");
    cudaStream_t s = (cudaStream_t)stream;
    int mu = 0;
    ed_status st;
    switch (dtype) {
        case ED_F64: st = tridiag_kind<0>(h, dtype, x, m, reorth != 0, s, alpha, beta, norm2, &mu); break;
        case ED_F32: st = tridiag_kind<1>(h, dtype, x, m, reorth != 0, s, alpha, beta, norm2, &mu); break;
        case ED_C128: st = tridiag_kind<2>(h, dtype, x, m, reorth != 0, s, alpha, beta, norm2, &mu); break;
        case ED_C64: st = tridiag_kind<3>(h, dtype, x, m, reorth != 0, s, alpha, beta, norm2, &mu); break;
        default: return fail(ED_ERR_ARG, "bad dtype");
    }
    if (m_used) *m_used = mu;
    return st;
}

extern "C" ed_status ed_time_evolve(const ed_hamiltonian* h, ed_dtype dtype, void* psi, double dt, int32_t m,
                                    ed_stream stream, double* err, int32_t* m_used) {
    using namespace ed;
    if (!h || !psi) return fail(ED_ERR_ARG, "null argument");
    if (m < 2 || m > 64) return fail(ED_ERR_ARG, "Krylov dimension out of range [2,64]");
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == ED_C128) return evolve_kind<2>(h, psi, dt, m, s, err, m_used);
    if (dtype == ED_C64) return evolve_kind<3>(h, psi, dt, m, s, err, m_used);
    return fail(ED_ERR_ARG, "time evolution needs complex vectors (ED_C128 or ED_C64)");
}

extern "C" ed_status ed_expectation(const ed_hamiltonian* h, ed_dtype dtype, const void* x, int32_t nvec,
                                    ed_stream stream, double* out) {
    using namespace ed;
    if (!h || !x || !out) return fail(ED_ERR_ARG, "null argument");
    if (nvec < 1 || nvec > 8) return fail(ED_ERR_ARG, "nvec out of range [1,8]");
    if ((dtype == ED_F64 || dtype == ED_F32) && !h->is_real)
        return fail(ED_ERR_ARG, "complex Hamiltonian or characters need a complex dtype");
    cudaStream_t s = (cudaStream_t)stream;
    switch (dtype_kind(dtype)) {
        case 0: return expectation_kind<0>(h, x, nvec, s, out);
        case 1: return expectation_kind<1>(h, x, nvec, s, out);
        case 2: return expectation_kind<2>(h, x, nvec, s, out);
        default: return expectation_kind<3>(h, x, nvec, s, out);
    }
}

extern "C" ed_status ed_tridiag_eigs(const double* alpha, const double* beta, int32_t n, int32_t k, double eps_vectors,
                                     int32_t filter, double* evals, int32_t* n_found) {
    using namespace ed;
    if (!alpha || (!beta && n > 1) || !evals || n < 1 || k < 1) return fail(ED_ERR_ARG, "bad argument");
    std::vector<double> a(alpha, alpha + n), b(n, 0.0);
    for (int i = 0; i + 1 < n; ++i) b[i] = beta[i];
    std::vector<double> lam;
    tridiag_lowest(a, b, n, k, filter != 0, eps_vectors, lam);
    for (size_t i = 0; i < lam.size(); ++i) evals[i] = lam[i];
    if (n_found) *n_found = (int32_t)lam.size();
    return ED_OK;
}
