/*
 * CPU oracle for the symmetry-adapted exact-diagonalization hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline arm load this library; the product path never does.
 * It shares no code with the CUDA library: plain, slow, obviously correct
 * brute force written from the thesis chapter "Symmetries and
 * Parallelization for Large-Scale Exact Diagonalization".
 *
 * Conventions:
 *  - a spin configuration is the integer sum_k sigma_k 2^(N-k), site 1 most
 *    significant, up = 1 (Eq. numberforspinconfig).  Site s (0-based) is
 *    bit N-1-s.
 *  - a group element acts actively: the spin on site i moves to site
 *    perm[g][i]; a spin-flip element then complements every spin
 *    (Eq. spinflipsymmetry, direct product Eq. tensorchar).
 *  - the representative of a state is the orbit element with the smallest
 *    integer (Eq. representativecondition), found by applying every group
 *    element (the "naive" approach of the sublattice-coding section).
 *  - a representative belongs to the sector of a 1-D irrep iff the
 *    projector sum_g chi(g)^* g |sigma> is non-zero, i.e. iff the sum of
 *    chi over its stabilizer is non-zero (Eq. symmetryadaptedwavefunction1d).
 *  - the norm of the symmetric state is N_sigma^2 = |G| |Stab(sigma)|.
 *  - matrix element between representatives: with the projector of
 *    Eq. symmetryadaptedwavefunction1d_lsed the element of Eq.
 *    matrixelementrepresentatives_lsed carries chi(g_tau)^*:
 *      <tau~|H_k|sigma~> = conj(chi(g_tau)) * N_tau/N_sigma * <tau|H_k|sigma~>.
 *  - vector entries for sampled checks come from SplitMix64 (Steele, Lea,
 *    Flood, OOPSLA 2014) keyed by the state integer.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- group action ------------------------------------------------------ */
static inline int get_spin(uint64_t s, int N, int site) { return (int)((s >> (N - 1 - site)) & 1u); }

uint64_t orc_apply(uint64_t s, int N, const int32_t* perm, int flip) {
    uint64_t out = 0;
    for (int i = 0; i < N; ++i) {
        int v = get_spin(s, N, i);
        if (flip) v ^= 1;
        if (v) out |= (uint64_t)1 << (N - 1 - perm[i]);
    }
    return out;
}

/* Representative by applying every element: rep, first minimising element,
 * number of minimising elements (= |Stab(rep)|), and the sum of chi over the
 * stabilizer of rep (computed from the minimisers: they form Stab(rep) g_0). */
void orc_rep(uint64_t s, int N, int G, const int32_t* perm, const uint8_t* flip, const double* chi,
             uint64_t* rep_out, int32_t* g_out, int32_t* nstab_out, double* stabsum_re, double* stabsum_im) {
    uint64_t best = ~(uint64_t)0;
    int gbest = -1;
    for (int g = 0; g < G; ++g) {
        uint64_t t = orc_apply(s, N, perm + (size_t)g * N, flip ? flip[g] : 0);
        if (t < best) { best = t; gbest = g; }
    }
    /* stabilizer of the representative: elements h with h rep = rep */
    int n = 0;
    double sr = 0.0, si = 0.0;
    for (int h = 0; h < G; ++h) {
        uint64_t t = orc_apply(best, N, perm + (size_t)h * N, flip ? flip[h] : 0);
        if (t == best) {
            ++n;
            if (chi) { sr += chi[2 * h]; si += chi[2 * h + 1]; }
        }
    }
    *rep_out = best;
    *g_out = gbest;
    *nstab_out = n;
    if (stabsum_re) *stabsum_re = sr;
    if (stabsum_im) *stabsum_im = si;
}

static int compatible(double sr, double si) { return sr * sr + si * si > 1e-12; }

/* next integer with the same popcount (Gosper's hack) */
static inline uint64_t next_same_popcount(uint64_t v) {
    uint64_t c = v & (~v + 1);
    uint64_t r = v + c;
    return (((r ^ v) >> 2) / c) | r;
}

/* Basis: every state with popcount n_up, in increasing integer order, kept iff
 * it is its own representative and compatible with the irrep.  The state space
 * is cut into chunks by the top `pb` bits so chunks can run in parallel; the
 * concatenation of chunks in prefix order is sorted.  Returns the dimension;
 * reps/stab may be NULL (count only), otherwise they must hold `cap` entries. */
int64_t orc_basis(int N, int n_up, int G, const int32_t* perm, const uint8_t* flip, const double* chi,
                  uint64_t* reps, int32_t* stab, int64_t cap) {
    int pb = N >= 12 ? 8 : 0;
    int nchunk = 1 << pb;
    int low = N - pb;
    int64_t* counts = (int64_t*)calloc((size_t)nchunk + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            if (!reps) break;
            int64_t acc = 0;
            for (int c = 0; c < nchunk; ++c) { int64_t t = counts[c]; counts[c] = acc; acc += t; }
            counts[nchunk] = acc;
            if (acc > cap) { free(counts); return -1; }
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < nchunk; ++c) {
            int pc = __builtin_popcount((unsigned)c);
            int rest = n_up - pc;
            if (rest < 0 || rest > low) continue;
            uint64_t prefix = (uint64_t)c << low;
            uint64_t lim = low == 64 ? ~(uint64_t)0 : ((uint64_t)1 << low);
            uint64_t v = rest == 0 ? 0 : (((uint64_t)1 << rest) - 1);
            int64_t k = 0, base = pass ? counts[c] : 0;
            while (1) {
                uint64_t s = prefix | v;
                uint64_t r; int32_t g, ns; double sr, si;
                orc_rep(s, N, G, perm, flip, chi, &r, &g, &ns, &sr, &si);
                if (r == s && compatible(sr, si)) {
                    if (pass) { reps[base + k] = s; stab[base + k] = ns; }
                    ++k;
                }
                if (rest == 0) break;
                v = next_same_popcount(v);
                if (v >= lim) break;
            }
            if (!pass) counts[c] = k;
        }
        if (!reps) {
            int64_t acc = 0;
            for (int c = 0; c < nchunk; ++c) acc += counts[c];
            free(counts);
            return acc;
        }
    }
    int64_t D = counts[nchunk];
    free(counts);
    return D;
}

static int64_t find_index(const uint64_t* reps, int64_t D, uint64_t s) {
    int64_t lo = 0, hi = D;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (reps[mid] < s) lo = mid + 1; else hi = mid;
    }
    return (lo < D && reps[lo] == s) ? lo : -1;
}

/* Terms are local operators on n_loc <= 3 sites given as dense complex
 * matrices M[a'][a] in the local basis a = sum_l spin(site_l) 2^(n_loc-1-l)
 * (first listed site most significant, matching the global encoding).
 * sites: [T][3], nloc: [T], mats: [T][8][8][2] (row a', column a). */
static void local_apply_targets(uint64_t s, int N, int nloc, const int32_t* sites, int* a_out) {
    int a = 0;
    for (int l = 0; l < nloc; ++l) a = (a << 1) | get_spin(s, N, sites[l]);
    *a_out = a;
}

static uint64_t local_set(uint64_t s, int N, int nloc, const int32_t* sites, int ap) {
    for (int l = 0; l < nloc; ++l) {
        int v = (ap >> (nloc - 1 - l)) & 1;
        uint64_t bit = (uint64_t)1 << (N - 1 - sites[l]);
        s = v ? (s | bit) : (s & ~bit);
    }
    return s;
}

/* Column-wise assembly of the symmetric-basis matrix in COO form:
 * for column sigma~ and every term, every local image tau contributes
 * M[a'][a] * conj(chi(g_tau)) * sqrt(stab_tau / stab_sigma) at row tau~.
 * Entries are emitted unsummed, for the columns c0 <= c < c1.  Returns the
 * number of entries or -1 if `cap` is too small.  With rows==NULL only counts. */
int64_t orc_coo_cols(int N, int G, const int32_t* perm, const uint8_t* flip, const double* chi,
                     const uint64_t* reps, const int32_t* stab, int64_t D, int64_t c0, int64_t c1,
                     int T, const int32_t* nloc, const int32_t* sites, const double* mats,
                     int64_t* rows, int64_t* cols, double* vals, int64_t cap) {
    int64_t n = 0;
    for (int64_t c = c0; c < c1; ++c) {
        uint64_t s = reps[c];
        for (int t = 0; t < T; ++t) {
            int nl = nloc[t];
            const int32_t* st = sites + 3 * t;
            const double* M = mats + (size_t)t * 128;
            int a;
            local_apply_targets(s, N, nl, st, &a);
            for (int ap = 0; ap < (1 << nl); ++ap) {
                double mr = M[(ap * 8 + a) * 2], mi = M[(ap * 8 + a) * 2 + 1];
                if (mr == 0.0 && mi == 0.0) continue;
                uint64_t tau = local_set(s, N, nl, st, ap);
                uint64_t r; int32_t g, ns; double sr, si;
                orc_rep(tau, N, G, perm, flip, chi, &r, &g, &ns, &sr, &si);
                if (!compatible(sr, si)) continue;
                int64_t j = find_index(reps, D, r);
                if (j < 0) continue; /* other popcount cannot happen for these terms */
                double cr = chi[2 * g], ci = -chi[2 * g + 1]; /* conj(chi(g_tau)) */
                double f = sqrt((double)ns / (double)stab[c]);
                if (rows) {
                    if (n >= cap) return -1;
                    rows[n] = j;
                    cols[n] = c;
                    vals[2 * n] = (mr * cr - mi * ci) * f;
                    vals[2 * n + 1] = (mr * ci + mi * cr) * f;
                }
                ++n;
            }
        }
    }
    return n;
}

/* The whole matrix: columns 0..D-1 (orc_coo_cols restricted to a column
 * range lets independent ranges be assembled concurrently). */
int64_t orc_coo(int N, int G, const int32_t* perm, const uint8_t* flip, const double* chi,
                const uint64_t* reps, const int32_t* stab, int64_t D,
                int T, const int32_t* nloc, const int32_t* sites, const double* mats,
                int64_t* rows, int64_t* cols, double* vals, int64_t cap) {
    return orc_coo_cols(N, G, perm, flip, chi, reps, stab, D, 0, D, T, nloc, sites, mats, rows, cols, vals, cap);
}

/* SplitMix64 finaliser and the keyed uniform used for sampled vectors. */
static inline uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline double keyed_uniform(uint64_t seed, int stream, uint64_t state) {
    uint64_t key = splitmix64(seed * 256u + (uint64_t)stream);
    return (double)(splitmix64(state ^ key) >> 11) * (1.0 / 9007199254740992.0);
}

/* Matrix-free rows: for each sampled representative sigma~ (which must be a
 * compatible representative), y(sigma~) = sum_j H[sigma~, j] x_j with
 * H[i,j] = conj(H[j,i]) (H Hermitian) and x_j = x(state_j) drawn from the
 * keyed SplitMix64 uniform in [-1,1) (imaginary part from stream 1 when
 * is_complex).  stab_sigma is recomputed here. */
void orc_rows(int N, int G, const int32_t* perm, const uint8_t* flip, const double* chi,
              int T, const int32_t* nloc, const int32_t* sites, const double* mats,
              const uint64_t* states, int64_t n_states, uint64_t seed, int is_complex, double* y_out) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < n_states; ++q) {
        uint64_t s = states[q];
        uint64_t r0; int32_t g0, ns0; double sr0, si0;
        orc_rep(s, N, G, perm, flip, chi, &r0, &g0, &ns0, &sr0, &si0);
        double yr = 0.0, yi = 0.0;
        for (int t = 0; t < T; ++t) {
            int nl = nloc[t];
            const int32_t* st = sites + 3 * t;
            const double* M = mats + (size_t)t * 128;
            int a;
            local_apply_targets(s, N, nl, st, &a);
            for (int ap = 0; ap < (1 << nl); ++ap) {
                double mr = M[(ap * 8 + a) * 2], mi = M[(ap * 8 + a) * 2 + 1];
                if (mr == 0.0 && mi == 0.0) continue;
                uint64_t tau = local_set(s, N, nl, st, ap);
                uint64_t r; int32_t g, ns; double sr, si;
                orc_rep(tau, N, G, perm, flip, chi, &r, &g, &ns, &sr, &si);
                if (!compatible(sr, si)) continue;
                /* H[j,i] = M * conj(chi(g)) * sqrt(ns/ns0); H[i,j] = conj of it */
                double cr = chi[2 * g], ci = -chi[2 * g + 1];
                double f = sqrt((double)ns / (double)ns0);
                double hr = (mr * cr - mi * ci) * f, hi = (mr * ci + mi * cr) * f;
                hi = -hi;
                double xr = 2.0 * keyed_uniform(seed, 0, r) - 1.0;
                double xi = is_complex ? 2.0 * keyed_uniform(seed, 1, r) - 1.0 : 0.0;
                yr += hr * xr - hi * xi;
                yi += hr * xi + hi * xr;
            }
        }
        y_out[2 * q] = yr;
        y_out[2 * q + 1] = yi;
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the following parallel regions (n >= 1); for the baseline's
 * single-thread figure. */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
