/*
 * ed.h -- C ABI of libed, a single-GPU (sm_103a) library for the matrix-free
 * Hamiltonian application y = H.x of spin-1/2 Heisenberg-type models in a
 * symmetry-adapted, fixed-Sz basis, and for Lanczos eigensolves built on it.
 *
 * The problem statement follows A. Wietek's thesis, chapter "Symmetries and
 * Parallelization for Large-Scale Exact Diagonalization":
 *   H = sum_b J_b S_i.S_j  (Eq. heisenbergallover)
 *     + sum_t Jchi_t S_i.(S_j x S_k)  (Eq. scalarchirality, Eq. chiralhamiltonian),
 *   a site-permutation group G with an optional spin flip (Eq. spinflipsymmetry,
 *   Eq. tensorchar) and a one-dimensional irrep chi of G
 *   (Eq. symmetryadaptedwavefunction1d), and a sector of fixed S^z_tot
 *   (Eq. sztotal).
 *
 * Conventions
 *   - A spin configuration is the integer sum_k sigma_k 2^(N-k), site 1 most
 *     significant, spin up = 1 (Eq. numberforspinconfig).  With 0-based sites,
 *     site s is bit N-1-s.
 *   - Group elements act actively: the spin on site i moves to site perm[g][i];
 *     a spin-flip element also complements every spin.
 *   - Sites are numbered so that sublattice X is the contiguous block
 *     [X*m, (X+1)*m), m = n_sites/n_sublat, with sublattice 0 in the most
 *     significant bits (sublattice-coding section, "Generic sublattice coding
 *     algorithm").  Every group element must map each block onto one block
 *     (sublattice stability).
 *   - The basis of a sector is the ascending list of orbit representatives
 *     (smallest integer in the orbit, Eq. representativecondition) whose
 *     projector sum_g conj(chi(g)) g|sigma> is non-zero; the index of a state is
 *     its position in that list.  The symmetric state of representative sigma
 *     has norm^2 = |G| |Stab(sigma)|.
 *   - Matrix elements between representatives (Eq. matrixelementrepresentatives
 *     with the projector of Eq. symmetryadaptedwavefunction1d_lsed):
 *       <tau~|H_k|sigma~> = conj(chi(g_tau)) sqrt(|Stab tau~|/|Stab sigma~|) <tau|H_k|sigma~>.
 *
 * Errors: every call returns an ed_status; ed_last_error() gives a message for
 * the calling thread.  No call throws.  Device pointers are CUDA device
 * pointers on the current device; host pointers are read only during the call.
 */
#ifndef ED_H
#define ED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ED_OK = 0,
    ED_ERR_ARG = 1,                     /* a null pointer, a size out of range, an unsupported dtype */
    ED_ERR_NOT_GROUP = 2,               /* perm/spinflip not closed under composition, or element 0 not the identity */
    ED_ERR_NOT_SYMMETRIC = 3,           /* some element does not map the bond or triangle set onto itself */
    ED_ERR_NOT_SUBLATTICE_STABLE = 4,   /* some element splits a sublattice block */
    ED_ERR_CHAR_NOT_HOMOMORPHISM = 5,   /* chi(gh) != chi(g)chi(h), |chi| != 1, or chi(identity) != 1 */
    ED_ERR_SPINFLIP_SZ = 6,             /* a spin-flip element with 2*n_up != n_sites */
    ED_ERR_EMPTY_SECTOR = 7,            /* the sector has dimension 0 */
    ED_ERR_NOMEM = 8,                   /* the allocator returned NULL */
    ED_ERR_INDEX_NOT_FOUND = 9,         /* a compatible representative was missing from the basis (internal error) */
    ED_ERR_TIMEOUT = 10,                /* a bounded device wait ran out */
    ED_ERR_NOT_CONVERGED = 11,          /* Lanczos reached max_iter before the tolerance */
    ED_ERR_CUDA = 12,                   /* a CUDA runtime call failed; the message holds its text */
    ED_ERR_TABLE_TOO_LARGE = 13         /* the sublattice tables do not fit the device's shared memory */
} ed_status;

/* Element type of vectors passed to ed_apply / ed_lanczos.
 * ED_F64/ED_F32 need a real Hamiltonian and real characters;
 * ED_C128/ED_C64 are interleaved (re, im) pairs. */
typedef enum { ED_F64 = 0, ED_F32 = 1, ED_C64 = 2, ED_C128 = 3 } ed_dtype;

/* A CUDA stream (cudaStream_t); NULL is the legacy default stream. */
typedef struct CUstream_st* ed_stream;

/* Device-memory provider.  alloc returns device memory of at least `bytes`
 * bytes, aligned to 256 bytes, usable on `stream`, or NULL; free releases it.
 * (Kernels read tables and vectors with 16-byte vector loads.)  When the allocator
 * pointer passed to a call is NULL the library uses cudaMalloc/cudaFree. */
typedef struct {
    void* (*alloc)(size_t bytes, ed_stream stream, void* ctx);
    void (*free)(void* ptr, size_t bytes, ed_stream stream, void* ctx);
    void* ctx;
} ed_allocator;

/* One symmetry sector.  All pointers are HOST pointers read during the call. */
typedef struct {
    int32_t n_sites;          /* N, 2 <= N <= 64 */
    int32_t n_up;             /* number of up spins, S^z = n_up - N/2 */
    int32_t n_sym;            /* |G| >= 1; element 0 must be the identity without flip */
    const int32_t* perm;      /* [n_sym][n_sites], row-major: spin on site i moves to perm[g][i] */
    const uint8_t* spinflip;  /* [n_sym] 0/1, or NULL for no flips */
    const double* chi;        /* [n_sym][2] = (Re, Im) of chi(g), |chi(g)| = 1 */
    int32_t n_sublat;         /* number of sublattice blocks, divides n_sites */
} ed_sector;

/* The Hamiltonian.  Host pointers, read during the call. */
typedef struct {
    int32_t n_bonds;
    const int32_t* bond;      /* [n_bonds][2] site pairs, i != j */
    const double* J;          /* [n_bonds] couplings of S_i.S_j */
    int32_t n_tri;
    const int32_t* tri;       /* [n_tri][3] sites (i, j, k) of S_i.(S_j x S_k), distinct */
    const double* Jchi;       /* [n_tri] couplings */
} ed_terms;

typedef struct ed_basis ed_basis;              /* opaque; owns device memory */
typedef struct ed_hamiltonian ed_hamiltonian;  /* opaque; basis + prepared terms */

/* ed_basis_build -- enumerate the sector's basis on the device.
 *
 * Validates the sector (group closure, identity first, chi a homomorphism,
 * spin flips only at S^z = 0, sublattice stability), prepares the
 * sublattice-coding lookup tables Rep_X, Sym_X and SymmetryAction_X
 * (Alg. "Preparation of lookup tables for sublattice coding algorithm",
 * Eqs. sublatsymdef, sublatrepdef, repsymdef, symactiondef), enumerates every
 * popcount-n_up state in increasing order, keeps those that are their own
 * representative (Alg. "Sublattice coding algorithm for finding the
 * representative") with a non-zero projector, and builds the prefix table
 * Limits (Alg. "Preparation of the distributed and symmetrized Hilbert space",
 * on one device and without the hash distribution).
 * Device memory comes from `alloc` (or cudaMalloc when NULL) and is owned by
 * the basis until ed_basis_free.  Runs on `stream` and synchronises it.
 * Returns ED_ERR_EMPTY_SECTOR (and no basis) for a zero-dimensional sector. */
ed_status ed_basis_build(const ed_sector* sector, const ed_allocator* alloc, ed_stream stream, ed_basis** out);

/* ---------------------------------------------------------------- SU(N) models
 * Sites carry one of n_colors colours; a configuration is the d-ary integer
 * sum_k sigma_k d^(N-k) (Eq. numberforspinconfig with local dimension d).
 * The library packs it into b = ceil(log2 d) bits per site (site 1 in the
 * most significant b bits), which keeps the order of the d-ary integers, so
 * representatives (orbit minima) and the sorted basis are those of the d-ary
 * encoding; ed_basis_export returns the packed words.  A sector fixes how
 * many sites carry each colour (the SU(N) analogue of fixed S^z). */
typedef struct {
    int32_t n_sites;          /* N >= 2, with N * b <= 64 */
    int32_t n_colors;         /* d, 2 <= d <= 16 */
    const int32_t* counts;    /* [n_colors] sites of each colour, summing to N (HOST) */
    int32_t n_sym;            /* |G| >= 1; element 0 must be the identity */
    const int32_t* perm;      /* [n_sym][n_sites]: the colour on site i moves to perm[g][i] (HOST) */
    const double* chi;        /* [n_sym][2] = (Re, Im) of chi(g) (HOST) */
    int32_t n_sublat;         /* blocks of N / n_sublat sites, every element maps blocks onto blocks;
                                 a block's bits (sites x b) at most 16 */
} ed_sector_sun;

/* ed_basis_build_sun -- the basis of an SU(N) sector on the device: every
 * colouring with the given counts, in increasing order, kept iff it is its
 * own representative with a non-zero projector (as ed_basis_build, with the
 * group acting on the b bits of each site together).  Validation errors as
 * ed_basis_build, ED_ERR_ARG for counts that do not add up to n_sites or more
 * than 64 bits. */
ed_status ed_basis_build_sun(const ed_sector_sun* sector, const ed_allocator* alloc, ed_stream stream,
                             ed_basis** out);

/* ed_hamiltonian_create_sun -- H = sum_b J_b P_(i_b j_b), P_ij the exchange of
 * the colours of sites i and j (Eq. sunexchangeop; the SU(N) Heisenberg model
 * of Eq. sunheisenbergringex without the ring term), on an SU(N) basis.  The
 * terms are `terms->bond`, `terms->J` (no triangles: ED_ERR_ARG).  Checks that
 * every element maps the bond set onto itself; a pair acts iff its colours
 * differ (amplitude J, element conj(chi(g_tau)) sqrt(|Stab tau~|/|Stab sigma~|) J)
 * and contributes J to the diagonal when they agree.  The Hamiltonian is
 * applied through its stored structure (ed_hamiltonian_store), built here
 * within max_bytes of device memory (ED_ERR_NOMEM above it); ed_apply,
 * ed_lanczos and the batch calls then work as for spin models.  Synchronous. */
ed_status ed_hamiltonian_create_sun(const ed_basis* basis, const ed_terms* terms, size_t max_bytes, ed_stream stream,
                                    ed_hamiltonian** out);

/* Dimension D of the sector. */
ed_status ed_basis_dim(const ed_basis* basis, int64_t* dim);

/* Copy the basis to HOST arrays: reps[D] as uint64 (ascending), stab[D] = |Stab(rep)|.
 * Either pointer may be NULL. */
ed_status ed_basis_export(const ed_basis* basis, uint64_t* reps, uint16_t* stab);

/* ed_sector_tables -- validate a sector and return its sublattice-coding
 * tables without touching the device (host only; for inspection and tests).
 * Performs the same checks as ed_basis_build and returns the same errors.
 * With m = n_sites/n_sublat and S = 2^m:
 *   rep[X*S + s] = Rep_X(s) (0xFFFF if no element maps block X onto block 0);
 *   sym_ids[sym_off[X*(S+1) + s] .. sym_off[X*(S+1) + s + 1]) = Sym_X(s);
 *   sa[(g*n_sublat + X)*S + s] = SymmetryAction_X(g, s), an m-bit substate of
 *   block dest[g*n_sublat + X].
 * Any output pointer may be NULL (call once with NULLs to learn *n_sym_ids).
 * Sizes: rep n_sublat*S, sym_off n_sublat*(S+1), sa n_sym*n_sublat*S,
 * dest n_sym*n_sublat, sym_ids *n_sym_ids. */
ed_status ed_sector_tables(const ed_sector* sector, uint16_t* rep, uint32_t* sym_off, uint16_t* sym_ids,
                           int64_t* n_sym_ids, uint16_t* sa, uint8_t* dest);

/* ed_representatives -- Alg. "Sublattice coding algorithm for finding the
 * representative" on the device for n caller-given states (HOST arrays, any
 * popcount; bits above n_sites are ignored).  Validates the sector like
 * ed_basis_build and uploads its tables for the duration of the call; n_up is
 * not used.  Outputs (HOST, any may be NULL): rep[n] the orbit minimum, g[n]
 * one element with g.state = rep, nstab[n] = |Stab(rep)|, compat[n] = 1 if the
 * representative's projector is non-zero in this sector.  Synchronous;
 * device memory from cudaMalloc, released before return. */
ed_status ed_representatives(const ed_sector* sector, const uint64_t* states, int64_t n, uint64_t* rep, int32_t* g,
                             int32_t* nstab, uint8_t* compat);

/* ed_representatives_noalloc -- the computation of ed_representatives for
 * callers that cannot allocate device memory.  Such callers include
 * applications whose device memory belongs to another runtime's pool (a
 * framework that reserves the GPU at start-up) and loops that must not call
 * cudaMalloc/cudaFree because those calls can synchronise the device.  This
 * entry point calls neither, nor any allocating library routine: the sector's
 * lookup-table image is copied into a file-scope device array of 224 KB
 * (229,376 bytes) that every GPU loading the library holds until exit, and
 * all other memory is the caller's.  (The thesis has no counterpart; this is
 * a deployment variant.)
 *   states: DEVICE uint64[n], n_sites-bit states (higher bits must be 0).
 *   rep, g, nstab, compat: DEVICE outputs [n], written in full; as in
 *   ed_representatives.  Inputs and outputs are owned by the caller.
 * Asynchronous on `stream`; the table upload is ordered on the same stream
 * and copies from a host buffer that lives only for the call, so the call
 * must not be made while `stream` is being captured into a CUDA graph: it
 * then returns ED_ERR_ARG before touching the device.  The first call on a
 * device looks up the array's device address (with that device current);
 * host threads may make it concurrently.  Every call shares the one array,
 * which keeps the last call's table image: calls that overlap on the GPU
 * (e.g. on different streams) race and must be serialised by the caller.  Nothing needs zeroing: each call rewrites every
 * byte of the array that its kernel reads.  Returns ED_ERR_TABLE_TOO_LARGE
 * if the table image exceeds 224 KB, and the validation errors of
 * ed_basis_build. */
ed_status ed_representatives_noalloc(const ed_sector* sector, const uint64_t* states, int64_t n, uint64_t* rep,
                                     int32_t* g, int32_t* nstab, uint8_t* compat, ed_stream stream);

/* ed_restrict -- write vectors of one sector in the basis of a subgroup's sector.
 *
 * `from` is a sector of group G with 1-D irrep chi; `to` a sector of a
 * subgroup H of G (every (perm, spin flip) of `to` is an element of `from`)
 * whose characters are chi restricted to H, with the same n_sites and n_up
 * (e.g. the translations of a space group, or the trivial group {e}, whose
 * basis is the plain fixed-Sz basis).  A state of G's sector lies in H's
 * sector: by Eq. symmetryadaptedwavefunctiontrafocharacter it transforms with
 * chi under every element of H.  Its coefficients in the normalised
 * projections of Eq. symmetryadaptedwavefunction1d are, for each
 * representative sigma_i of `to` with G-representative r = g.sigma_i at
 * index j of `from`,
 *   y_i = chi(g) sqrt(|Stab_G(r)| |H| / (|G| |Stab_H(sigma_i)|)) x_j,
 * and 0 when r's projector vanishes in G's sector.  Norms are preserved.
 *   x: DEVICE [nvec][D_from], y: DEVICE [nvec][D_to], `dtype`, caller-owned,
 *   column-major as for ed_apply, 1 <= nvec <= 8; y is overwritten.
 * Errors: ED_ERR_ARG for null pointers, different n_sites/n_up, an element of
 * `to` that is not in `from`, characters that differ from the restriction
 * (by more than 1e-9), or a real dtype with complex characters of `from`;
 * ED_ERR_INDEX_NOT_FOUND if a compatible representative is missing from
 * `from` (internal error).  Runs on `stream` and synchronises it (one 8-byte
 * device counter from `to`'s allocator). */
ed_status ed_restrict(const ed_basis* from, const ed_basis* to, ed_dtype dtype, const void* x, void* y, int32_t nvec,
                      ed_stream stream);

/* ed_apply_sz -- y = O x for the one-site sum O = sum_i c_i S^z_i (e.g. the
 * Fourier component S^z(q) = N^-1/2 sum_i exp(i q.r_i) S^z_i probed by the
 * dynamical spin structure factor) from the sector of `from` into the sector
 * of `to`.  c: HOST [n_sites][2] = (Re, Im) of c_i.  The two sectors have the
 * same group (the same elements, in any order) and n_up, and O must map one
 * onto the other: for every element g, s_g c_{g^-1(j)} = lambda(g) c_j for all
 * sites j (s_g = -1 for an element with spin flip, +1 otherwise), |lambda(g)| = 1,
 * and chi_to(g) = lambda(g) chi_from(g) (within 1e-9).  With the normalised
 * projections of Eq. symmetryadaptedwavefunction1d in both sectors,
 *   y_sigma = f(sigma) x_j,  f(sigma) = sum_i c_i s^z_i(sigma), s^z = +-1/2,
 * for each representative sigma of `to` at index j of `from` (0 when sigma is
 * not in `from`'s basis: its projector vanishes there).
 *   x: DEVICE [nvec][D_from], y: DEVICE [nvec][D_to], `dtype`, caller-owned,
 *   column-major as for ed_apply, 1 <= nvec <= 8; y is overwritten.
 * Errors: ED_ERR_ARG for null pointers, sectors that differ in n_sites, n_up
 * or group, coefficients that are all zero or that violate the condition
 * above, characters that are not lambda chi, or a real dtype with complex
 * coefficients or characters.  Runs on `stream` and synchronises it (N
 * coefficients in device memory from `to`'s allocator). */
ed_status ed_apply_sz(const ed_basis* from, const ed_basis* to, const double* c, ed_dtype dtype, const void* x,
                      void* y, int32_t nvec, ed_stream stream);

void ed_basis_free(ed_basis* basis);

/* ed_hamiltonian_create -- bind terms to a basis.
 * Checks that every group element maps the bond set (with couplings) and the
 * triangle set (with orientation and coupling) onto itself, splits each
 * S_i.S_j into its Ising part and the exchange 1/2(S+_i S-_j + S-_i S+_j)
 * (non-branching terms, Eq. nonbranchingcondition) and each chirality term
 * into spin-pair flips weighted by the third spin, and uploads the flip list.
 * The basis must outlive the Hamiltonian.  Complex terms (any Jchi != 0) or
 * complex characters need ED_C64/ED_C128 vectors. */
ed_status ed_hamiltonian_create(const ed_basis* basis, const ed_terms* terms, ed_hamiltonian** out);

/* 1 if the Hamiltonian in this sector is real symmetric (real vectors allowed). */
ed_status ed_hamiltonian_is_real(const ed_hamiltonian* h, int32_t* is_real);

void ed_hamiltonian_free(ed_hamiltonian* h);

/* ed_apply -- y = H x for nvec vectors (1 <= nvec <= 8).
 *
 * x and y are DEVICE arrays of `dtype`, column-major [nvec][D] (vector v
 * starts at element v*D), owned by the caller; y is overwritten; x and y must
 * not overlap.  Matrix-free (section "Distributed and hybrid memory
 * parallelization", Eqs. branchingsum, outputvector): each row sigma_i of y is
 * produced by one owner from the non-branching terms applied to sigma_i, the
 * representative and g_tau of each image by sublattice coding, and the index
 * of the representative by Limits + binary search (Alg. "Parallel
 * matrix-vector multiply for a non-branching term", restated in pull form:
 * y_i = sum_j conj(H_ji) x_j, valid because H is Hermitian).
 * Asynchronous on `stream`. */
ed_status ed_apply(const ed_hamiltonian* h, ed_dtype dtype, const void* x, void* y, int32_t nvec, ed_stream stream);

/* ed_hamiltonian_store -- compute H's sparsity structure once and keep it on
 * the device, so that later ed_apply calls (and everything built on them:
 * ed_lanczos, ed_expectation, ed_time_evolve, ed_lanczos_tridiag) stream it
 * instead of repeating the representative search (Alg. "Sublattice coding
 * algorithm for finding the representative") and the Limits + binary search
 * for every element.  The thesis recomputes elements in every
 * matrix-vector multiply because its sectors (D ~ 10^11) leave no room for the
 * matrix; sectors that fit one GPU usually leave room for it, and H stays the
 * same across all Lanczos steps.  What is stored: for every row sigma_i and
 * every non-zero off-diagonal element of the pull form y_i = sum_j conj(H_ji) x_j
 * (same elements, same order as the matrix-free kernel), the column j and a
 * one-byte code of conj(h) chi(g_tau) sqrt(|Stab tau~|); per row the Ising
 * part (FP64); the coefficients of at most 256 codes.  Columns are cut into
 * segments of 2^seg_log2 elements and ed_apply runs one pass per segment, so
 * each pass gathers x from one slice of about the size of L2.  seg_log2 = 0
 * picks 128 MB of `dtype` elements, at most 2^24; otherwise 5 <= seg_log2 <= 28,
 * with at most 128 segments, and a stored element keeps its code in the bits
 * above the column offset (ED_ERR_TABLE_TOO_LARGE if the codes that occur do
 * not fit beside a seg_log2-bit offset).  Results of
 * ed_apply are the same H x up to the summation order across segments; with
 * one segment and real vectors they are bit-identical to the matrix-free
 * kernel's.  Device memory (about 4 bytes per element plus 9 bytes per row
 * per segment... exactly *bytes) comes from the basis's allocator; if the
 * structure would need more than max_bytes, nothing is kept and
 * ED_ERR_NOMEM is returned (ed_apply stays matrix-free).  Also
 * ED_ERR_TABLE_TOO_LARGE when more than 256 distinct coefficients occur,
 * ED_ERR_ARG for more than 255 flip terms.  Synchronous on `stream`.
 * A second call replaces the stored structure. */
ed_status ed_hamiltonian_store(ed_hamiltonian* h, ed_dtype dtype, int32_t seg_log2, size_t max_bytes,
                               ed_stream stream, size_t* bytes);

/* ed_hamiltonian_store_autotune -- ed_hamiltonian_store with the column
 * segment and the one-vector schedule chosen by timing: the structure is built
 * for segments of half, one and two times the default size (within
 * 2^5..2^26 elements and 128 segments); for each, one-vector ed_apply is timed on
 * scratch vectors (2 D elements of `dtype` from the basis's allocator,
 * released on return) with 1, 2, 4 and 8 lanes per row
 * (ed_hamiltonian_store_set_lanes), and the fastest pair is kept (the
 * structure built again if it was not the last one tried).  Fewer, larger
 * segments save the per-row work of each pass; smaller ones keep the gathered
 * part of x in L2; several lanes per row balance long rows across a warp.
 * *seg_log2 (if non-NULL) receives the chosen log2 segment size, *bytes the
 * structure's size (ed_hamiltonian_store_schedule reports both choices).
 * Errors as ed_hamiltonian_store.  Synchronous. */
ed_status ed_hamiltonian_store_autotune(ed_hamiltonian* h, ed_dtype dtype, size_t max_bytes, ed_stream stream,
                                        int32_t* seg_log2, size_t* bytes);

/* ed_hamiltonian_store_set_lanes -- work split of the stored pass for ONE
 * vector (several vectors always take one lane per row): lanes_per_row = 1
 * (the default after every ed_hamiltonian_store: one lane per row, a row's
 * elements summed in stored order, one warp per 32 rows) or 2, 4, 8 (groups of
 * that many consecutive lanes share a row; element k goes to lane k mod L of
 * the group and a butterfly of warp shuffles combines the lanes' sums; a warp
 * still owns 32 rows and takes them in L rounds).  Results differ from one
 * lane per row only by summation order (the bit-identity with the
 * matrix-free kernel holds for one lane per row).  ED_ERR_ARG for other
 * values or without a stored structure. */
ed_status ed_hamiltonian_store_set_lanes(ed_hamiltonian* h, int32_t lanes_per_row);

/* The stored structure's schedule: log2 column-segment size and lanes per row
 * of the one-vector pass (both 0 without a stored structure).  Either pointer
 * may be NULL. */
ed_status ed_hamiltonian_store_schedule(const ed_hamiltonian* h, int32_t* seg_log2, int32_t* lanes_per_row);

/* Size of the stored structure: entries (off-diagonal elements), column
 * segments, distinct coefficient codes, device bytes; all 0 when none. */
ed_status ed_hamiltonian_store_info(const ed_hamiltonian* h, int64_t* entries, int32_t* segments, int32_t* codes,
                                    size_t* bytes);

/* Release the stored structure (ed_apply becomes matrix-free again). */
void ed_hamiltonian_store_free(ed_hamiltonian* h);

/* Counters of the most recent ed_apply on this Hamiltonian (synchronises stream):
 * number of off-diagonal terms whose representative was found (gathers per
 * vector) and number of images skipped as incompatible. */
ed_status ed_apply_counters(const ed_hamiltonian* h, ed_stream stream, int64_t* gathers, int64_t* skipped);

/* Time ed_apply on (x, y) with the launch sized for 1, 2, ... resident blocks
 * per SM, up to the most the kernel's registers allow (one vector: 6 for real
 * vectors and N <= 32, 4 for real vectors and N > 32 or complex FP32, 2 for
 * complex FP64; several vectors: 2), and keep the fastest for this
 * dtype and nvec class (nvec == 1 or > 1) in `h`.  Fewer resident blocks let
 * each block keep more of the sublattice tables in shared memory; more
 * blocks hide more memory latency.  Results of ed_apply do not depend on the
 * choice (every row is computed by one thread in a fixed order).  Overwrites
 * y; synchronous.  Writes the chosen count to *blocks_per_sm if non-NULL.
 * Without a call, ed_apply uses the most blocks the registers allow. */
ed_status ed_apply_autotune(ed_hamiltonian* h, ed_dtype dtype, const void* x, void* y, int32_t nvec,
                            ed_stream stream, int32_t* blocks_per_sm);

/* Set the resident blocks per SM that ed_apply sizes its launch for (for this
 * dtype and nvec class); 0 restores the default.  ED_ERR_ARG unless
 * 0 <= blocks_per_sm <= the limit listed at ed_apply_autotune. */
ed_status ed_apply_set_blocks(ed_hamiltonian* h, ed_dtype dtype, int32_t nvec, int32_t blocks_per_sm);

typedef struct {
    ed_dtype dtype;        /* vector type: F64/C128 plain, F32/C64 mixed (FP64 reductions) */
    int32_t n_eig;         /* lowest eigenvalues wanted, 1..8 */
    double tol;            /* convergence tolerance on eigenvalues (relative, e.g. 1e-10); with F32/C64
                              vectors and refine > 0, tol applies to the refined values */
    int32_t max_iter;      /* Lanczos steps at most (<= 2000) */
    int32_t reorth;        /* 1 = full reorthogonalisation (classical Gram-Schmidt against all stored
                              vectors, then again against the last two; max_iter + 1 vectors are stored);
                              0 = the plain three-term recursion (three vectors in memory): spurious
                              copies of converged eigenvalues are removed from the Ritz values (Cullum-Willoughby
                              test) and Ritz vectors come from a second pass of the recursion */
    uint64_t seed;         /* start vector v1(state) = keyed SplitMix64 uniform in [-1,1), normalised */
    int32_t refine;        /* mixed precision (F32/C64), 0 = no refinement: the FP32 phase runs until each
                              Ritz pair's residual bound allows (or reaches the FP32 noise floor), then the
                              Ritz vectors in FP64 get one FP64 H.x and their Rayleigh quotients; if
                              r^2/gap misses tol, at most this many FP64 Lanczos steps from their sum */
    int32_t check_every;   /* T-matrix eigensolve every this many steps (>= 1) */
    int32_t host_vectors;  /* plain recursion only (reorth = 0), where the Ritz vectors are needed:
                              1 = keep every Lanczos vector in host (system) memory as it is made, on a
                              second stream, and form the Ritz vectors (evecs, and the mixed refinement's
                              start) from there instead of by a second pass of iters H.x.  Needs a device
                              that reads pageable host memory (e.g. over NVLink-C2C); elsewhere the second
                              pass is used.  Host memory: (iters + 1) vectors of the dtype, reserved for
                              max_iter + 1 and released on return.  2 = keep them in device memory
                              ((max_iter + 1) vectors of the dtype from the allocator).  0 = second pass */
} ed_lanczos_opts;

typedef struct {
    int32_t iters;             /* Lanczos steps taken */
    int32_t converged;         /* 1 if all n_eig reached tol */
    int32_t n_apply;           /* H.x applications (including refinement) */
    double ritz[8];            /* T-matrix eigenvalues at exit (in the vector dtype's precision) */
    double resid_bound[8];     /* beta_n |s_n,k|: Lanczos residual bound of each Ritz pair */
    double refined[8];         /* eigenvalues after the FP64 refinement (when refine) */
    double refined_resid[8];   /* |H y - E y| / |y| of the Rayleigh quotient, or the FP64 polish's Lanczos
                                  residual bound (when refine) */
    double seconds;            /* wall time of the call */
} ed_lanczos_report;

/* ed_lanczos -- lowest eigenvalues of H by the Lanczos recursion
 * (Eqs. lanczosrecursionabbrev, tmatrix; Algs. "Real-symmetric Lanczos step"
 * and "Complex-Hermitian Lanczos step") with FP64 inner products,
 * optional full reorthogonalisation, and the tridiagonal eigenproblem solved in
 * FP64 every check_every steps.  evals: HOST [n_eig] (refined values when
 * opts.refine and the vectors are FP32, else Ritz values).  Converged means,
 * for each wanted Ritz value theta, |theta_n - theta_{n-c}| <= tol max(1,|theta|)
 * between checks and a Lanczos residual bound r = beta |s_last| with
 * min(r, r^2/gap) <= tol max(1,|theta|).  evecs: DEVICE [n_eig][D] of the vector dtype
 * (normalised Ritz vectors), or NULL.  Without reorthogonalisation the Ritz
 * vectors and the refinement's start vector cost a second pass of `iters`
 * H.x applications.  Workspace comes from the basis's allocator
 * and is released before return.  Synchronous.  Returns
 * ED_ERR_NOT_CONVERGED if max_iter is reached first (results still written). */
ed_status ed_lanczos(const ed_hamiltonian* h, const ed_lanczos_opts* opts, double* evals, void* evecs,
                     ed_lanczos_report* report, ed_stream stream);

/* ed_expectation -- <x_v|H|x_v> and <x_v|x_v> for nvec (1..8) DEVICE vectors
 * laid out as for ed_apply, with FP64 reductions: out (HOST) [nvec][3] =
 * (Re <x|Hx>, Im <x|Hx>, <x|x>).  One ed_apply into a workspace from the
 * basis's allocator.  With H the orbit average of a bond operator,
 * (1/|orbit|) sum over the bonds {i', j'} of the symmetry orbit of {i, j} of
 * S_i'.S_j', this gives the spin correlation <S_i.S_j> of a state of the
 * sector (the correlations behind the static structure factor, Eq.
 * structurefactor): <psi|g O g^-1|psi> = <psi|O|psi> for a state of a
 * one-dimensional irrep.  Synchronous on `stream`. */
ed_status ed_expectation(const ed_hamiltonian* h, ed_dtype dtype, const void* x, int32_t nvec, ed_stream stream,
                         double* out);

/* ed_time_evolve -- psi <- exp(-i H dt) psi by one Krylov step: m (2..64)
 * Lanczos vectors from psi with full reorthogonalisation, the m x m
 * tridiagonal T = V^H H V (Eq. tmatrix) diagonalised on the host, and
 * psi_new = |psi| V exp(-i T dt) e_1 (the Krylov propagator behind the
 * thesis's Lanczos time evolution).  psi: DEVICE [D] of ED_C128 or ED_C64,
 * overwritten.  *err (if non-NULL) = |psi| beta_m |(exp(-i T dt) e_1)_m|,
 * the standard estimate of the step's error; *m_used (if non-NULL) the
 * Krylov dimension used (smaller when psi spans an invariant subspace).
 * Workspace (m + 1 vectors) from the basis's allocator.  Synchronous. */
ed_status ed_time_evolve(const ed_hamiltonian* h, ed_dtype dtype, void* psi, double dt, int32_t m, ed_stream stream,
                         double* err, int32_t* m_used);

/* ed_lanczos_tridiag -- the Lanczos recursion (Eqs. lanczosrecursion, tmatrix)
 * started from a given DEVICE vector x [D] of `dtype` (not modified, need not
 * be normalised): v_0 = x/|x|, alpha[n] = <v_n|H v_n>, beta[n] = |w_n| with
 * w_n = H v_n - alpha[n] v_n - beta[n-1] v_{n-1}, v_{n+1} = w_n/beta[n], for
 * n < *m_used <= m.  T has diagonal alpha[0..m_used-1] and off-diagonal
 * beta[0..m_used-2]; beta[m_used-1] is the norm of the last residual.  The
 * recursion stops early when beta[n] < 1e-14 (|alpha[n]| + 1) (x lies in an
 * invariant subspace of that dimension).  *norm2 (if non-NULL) = <x|x>.
 * The continued-fraction expansion <x|(z - H)^-1|x> =
 * norm2 / (z - alpha[0] - beta[0]^2 / (z - alpha[1] - ...)) of a dynamical
 * correlation function needs only these numbers.  reorth = 1 keeps all
 * m+1 vectors (m capped at D) and orthogonalises each new one against them
 * (classical Gram-Schmidt twice, the second pass against the last two);
 * reorth = 0 is the plain three-term recursion with three vectors.
 * alpha, beta: HOST [m].  1 <= m <= 100000 (m <= 65534 with reorth).  Workspace from the basis's
 * allocator; FP64 reductions.  Synchronous. */
ed_status ed_lanczos_tridiag(const ed_hamiltonian* h, ed_dtype dtype, const void* x, int32_t m, int32_t reorth,
                             ed_stream stream, double* alpha, double* beta, double* norm2, int32_t* m_used);

/* Lowest k eigenvalues of a Lanczos T-matrix (Eq. tmatrix: diagonal alpha[n],
 * off-diagonal beta[n-1], HOST arrays) by Sturm bisection in FP64, the solver
 * ed_lanczos uses.  filter = 1 applies its treatment of the plain recursion:
 * Ritz values within 100 eps_vectors |T| of each other count once, and a
 * value without such copies that is also an eigenvalue of T without its first
 * row and column (within 1e3 eps_64 |T|) is dropped as spurious; eps_vectors
 * is the unit roundoff of the Lanczos vectors (2^-53 for FP64, 2^-24 for FP32,
 * or their epsilon).  Writes at most k values, ascending, to evals (HOST) and
 * their number to *n_found.  Host only; no device is touched. */
ed_status ed_tridiag_eigs(const double* alpha, const double* beta, int32_t n, int32_t k, double eps_vectors,
                          int32_t filter, double* evals, int32_t* n_found);

/* ed_band_eigs -- lowest k eigenpairs of a Hermitian band matrix T (the block
 * tridiagonal T of block Lanczos has bandwidth 2 block - 1), the host solver
 * ed_lanczos_batch uses.  band: HOST [n][bw+1][2], entry (i, q) = (Re, Im) of
 * T[i][i-q] for q <= i (the lower band; the diagonal's imaginary part is
 * ignored).  Eigenvalues by bisection on the inertia of T - x (banded LDL^H,
 * FP64), ascending, into evals[k]; eigenvectors (evecs: HOST [k][n][2] or
 * NULL) by inverse iteration with pivoting inside the band, each
 * orthogonalised against the earlier ones (so degenerate values get
 * orthonormal vectors).  *n_found = min(k, n).  Host only; no device is
 * touched. */
ed_status ed_band_eigs(const double* band, int32_t n, int32_t bw, int32_t k, double* evals, double* evecs,
                       int32_t* n_found);

/* ---------------------------------------------------------------- batches of sectors
 * A batch groups Hamiltonians of several sectors of one cluster (same number
 * of sites, state word and sublattice blocks, e.g. every momentum/irrep
 * sector) so that one launch applies all of them and block Lanczos runs on
 * all of them at once.  Vectors of a batch are concatenated: sector s owns rows
 * [row_off[s], row_off[s+1]) (ed_batch_rows), and a block of nvec vectors of
 * sector s starts at element nvec*row_off[s], column-major within the sector.
 * The Hamiltonians must outlive the batch. */
typedef struct ed_batch ed_batch;

ed_status ed_batch_create(const ed_hamiltonian* const* h, int32_t n, ed_batch** out);

/* HOST row_off[n+1]. */
ed_status ed_batch_rows(const ed_batch* batch, int64_t* row_off);

/* y_s = H_s x_s for every sector s, nvec (1..8) vectors each, in one persistent
 * launch: every block takes a contiguous range of the batch's rows and stages
 * each sector's tables as it reaches its rows.  x, y: DEVICE, caller-owned.
 * Asynchronous on `stream`. */
ed_status ed_apply_batch(const ed_batch* batch, ed_dtype dtype, const void* x, void* y, int32_t nvec, ed_stream stream);

/* Time ed_apply_batch for grids of 1, 2, 4, 8, 16 waves of resident blocks
 * (shorter row ranges per block balance uneven sectors, longer ones restage
 * fewer tables) and keep the fastest for this dtype and nvec.  Overwrites y.
 * Synchronous; call it before capturing work that uses the batch. */
ed_status ed_batch_autotune(ed_batch* batch, ed_dtype dtype, const void* x, void* y, int32_t nvec, ed_stream stream,
                            int32_t* waves);

void ed_batch_free(ed_batch* batch);

typedef struct {
    ed_dtype dtype;        /* ED_F64 (all sectors real) or ED_C128; or FP32 vectors, ED_F32 (all sectors
                              real) or ED_C64, which need reorth = 1 and n_eig <= 8: the block
                              Gram-Schmidt then runs in FP32 arithmetic (sums across row tiles and the
                              b x b matrices in FP64), a sector stops when its values settle to tol or to
                              the FP32 noise of T (8 eps_32 |T|), and the values are refined in FP64 */
    int32_t block;         /* right-hand sides per sector, 1..8 */
    int32_t n_eig;         /* lowest eigenvalues per sector */
    double tol;            /* convergence: each eigenvalue changed by at most tol/10 (relative) since the
                              previous check, on two checks in a row, and its Ritz residual bound r
                              (beta |s_last| for block = 1, |B_last z_last| for a Ritz vector z of the
                              block T) within min(r, r^2/gap) <= tol (relative) */
    int32_t max_iter;      /* block steps at most (2..400) */
    uint64_t seed;         /* Gaussian start blocks from keyed SplitMix64 of (seed, column, state) */
    int32_t use_graph;     /* 1: capture one step (all kernels, all sectors) as a CUDA graph and replay it */
    int32_t check_every;   /* eigenvalue check every this many steps */
    int32_t reorth;        /* 1: full reorthogonalisation (classical Gram-Schmidt against all stored blocks
                              and a second pass against the last two); 0: the plain recursion (only the
                              last two vectors), spurious copies
                              of converged eigenvalues removed as in ed_lanczos; needs block = 1 (with
                              larger blocks copies could not be told from multiplicities: ED_ERR_ARG) */
} ed_block_lanczos_opts;

typedef struct {
    int32_t iters;             /* block steps taken */
    int32_t converged_sectors; /* sectors whose n_eig values were steady for two checks (FP32
                                  vectors: whose refined values are certified) */
    int32_t krylov_dim;        /* iters * block */
    int32_t used_graph;
    double seconds;            /* wall time of the call */
    double step_seconds;       /* time inside the steps (graph launches + sync) */
} ed_block_lanczos_report;

/* ed_lanczos_batch -- block Lanczos (the block form of Eqs.
 * lanczosrecursionabbrev and tmatrix with b x b blocks) on every sector of the
 * batch at once, with full reorthogonalisation (classical Gram-Schmidt against
 * all stored blocks, then again against the last two, where the new block's
 * large components lie) or the plain recursion (opts.reorth) and
 * Cholesky QR twice for the new block; a sector whose values have settled
 * stops iterating (its rows are skipped by later steps); inner
 * products in FP64 with a fixed reduction order.  evals: HOST [n][n_eig]
 * (sector-major), lowest eigenvalues of each sector's block tridiagonal T
 * (degenerate eigenvalues appear with their multiplicity up to the block size).
 * With FP32 vectors the values are then refined as ed_lanczos refines its
 * mixed-precision run: per sector the Ritz vectors of the n_eig lowest values
 * of T (inverse iteration on the band T) are formed in FP64 from the FP32
 * blocks, one FP64 batched H.x is applied to all of them, and Rayleigh-Ritz
 * on their span (which resolves degenerate copies) gives the returned values
 * E and vectors y.  A sector counts as converged when every residual
 * r = |Hy - E y| / |y| satisfies r <= tol |E| or r^2 / gap <= tol |E| (gap:
 * the distance from E to the nearest Ritz value of T of another level, less r,
 * values within max(10 r, 1e-6 |E|) of E counting as copies of its own level;
 * the Rayleigh quotient's error is at most r^2 / gap).  Sectors not certified
 * this way (a close next level) continue in FP64: block Lanczos from their
 * refined vectors, with only those sectors iterating (at most 60 steps).
 * Workspace from the batch's allocator (or cudaMalloc), released before
 * return.  Synchronous (uses an internal stream).
 * ED_ERR_NOT_CONVERGED if some sector did not settle within max_iter, or (FP32
 * vectors) its refined values are not certified (values still written). */
ed_status ed_lanczos_batch(const ed_batch* batch, const ed_block_lanczos_opts* opts, double* evals,
                           ed_block_lanczos_report* report, ed_stream stream);

/* Message of the last error on the calling thread ("" if none). */
const char* ed_last_error(void);

/* Library version string. */
const char* ed_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ED_H */
