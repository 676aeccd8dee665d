// Internal declarations of libed (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ed.h"

namespace ed {

// ---------------------------------------------------------------- errors
void set_error(ed_status st, const char* fmt, ...);
ed_status fail(ed_status st, const char* fmt, ...);
ed_status cuda_fail(cudaError_t e, const char* what);

#define ED_CUDA(call)                                  \
    do {                                               \
        cudaError_t _e = (call);                       \
        if (_e != cudaSuccess) return ed::cuda_fail(_e, #call); \
    } while (0)

// ---------------------------------------------------------------- memory
struct Alloc {
    ed_allocator a{};
    bool custom = false;
    void* get(size_t bytes, cudaStream_t s) const;
    void put(void* p, size_t bytes, cudaStream_t s) const;
};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// ---------------------------------------------------------------- sublattice-coding tables (host)
// Table layouts (m = bits per sublattice block, S = 2^m substates):
//   rep[X*S + s]                 Rep_X(s)                      (Eq. sublatrepdef)
//   sym_off[X*(S+1) + s .. +1]   range of Sym_X(s) in sym_ids  (Eq. repsymdef)
//   sa[(g*n_sub + X)*S + s]      SymmetryAction_X(g, s) as an m-bit substate of
//                                block dest[g*n_sub + X]       (Eq. symactiondef)
//   src[g*n_sub + Z]             the block X with dest(g, X) = Z
struct HostTables {
    int N = 0, n_up = 0, G = 0, n_sub = 0, m = 0;
    std::vector<int32_t> perm;      // [G][N]
    std::vector<uint8_t> flip;      // [G]
    std::vector<double> chi;        // [G][2]
    std::vector<uint8_t> dest, src; // [G][n_sub]
    std::vector<uint16_t> rep;      // [n_sub][S]
    std::vector<uint32_t> sym_off;  // [n_sub][S+1]
    std::vector<uint16_t> sym_ids;
    std::vector<uint16_t> sa;       // [G][n_sub][S]
    std::vector<uint16_t> chi_cls;  // [G] id of the value chi(g); equal ids <=> equal characters
    bool real_chars = true;
    // SymmetryAction stored once per distinct local block map (a permutation of
    // the m positions of a block plus the flip bit): srclid[g*n_sub + Z] packs
    // the source block X = src(g, Z) (low 8 bits) and the map id (high bits).
    // For m <= 8 a map is one table of S bytes; for m > 8 it is two chunk
    // tables (high m - c and low c = m/2 bits) of uint16 images that are OR-ed.
    int n_lmap = 0;
    std::vector<uint32_t> srclid;   // [G][n_sub]
    // Per element and DESTINATION block Z: (source block X << 12) | map id,
    // padded to dl_stride (a multiple of 4) entries per element; empty when a
    // map id does not fit 12 bits or there are more than 16 blocks.
    std::vector<uint16_t> dl;
    int dl_stride = 0;
    std::vector<uint8_t> chi_neg;   // [G] real chi(g) < 0
    std::vector<uint16_t> lmap_tab; // [n_lmap][table entries per map]
    int chunk_lo = 0;               // c (0 when m <= 8)
};

ed_status build_host_tables(const ed_sector* sec, HostTables& t);

// Device copy of the tables, in the order they are staged into shared memory.
struct DevTables {
    int N, G, n_sub, m;
    int sa_bytes;            // 1 (m <= 8) or 2
    const uint8_t* blob;     // contiguous device image (see tables_blob layout)
    size_t blob_bytes;
    // offsets (bytes) inside the blob
    uint32_t off_rep, off_symoff, off_symids, off_sa, off_src, off_chi, off_chicls, off_sqrt;
    uint32_t off_chif, off_sqrtf;   // float copies of chi and sqrt tables for FP32 vectors
    int chunk_lo;                   // low chunk bits of SymmetryAction maps (0: single table)
    int lmap_stride;                // entries per map
    uint32_t off_dl, off_chineg;
    int dl_stride;
};

// ---------------------------------------------------------------- flip terms (host + device)
// Off-diagonal non-branching terms grouped by site pair (a, b):
//   h(sigma) = jhalf + i * sum_t k_t * s^z_{c_t} * (spin a down ? +1 : -1)
// where jhalf = sum of J/2 over the bonds on {a,b} (exchange part of S_a.S_b)
// and each chirality triangle containing the pair contributes k = +-Jchi/2
// (sign + when (a, b, c) is a cyclic rotation of the triangle's order).
struct FlipTerm {
    int8_t pa, pb;   // bit positions (N-1-site)
    int8_t pc0, pc1; // bit positions of the third sites, -1 if absent
    float pad;
    double jhalf;
    double k0, k1;
};

struct DiagClass {          // Ising part grouped by coupling: sum_b J_b s^z_i s^z_j
    double J;               // coupling of this class
    int first, count;       // range in the bond-position list
};

}  // namespace ed

// ---------------------------------------------------------------- opaque handles
struct ed_basis {
    ed::Alloc alloc;
    ed::HostTables ht;
    ed::DevTables dt{};
    ed::DevBuf tables;          // blob
    int64_t dim = 0;
    int word = 4;               // bytes per state word (4 if N <= 32 else 8)
    ed::DevBuf reps;            // [dim] uint32 or uint64, ascending
    ed::DevBuf stab;            // [dim] uint16
    int prefix_bits = 0;        // L = N - m: bits below the top sublattice block
    // Two-level Limits directory, one device allocation:
    //   base[S+1] (uint32): first key of top-block value v
    //   q[S] (uint8, padded to 16 bytes): bucket bits used below the top block for v
    //   limits[n_keys+1] (uint2, 16-byte aligned): .x first basis index of the
    //     bucket, .y byte p = fingerprint state_fp() of its state p < 4
    ed::DevBuf limits;
    uint64_t n_keys = 0;
    int device = 0;
    // SU(N) basis (ed_basis_build_sun): colours in sun_b bits per site; the
    // tables above act on the n_sites * sun_b bit positions
    int sun_d = 0;                      // number of colours (0: spin-1/2 basis)
    int sun_b = 1;                      // bits per site
    int sun_N = 0;                      // sites
    std::vector<int32_t> sun_perm;      // [G][sun_N] site permutations
    std::vector<int32_t> sun_counts;    // [sun_d]
    size_t dir_q_off() const { return (size_t)((1 << ht.m) + 1) * 4; }
    size_t dir_lim_off() const { return (dir_q_off() + (size_t)(((1 << ht.m) + 15) & ~15) + 15) & ~(size_t)15; }
};

namespace ed {
// Stored structure of H (csrc/ed_cache.cu): per column segment b, entry
// counts per row, per-slice offsets and the entries (code << 24 | column
// offset), the per-row Ising part, and the coefficient table of the codes.
struct HCache {
    bool valid = false;
    int seg_bits = 0, nb = 0, n_code = 0, sms = 0, off_bits = 24;
    bool axis_d = false, axis_f = false;  // complex codes all real or purely imaginary (FP64 / FP32 table)
    int n_re = 0;                         // codes below n_re have real coefficients
    int lanes = 1;                        // lanes per row of the one-vector pass (1, 2, 4, 8)
    int64_t ns = 0;                 // slices of 32 rows
    DevBuf counts, boff, ent, diag, ctab, ctr;
    std::vector<uint64_t> bbase;    // [nb+1] first entry of each segment
    uint64_t n_ent = 0, n_skip = 0;
    size_t bytes = 0;
};
}  // namespace ed

struct ed_hamiltonian {
    const ed_basis* basis = nullptr;
    bool is_real = true;
    int n_flip = 0;
    int n_diag_bonds = 0;
    std::vector<ed::FlipTerm> flips;
    std::vector<int8_t> diag_pos;       // [2*n_diag_bonds] bit positions
    std::vector<ed::DiagClass> diag_cls;
    ed::DevBuf d_flips, d_diag_pos, d_diag_cls, d_counters;
    int n_diag_cls = 0;
    // real coefficients: jhs[c][n] = jhalf_c * sqrt(n) for the distinct jhalf values c
    int n_jc = 0;
    std::vector<double> jhs;
    std::vector<uint8_t> jcls;          // [n_flip]
    ed::DevBuf d_jhs, d_jcls;
    int tuned_blocks[4][2] = {};        // resident H.x blocks per SM by dtype, nvec == 1 / > 1 (0: default)
    bool sun = false;                   // SU(N) exchange model: applied through its stored structure only
    ed::HCache cache;                   // stored structure, when built (ed_hamiltonian_store)
};

namespace ed {
// Arguments of one sector's H.x (device pointers; see ed_apply.cu).
struct HxArgs {
    DevTables dt;
    const void* reps;
    const uint16_t* stab;
    const uint32_t* dir_base;
    const uint8_t* dir_q;
    const uint2* limits;
    int L, S;
    int blocks;                   // resident blocks per SM the launch is sized for (drives the staging plan)
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
HxArgs make_args(const ed_hamiltonian* h);
// One sector's stored structure as the batched stored-structure kernel reads
// it (one column segment; see csrc/ed_cache.cu).
struct CacheSector {
    const uint8_t* counts;     // [32 ns] entries per row
    const uint32_t* boff;      // [ns] first entry of each slice
    const uint32_t* ent;       // entries: (code << off_bits) | column
    const double* diag;        // [D] Ising part
    const uint16_t* stab;      // [D] |Stab sigma_i|
    const uint8_t* ctab;       // coefficients: [256] double2, [256] double, [256] float2, [256] float
    const uint8_t* sq;         // sqrt(k) then 1/sqrt(k), k = 0..G (double)
    const uint8_t* sqf;        // the same in float
    int64_t D, ns, slice0;     // rows, slices, first slice of the sector in the batch's slice list
    int G1;                    // G + 1
    uint32_t off_bits;
};
// One batched H.x launch (all sectors of a batch).
struct BatchLaunch {
    const HxArgs* desc;        // device [n_sec]
    const int64_t* row_off;    // device [n_sec+1]
    int n_sec;
    int64_t total_rows;
    size_t smem;
    bool w8, chunked, ns_ok;
    int n_sub;
    ed_dtype dtype;
    int nvec;
    const void* x;
    void* y;
    const int* x_step;         // device step index or null
    int64_t x_step_elems;
    unsigned long long* counters;
    int waves;                 // grid = SMs x resident blocks x waves
    int blocks;                // resident blocks per SM (staging plan of every sector)
    const int* active;         // device [n_sec]: rows of sectors with 0 are skipped (null: all)
    const CacheSector* stored; // device [n_sec]: every sector's stored structure, or null (matrix-free)
    int64_t stored_slices;     // slices of 32 rows over all sectors
};
ed_status apply_batch_launch(const BatchLaunch& L, cudaStream_t s);
// implemented in ed_cache.cu: the batched stored-structure H.x, and the
// descriptor of one Hamiltonian's structure (false unless stored in one segment)
ed_status cache_batch_launch(const BatchLaunch& L, cudaStream_t s);
bool cache_sector_desc(const ed_hamiltonian* h, CacheSector& d);
size_t hx_smem_bytes(const ed_hamiltonian* h, ed_dtype dt, bool ns_ok, int nvec, int blocks);
int hx_default_blocks(const ed_hamiltonian* h, ed_dtype dt, bool ns_ok, int nvec);
// implemented in ed_basis.cu
ed_status basis_build_device(ed_basis* b, cudaStream_t s);
ed_status upload_tables(ed_basis* b, cudaStream_t s);
void make_blob(const HostTables& t, DevTables& d, std::vector<uint8_t>& image);
ed_status representatives_device(const ed_basis* b, const uint64_t* states, int64_t n, uint64_t* rep, int32_t* g,
                                 int32_t* nstab, uint8_t* compat, cudaStream_t s);
ed_status representatives_static(const ed_sector* sector, const uint64_t* states, int64_t n, uint64_t* rep, int32_t* g,
                                 int32_t* nstab, uint8_t* compat, cudaStream_t s);
ed_status exclusive_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* total, const Alloc& A,
                             cudaStream_t s);
// implemented in ed_apply.cu; uses the stored structure when there is one and use_cache is set
ed_status apply_launch(const ed_hamiltonian* h, ed_dtype dt, const void* x, void* y, int nvec, cudaStream_t s,
                       bool use_cache = true);
// implemented in ed_cache.cu
ed_status cache_build(ed_hamiltonian* h, ed_dtype dtype, int seg_log2, size_t max_bytes, cudaStream_t s);
ed_status cache_apply(const ed_hamiltonian* h, ed_dtype dt, const void* x, void* y, int nvec, cudaStream_t s);
void cache_free(ed_hamiltonian* h);
// implemented in ed_lanczos.cu
void tridiag_lowest(const std::vector<double>& a, const std::vector<double>& b, int n, int k, bool filter,
                    double eps_v, std::vector<double>& lam, std::vector<double>* last = nullptr);
ed_status lanczos_run(const ed_hamiltonian* h, const ed_lanczos_opts* o, double* evals, void* evecs,
                      ed_lanczos_report* rep, cudaStream_t s);
}  // namespace ed
