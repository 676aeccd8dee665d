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
#include "ed_apply_impl.cuh"

namespace ed {

// instantiated in ed_apply_k0..k3.cu
extern template ed_status apply_launch_kind<0>(const HxArgs&, size_t, int, bool, bool, bool, cudaStream_t);
extern template ed_status apply_launch_kind<1>(const HxArgs&, size_t, int, bool, bool, bool, cudaStream_t);
extern template ed_status apply_launch_kind<2>(const HxArgs&, size_t, int, bool, bool, bool, cudaStream_t);
extern template ed_status apply_launch_kind<3>(const HxArgs&, size_t, int, bool, bool, bool, cudaStream_t);
extern template ed_status apply_batch_kind<0>(const BatchLaunch&, cudaStream_t);
extern template ed_status apply_batch_kind<1>(const BatchLaunch&, cudaStream_t);
extern template ed_status apply_batch_kind<2>(const BatchLaunch&, cudaStream_t);
extern template ed_status apply_batch_kind<3>(const BatchLaunch&, cudaStream_t);

// Must agree with the kernel's template choice (launch_ns / batch_nv): the
// block-count-specialised search runs for 2..4 blocks with packed entries.
static bool generic_search(const ed_basis* b, bool ns_ok) {
    return !(ns_ok && b->ht.n_sub >= 2 && b->ht.n_sub <= 4);
}

static int kind_of(ed_dtype dt) { return dt == ED_F64 ? 0 : dt == ED_F32 ? 1 : dt == ED_C128 ? 2 : 3; }

static SmemLayout layout_for(const ed_hamiltonian* h, ed_dtype dt, bool ns_ok) {
    const ed_basis* b = h->basis;
    return smem_layout(hot_bytes(b->dt, kind_of(dt), generic_search(b, ns_ok)), h->n_flip, h->n_jc, b->dt.G,
                       1 << b->ht.m);
}

size_t apply_smem_bytes(const ed_hamiltonian* h, ed_dtype dt) {
    return layout_for(h, dt, h->basis->dt.dl_stride == 4).total;
}

HxArgs make_args(const ed_hamiltonian* h) {
    const ed_basis* b = h->basis;
    HxArgs a{};
    a.dt = b->dt;
    a.reps = b->reps.p;
    a.stab = (const uint16_t*)b->stab.p;
    const uint8_t* dir = (const uint8_t*)b->limits.p;
    a.dir_base = (const uint32_t*)dir;
    a.dir_q = dir + b->dir_q_off();
    a.limits = (const uint32_t*)(dir + b->dir_lim_off());
    a.bkt = b->bkt.p;
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
    a.D = b->dim;
    a.nvec = 1;
    return a;
}

size_t hx_smem_bytes(const ed_hamiltonian* h, ed_dtype dt, bool ns_ok) { return layout_for(h, dt, ns_ok).total; }

ed_status apply_batch_launch(const BatchLaunch& L, cudaStream_t s) {
    switch (L.dtype) {
        case ED_F64: return apply_batch_kind<0>(L, s);
        case ED_F32: return apply_batch_kind<1>(L, s);
        case ED_C128: return apply_batch_kind<2>(L, s);
        case ED_C64: return apply_batch_kind<3>(L, s);
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
    a.bkt = b->bkt.p;
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
    const bool w8 = b->word == 8, ch = b->dt.chunk_lo > 0;
    const bool ns_ok = b->dt.dl_stride == 4;
    const size_t smem = layout_for(h, dt, ns_ok).total;
    const int n_sub = b->ht.n_sub;
    switch (dt) {
        case ED_F64: return apply_launch_kind<0>(a, smem, n_sub, ns_ok, w8, ch, s);
        case ED_F32: return apply_launch_kind<1>(a, smem, n_sub, ns_ok, w8, ch, s);
        case ED_C128: return apply_launch_kind<2>(a, smem, n_sub, ns_ok, w8, ch, s);
        case ED_C64: return apply_launch_kind<3>(a, smem, n_sub, ns_ok, w8, ch, s);
    }
    return fail(ED_ERR_ARG, "bad dtype");
}

}  // namespace ed
