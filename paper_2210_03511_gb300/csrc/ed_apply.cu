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

static HxPlan plan_for(const ed_hamiltonian* h, ed_dtype dt, bool ns_ok, int blocks) {
    const ed_basis* b = h->basis;
    return hx_plan(b->dt, kind_of(dt), generic_search(b, ns_ok), blocks, h->n_flip, h->n_jc, 1 << b->ht.m);
}

size_t hx_smem_bytes(const ed_hamiltonian* h, ed_dtype dt, bool ns_ok, int nvec, int blocks) {
    (void)nvec;
    return plan_for(h, dt, ns_ok, blocks).lay.total;
}

// Default resident blocks per SM: the most the registers allow (see
// hx_min_blocks); the staging plan keeps in shared memory what fits
// beside them and reads the rest through L1/L2.  (Measured on the
// workloads: occupancy pays more than staging the Rep/Sym tables.)
int hx_default_blocks(const ed_hamiltonian* h, ed_dtype dt, bool ns_ok, int nvec) {
    (void)ns_ok;
    return hx_min_blocks(h->basis->word, nvec == 1 ? 1 : MAXV, kind_of(dt));
}

static int blocks_for(const ed_hamiltonian* h, ed_dtype dt, bool ns_ok, int nvec) {
    const int t = h->tuned_blocks[kind_of(dt)][nvec > 1 ? 1 : 0];
    return t > 0 ? t : hx_default_blocks(h, dt, ns_ok, nvec);
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
    a.limits = (const uint2*)(dir + b->dir_lim_off());
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
    a.blocks = 1;  // set per launch
    return a;
}


ed_status apply_batch_launch(const BatchLaunch& L, cudaStream_t s) {
    if (L.stored) return cache_batch_launch(L, s);
    switch (L.dtype) {
        case ED_F64: return apply_batch_kind<0>(L, s);
        case ED_F32: return apply_batch_kind<1>(L, s);
        case ED_C128: return apply_batch_kind<2>(L, s);
        case ED_C64: return apply_batch_kind<3>(L, s);
    }
    return fail(ED_ERR_ARG, "bad dtype");
}

ed_status apply_launch(const ed_hamiltonian* h, ed_dtype dt, const void* x, void* y, int nvec, cudaStream_t s,
                       bool use_cache) {
    if (use_cache && h->cache.valid) return cache_apply(h, dt, x, y, nvec, s);
    if (h->sun)
        return fail(ED_ERR_ARG, "an SU(N) Hamiltonian is applied through its stored structure, which was released");
    const ed_basis* b = h->basis;
    if (h->n_flip > 256) return fail(ED_ERR_ARG, "more than 256 flip terms are not supported");
    HxArgs a = make_args(h);
    a.x = x;
    a.y = y;
    a.nvec = nvec;
    a.counters = (unsigned long long*)h->d_counters.p;
    ED_CUDA(cudaMemsetAsync(h->d_counters.p, 0, 24, s));
    const bool w8 = b->word == 8, ch = b->dt.chunk_lo > 0;
    const bool ns_ok = b->dt.dl_stride == 4;
    a.blocks = blocks_for(h, dt, ns_ok, nvec);
    const size_t smem = plan_for(h, dt, ns_ok, a.blocks).lay.total;
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

extern "C" ed_status ed_apply_autotune(ed_hamiltonian* h, ed_dtype dtype, const void* x, void* y, int32_t nvec,
                                       ed_stream stream, int32_t* blocks_out) {
    using namespace ed;
    if (!h || !x || !y) return fail(ED_ERR_ARG, "null argument");
    if (nvec < 1 || nvec > MAXV) return fail(ED_ERR_ARG, "nvec out of range [1,8]");
    if (h->sun) return fail(ED_ERR_ARG, "an SU(N) Hamiltonian has no matrix-free kernel to tune");
    cudaStream_t s = (cudaStream_t)stream;
    int& slot = h->tuned_blocks[kind_of(dtype)][nvec > 1 ? 1 : 0];
    const int top = hx_min_blocks(h->basis->word, nvec == 1 ? 1 : MAXV, kind_of(dtype));
    cudaEvent_t e0, e1;
    ED_CUDA(cudaEventCreate(&e0));
    ED_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_b = 0;
    ed_status st = ED_OK;
    for (int b = 1; b <= top && st == ED_OK; ++b) {
        slot = b;
        st = apply_launch(h, dtype, x, y, nvec, s, false);  // warm-up (configures the instantiation)
        if (st != ED_OK) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = fail(ED_ERR_CUDA, "event record"); break; }
        st = apply_launch(h, dtype, x, y, nvec, s, false);
        if (st != ED_OK) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            st = fail(ED_ERR_CUDA, "event wait");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_b = b; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    slot = st == ED_OK ? best_b : 0;
    if (blocks_out) *blocks_out = slot;
    return st;
}

extern "C" ed_status ed_apply_set_blocks(ed_hamiltonian* h, ed_dtype dtype, int32_t nvec, int32_t blocks) {
    using namespace ed;
    if (!h) return fail(ED_ERR_ARG, "null argument");
    if (nvec < 1 || nvec > MAXV) return fail(ED_ERR_ARG, "nvec out of range [1,8]");
    if ((int)dtype < 0 || (int)dtype > 3) return fail(ED_ERR_ARG, "bad dtype");
    const int top = hx_min_blocks(h->basis->word, nvec == 1 ? 1 : MAXV, kind_of(dtype));
    if (blocks < 0 || blocks > top) return fail(ED_ERR_ARG, "blocks per SM out of range [0,%d]", top);
    h->tuned_blocks[kind_of(dtype)][nvec > 1 ? 1 : 0] = blocks;
    return ED_OK;
}
