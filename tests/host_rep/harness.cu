// Test harness: the library's representative search (Alg. "Sublattice coding
// algorithm for finding the representative") compiled for the host.  The
// search functions are __host__ __device__, so the code the kernels run is
// exercised here on the CPU against the oracle, over the library's own table
// image (build_host_tables + make_blob, linked from libed.so).
#include <vector>

#include "ed_device.cuh"

namespace {

template <typename W, bool CH>
int run(const ed::TabView<CH>& t, const uint64_t* states, int64_t n, int n_sub, int variant, uint64_t* rep,
        int32_t* g, int32_t* nst, uint8_t* cp, uint8_t* own) {
    for (int64_t i = 0; i < n; ++i) {
        W r;
        int gb, ns;
        bool c;
        const W s = (W)states[i];
        if (variant == 1 && n_sub == 2) ed::find_rep_ns<W, CH, 2>(s, t, r, gb, ns, c);
        else if (variant == 1 && n_sub == 3) ed::find_rep_ns<W, CH, 3>(s, t, r, gb, ns, c);
        else if (variant == 1 && n_sub == 4) ed::find_rep_ns<W, CH, 4>(s, t, r, gb, ns, c);
        else if (variant == 1) return -2;
        else ed::find_rep<W, CH>(s, t, r, gb, ns, c);
        rep[i] = (uint64_t)r;
        g[i] = gb;
        nst[i] = ns;
        cp[i] = c ? 1 : 0;
        int ns2;
        bool c2;
        own[i] = ed::is_rep<W, CH>(s, t, ns2, c2) ? 1 : 0;
        if (own[i] && (ns2 != ns || c2 != c)) return -3;  // the two searches disagree
    }
    return 0;
}

}  // namespace

// variant 0: generic search; 1: the block-count-specialised search (2..4
// blocks, packed per-element entries required).  Returns 0, an ed_status
// (> 0) from the table builder, -1 when variant 1 has no packed entries, -2
// for a block count it does not cover, -3 when is_rep disagrees.
extern "C" int harness_representatives(const ed_sector* sec, const uint64_t* states, int64_t n, int variant,
                                       uint64_t* rep, int32_t* g, int32_t* nst, uint8_t* cp, uint8_t* own) {
    ed::HostTables ht;
    const ed_status st = ed::build_host_tables(sec, ht);
    if (st != ED_OK) return (int)st;
    ed::DevTables dt{};
    std::vector<uint8_t> img;
    ed::make_blob(ht, dt, img);
    dt.blob = img.data();
    if (variant == 1 && dt.dl_stride != 4) return -1;
    const bool w8 = ht.N > 32, ch = dt.chunk_lo > 0;
    if (ch) {
        const ed::TabView<true> t = ed::tab_view<true>(img.data(), dt);
        return w8 ? run<uint64_t, true>(t, states, n, ht.n_sub, variant, rep, g, nst, cp, own)
                  : run<uint32_t, true>(t, states, n, ht.n_sub, variant, rep, g, nst, cp, own);
    }
    const ed::TabView<false> t = ed::tab_view<false>(img.data(), dt);
    return w8 ? run<uint64_t, false>(t, states, n, ht.n_sub, variant, rep, g, nst, cp, own)
              : run<uint32_t, false>(t, states, n, ht.n_sub, variant, rep, g, nst, cp, own);
}
