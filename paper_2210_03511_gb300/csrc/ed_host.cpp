// Host side of libed: errors, allocation, sector validation, sublattice-coding
// table preparation, term preparation and the C ABI entry points.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "ed_internal.h"
#include "ed_transfer.h"

namespace ed {

static thread_local std::string g_err;

void set_error(ed_status, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

ed_status fail(ed_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

ed_status cuda_fail(cudaError_t e, const char* what) {
    return fail(ED_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* Alloc::get(size_t bytes, cudaStream_t s) const {
    if (bytes == 0) bytes = 16;
    if (custom) return a.alloc(bytes, (ed_stream)s, a.ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Alloc::put(void* p, size_t bytes, cudaStream_t s) const {
    if (!p) return;
    if (custom) a.free(p, bytes, (ed_stream)s, a.ctx);
    else cudaFree(p);
}

// ------------------------------------------------------------------ sector validation + Alg. 1
static std::string elem_key(const int32_t* p, int N, uint8_t f) {
    std::string k((const char*)p, (size_t)N * sizeof(int32_t));
    k.push_back((char)f);
    return k;
}

ed_status build_host_tables(const ed_sector* sec, HostTables& t) {
    if (!sec || !sec->perm || !sec->chi) return fail(ED_ERR_ARG, "sector, perm and chi must be non-null");
    const int N = sec->n_sites, G = sec->n_sym, n_sub = sec->n_sublat;
    if (N < 2 || N > 64) return fail(ED_ERR_ARG, "n_sites=%d out of range [2,64]", N);
    if (sec->n_up < 0 || sec->n_up > N) return fail(ED_ERR_ARG, "n_up=%d out of range", sec->n_up);
    if (G < 1 || G > 65535) return fail(ED_ERR_ARG, "n_sym=%d out of range [1,65535]", G);
    if (n_sub < 1 || N % n_sub) return fail(ED_ERR_ARG, "n_sublat=%d must divide n_sites=%d", n_sub, N);
    const int m = N / n_sub;
    if (m > 16) return fail(ED_ERR_TABLE_TOO_LARGE, "sublattice block of %d sites exceeds 16", m);
    t.N = N; t.n_up = sec->n_up; t.G = G; t.n_sub = n_sub; t.m = m;
    t.perm.assign(sec->perm, sec->perm + (size_t)G * N);
    t.flip.assign(G, 0);
    if (sec->spinflip) for (int g = 0; g < G; ++g) t.flip[g] = sec->spinflip[g] ? 1 : 0;
    t.chi.assign(sec->chi, sec->chi + 2 * (size_t)G);
    // permutations
    for (int g = 0; g < G; ++g) {
        std::vector<char> seen(N, 0);
        for (int i = 0; i < N; ++i) {
            int j = t.perm[(size_t)g * N + i];
            if (j < 0 || j >= N || seen[j]) return fail(ED_ERR_NOT_GROUP, "perm[%d] is not a permutation", g);
            seen[j] = 1;
        }
    }
    for (int i = 0; i < N; ++i)
        if (t.perm[i] != i || t.flip[0]) return fail(ED_ERR_NOT_GROUP, "element 0 is not the identity");
    for (int g = 0; g < G; ++g)
        if (t.flip[g] && 2 * t.n_up != N)
            return fail(ED_ERR_SPINFLIP_SZ, "spin flip needs n_up = N/2 (n_up=%d, N=%d)", t.n_up, N);
    // characters, grouped into classes of equal value (class 0 = the value 1)
    t.chi_cls.assign(G, 0);
    t.real_chars = true;
    {
        double re0 = t.chi[0], im0 = t.chi[1];
        if (fabs(re0 - 1.0) > 1e-9 || fabs(im0) > 1e-9) return fail(ED_ERR_CHAR_NOT_HOMOMORPHISM, "chi(identity) != 1");
    }
    std::vector<std::pair<double, double>> cls_val;
    for (int g = 0; g < G; ++g) {
        double re = t.chi[2 * g], im = t.chi[2 * g + 1];
        if (fabs(re * re + im * im - 1.0) > 1e-9) return fail(ED_ERR_CHAR_NOT_HOMOMORPHISM, "|chi(%d)| != 1", g);
        if (fabs(im) > 1e-12) t.real_chars = false;
        int c = -1;
        for (size_t k = 0; k < cls_val.size(); ++k)
            if (fabs(cls_val[k].first - re) < 1e-9 && fabs(cls_val[k].second - im) < 1e-9) { c = (int)k; break; }
        if (c < 0) { c = (int)cls_val.size(); cls_val.push_back({re, im}); }
        t.chi_cls[g] = (uint16_t)c;
    }
    // closure and homomorphism
    std::unordered_map<std::string, int> index;
    index.reserve((size_t)G * 2);
    for (int g = 0; g < G; ++g) {
        auto r = index.emplace(elem_key(&t.perm[(size_t)g * N], N, t.flip[g]), g);
        if (!r.second) return fail(ED_ERR_NOT_GROUP, "elements %d and %d coincide", r.first->second, g);
    }
    std::vector<int32_t> comp(N);
    for (int a = 0; a < G; ++a) {
        for (int b = 0; b < G; ++b) {
            // (a o b): spin at i moves to perm_b[i], then to perm_a[perm_b[i]]
            for (int i = 0; i < N; ++i) comp[i] = t.perm[(size_t)a * N + t.perm[(size_t)b * N + i]];
            auto it = index.find(elem_key(comp.data(), N, t.flip[a] ^ t.flip[b]));
            if (it == index.end()) return fail(ED_ERR_NOT_GROUP, "product of elements %d and %d is missing", a, b);
            int c = it->second;
            double pr = t.chi[2 * a] * t.chi[2 * b] - t.chi[2 * a + 1] * t.chi[2 * b + 1];
            double pi = t.chi[2 * a] * t.chi[2 * b + 1] + t.chi[2 * a + 1] * t.chi[2 * b];
            if (fabs(pr - t.chi[2 * c]) > 1e-9 || fabs(pi - t.chi[2 * c + 1]) > 1e-9)
                return fail(ED_ERR_CHAR_NOT_HOMOMORPHISM, "chi(%d)chi(%d) != chi(%d)", a, b, c);
        }
    }
    // sublattice stability: destination block of every block
    t.dest.assign((size_t)G * n_sub, 0);
    t.src.assign((size_t)G * n_sub, 0);
    for (int g = 0; g < G; ++g) {
        std::vector<char> hit(n_sub, 0);
        for (int X = 0; X < n_sub; ++X) {
            int Z = t.perm[(size_t)g * N + X * m] / m;
            for (int l = 1; l < m; ++l)
                if (t.perm[(size_t)g * N + X * m + l] / m != Z)
                    return fail(ED_ERR_NOT_SUBLATTICE_STABLE, "element %d splits sublattice %d", g, X);
            t.dest[(size_t)g * n_sub + X] = (uint8_t)Z;
            t.src[(size_t)g * n_sub + Z] = (uint8_t)X;
            hit[Z] = 1;
        }
        for (int Z = 0; Z < n_sub; ++Z)
            if (!hit[Z]) return fail(ED_ERR_NOT_SUBLATTICE_STABLE, "element %d merges sublattices", g);
    }
    // SymmetryAction_X(g, s): image of substate s of block X, read in block dest(g, X)
    const int S = 1 << m;
    t.sa.assign((size_t)G * n_sub * S, 0);
    for (int g = 0; g < G; ++g)
        for (int X = 0; X < n_sub; ++X) {
            const int Z = t.dest[(size_t)g * n_sub + X];
            uint16_t* row = &t.sa[((size_t)g * n_sub + X) * S];
            for (int s = 0; s < S; ++s) {
                uint32_t img = 0;
                for (int l = 0; l < m; ++l) {
                    int bit = (s >> (m - 1 - l)) & 1;
                    if (t.flip[g]) bit ^= 1;
                    if (bit) {
                        int lp = t.perm[(size_t)g * N + X * m + l] - Z * m;
                        img |= 1u << (m - 1 - lp);
                    }
                }
                row[s] = (uint16_t)img;
            }
        }
    // Rep_X and Sym_X over G_X = {g : g maps X onto block 0}
    t.rep.assign((size_t)n_sub * S, 0xFFFF);
    t.sym_off.assign((size_t)n_sub * (S + 1), 0);
    t.sym_ids.clear();
    for (int X = 0; X < n_sub; ++X) {
        for (int s = 0; s < S; ++s) {
            uint32_t best = 0xFFFFFFFFu;
            for (int g = 0; g < G; ++g)
                if (t.dest[(size_t)g * n_sub + X] == 0) best = std::min<uint32_t>(best, t.sa[((size_t)g * n_sub + X) * S + s]);
            t.sym_off[(size_t)X * (S + 1) + s] = (uint32_t)t.sym_ids.size();
            if (best != 0xFFFFFFFFu) {
                t.rep[(size_t)X * S + s] = (uint16_t)best;
                for (int g = 0; g < G; ++g)
                    if (t.dest[(size_t)g * n_sub + X] == 0 && t.sa[((size_t)g * n_sub + X) * S + s] == best)
                        t.sym_ids.push_back((uint16_t)g);
            }
        }
        t.sym_off[(size_t)X * (S + 1) + S] = (uint32_t)t.sym_ids.size();
    }
    // distinct local block maps (positions + flip) and their SymmetryAction tables
    t.chunk_lo = m <= 8 ? 0 : m / 2;
    const int c_lo = t.chunk_lo, c_hi = m - c_lo;
    const int stride = m <= 8 ? S : (1 << c_hi) + (1 << c_lo);
    std::map<std::vector<int>, int> lmap_id;
    t.srclid.assign((size_t)G * n_sub, 0);
    t.lmap_tab.clear();
    for (int g = 0; g < G; ++g)
        for (int X = 0; X < n_sub; ++X) {
            const int Z = t.dest[(size_t)g * n_sub + X];
            std::vector<int> key(m + 1);
            for (int l = 0; l < m; ++l) key[l] = t.perm[(size_t)g * N + X * m + l] - Z * m;
            key[m] = t.flip[g];
            auto it = lmap_id.find(key);
            int id;
            if (it == lmap_id.end()) {
                id = (int)lmap_id.size();
                lmap_id[key] = id;
                // image of a set of local bits (complemented first for a flip element)
                auto img = [&](uint32_t bits, uint32_t within) {
                    uint32_t out = 0;
                    for (int l = 0; l < m; ++l) {
                        if (!((within >> (m - 1 - l)) & 1)) continue;
                        int bit = (bits >> (m - 1 - l)) & 1;
                        if (key[m]) bit ^= 1;
                        if (bit) out |= 1u << (m - 1 - key[l]);
                    }
                    return (uint16_t)out;
                };
                const uint32_t full = (1u << m) - 1;
                if (m <= 8) {
                    for (int s2 = 0; s2 < S; ++s2) t.lmap_tab.push_back(img((uint32_t)s2, full));
                } else {
                    const uint32_t hi_mask = full & ~((1u << c_lo) - 1), lo_mask = (1u << c_lo) - 1;
                    for (int h = 0; h < (1 << c_hi); ++h) t.lmap_tab.push_back(img((uint32_t)h << c_lo, hi_mask));
                    for (int l2 = 0; l2 < (1 << c_lo); ++l2) t.lmap_tab.push_back(img((uint32_t)l2, lo_mask));
                }
            } else {
                id = it->second;
            }
            t.srclid[(size_t)g * n_sub + Z] = (uint32_t)X | ((uint32_t)id << 8);
        }
    t.n_lmap = (int)lmap_id.size();
    (void)stride;
    t.dl.clear();
    t.dl_stride = 0;
    if (t.n_lmap < 4096 && n_sub <= 16) {
        t.dl_stride = (n_sub + 3) & ~3;
        t.dl.assign((size_t)G * t.dl_stride, 0);
        for (int g = 0; g < G; ++g)
            for (int Z = 0; Z < n_sub; ++Z) {
                const uint32_t e = t.srclid[(size_t)g * n_sub + Z];
                const int X = (int)(e & 0xFFu), lid = (int)(e >> 8);
                t.dl[(size_t)g * t.dl_stride + Z] = (uint16_t)((X << 12) | lid);
            }
    }
    t.chi_neg.assign(G, 0);
    for (int g = 0; g < G; ++g) t.chi_neg[g] = t.chi[2 * g] < 0.0 ? 1 : 0;
    return ED_OK;
}

// ------------------------------------------------------------------ terms
static void canon_bond(int i, int j, int& a, int& b) { a = std::min(i, j); b = std::max(i, j); }

// canonical oriented triangle: rotate so the smallest site comes first; if the
// remaining two are descending, store the reversed orientation with sign -1
static void canon_tri(int i, int j, int k, int key[3], int& sign) {
    int v[3] = {i, j, k};
    int r = 0;
    if (v[1] < v[r]) r = 1;
    if (v[2] < v[r]) r = 2;
    int a = v[r], b = v[(r + 1) % 3], c = v[(r + 2) % 3];
    if (b < c) { key[0] = a; key[1] = b; key[2] = c; sign = 1; }
    else { key[0] = a; key[1] = c; key[2] = b; sign = -1; }
}

static bool maps_close(const std::map<std::vector<int>, double>& A, const std::map<std::vector<int>, double>& B) {
    if (A.size() != B.size()) return false;
    auto ia = A.begin();
    auto ib = B.begin();
    for (; ia != A.end(); ++ia, ++ib) {
        if (ia->first != ib->first) return false;
        if (fabs(ia->second - ib->second) > 1e-12 * (1.0 + fabs(ia->second))) return false;
    }
    return true;
}

static ed_status prepare_terms(const ed_basis* b, const ed_terms* tm, ed_hamiltonian* h) {
    const HostTables& t = b->ht;
    const int N = t.N;
    if (tm->n_bonds < 0 || tm->n_tri < 0) return fail(ED_ERR_ARG, "negative term counts");
    if (tm->n_bonds && (!tm->bond || !tm->J)) return fail(ED_ERR_ARG, "bond/J null");
    if (tm->n_tri && (!tm->tri || !tm->Jchi)) return fail(ED_ERR_ARG, "tri/Jchi null");
    std::map<std::vector<int>, double> bonds, tris;
    for (int q = 0; q < tm->n_bonds; ++q) {
        int i = tm->bond[2 * q], j = tm->bond[2 * q + 1];
        if (i < 0 || i >= N || j < 0 || j >= N || i == j) return fail(ED_ERR_ARG, "bad bond %d (%d,%d)", q, i, j);
        int a, c;
        canon_bond(i, j, a, c);
        bonds[{a, c}] += tm->J[q];
    }
    for (int q = 0; q < tm->n_tri; ++q) {
        int i = tm->tri[3 * q], j = tm->tri[3 * q + 1], k = tm->tri[3 * q + 2];
        if (i < 0 || i >= N || j < 0 || j >= N || k < 0 || k >= N || i == j || j == k || i == k)
            return fail(ED_ERR_ARG, "bad triangle %d", q);
        int key[3], sg;
        canon_tri(i, j, k, key, sg);
        tris[{key[0], key[1], key[2]}] += sg * tm->Jchi[q];
    }
    // invariance under every element (spin flip is a pi rotation in spin space:
    // it leaves both S.S and the scalar triple product unchanged)
    for (int g = 0; g < t.G; ++g) {
        const int32_t* p = &t.perm[(size_t)g * N];
        std::map<std::vector<int>, double> b2, t2;
        for (auto& kv : bonds) {
            int a, c;
            canon_bond(p[kv.first[0]], p[kv.first[1]], a, c);
            b2[{a, c}] += kv.second;
        }
        for (auto& kv : tris) {
            int key[3], sg;
            canon_tri(p[kv.first[0]], p[kv.first[1]], p[kv.first[2]], key, sg);
            t2[{key[0], key[1], key[2]}] += sg * kv.second;
        }
        if (!maps_close(bonds, b2) || !maps_close(tris, t2))
            return fail(ED_ERR_NOT_SYMMETRIC, "element %d does not map the terms onto themselves", g);
    }
    // Ising part grouped by coupling
    std::map<double, std::vector<std::pair<int, int>>> cls;
    for (auto& kv : bonds)
        if (kv.second != 0.0) cls[kv.second].push_back({kv.first[0], kv.first[1]});
    h->diag_pos.clear();
    h->diag_cls.clear();
    for (auto& kv : cls) {
        DiagClass d;
        d.J = kv.first;
        d.first = (int)h->diag_pos.size() / 2;
        d.count = (int)kv.second.size();
        for (auto& pr : kv.second) {
            h->diag_pos.push_back((int8_t)(N - 1 - pr.first));
            h->diag_pos.push_back((int8_t)(N - 1 - pr.second));
        }
        h->diag_cls.push_back(d);
    }
    h->n_diag_bonds = (int)h->diag_pos.size() / 2;
    h->n_diag_cls = (int)h->diag_cls.size();
    // flip terms per site pair
    struct Acc {
        double jhalf = 0.0;
        std::vector<std::pair<int, double>> tri;  // (third site, k)
    };
    std::map<std::pair<int, int>, Acc> pairs;
    for (auto& kv : bonds)
        if (kv.second != 0.0) pairs[{kv.first[0], kv.first[1]}].jhalf += 0.5 * kv.second;
    bool cplx_terms = false;
    for (auto& kv : tris) {
        if (kv.second == 0.0) continue;
        cplx_terms = true;
        const int v[3] = {kv.first[0], kv.first[1], kv.first[2]};
        for (int r = 0; r < 3; ++r) {
            int a = v[r], bb = v[(r + 1) % 3], c = v[(r + 2) % 3];
            // S_i.(S_j x S_k) = (i/2) sum_cyclic(a,b,c) S^z_c (S+_a S-_b - S-_a S+_b);
            // stored with the smaller site first: a reversed pair flips the sign
            int lo = std::min(a, bb), hi = std::max(a, bb);
            double k = 0.5 * kv.second * (lo == a ? 1.0 : -1.0);
            pairs[{lo, hi}].tri.push_back({c, k});
        }
    }
    h->flips.clear();
    for (auto& kv : pairs) {
        const Acc& A = kv.second;
        size_t q = 0;
        bool first = true;
        while (first || q < A.tri.size()) {
            FlipTerm f{};
            f.pa = (int8_t)(N - 1 - kv.first.first);
            f.pb = (int8_t)(N - 1 - kv.first.second);
            f.jhalf = first ? A.jhalf : 0.0;
            f.pc0 = f.pc1 = -1;
            if (q < A.tri.size()) { f.pc0 = (int8_t)(N - 1 - A.tri[q].first); f.k0 = A.tri[q].second; ++q; }
            if (q < A.tri.size()) { f.pc1 = (int8_t)(N - 1 - A.tri[q].first); f.k1 = A.tri[q].second; ++q; }
            first = false;
            if (f.jhalf != 0.0 || f.pc0 >= 0) h->flips.push_back(f);
        }
    }
    h->n_flip = (int)h->flips.size();
    h->is_real = t.real_chars && !cplx_terms;
    // coefficient classes by exchange amplitude
    std::vector<double> vals;
    h->jcls.assign(h->n_flip, 0);
    for (int f = 0; f < h->n_flip; ++f) {
        int c = -1;
        for (size_t k = 0; k < vals.size(); ++k)
            if (vals[k] == h->flips[f].jhalf) { c = (int)k; break; }
        if (c < 0) { c = (int)vals.size(); vals.push_back(h->flips[f].jhalf); }
        if (c > 255) return fail(ED_ERR_ARG, "more than 256 distinct couplings");
        h->jcls[f] = (uint8_t)c;
    }
    h->n_jc = (int)vals.size();
    h->jhs.assign((size_t)h->n_jc * (t.G + 1), 0.0);
    for (int c = 0; c < h->n_jc; ++c)
        for (int n = 0; n <= t.G; ++n) h->jhs[(size_t)c * (t.G + 1) + n] = vals[c] * sqrt((double)n);
    return ED_OK;
}

// SU(N) exchange model H = sum_b J_b P_(i_b j_b) (Eq. sunexchangeop): each
// site pair is one non-branching term; P swaps the two sites' colours, so a
// term acts iff the colours differ, with amplitude J, and contributes J to the
// diagonal when they agree.  The flip positions are the lowest bits of the two
// sites' packed colours.
static ed_status prepare_terms_sun(const ed_basis* b, const ed_terms* tm, ed_hamiltonian* h) {
    const int N = b->sun_N, bits = b->sun_b, G = b->ht.G;
    if (tm->n_bonds < 0) return fail(ED_ERR_ARG, "negative term counts");
    if (tm->n_tri) return fail(ED_ERR_ARG, "the SU(N) exchange model takes pair terms only");
    if (tm->n_bonds && (!tm->bond || !tm->J)) return fail(ED_ERR_ARG, "bond/J null");
    std::map<std::vector<int>, double> bonds;
    for (int q = 0; q < tm->n_bonds; ++q) {
        int i = tm->bond[2 * q], j = tm->bond[2 * q + 1];
        if (i < 0 || i >= N || j < 0 || j >= N || i == j) return fail(ED_ERR_ARG, "bad bond %d (%d,%d)", q, i, j);
        int a, c;
        canon_bond(i, j, a, c);
        bonds[{a, c}] += tm->J[q];
    }
    for (int g = 0; g < G; ++g) {
        const int32_t* p = &b->sun_perm[(size_t)g * N];
        std::map<std::vector<int>, double> b2;
        for (auto& kv : bonds) {
            int a, c;
            canon_bond(p[kv.first[0]], p[kv.first[1]], a, c);
            b2[{a, c}] += kv.second;
        }
        if (!maps_close(bonds, b2)) return fail(ED_ERR_NOT_SYMMETRIC, "element %d does not map the terms onto themselves", g);
    }
    h->flips.clear();
    std::vector<double> vals;
    h->jcls.clear();
    for (auto& kv : bonds) {
        if (kv.second == 0.0) continue;
        FlipTerm f{};
        f.pa = (int8_t)((N - 1 - kv.first[0]) * bits);
        f.pb = (int8_t)((N - 1 - kv.first[1]) * bits);
        f.pc0 = f.pc1 = -1;
        f.jhalf = kv.second;  // the amplitude of P_ij
        int c = -1;
        for (size_t k = 0; k < vals.size(); ++k)
            if (vals[k] == kv.second) { c = (int)k; break; }
        if (c < 0) { c = (int)vals.size(); vals.push_back(kv.second); }
        if (c > 255) return fail(ED_ERR_ARG, "more than 256 distinct couplings");
        h->flips.push_back(f);
        h->jcls.push_back((uint8_t)c);
    }
    h->n_flip = (int)h->flips.size();
    h->n_diag_bonds = 0;
    h->n_diag_cls = 0;
    h->diag_pos.clear();
    h->diag_cls.clear();
    h->is_real = b->ht.real_chars;
    h->sun = true;
    h->n_jc = (int)vals.size();
    h->jhs.assign((size_t)h->n_jc * (G + 1), 0.0);
    for (int c = 0; c < h->n_jc; ++c)
        for (int n = 0; n <= G; ++n) h->jhs[(size_t)c * (G + 1) + n] = vals[c] * sqrt((double)n);
    return ED_OK;
}

static ed_status upload_terms(const ed_basis* basis, ed_hamiltonian* h) {
    const Alloc& A = basis->alloc;
    auto up = [&](DevBuf& d, const void* src, size_t bytes) -> bool {
        d.bytes = bytes ? bytes : 16;
        d.p = A.get(d.bytes, 0);
        if (!d.p) return false;
        if (bytes && cudaMemcpy(d.p, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return false;
        return true;
    };
    bool ok = up(h->d_flips, h->flips.data(), h->flips.size() * sizeof(FlipTerm)) &&
              up(h->d_diag_pos, h->diag_pos.data(), h->diag_pos.size()) &&
              up(h->d_diag_cls, h->diag_cls.data(), h->diag_cls.size() * sizeof(DiagClass)) &&
              up(h->d_jhs, h->jhs.data(), h->jhs.size() * sizeof(double)) &&
              up(h->d_jcls, h->jcls.data(), h->jcls.size());
    if (ok) {
        h->d_counters.bytes = 32;
        h->d_counters.p = A.get(32, 0);
        ok = h->d_counters.p && cudaMemset(h->d_counters.p, 0, 32) == cudaSuccess;
    }
    return ok ? ED_OK : fail(ED_ERR_NOMEM, "device allocation for terms failed");
}

}  // namespace ed

using namespace ed;

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* ed_last_error(void) { return g_err.c_str(); }
const char* ed_version(void) { return "libed 0.1 (sm_103a)"; }

ed_status ed_basis_build(const ed_sector* sector, const ed_allocator* alloc, ed_stream stream, ed_basis** out) {
    if (!out) return fail(ED_ERR_ARG, "out is null");
    *out = nullptr;
    ed_basis* b = new ed_basis();
    if (alloc) {
        if (!alloc->alloc || !alloc->free) { delete b; return fail(ED_ERR_ARG, "allocator callbacks null"); }
        b->alloc.a = *alloc;
        b->alloc.custom = true;
    }
    ed_status st = build_host_tables(sector, b->ht);
    if (st == ED_OK) st = basis_build_device(b, (cudaStream_t)stream);
    if (st != ED_OK) {
        ed_basis_free(b);
        return st;
    }
    *out = b;
    return ED_OK;
}

ed_status ed_basis_build_sun(const ed_sector_sun* sector, const ed_allocator* alloc, ed_stream stream,
                             ed_basis** out) {
    if (!out) return fail(ED_ERR_ARG, "out is null");
    *out = nullptr;
    if (!sector || !sector->counts || !sector->perm || !sector->chi) return fail(ED_ERR_ARG, "null argument");
    const int N = sector->n_sites, d = sector->n_colors, G = sector->n_sym;
    if (d < 2 || d > 16) return fail(ED_ERR_ARG, "n_colors=%d out of range [2,16]", d);
    int bits = 1;
    while ((1 << bits) < d) ++bits;
    if (N < 2 || N * bits > 64) return fail(ED_ERR_ARG, "%d sites of %d bits exceed 64 bits", N, bits);
    if (G < 1) return fail(ED_ERR_ARG, "n_sym=%d", G);
    int tot = 0, pop = 0;
    for (int c = 0; c < d; ++c) {
        if (sector->counts[c] < 0) return fail(ED_ERR_ARG, "negative count of colour %d", c);
        tot += sector->counts[c];
        pop += sector->counts[c] * __builtin_popcount((unsigned)c);
    }
    if (tot != N) return fail(ED_ERR_ARG, "colour counts add up to %d, not %d sites", tot, N);
    for (int64_t q = 0; q < (int64_t)G * N; ++q)
        if (sector->perm[q] < 0 || sector->perm[q] >= N) return fail(ED_ERR_NOT_GROUP, "perm entry out of range");
    // the same group acting on bit positions: bit t of site s moves to bit t of site perm[g][s]
    std::vector<int32_t> bperm((size_t)G * N * bits);
    for (int g = 0; g < G; ++g)
        for (int s2 = 0; s2 < N; ++s2)
            for (int t = 0; t < bits; ++t)
                bperm[((size_t)g * N + s2) * bits + t] = sector->perm[(size_t)g * N + s2] * bits + t;
    ed_sector bs{};
    bs.n_sites = N * bits;
    bs.n_up = pop;
    bs.n_sym = G;
    bs.perm = bperm.data();
    bs.spinflip = nullptr;
    bs.chi = sector->chi;
    bs.n_sublat = sector->n_sublat;
    ed_basis* b = new ed_basis();
    if (alloc) {
        if (!alloc->alloc || !alloc->free) { delete b; return fail(ED_ERR_ARG, "allocator callbacks null"); }
        b->alloc.a = *alloc;
        b->alloc.custom = true;
    }
    b->sun_d = d;
    b->sun_b = bits;
    b->sun_N = N;
    b->sun_perm.assign(sector->perm, sector->perm + (size_t)G * N);
    b->sun_counts.assign(sector->counts, sector->counts + d);
    ed_status st = build_host_tables(&bs, b->ht);
    if (st == ED_OK) st = basis_build_device(b, (cudaStream_t)stream);
    if (st != ED_OK) {
        ed_basis_free(b);
        return st;
    }
    *out = b;
    return ED_OK;
}

ed_status ed_hamiltonian_create_sun(const ed_basis* basis, const ed_terms* terms, size_t max_bytes, ed_stream stream,
                                    ed_hamiltonian** out) {
    if (!basis || !terms || !out) return fail(ED_ERR_ARG, "null argument");
    *out = nullptr;
    if (!basis->sun_d) return fail(ED_ERR_ARG, "not an SU(N) basis (ed_basis_build_sun)");
    ed_hamiltonian* h = new ed_hamiltonian();
    h->basis = basis;
    ed_status st = prepare_terms_sun(basis, terms, h);
    if (st == ED_OK) {
        cudaSetDevice(basis->device);
        st = upload_terms(basis, h);
    }
    if (st == ED_OK) st = cache_build(h, h->is_real ? ED_F64 : ED_C128, 0, max_bytes, (cudaStream_t)stream);
    if (st != ED_OK) {
        ed_hamiltonian_free(h);
        return st;
    }
    *out = h;
    return ED_OK;
}

ed_status ed_basis_dim(const ed_basis* b, int64_t* dim) {
    if (!b || !dim) return fail(ED_ERR_ARG, "null argument");
    *dim = b->dim;
    return ED_OK;
}

ed_status ed_basis_export(const ed_basis* b, uint64_t* reps, uint16_t* stab) {
    if (!b) return fail(ED_ERR_ARG, "null basis");
    cudaSetDevice(b->device);
    if (reps) {
        if (b->word == 8) {
            ED_CUDA(cudaMemcpy(reps, b->reps.p, (size_t)b->dim * 8, cudaMemcpyDeviceToHost));
        } else {
            std::vector<uint32_t> tmp((size_t)b->dim);
            ED_CUDA(cudaMemcpy(tmp.data(), b->reps.p, (size_t)b->dim * 4, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < b->dim; ++i) reps[i] = tmp[(size_t)i];
        }
    }
    if (stab) ED_CUDA(cudaMemcpy(stab, b->stab.p, (size_t)b->dim * 2, cudaMemcpyDeviceToHost));
    return ED_OK;
}

ed_status ed_sector_tables(const ed_sector* sector, uint16_t* rep, uint32_t* sym_off, uint16_t* sym_ids,
                           int64_t* n_sym_ids, uint16_t* sa, uint8_t* dest) {
    HostTables t;
    ed_status st = build_host_tables(sector, t);
    if (st != ED_OK) return st;
    if (rep) memcpy(rep, t.rep.data(), t.rep.size() * 2);
    if (sym_off) memcpy(sym_off, t.sym_off.data(), t.sym_off.size() * 4);
    if (sym_ids) memcpy(sym_ids, t.sym_ids.data(), t.sym_ids.size() * 2);
    if (n_sym_ids) *n_sym_ids = (int64_t)t.sym_ids.size();
    if (sa) memcpy(sa, t.sa.data(), t.sa.size() * 2);
    if (dest) memcpy(dest, t.dest.data(), t.dest.size());
    return ED_OK;
}

ed_status ed_representatives(const ed_sector* sector, const uint64_t* states, int64_t n, uint64_t* rep, int32_t* g,
                             int32_t* nstab, uint8_t* compat) {
    if (!sector || (n > 0 && !states) || n < 0) return fail(ED_ERR_ARG, "bad arguments");
    ed_basis tmp;
    ed_status st = build_host_tables(sector, tmp.ht);
    if (st != ED_OK || n == 0) return st;
    ED_CUDA(cudaGetDevice(&tmp.device));
    tmp.word = tmp.ht.N <= 32 ? 4 : 8;
    st = upload_tables(&tmp, 0);
    if (st != ED_OK) return st;
    const size_t per = 8 + 8 + 4 + 4 + 1;
    uint8_t* d = (uint8_t*)tmp.alloc.get((size_t)n * per + 64, 0);
    if (!d) {
        tmp.alloc.put(tmp.tables.p, tmp.tables.bytes, 0);
        return fail(ED_ERR_NOMEM, "scratch for %lld states", (long long)n);
    }
    uint64_t* ds = (uint64_t*)d;
    uint64_t* dr = ds + n;
    int32_t* dg = (int32_t*)(dr + n);
    int32_t* dn = dg + n;
    uint8_t* dc = (uint8_t*)(dn + n);
    const uint64_t mask = tmp.ht.N == 64 ? ~0ull : ((1ull << tmp.ht.N) - 1);
    std::vector<uint64_t> clean(states, states + n);
    for (auto& v : clean) v &= mask;
    if (cudaMemcpy(ds, clean.data(), (size_t)n * 8, cudaMemcpyHostToDevice) != cudaSuccess) st = fail(ED_ERR_CUDA, "copy");
    if (st == ED_OK) st = representatives_device(&tmp, ds, n, dr, dg, dn, dc, 0);
    if (st == ED_OK && cudaDeviceSynchronize() != cudaSuccess) st = fail(ED_ERR_CUDA, "representative kernel failed");
    if (st == ED_OK && rep) cudaMemcpy(rep, dr, (size_t)n * 8, cudaMemcpyDeviceToHost);
    if (st == ED_OK && g) cudaMemcpy(g, dg, (size_t)n * 4, cudaMemcpyDeviceToHost);
    if (st == ED_OK && nstab) cudaMemcpy(nstab, dn, (size_t)n * 4, cudaMemcpyDeviceToHost);
    if (st == ED_OK && compat) cudaMemcpy(compat, dc, (size_t)n, cudaMemcpyDeviceToHost);
    tmp.alloc.put(d, (size_t)n * per + 64, 0);
    tmp.alloc.put(tmp.tables.p, tmp.tables.bytes, 0);
    tmp.tables.p = nullptr;
    return st;
}

ed_status ed_representatives_noalloc(const ed_sector* sector, const uint64_t* states, int64_t n, uint64_t* rep,
                                     int32_t* g, int32_t* nstab, uint8_t* compat, ed_stream stream) {
    return representatives_static(sector, states, n, rep, g, nstab, compat, (cudaStream_t)stream);
}

ed_status ed_restrict(const ed_basis* from, const ed_basis* to, ed_dtype dtype, const void* x, void* y, int32_t nvec,
                      ed_stream stream) {
    if (from && to && (from->sun_d || to->sun_d)) return fail(ED_ERR_ARG, "ed_restrict takes spin-1/2 bases");
    return restrict_vectors(from, to, dtype, x, y, nvec, (cudaStream_t)stream);
}

ed_status ed_apply_sz(const ed_basis* from, const ed_basis* to, const double* c, ed_dtype dtype, const void* x, void* y,
                      int32_t nvec, ed_stream stream) {
    if (from && to && (from->sun_d || to->sun_d)) return fail(ED_ERR_ARG, "ed_apply_sz takes spin-1/2 bases");
    return sz_transfer(from, to, c, dtype, x, y, nvec, (cudaStream_t)stream);
}

void ed_basis_free(ed_basis* b) {
    if (!b) return;
    b->alloc.put(b->reps.p, b->reps.bytes, 0);
    b->alloc.put(b->stab.p, b->stab.bytes, 0);
    b->alloc.put(b->limits.p, b->limits.bytes, 0);
    b->alloc.put(b->tables.p, b->tables.bytes, 0);
    delete b;
}

ed_status ed_hamiltonian_create(const ed_basis* basis, const ed_terms* terms, ed_hamiltonian** out) {
    if (!basis || !terms || !out) return fail(ED_ERR_ARG, "null argument");
    *out = nullptr;
    if (basis->sun_d) return fail(ED_ERR_ARG, "an SU(N) basis takes ed_hamiltonian_create_sun");
    ed_hamiltonian* h = new ed_hamiltonian();
    h->basis = basis;
    ed_status st = prepare_terms(basis, terms, h);
    if (st != ED_OK) { delete h; return st; }
    cudaSetDevice(basis->device);
    st = upload_terms(basis, h);
    if (st != ED_OK) {
        ed_hamiltonian_free(h);
        return st;
    }
    *out = h;
    return ED_OK;
}

ed_status ed_hamiltonian_is_real(const ed_hamiltonian* h, int32_t* is_real) {
    if (!h || !is_real) return fail(ED_ERR_ARG, "null argument");
    *is_real = h->is_real ? 1 : 0;
    return ED_OK;
}

void ed_hamiltonian_free(ed_hamiltonian* h) {
    if (!h) return;
    cache_free(h);
    const Alloc& A = h->basis->alloc;
    A.put(h->d_flips.p, h->d_flips.bytes, 0);
    A.put(h->d_diag_pos.p, h->d_diag_pos.bytes, 0);
    A.put(h->d_diag_cls.p, h->d_diag_cls.bytes, 0);
    A.put(h->d_counters.p, h->d_counters.bytes, 0);
    A.put(h->d_jhs.p, h->d_jhs.bytes, 0);
    A.put(h->d_jcls.p, h->d_jcls.bytes, 0);
    delete h;
}

ed_status ed_apply(const ed_hamiltonian* h, ed_dtype dtype, const void* x, void* y, int32_t nvec, ed_stream stream) {
    if (!h || !x || !y) return fail(ED_ERR_ARG, "null argument");
    if (nvec < 1 || nvec > 8) return fail(ED_ERR_ARG, "nvec=%d out of range [1,8]", nvec);
    if (dtype != ED_F64 && dtype != ED_F32 && dtype != ED_C64 && dtype != ED_C128)
        return fail(ED_ERR_ARG, "unknown dtype %d", (int)dtype);
    if ((dtype == ED_F64 || dtype == ED_F32) && !h->is_real)
        return fail(ED_ERR_ARG, "complex Hamiltonian or characters need a complex dtype");
    return apply_launch(h, dtype, x, y, nvec, (cudaStream_t)stream);
}

ed_status ed_apply_counters(const ed_hamiltonian* h, ed_stream stream, int64_t* gathers, int64_t* skipped) {
    if (!h) return fail(ED_ERR_ARG, "null argument");
    unsigned long long c[3];
    ED_CUDA(cudaMemcpyAsync(c, h->d_counters.p, 24, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    ED_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (gathers) *gathers = (int64_t)c[0];
    if (skipped) *skipped = (int64_t)c[1];
    if (c[2]) return fail(ED_ERR_INDEX_NOT_FOUND, "%llu compatible representatives were missing from the basis", c[2]);
    return ED_OK;
}

ed_status ed_lanczos(const ed_hamiltonian* h, const ed_lanczos_opts* opts, double* evals, void* evecs,
                     ed_lanczos_report* report, ed_stream stream) {
    if (!h || !opts || !evals) return fail(ED_ERR_ARG, "null argument");
    if (opts->n_eig < 1 || opts->n_eig > 8) return fail(ED_ERR_ARG, "n_eig out of range [1,8]");
    if (opts->max_iter < 1 || opts->max_iter > 2000) return fail(ED_ERR_ARG, "max_iter out of range [1,2000]");
    if ((opts->dtype == ED_F64 || opts->dtype == ED_F32) && !h->is_real)
        return fail(ED_ERR_ARG, "complex Hamiltonian or characters need a complex dtype");
    return lanczos_run(h, opts, evals, evecs, report, (cudaStream_t)stream);
}

}  // extern "C"
