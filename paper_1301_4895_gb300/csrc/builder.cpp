// Host term-list builder (runs once per nucleus; no device involvement).
//
// Steps (arXiv:1301.4895):
//   * G^B tensors, eq. def_g, for the nucleon operators of Sec. 7;
//   * their antisymmetric components (Sec. 3 tuples, Sec. 4);
//   * L^(A) by the bullet recursion, eq. recr_L / rec_L_P / rec_L_N, with
//     the product of eq. antis_product_2 and sgn(x|y) of Sec. 3;
//   * the components of interest (all independent spin components, Sec. 4,
//     or listed (sink set, source set) pairs, Sec. 5 / Sec. 8);
//   * backward pruning into the operation lists Lambda^(m) (Sec. 3, Fig. 1,
//     Sec. 4 end): every split of a needed component is one operation;
//   * compaction of every stage to dense indices and z-major op arrays.
//
// Index spaces. A component is a tuple of four sets (Sec. 3): proton spins,
// neutron spins (values < dim), u and d spinor-colour indices (values
// < nxi = 3 * dim: with the nonrelativistic projector only spins 0, 1 occur).
// A stage with set sizes (kp, kn, ku, kd) is enumerated densely by the
// colex ranks of its four sets, proton set slowest and d set fastest; its
// size is the bound P(n_P, n_N) of Sec. 7.

#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <numeric>
#include <stdexcept>
#include <vector>

#include "mbc_internal.h"

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using u32 = uint32_t;
using i64 = int64_t;

i64 binom(int n, int k) {
    if (k < 0 || n < 0 || k > n) return 0;
    i64 r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// multinomial (a+b+c)! / (a! b! c!), zero if any part is negative
i64 multinom3(int a, int b, int c) {
    if (a < 0 || b < 0 || c < 0) return 0;
    return binom(a + b + c, a) * binom(b + c, b);
}

struct Binom {
    i64 c[25][25];
    Binom() {
        for (int n = 0; n < 25; ++n)
            for (int k = 0; k < 25; ++k) c[n][k] = binom(n, k);
    }
};
const Binom &B() {
    static Binom b;
    return b;
}

// colex rank of a set given as a bitmask: sum over its t-th element p of C(p, t+1)
inline i64 colex_rank(u32 m) {
    i64 r = 0;
    int t = 1;
    while (m) {
        int p = __builtin_ctz(m);
        r += B().c[p][t++];
        m &= m - 1;
    }
    return r;
}

inline u32 colex_unrank(i64 r, int k, int n) {
    u32 m = 0;
    for (int t = k; t >= 1; --t) {
        int p = t - 1;
        while (p + 1 < n && B().c[p + 1][t] <= r) ++p;
        r -= B().c[p][t];
        m |= 1u << p;
    }
    return m;
}

// A component key: four sets.
struct Key {
    u32 dp, dn, u, d;
};
inline bool disjoint(const Key &a, const Key &b) {
    return !(a.dp & b.dp) && !(a.dn & b.dn) && !(a.u & b.u) && !(a.d & b.d);
}
inline Key unite(const Key &a, const Key &b) { return {a.dp | b.dp, a.dn | b.dn, a.u | b.u, a.d | b.d}; }
inline Key minus(const Key &a, const Key &b) { return {a.dp & ~b.dp, a.dn & ~b.dn, a.u & ~b.u, a.d & ~b.d}; }

// sgn(x|y) of one index group: (-1)^{#(i in x, j in y, i > j)}  (Sec. 3)
inline int group_parity(u32 x, u32 y) {
    int n = 0;
    while (y) {
        int j = __builtin_ctz(y);
        n += __builtin_popcount(x >> (j + 1));
        y &= y - 1;
    }
    return n & 1;
}
inline int key_sign(const Key &x, const Key &y) {
    int p = group_parity(x.dp, y.dp) ^ group_parity(x.dn, y.dn) ^ group_parity(x.u, y.u) ^ group_parity(x.d, y.d);
    return p ? -1 : 1;
}

// Dense enumeration of a stage with fixed set sizes.
struct Space {
    int dim = 4, nxi = 12;
    int kp = 0, kn = 0, ku = 0, kd = 0;
    i64 np_ = 1, nn_ = 1, nu_ = 1, nd_ = 1;
    void init(int dim_, int nxi_, int kp_, int kn_, int ku_, int kd_) {
        dim = dim_; nxi = nxi_; kp = kp_; kn = kn_; ku = ku_; kd = kd_;
        np_ = binom(dim, kp); nn_ = binom(dim, kn); nu_ = binom(nxi, ku); nd_ = binom(nxi, kd);
    }
    i64 size() const { return np_ * nn_ * nu_ * nd_; }
    i64 index(const Key &k) const {
        return ((colex_rank(k.dp) * nn_ + colex_rank(k.dn)) * nu_ + colex_rank(k.u)) * nd_ + colex_rank(k.d);
    }
    Key key(i64 i) const {
        Key k;
        i64 rd = i % nd_; i /= nd_;
        i64 ru = i % nu_; i /= nu_;
        i64 rn = i % nn_; i /= nn_;
        k.d = colex_unrank(rd, kd, nxi);
        k.u = colex_unrank(ru, ku, nxi);
        k.dn = colex_unrank(rn, kn, dim);
        k.dp = colex_unrank(i, kp, dim);
        return k;
    }
};

// Quark content of the baryons (Sec. 7): proton (u,u,d), neutron (d,u,d).
inline int n_u_of(int b) { return b == MBC_PROTON ? 2 : 1; }
inline int n_d_of(int b) { return b == MBC_PROTON ? 1 : 2; }

// Block component index of y (one baryon): [spin][pair rank][single], where
// for the proton the pair is the u pair and the single the d index, for the
// neutron the pair is the d pair and the single the u index.
inline i64 block_index(const Key &y, int b, int nxi) {
    i64 npair = binom(nxi, 2);
    if (b == MBC_PROTON) {
        int s = __builtin_ctz(y.dp);
        return (s * npair + colex_rank(y.u)) * nxi + __builtin_ctz(y.d);
    }
    int s = __builtin_ctz(y.dn);
    return (s * npair + colex_rank(y.d)) * nxi + __builtin_ctz(y.u);
}

// Enumerate every split z = x + y where y is a component of one baryon of
// type b (Sec. 3): y takes one spin of its species, n_u_of(b) u indices and
// n_d_of(b) d indices out of z. The order is fixed (spin, u choice, d choice).
template <class F>
inline void for_splits(const Key &z, int b, F &&f) {
    u32 ds = b == MBC_PROTON ? z.dp : z.dn;
    int up[24], dq[24];
    int nu = 0, nd = 0;
    for (u32 m = z.u; m; m &= m - 1) up[nu++] = __builtin_ctz(m);
    for (u32 m = z.d; m; m &= m - 1) dq[nd++] = __builtin_ctz(m);
    for (u32 m = ds; m; m &= m - 1) {
        u32 sbit = m & (~m + 1);
        if (b == MBC_PROTON) {
            for (int i = 0; i < nu; ++i)
                for (int j = i + 1; j < nu; ++j)
                    for (int k = 0; k < nd; ++k) {
                        Key y{sbit, 0, (1u << up[i]) | (1u << up[j]), 1u << dq[k]};
                        f(y);
                    }
        } else {
            for (int j = 0; j < nu; ++j)
                for (int i = 0; i < nd; ++i)
                    for (int k = i + 1; k < nd; ++k) {
                        Key y{0, sbit, 1u << up[j], (1u << dq[i]) | (1u << dq[k])};
                        f(y);
                    }
        }
    }
}

// Index spaces larger than this are tracked as sorted index lists instead of
// dense marks (two relativistic quark sources: C(24, 6)^2 quark sets alone).
constexpr i64 kDenseLimit = (i64)1 << 27;

inline int omp_threads() {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
inline int omp_thread() {
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

// ---- Gamma matrices and G (eq. def_g) -------------------------------------

struct SpinEntry {
    int r, c, v;
};

// Gamma_1 (Sec. 1 / Sec. 7): identity (rel) or P_nr = diag(1,1,0,0) (nonrel).
std::vector<SpinEntry> gamma1(int dim) {
    std::vector<SpinEntry> g;
    for (int s = 0; s < dim; ++s) g.push_back({s, s, 1});
    return g;
}
// Gamma_2 = C gamma_5 (Euclidean Dirac representation, C = gamma_2 gamma_4):
// entries (0,1) = -1, (1,0) = +1, (2,3) = -1, (3,2) = +1; the nonrelativistic
// C gamma_5 P_nr keeps the upper-left block only.
std::vector<SpinEntry> gamma2(int dim) {
    std::vector<SpinEntry> g = {{0, 1, -1}, {1, 0, 1}};
    if (dim == 4) {
        g.push_back({2, 3, -1});
        g.push_back({3, 2, 1});
    }
    return g;
}
int levi(int a, int b, int c) {
    if (a == b || b == c || a == c) return 0;
    int inv = (a > b) + (a > c) + (b > c);
    return (inv & 1) ? -1 : 1;
}

// G(alpha; xi1, xi2, xi3) nonzeros for one alpha
struct GEntry {
    int x1, x2, x3, v;
};
std::vector<GEntry> g_entries(int dim, int alpha) {
    std::vector<GEntry> out;
    for (auto &a : gamma1(dim)) {
        if (a.r != alpha) continue;
        for (auto &b : gamma2(dim))
            for (int c1 = 0; c1 < 3; ++c1)
                for (int c2 = 0; c2 < 3; ++c2)
                    for (int c3 = 0; c3 < 3; ++c3) {
                        int e = levi(c1, c2, c3);
                        if (!e) continue;
                        out.push_back({3 * a.c + c1, 3 * b.r + c2, 3 * b.c + c3, a.v * b.v * e});
                    }
    }
    return out;
}

// Antisymmetric components of G_B (Sec. 3-4): sum over the orderings of the
// baryon's same-flavour slots with the sign of the ordering.
struct SparseEntry {
    Key k;
    i64 v;
};
// With ns quark sources (Sec. 6 eq. G_tilde) the source baryon index is
// chi = ns * alpha + s and a quark index xi = ns * kappa + s: G~ is G on
// (alpha; kappa1, kappa2, kappa3) when all three quarks come from source s.
std::vector<SparseEntry> g_minus(int dim, int b, int ns = 1) {
    std::vector<SparseEntry> out;
    for (int chi = 0; chi < dim * ns; ++chi) {
        const int a = chi / ns, src = chi % ns;
        auto ge = g_entries(dim, a);
        for (auto &e : ge) {
            e.x1 = e.x1 * ns + src;
            e.x2 = e.x2 * ns + src;
            e.x3 = e.x3 * ns + src;
        }
        std::vector<SparseEntry> acc;
        for (auto &e : ge) {
            Key k;
            int sign = 1;
            if (b == MBC_PROTON) {  // u at slots 1, 2; d at slot 3
                if (e.x1 == e.x2) continue;
                k = {1u << chi, 0, (1u << e.x1) | (1u << e.x2), 1u << e.x3};
                if (e.x1 > e.x2) sign = -1;
            } else {  // d at slots 1, 3; u at slot 2
                if (e.x1 == e.x3) continue;
                k = {0, 1u << chi, 1u << e.x2, (1u << e.x1) | (1u << e.x3)};
                if (e.x1 > e.x3) sign = -1;
            }
            bool found = false;
            for (auto &c : acc)
                if (c.k.dp == k.dp && c.k.dn == k.dn && c.k.u == k.u && c.k.d == k.d) {
                    c.v += sign * e.v;
                    found = true;
                    break;
                }
            if (!found) acc.push_back({k, (i64)(sign * e.v)});
        }
        for (auto &c : acc)
            if (c.v) out.push_back(c);
    }
    return out;
}

struct StageCounts {
    int kp, kn, ku, kd;
};
StageCounts counts_after(const int8_t *path, int m) {  // stage m (1-based)
    StageCounts c{0, 0, 0, 0};
    for (int i = 0; i < m; ++i) {
        if (path[i] == MBC_PROTON) ++c.kp; else ++c.kn;
        c.ku += n_u_of(path[i]);
        c.kd += n_d_of(path[i]);
    }
    return c;
}

// Sec. 7 bounds: P(n_P, n_N) and Q_P / Q_N for adding baryon b.
// dim: spin (or spin-sink) values of a baryon index, n3: quark index values
// (Sec. 7 with D; Sec. 6 with 4 N_s and 12 N_s)
i64 p_bound(int dim, int np, int nn, int n3) {
    return binom(dim, np) * binom(dim, nn) * binom(n3, 2 * np + nn) * binom(n3, np + 2 * nn);
}
i64 q_bound(int dim, int np, int nn, int b, int n3) {
    int nu = 2 * np + nn, nd = np + 2 * nn;
    if (b == MBC_PROTON)
        return multinom3(np, 1, dim - 1 - np) * multinom3(nn, 0, dim - nn) * multinom3(nu, 2, n3 - 2 - nu) *
               multinom3(nd, 1, n3 - 1 - nd);
    return multinom3(np, 0, dim - np) * multinom3(nn, 1, dim - 1 - nn) * multinom3(nu, 1, n3 - 1 - nu) *
           multinom3(nd, 2, n3 - 2 - nd);
}

double factorial(int n) {
    double f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// One nucleus of a (possibly combined) list: its requested components and the
// terms (projection, sink spins, source spins, weight) that define them.
struct Term {
    int proj;           // output component within the part
    const int8_t *snk, *src;
    double w;
};
struct PartReq {
    int np = 0, nn = 0, A = 0;
    int n_comp = 0;
    std::vector<int8_t> snk, src;  // n_comp * A labels (-1 for projections)
    std::vector<Term> terms;
    bool forbidden = false;
};

// Requested components of one nucleus (Sec. 4 all independent components,
// Sec. 5 / Sec. 8 listed pairs or projections).
void part_requests(const mbc_op_spec *spec, int dim, int dim_src, int nxi, PartReq &R) {
    const int np = spec->n_p, nn = spec->n_n, A = np + nn;
    R.np = np; R.nn = nn; R.A = A;
    auto sets = [&](int k, int n) {
        std::vector<std::vector<int8_t>> out;
        for (i64 r = 0; r < binom(n, k); ++r) {
            u32 m = colex_unrank(r, k, n);
            std::vector<int8_t> v;
            for (int s = 0; s < n; ++s)
                if (m & (1u << s)) v.push_back((int8_t)s);
            out.push_back(v);
        }
        return out;
    };
    R.forbidden = np > std::min(dim, dim_src) || nn > std::min(dim, dim_src) || 2 * np + nn > nxi ||
                  np + 2 * nn > nxi;
    if (spec->spin_mode == MBC_SPIN_ALL) {
        std::vector<std::vector<int8_t>> snk_comps, src_comps;
        if (!R.forbidden) {
            for (auto &p : sets(np, dim))
                for (auto &n : sets(nn, dim)) {
                    std::vector<int8_t> v = p;
                    v.insert(v.end(), n.begin(), n.end());
                    snk_comps.push_back(v);
                }
            for (auto &p : sets(np, dim_src))
                for (auto &n : sets(nn, dim_src)) {
                    std::vector<int8_t> v = p;
                    v.insert(v.end(), n.begin(), n.end());
                    src_comps.push_back(v);
                }
        }
        for (auto &a : snk_comps)
            for (auto &b : src_comps) {
                R.snk.insert(R.snk.end(), a.begin(), a.end());
                R.src.insert(R.src.end(), b.begin(), b.end());
            }
        R.n_comp = (int)(snk_comps.size() * src_comps.size());
    } else if (spec->spin_mode == MBC_SPIN_LISTED) {
        R.n_comp = spec->n_spin_sel;
        R.snk.assign(spec->snk_spins, spec->snk_spins + (size_t)A * spec->n_spin_sel);
        R.src.assign(spec->src_spins, spec->src_spins + (size_t)A * spec->n_spin_sel);
    } else {  // MBC_SPIN_PROJECTED: one output per projection; labels are not single spin tuples
        R.n_comp = spec->n_proj;
        R.snk.assign((size_t)A * spec->n_proj, (int8_t)-1);
        R.src.assign((size_t)A * spec->n_proj, (int8_t)-1);
    }
    if (spec->spin_mode == MBC_SPIN_PROJECTED) {
        for (int t = 0; t < spec->n_spin_sel; ++t)
            R.terms.push_back({spec->term_proj[t], spec->snk_spins + (size_t)A * t, spec->src_spins + (size_t)A * t,
                               spec->term_coef[t]});
    } else {
        for (int c = 0; c < R.n_comp; ++c)
            R.terms.push_back({c, R.snk.data() + (size_t)A * c, R.src.data() + (size_t)A * c, 1.0});
    }
}

// Build a term list for n nuclei that lie on one path (Sec. 7: smaller
// nuclei on the path of the largest one reuse its stages). specs[0..n) share
// dirac_dim, n_sources and n_sinks; the largest nucleus fixes the path and
// every other one must be the nucleus of a prefix of it. With n = 1 this is
// the list of one nucleus.
mbc_status build(const mbc_op_spec *specs, int n_specs, mbc_term_list *L) {
    int big = 0;
    for (int j = 1; j < n_specs; ++j)
        if (specs[j].n_p + specs[j].n_n > specs[big].n_p + specs[big].n_n) big = j;
    const mbc_op_spec *spec = &specs[big];
    const int np = spec->n_p, nn = spec->n_n, A = np + nn, D = spec->dirac_dim;
    bool list_free = false;
    for (int j = 0; j < n_specs; ++j) list_free = list_free || specs[j].list_free != 0;
    const int ns = std::max(1, spec->n_sources), nk = std::max(1, spec->n_sinks);
    const int dim = D * nk;        // sink baryon index: spin x sink function (Sec. 6 psi)
    const int dim_src = D * ns;    // source baryon index: spin x source (Sec. 6 chi)
    const int nxi = 3 * D * ns;    // quark index: spinor-colour x source
    L->A = A; L->n_p = np; L->n_n = nn; L->dim = D; L->n_sources = ns; L->n_sinks = nk; L->nxi = nxi;
    L->dim_snk = dim; L->dim_src = dim_src;
    L->block_size = (i64)dim * binom(nxi, 2) * nxi;
    L->norm = factorial(np) * factorial(nn);
    L->norm *= L->norm;
    if (spec->path) {
        for (int i = 0; i < A; ++i) L->path[i] = spec->path[i];
    } else {
        int first = np > nn ? MBC_PROTON : MBC_NEUTRON;  // Sec. 7 rule, ties: neutrons first
        int nf = first == MBC_PROTON ? np : nn;
        for (int i = 0; i < A; ++i) L->path[i] = (int8_t)(i < nf ? first : 1 - first);
    }
    for (int i = 0; i < A; ++i) L->need_block[L->path[i]] = true;

    // every nucleus must be a prefix of the path, with the same operators
    std::vector<PartReq> parts((size_t)n_specs);
    for (int j = 0; j < n_specs; ++j) {
        const mbc_op_spec &s = specs[j];
        const int Aj = s.n_p + s.n_n;
        if (s.dirac_dim != D || std::max(1, s.n_sources) != ns || std::max(1, s.n_sinks) != nk)
            return MBC_ERR_INVALID_ARG;
        auto c = counts_after(L->path, Aj);
        if (c.kp != s.n_p || c.kn != s.n_n) return MBC_ERR_INVALID_ARG;  // not on the path
        if (s.path)
            for (int i = 0; i < Aj; ++i)
                if (s.path[i] != L->path[i]) return MBC_ERR_INVALID_ARG;
        part_requests(&s, dim, dim_src, nxi, parts[(size_t)j]);
    }
    bool forbidden = false;
    int n_comp = 0;
    for (auto &R : parts) {
        forbidden = forbidden || R.forbidden;
        n_comp += R.n_comp;
    }
    L->n_comp = n_comp;
    L->parts.clear();
    {
        int c0 = 0;
        for (auto &R : parts) {
            double nrm = factorial(R.np) * factorial(R.nn);
            L->parts.push_back({R.np, R.nn, R.A, c0, c0 + R.n_comp, nrm * nrm});
            c0 += R.n_comp;
            // labels padded to A entries per component
            for (int c = 0; c < R.n_comp; ++c) {
                for (int i = 0; i < A; ++i) {
                    L->comp_snk.push_back(i < R.A ? R.snk[(size_t)c * R.A + i] : (int8_t)-1);
                    L->comp_src.push_back(i < R.A ? R.src[(size_t)c * R.A + i] : (int8_t)-1);
                }
            }
        }
    }
    L->fin_off.assign((size_t)L->n_comp + 1, 0);
    // a spin tuple of one species -> (set bitmask, sign of the sorting
    // permutation); repeated or out-of-range spins give the Pauli zero (Sec. 3)
    auto spin_set = [&](const int8_t *s, int off, int n, int range, u32 &mask, int &sign) {
        mask = 0;
        int inv = 0;
        for (int i = 0; i < n; ++i) {
            const int v = s[off + i];
            if (v < 0 || v >= range || (mask & (1u << v))) return false;
            for (int j = 0; j < i; ++j) inv += s[off + j] > v;
            mask |= 1u << v;
        }
        sign = (inv & 1) ? -1 : 1;
        return true;
    };

    mbc_list_stats &st = L->stats;
    std::memset(&st, 0, sizeof(st));
    st.A = A; st.n_steps = A - 1;
    for (int i = 0; i < A; ++i) st.path[i] = L->path[i];
    st.block_size = L->block_size;
    st.n_comp = L->n_comp;
    st.norm = L->norm;
    st.n_parts = n_specs;
    for (int m = 1; m <= A; ++m) {
        auto c = counts_after(L->path, m);
        st.stage_bound[m - 1] = p_bound(dim, c.kp, c.kn, nxi);
        if (m < A) st.q_bound[m - 1] = q_bound(dim, c.kp, c.kn, L->path[m], nxi);
    }
    if (forbidden) {
        if (n_specs > 1) return MBC_ERR_INVALID_ARG;  // a combined path through a forbidden nucleus
        L->pauli_forbidden = true;
        return MBC_ERR_PAULI_FORBIDDEN;
    }
    std::vector<bool> stage_wanted((size_t)A + 1, false);
    for (auto &R : parts) stage_wanted[(size_t)R.A] = true;

    // ---- L^(m) by the bullet recursion (eq. recr_L), kept where a nucleus ends
    std::vector<std::vector<SparseEntry>> Lm((size_t)A + 1);
    std::vector<SparseEntry> gm[2] = {g_minus(D, MBC_PROTON, ns), g_minus(D, MBC_NEUTRON, ns)};
    std::vector<SparseEntry> cur = gm[L->path[0]];
    if (stage_wanted[1]) Lm[1] = cur;
    for (int m = 1; m < A; ++m) {
        int b = L->path[m];
        auto c = counts_after(L->path, m + 1);
        Space sp;
        sp.init(dim_src, nxi, c.kp, c.kn, c.ku, c.kd);  // L lives on source-side baryon indices
        const auto &g = gm[b];
        if (sp.size() > kDenseLimit) {
            // index space too large for dense marks (two relativistic sources):
            // products collected per thread, sorted by index, equal keys added
            std::vector<std::vector<std::pair<i64, i64>>> parts_t((size_t)omp_threads());
#pragma omp parallel for schedule(dynamic, 64)
            for (i64 i = 0; i < (i64)cur.size(); ++i) {
                auto &out = parts_t[(size_t)omp_thread()];
                for (auto &y : g)
                    if (disjoint(cur[i].k, y.k))
                        out.push_back({sp.index(unite(cur[i].k, y.k)), cur[i].v * y.v * key_sign(cur[i].k, y.k)});
            }
            std::vector<std::pair<i64, i64>> all;
            for (auto &v : parts_t) {
                all.insert(all.end(), v.begin(), v.end());
                std::vector<std::pair<i64, i64>>().swap(v);
            }
            std::sort(all.begin(), all.end(), [](const std::pair<i64, i64> &a, const std::pair<i64, i64> &b2) {
                return a.first < b2.first;
            });
            std::vector<SparseEntry> nxt;
            for (size_t i = 0; i < all.size();) {
                size_t j = i;
                i64 v = 0;
                while (j < all.size() && all[j].first == all[i].first) v += all[j++].second;
                if (v) nxt.push_back({sp.key(all[i].first), v});
                i = j;
            }
            cur.swap(nxt);
            if (stage_wanted[(size_t)m + 1]) Lm[(size_t)m + 1] = cur;
            continue;
        }
        std::vector<std::atomic<i64>> dense((size_t)sp.size());
        for (auto &d : dense) d.store(0, std::memory_order_relaxed);
#pragma omp parallel for schedule(dynamic, 256)
        for (i64 i = 0; i < (i64)cur.size(); ++i)
            for (auto &y : g)
                if (disjoint(cur[i].k, y.k)) {
                    Key z = unite(cur[i].k, y.k);
                    dense[(size_t)sp.index(z)].fetch_add(cur[i].v * y.v * key_sign(cur[i].k, y.k),
                                                         std::memory_order_relaxed);
                }
        std::vector<SparseEntry> nxt;
        for (i64 i = 0; i < sp.size(); ++i) {
            i64 v = dense[(size_t)i].load(std::memory_order_relaxed);
            if (v) nxt.push_back({sp.key(i), v});
        }
        cur.swap(nxt);
        if (stage_wanted[(size_t)m + 1]) Lm[(size_t)m + 1] = cur;
    }
    // Lm[m]: nonzero L^(m) entries, in dense-index order of the stage-m space

    // ---- components of interest and the needed set of every stage ----------
    std::vector<Space> spaces((size_t)A + 1);
    for (int m = 1; m <= A; ++m) {
        auto c = counts_after(L->path, m);
        spaces[(size_t)m].init(dim, nxi, c.kp, c.kn, c.ku, c.kd);
    }
    // needed components per stage: dense marks, or for index spaces beyond
    // kDenseLimit a list of full indices (sorted and made unique when read)
    std::vector<bool> sparse((size_t)A + 1, false);
    for (int m = 1; m <= A; ++m) sparse[(size_t)m] = spaces[(size_t)m].size() > kDenseLimit;
    if (list_free)
        for (int m = 1; m <= A; ++m)
            if (sparse[(size_t)m]) return MBC_ERR_UNSUPPORTED;  // list-free steps rank dense spaces
    std::vector<std::vector<uint8_t>> need((size_t)A + 1);  // dense marks, allocated when first used
    std::vector<std::vector<i64>> need_sp((size_t)A + 1);
    for (int m = 1; m <= A; ++m)
        if (stage_wanted[(size_t)m] && !sparse[(size_t)m]) need[(size_t)m].assign((size_t)spaces[(size_t)m].size(), 0);
    struct FinEntry {
        i64 zfull;
        double l;
    };
    // modified list of each output (Sec. 5): L_M(sink set; U, D) = sum over the
    // output's terms of weight * sign(sink order) * sign(source order) * L(source set; U, D)
    std::vector<std::vector<FinEntry>> fin((size_t)L->n_comp);
    for (size_t j = 0; j < parts.size(); ++j) {
        const PartReq &R = parts[j];
        const int c0 = L->parts[j].c0;
        const Space &spA = spaces[(size_t)R.A];
        for (const Term &tm : R.terms) {
            u32 sp_, sn_, ap_, an_;
            int g1, g2, g3, g4;
            if (!spin_set(tm.snk, 0, R.np, dim, sp_, g1) || !spin_set(tm.snk, R.np, R.nn, dim, sn_, g2) ||
                !spin_set(tm.src, 0, R.np, dim_src, ap_, g3) || !spin_set(tm.src, R.np, R.nn, dim_src, an_, g4))
                continue;  // a repeated or out-of-range spin: Pauli zero term
            const double w = tm.w * g1 * g2 * g3 * g4;
            for (auto &e : Lm[(size_t)R.A]) {
                if (e.k.dp != ap_ || e.k.dn != an_) continue;
                Key z{sp_, sn_, e.k.u, e.k.d};
                fin[(size_t)(c0 + tm.proj)].push_back({spA.index(z), w * (double)e.v});
            }
        }
        for (int c = c0; c < c0 + R.n_comp; ++c) {  // add equal keys, drop exact cancellations
            auto &v = fin[(size_t)c];
            std::sort(v.begin(), v.end(), [](const FinEntry &a, const FinEntry &b) { return a.zfull < b.zfull; });
            size_t w = 0;
            for (size_t i = 0; i < v.size();) {
                size_t k = i;
                double sum = 0.0;
                while (k < v.size() && v[k].zfull == v[i].zfull) sum += v[k++].l;
                if (sum != 0.0) v[w++] = {v[i].zfull, sum};
                i = k;
            }
            v.resize(w);
            for (auto &e : v) {
                if (sparse[(size_t)R.A])
                    need_sp[(size_t)R.A].push_back(e.zfull);
                else
                    need[(size_t)R.A][(size_t)e.zfull] = 1;
            }
        }
    }
    Lm.clear();

    // ---- backward pruning (Sec. 3): stage m needs every x of every split of
    // the needed components of stage m + 1, plus its own nuclei's components
    std::vector<std::vector<i64>> members((size_t)A + 1);  // needed full indices, ascending
    std::vector<std::vector<int32_t>> compact((size_t)A + 1);
    for (int m = A; m >= 1; --m) {
        auto &mem = members[(size_t)m];
        if (sparse[(size_t)m]) {
            mem.swap(need_sp[(size_t)m]);
            std::sort(mem.begin(), mem.end());
            mem.erase(std::unique(mem.begin(), mem.end()), mem.end());
        } else {
            auto &nd = need[(size_t)m];
            for (i64 i = 0; i < (i64)nd.size(); ++i)
                if (nd[(size_t)i]) mem.push_back(i);
            std::vector<uint8_t>().swap(nd);
        }
        if (m == 1) break;
        const Space &sz = spaces[(size_t)m], &sx = spaces[(size_t)m - 1];
        int b = L->path[m - 1];
        if (sparse[(size_t)m - 1]) {
            std::vector<std::vector<i64>> parts_t((size_t)omp_threads());
#pragma omp parallel for schedule(dynamic, 256)
            for (i64 i = 0; i < (i64)mem.size(); ++i) {
                auto &out = parts_t[(size_t)omp_thread()];
                Key z = sz.key(mem[(size_t)i]);
                for_splits(z, b, [&](const Key &y) { out.push_back(sx.index(minus(z, y))); });
            }
            auto &nx = need_sp[(size_t)m - 1];
            for (auto &v : parts_t) nx.insert(nx.end(), v.begin(), v.end());
            continue;
        }
        auto &nx = need[(size_t)m - 1];
        if (nx.empty()) nx.assign((size_t)sx.size(), 0);
#pragma omp parallel for schedule(dynamic, 256)
        for (i64 i = 0; i < (i64)mem.size(); ++i) {
            Key z = sz.key(mem[(size_t)i]);
            for_splits(z, b, [&](const Key &y) {
                __atomic_store_n(&nx[(size_t)sx.index(minus(z, y))], (uint8_t)1, __ATOMIC_RELAXED);
            });
        }
    }
    for (int m = 1; m <= A; ++m) st.stage_size[m - 1] = (i64)members[(size_t)m].size();

    // compact index of every needed component; stage 1 uses block indices.
    // Sparse stages keep no map: the compact index is the position in the
    // sorted member list.
    auto compact_index = [&](int m, i64 full) -> i64 {
        if (!sparse[(size_t)m]) return (i64)compact[(size_t)m][(size_t)full];
        const auto &mem = members[(size_t)m];
        auto it = std::lower_bound(mem.begin(), mem.end(), full);
        return (it != mem.end() && *it == full) ? (i64)(it - mem.begin()) : -1;
    };
    for (int m = 2; m <= A; ++m) {
        if (sparse[(size_t)m]) continue;
        auto &cm = compact[(size_t)m];
        cm.assign((size_t)spaces[(size_t)m].size(), -1);
        auto &mem = members[(size_t)m];
        for (i64 i = 0; i < (i64)mem.size(); ++i) cm[(size_t)mem[(size_t)i]] = (int32_t)i;
    }

    // ---- operation lists (z-major) -----------------------------------------
    L->steps.resize((size_t)A - 1);
    for (int m = 1; m < A; ++m) {
        mbc::Step &s = L->steps[(size_t)m - 1];
        int b = L->path[m];
        s.baryon = b;
        const Space &sz = spaces[(size_t)m + 1], &sx = spaces[(size_t)m];
        auto &mem = members[(size_t)m + 1];
        s.n_z = (i64)mem.size();
        s.n_x = m == 1 ? L->block_size : (i64)members[(size_t)m].size();
        i64 k = 0;
        if (s.n_z) for_splits(sz.key(mem[0]), b, [&](const Key &) { ++k; });
        s.k = k;
        st.ops_per_z[m - 1] = k;
        st.n_ops[m - 1] = k * s.n_z;
        st.n_ops_total += k * s.n_z;
        s.dense = s.n_z == sz.size() && (m == 1 || (i64)members[(size_t)m].size() == sx.size());
        if (s.dense) st.dense_mask |= 1u << (m - 1);
        s.zk[0] = sz.kp; s.zk[1] = sz.kn; s.zk[2] = sz.ku; s.zk[3] = sz.kd;
        s.xk[0] = sx.kp; s.xk[1] = sx.kn; s.xk[2] = sx.ku; s.xk[3] = sx.kd;
        if (list_free) {
            // splits regenerated from the output key on the device; two index
            // tables stand in for the op arrays where a stage is not dense
            s.generated = true;
            if (s.n_z != sz.size()) s.zrank.assign(mem.begin(), mem.end());
            if (m > 1 && (i64)members[(size_t)m].size() != sx.size()) s.xmap = compact[(size_t)m];
            st.op_bytes += (i64)(s.zrank.size() * sizeof(int64_t) + s.xmap.size() * sizeof(int32_t));
            continue;
        }
        st.op_bytes += k * s.n_z * (i64)(sizeof(uint32_t) + sizeof(uint16_t));
        s.x.resize((size_t)(k * s.n_z));
        s.ys.resize((size_t)(k * s.n_z));
        int bprev = L->path[0];
        std::atomic<bool> bad{false};
#pragma omp parallel for schedule(dynamic, 256)
        for (i64 i = 0; i < s.n_z; ++i) {
            Key z = sz.key(mem[(size_t)i]);
            i64 j = 0;
            for_splits(z, b, [&](const Key &y) {
                Key x = minus(z, y);
                i64 xi = m == 1 ? block_index(x, bprev, nxi) : compact_index(m, sx.index(x));
                if (xi < 0 || j >= k) {
                    bad = true;
                    return;
                }
                size_t o = (size_t)(i * k + j);
                s.x[o] = (uint32_t)xi;
                s.ys[o] = (uint16_t)(block_index(y, b, nxi) | (key_sign(x, y) < 0 ? 0x8000u : 0u));
                ++j;
            });
            if (j != k) bad = true;
        }
        if (bad) return MBC_ERR_INVALID_ARG;
    }

    // ---- contraction lists (eq. C_final), each at its nucleus' stage -------
    L->final_size = A == 1 ? L->block_size : (i64)members[(size_t)A].size();
    for (size_t j = 0; j < parts.size(); ++j) {
        const mbc_term_list::Part &pt = L->parts[j];
        const int Aj = pt.A;
        for (int c = pt.c0; c < pt.c1; ++c) {
            for (auto &e : fin[(size_t)c]) {
                i64 zi = Aj == 1 ? block_index(spaces[1].key(e.zfull), L->path[0], nxi) : compact_index(Aj, e.zfull);
                L->fin_z.push_back((uint32_t)zi);
                L->fin_l.push_back(e.l);
            }
            L->fin_off[(size_t)c + 1] = (i64)L->fin_z.size();
        }
    }
    st.n_l_total = (i64)L->fin_z.size();
    return MBC_OK;
}

}  // namespace

extern "C" {

const char *mbc_status_string(mbc_status s) {
    switch (s) {
        case MBC_OK: return "MBC_OK";
        case MBC_ERR_INVALID_ARG: return "MBC_ERR_INVALID_ARG";
        case MBC_ERR_PAULI_FORBIDDEN: return "MBC_ERR_PAULI_FORBIDDEN";
        case MBC_ERR_OOM: return "MBC_ERR_OOM";
        case MBC_ERR_CUDA: return "MBC_ERR_CUDA";
        case MBC_ERR_TIMEOUT: return "MBC_ERR_TIMEOUT";
        case MBC_ERR_UNSUPPORTED: return "MBC_ERR_UNSUPPORTED";
    }
    return "MBC_ERR_UNKNOWN";
}

}  // extern "C"

namespace {

// Argument checks of one spec (no allocation).
mbc_status check_spec(const mbc_op_spec *spec) {
    const int A = spec->n_p + spec->n_n;
    if (spec->n_p < 0 || spec->n_n < 0 || A < 1 || A > MBC_MAX_A) return MBC_ERR_INVALID_ARG;
    if (spec->dirac_dim != 2 && spec->dirac_dim != 4) return MBC_ERR_INVALID_ARG;
    // quark indices (3 dirac_dim n_sources values) must fit the 24-value index tables
    if (spec->n_sources < 1 || 3 * spec->dirac_dim * spec->n_sources > 24) return MBC_ERR_UNSUPPORTED;
    if (spec->n_sinks < 0 || spec->dirac_dim * std::max(1, spec->n_sinks) > 16) return MBC_ERR_UNSUPPORTED;
    if (spec->spin_mode != MBC_SPIN_ALL && spec->spin_mode != MBC_SPIN_LISTED && spec->spin_mode != MBC_SPIN_PROJECTED)
        return MBC_ERR_INVALID_ARG;
    if (spec->spin_mode == MBC_SPIN_PROJECTED) {
        if (spec->n_proj < 1 || spec->n_spin_sel < 1 || !spec->snk_spins || !spec->src_spins || !spec->term_proj ||
            !spec->term_coef)
            return MBC_ERR_INVALID_ARG;
        for (int t = 0; t < spec->n_spin_sel; ++t)
            if (spec->term_proj[t] < 0 || spec->term_proj[t] >= spec->n_proj) return MBC_ERR_INVALID_ARG;
    }
    if (spec->spin_mode == MBC_SPIN_LISTED &&
        (spec->n_spin_sel < 1 || !spec->snk_spins || !spec->src_spins))
        return MBC_ERR_INVALID_ARG;
    if (spec->path) {
        if (spec->path_len != A) return MBC_ERR_INVALID_ARG;
        int cp = 0;
        for (int i = 0; i < A; ++i) {
            if (spec->path[i] != MBC_PROTON && spec->path[i] != MBC_NEUTRON) return MBC_ERR_INVALID_ARG;
            cp += spec->path[i] == MBC_PROTON;
        }
        if (cp != spec->n_p) return MBC_ERR_INVALID_ARG;
    }
    return MBC_OK;
}

mbc_status build_checked(const mbc_op_spec *specs, int32_t n_specs, mbc_term_list **out) {
    if (!out) return MBC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!specs || n_specs < 1 || n_specs > 64) return MBC_ERR_INVALID_ARG;
    for (int j = 0; j < n_specs; ++j) {
        mbc_status cs = check_spec(&specs[j]);
        if (cs != MBC_OK) return cs;
    }
    mbc_term_list *L = new (std::nothrow) mbc_term_list();
    if (!L) return MBC_ERR_OOM;
    mbc_status s;
    try {
        s = build(specs, n_specs, L);
    } catch (const std::bad_alloc &) {
        s = MBC_ERR_OOM;
    } catch (...) {
        s = MBC_ERR_INVALID_ARG;
    }
    if (s == MBC_OK || s == MBC_ERR_PAULI_FORBIDDEN) {
        *out = L;
    } else {
        delete L;
    }
    return s;
}

}  // namespace

extern "C" {

mbc_status mbc_build_term_list(const mbc_op_spec *spec, mbc_term_list **out) {
    return build_checked(spec, 1, out);
}

mbc_status mbc_build_combined(const mbc_op_spec *specs, int32_t n_specs, mbc_term_list **out) {
    return build_checked(specs, n_specs, out);
}

mbc_status mbc_term_list_part(const mbc_term_list *list, int32_t j, mbc_list_part *part) {
    if (!list || !part || j < 0 || j >= (int32_t)list->parts.size()) return MBC_ERR_INVALID_ARG;
    const auto &p = list->parts[(size_t)j];
    part->n_p = p.n_p;
    part->n_n = p.n_n;
    part->c0 = p.c0;
    part->c1 = p.c1;
    return MBC_OK;
}

mbc_status mbc_term_list_stats(const mbc_term_list *list, mbc_list_stats *st) {
    if (!list || !st) return MBC_ERR_INVALID_ARG;
    *st = list->stats;
    return MBC_OK;
}

mbc_status mbc_term_list_components(const mbc_term_list *list, int8_t *snk, int8_t *src) {
    if (!list || (!snk && !src)) return MBC_ERR_INVALID_ARG;
    if (snk) std::copy(list->comp_snk.begin(), list->comp_snk.end(), snk);
    if (src) std::copy(list->comp_src.begin(), list->comp_src.end(), src);
    return MBC_OK;
}

int64_t mbc_term_list_n_l(const mbc_term_list *list, int32_t c) {
    if (!list || c < 0 || c >= list->n_comp || list->fin_off.empty()) return 0;
    return list->fin_off[(size_t)c + 1] - list->fin_off[(size_t)c];
}

void mbc_free_term_list(mbc_term_list *list) {
    if (!list) return;
    mbc::free_device_cache(list);
    delete list;
}

const char *mbc_version(void) { return "mbc 0.1 (sm_103a)"; }

}  // extern "C"
