// Host check of the list-free split generator: every operation that
// gen_ops.cuh regenerates from an output key is compared with the stored
// operation arrays of the same list built by the host builder, and every
// input index is checked against its stage. The device functions are compiled
// for the host with plain C++ stand-ins for the CUDA intrinsics they use.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#define __device__
#define __forceinline__ inline
#define __constant__
static inline int __ffs(uint32_t x) { return __builtin_ffs((int)x); }
static inline int __popc(uint32_t x) { return __builtin_popcount(x); }
template <class T>
static inline T __ldg(const T *p) { return *p; }

#include "../../paper_1301_4895_gb300/csrc/builder.cpp"
#include "../../paper_1301_4895_gb300/csrc/gen_ops.cuh"

namespace mbc {
void free_device_cache(mbc_term_list *) {}
}  // namespace mbc

static int64_t bn(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// returns the number of mismatching or out-of-range operations (-1: build failed)
static int64_t check(int np, int nn, int D, const int8_t *snk, const int8_t *src, int nsel, int ns, int nk) {
    mbc_op_spec sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.n_p = np;
    sp.n_n = nn;
    sp.dirac_dim = D;
    sp.n_sources = ns;
    sp.n_sinks = nk;
    sp.spin_mode = nsel ? MBC_SPIN_LISTED : MBC_SPIN_ALL;
    sp.n_spin_sel = nsel;
    sp.snk_spins = snk;
    sp.src_spins = src;
    mbc_term_list *L = nullptr, *F = nullptr;
    if (mbc_build_term_list(&sp, &L) != MBC_OK) return -1;
    sp.list_free = 1;
    if (mbc_build_term_list(&sp, &F) != MBC_OK) return -1;
    for (int n = 0; n < 25; ++n)
        for (int k = 0; k < 25; ++k) mbc::c_binom[n][k] = (uint32_t)bn(n, k);
    int64_t bad = 0, tot = 0;
    for (size_t m = 0; m < F->steps.size(); ++m) {
        const auto &s = F->steps[m], &r = L->steps[m];
        mbc::GenStep g;
        std::memset(&g, 0, sizeof(g));
        g.b = s.baryon;
        g.bprev = F->path[0];
        g.x_block = m == 0;
        g.nxi = F->nxi;
        g.npair = (int)bn(F->nxi, 2);
        g.dim = F->dim_snk;
        for (int i = 0; i < 4; ++i) {
            g.zk[i] = s.zk[i];
            g.xk[i] = s.xk[i];
            const int n = i < 2 ? F->dim_snk : F->nxi;
            g.zr[i] = bn(n, s.zk[i]);
            g.xr[i] = bn(n, s.xk[i]);
        }
        g.zrank = s.zrank.empty() ? nullptr : s.zrank.data();
        g.xmap = s.xmap.empty() ? nullptr : s.xmap.data();
        for (int64_t z = 0; z < s.n_z; ++z) {
            uint32_t key[4];
            mbc::g_key(g, z, key);
            for (int64_t j = 0; j < s.k; ++j) {
                uint32_t ox, oy;
                mbc::g_op(g, key, j, ox, oy);
                ++tot;
                const size_t o = (size_t)(z * s.k + j);
                if ((int64_t)ox >= s.n_x || ox != r.x[o] || oy != r.ys[o]) ++bad;
            }
        }
    }
    std::printf("(%d,%d) D=%d sources %d sinks %d: %lld operations, %lld mismatches\n", np, nn, D, ns, nk,
                (long long)tot, (long long)bad);
    mbc_free_term_list(L);
    mbc_free_term_list(F);
    return bad;
}

int main() {
    int64_t bad = 0;
    auto add = [&](int64_t b) { bad += b < 0 ? 1 : b; };
    add(check(1, 1, 2, nullptr, nullptr, 0, 1, 1));
    add(check(2, 1, 2, nullptr, nullptr, 0, 1, 1));
    add(check(1, 2, 2, nullptr, nullptr, 0, 1, 1));
    add(check(2, 2, 2, nullptr, nullptr, 0, 1, 1));
    add(check(1, 1, 4, nullptr, nullptr, 0, 1, 1));
    const int8_t a[4] = {0, 1, 0, 1}, s2[8] = {0, 1, 0, 1, 0, 2, 1, 3}, r2[8] = {0, 1, 0, 1, 0, 1, 0, 1};
    add(check(2, 2, 4, a, a, 1, 1, 1));
    add(check(2, 2, 4, s2, r2, 2, 1, 1));
    const int8_t c[3] = {0, 1, 2}, d[3] = {1, 2, 3};
    add(check(0, 3, 4, c, d, 1, 1, 1));
    const int8_t e[4] = {0, 1, 2, 3}, f[4] = {0, 2, 0, 2};
    add(check(2, 2, 2, e, f, 1, 2, 2));
    std::printf("%s\n", bad ? "FAIL" : "OK");
    return bad ? 1 : 0;
}
