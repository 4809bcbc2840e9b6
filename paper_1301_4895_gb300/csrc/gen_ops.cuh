// List-free recursion steps: the splits z = x + y of an output component are
// regenerated on the device from the component's key instead of being read
// from stored operation arrays (Sec. 3: a component is a tuple of four sets,
// proton spins, neutron spins, u and d indices, each enumerated by its colex
// rank; every split of a needed component is one operation).
//
// The enumeration order is the builder's (spin of the added baryon, then its
// u choice, then its d choice, each ascending), so a generated step performs
// the same operations in the same order as the stored list.
#pragma once

#include <cstdint>

namespace mbc {

// C(n, k) for n, k <= 24 (quark index values of up to two sources)
__constant__ uint32_t c_binom[25][25];

struct GenStep {
    int32_t b;          // baryon added: MBC_PROTON (0) or MBC_NEUTRON (1)
    int32_t bprev;      // first baryon of the path (x is its block when x_block)
    int32_t x_block;    // the input stage is the first baryon's block (step 1)
    int32_t nxi, npair; // quark index values, C(nxi, 2)
    int32_t dim;        // sink baryon index values
    int32_t zk[4], xk[4];    // set sizes of the output and input stages
    int64_t zr[4], xr[4];    // radices C(dim, kp), C(dim, kn), C(nxi, ku), C(nxi, kd)
    const int64_t *zrank;    // dense rank of each output (NULL: output stage dense)
    const int32_t *xmap;     // compact index of each dense input rank (NULL: dense)
};

__device__ __forceinline__ int64_t g_colex_rank(uint32_t m) {
    int64_t r = 0;
    int t = 1;
    while (m) {
        const int p = __ffs(m) - 1;
        r += c_binom[p][t++];
        m &= m - 1;
    }
    return r;
}

__device__ __forceinline__ uint32_t g_colex_unrank(int64_t r, int k, int n) {
    uint32_t m = 0;
    for (int t = k; t >= 1; --t) {
        int p = t - 1;
        while (p + 1 < n && (int64_t)c_binom[p + 1][t] <= r) ++p;
        r -= c_binom[p][t];
        m |= 1u << p;
    }
    return m;
}

// position of the i-th (0-based) set bit of m
__device__ __forceinline__ int g_select(uint32_t m, int i) {
    for (int t = 0; t < i; ++t) m &= m - 1;
    return __ffs(m) - 1;
}

// (i, j), i < j, of the idx-th pair of n elements in lexicographic order
__device__ __forceinline__ void g_lex_pair(int idx, int n, int &i, int &j) {
    i = 0;
    while (idx >= n - 1 - i) {
        idx -= n - 1 - i;
        ++i;
    }
    j = i + 1 + idx;
}

// (-1)^{#(i in x, j in y, i > j)} of one index group, as a parity bit
__device__ __forceinline__ uint32_t g_parity(uint32_t x, uint32_t y) {
    uint32_t n = 0;
    while (y) {
        const int j = __ffs(y) - 1;
        n += __popc(x >> (j + 1));
        y &= y - 1;
    }
    return n & 1u;
}

// block component index [spin][pair rank][single] of one baryon's key
__device__ __forceinline__ uint32_t g_block_index(uint32_t dp, uint32_t dn, uint32_t u, uint32_t d, int b, int nxi,
                                                  int npair) {
    if (b == 0) return (uint32_t)(((__ffs(dp) - 1) * npair + g_colex_rank(u)) * nxi + (__ffs(d) - 1));
    return (uint32_t)(((__ffs(dn) - 1) * npair + g_colex_rank(d)) * nxi + (__ffs(u) - 1));
}

// key (dp, dn, u, d) of output component z
__device__ __forceinline__ void g_key(const GenStep &g, int64_t z, uint32_t key[4]) {
    int64_t i = g.zrank ? __ldg(g.zrank + z) : z;
    const int64_t rd = i % g.zr[3];
    i /= g.zr[3];
    const int64_t ru = i % g.zr[2];
    i /= g.zr[2];
    const int64_t rn = i % g.zr[1];
    i /= g.zr[1];
    key[3] = g_colex_unrank(rd, g.zk[3], g.nxi);
    key[2] = g_colex_unrank(ru, g.zk[2], g.nxi);
    key[1] = g_colex_unrank(rn, g.zk[1], g.dim);
    key[0] = g_colex_unrank(i, g.zk[0], g.dim);
}

// Operation j of output key z: x index (into the input stage) and
// y block index | sign << 15, as in the stored lists.
__device__ __forceinline__ void g_op(const GenStep &g, const uint32_t z[4], int64_t j, uint32_t &ox, uint32_t &oy) {
    const int nu = __popc(z[2]), nd = __popc(z[3]);
    uint32_t y[4] = {0, 0, 0, 0};
    if (g.b == 0) {  // proton: one spin, a u pair, one d
        const int64_t per_spin = (int64_t)(nu * (nu - 1) / 2) * nd;
        const int s = (int)(j / per_spin);
        const int64_t rem = j % per_spin;
        int i1, i2;
        g_lex_pair((int)(rem / nd), nu, i1, i2);
        y[0] = 1u << g_select(z[0], s);
        y[2] = (1u << g_select(z[2], i1)) | (1u << g_select(z[2], i2));
        y[3] = 1u << g_select(z[3], (int)(rem % nd));
    } else {  // neutron: one spin, one u, a d pair
        const int64_t npd = nd * (nd - 1) / 2;
        const int64_t per_spin = (int64_t)nu * npd;
        const int s = (int)(j / per_spin);
        const int64_t rem = j % per_spin;
        int i1, i2;
        g_lex_pair((int)(rem % npd), nd, i1, i2);
        y[1] = 1u << g_select(z[1], s);
        y[2] = 1u << g_select(z[2], (int)(rem / npd));
        y[3] = (1u << g_select(z[3], i1)) | (1u << g_select(z[3], i2));
    }
    const uint32_t x[4] = {z[0] & ~y[0], z[1] & ~y[1], z[2] & ~y[2], z[3] & ~y[3]};
    if (g.x_block) {
        ox = g_block_index(x[0], x[1], x[2], x[3], g.bprev, g.nxi, g.npair);
    } else {
        const int64_t r =
            ((g_colex_rank(x[0]) * g.xr[1] + g_colex_rank(x[1])) * g.xr[2] + g_colex_rank(x[2])) * g.xr[3] +
            g_colex_rank(x[3]);
        ox = g.xmap ? (uint32_t)__ldg(g.xmap + r) : (uint32_t)r;
    }
    const uint32_t sgn = g_parity(x[0], y[0]) ^ g_parity(x[1], y[1]) ^ g_parity(x[2], y[2]) ^ g_parity(x[3], y[3]);
    oy = g_block_index(y[0], y[1], y[2], y[3], g.b, g.nxi, g.npair) | (sgn << 15);
}

}  // namespace mbc
