// Small-stage contraction kernel: every stage of one site fits in shared
// memory (the nonrelativistic nuclei, where the largest stage has 225
// components, Sec. 7 P(n_P, n_N) with D = 2).
//
// One warp owns one sink site at a time; a CTA holds T = warps-per-CTA sites
// (one tile). Per site, in the warp's shared-memory region:
//   1. the nxi x nxi propagator tile (rows: sink spinor-colour indices that
//      Gamma_1/Gamma_2 can reach, cols: source indices that L can reach);
//      MIXED scales it by an exact power of two so its largest entry is O(1);
//   2. the diquark Q and the antisymmetric block components f_P, f_N
//      (Sec. 2 blocks; Sec. 4: antisymmetrised by the two orderings of the
//      same-flavour slots);
//   3. every step F^(m+1)[z] = sum_j s_j F^(m)[x_j] f[y_j] (eq. recr_F) over
//      the z-major lists; g lanes share one z and combine by xor shuffles;
//   4. the contraction with L (eq. C_final) into FP64;
// then the CTA multiplies each site's components by the momentum phases and
// sums its T sites in a fixed order into one partial per (tile, mom, comp).
#pragma once

#include "device_common.cuh"

namespace mbc {

constexpr int kMaxMom = 32;
constexpr int kSmallMaxComp = 64;

struct SmallStepDesc {
    int32_t n_z, k, g, x_off, y_off, z_off;
    int64_t op_off;   // warp-per-site layout [round][z][sub-lane]: outputs [0, n_main) with g lanes each
    int64_t zop_off;  // lanes-are-sites layout: z-major, k ops per z
    int32_t n_main;   // outputs in whole rounds of 32 / g; the rest take g2 lanes each
    int32_t g2;
    int64_t op_off2;  // the rest's ops, [round][z - n_main][sub-lane] with g2
};

struct SmallPlan {
    int32_t A, dim, nxi, n_g2, n_comp, n_steps;
    int32_t path0;
    int32_t need_blk[2], blk_off[2];
    int32_t s_off, q_off;               // entry offsets in the per-site region
    int32_t site_entries;               // per-site region size (entries)
    int32_t block_size, npair;
    int32_t fin_g;                      // lanes per component in the contraction
    SmallStepDesc step[16];
    const uint32_t *ops;                // packed: x | y << 16 | sign << 31
    const uint32_t *zops;               // the same ops, z-major
    int32_t part_off;                   // lanes-are-sites: split partials (64 entries)
    const int64_t *fin_off;             // n_comp + 1
    const uint32_t *fin_z;              // entry offsets in the per-site region
    const double *fin_l;                // integer L values
    const double *comp_inv_norm;        // per component: 1 / (n_P! n_N!)^2 of its nucleus
    const int32_t *comp_deg;            // per component: 3 A of its nucleus (homogeneity degree)
};

// A batch of term lists contracted by one persistent launch: the work items
// are (list, tile) pairs, numbered list by list in the order given (the host
// puts the most expensive list first), handed out by an atomic counter. In a
// shared batch (lists with the same tile shape and buffer offsets of the S
// tile, diquark and blocks) an item is a tile and covers every list: the
// tile and the blocks (of the baryons any list needs) are computed once per
// site, then each list runs its steps and contraction.
constexpr int kMaxBatch = 8;
struct SmallBatch {
    int32_t n_lists;
    int32_t site_stride;      // warp-per-site kernel: entries of one site region (max over lists)
    int32_t comp_stride;      // warp-per-site kernel: components per site in the C area (max)
    int32_t tiles_per_slab;
    int32_t shared;           // items are tiles covering every list
    int32_t need_union[2];    // shared: blocks some list needs
    int64_t total_items;
    int64_t item_base[kMaxBatch + 1];
    int64_t partial_off[kMaxBatch];  // in double2 units
    unsigned long long *counter;     // zeroed before the launch
    SmallPlan plan[kMaxBatch];
};

// next work item of the CTA (thread 0 draws, everyone reads); returns the list
__device__ __forceinline__ int next_item(const SmallBatch &B, int64_t &tile) {
    __shared__ long long s_item;
    __syncthreads();
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(B.counter, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= B.total_items) return -1;
    if (B.shared) {
        tile = item;
        return 0;
    }
    int l = 0;
    while (l + 1 < B.n_lists && item >= B.item_base[l + 1]) ++l;
    tile = item - B.item_base[l];
    return l;
}

struct FieldDesc {
    const void *s;        // u = d field
    int32_t dtype;        // 0: complex double, 1: complex float
    int32_t n_cfg, nt, lx, ly, lz;
    int64_t stride_cfg, stride_t;  // in complex elements
    int32_t t0, n_t;               // evaluated slices [t0, t0 + n_t)
    int32_t n_src;                 // quark sources per site: a site holds n_src 12 x 12 matrices
};

// complex elements of one site (all sources)
__device__ __forceinline__ int64_t site_elems(const FieldDesc &f) { return 144LL * f.n_src; }

// Entry e of a site's propagator tile with nrow x ncol entries: row r = e / ncol
// is the sink index, column c = e % ncol the source quark index
// xi = n_src * kappa + s (Sec. 6), read from source s's 12 x 12 matrix.
__device__ __forceinline__ int tile_index(const FieldDesc &f, int e, int ncol) {
    const int r = e / ncol, c = e % ncol;
    return (c % f.n_src) * 144 + r * 12 + c / f.n_src;
}

struct MomDesc {
    int32_t n_mom;
    int32_t mom[kMaxMom][3];
};

__device__ __forceinline__ double2 load_prop(const FieldDesc &f, int64_t base, int idx) {
    if (f.dtype == 0) {
        const double2 *p = reinterpret_cast<const double2 *>(f.s) + base + idx;
        return __ldg(p);
    }
    const float2 *p = reinterpret_cast<const float2 *>(f.s) + base + idx;
    float2 v = __ldg(p);
    return make_double2(v.x, v.y);
}

// phase exp(-2 pi i (n_x x / L_x + n_y y / L_y + n_z z / L_z))
__device__ __forceinline__ double2 mom_phase(const int32_t *n, int x, int y, int z, int lx, int ly, int lz) {
    // reduce each product modulo its extent in integers, then one turn fraction
    int rx = ((n[0] * x) % lx + lx) % lx, ry = ((n[1] * y) % ly + ly) % ly, rz = ((n[2] * z) % lz + lz) % lz;
    double turns = (double)rx / lx + (double)ry / ly + (double)rz / lz;
    double s, c;
    sincospi(-2.0 * turns, &s, &c);
    return make_double2(c, s);
}

// Outputs [z_begin, z_begin + n) of a step with g lanes per output. Their ops
// are stored as [round j][z - z_begin][sub-lane]: in round j the g lanes of
// output z read ops j*g + sub, so a warp reads 32 consecutive words.
template <class Tr>
__device__ __forceinline__ void small_step_part(const typename Tr::V *X, const typename Tr::V *Y, typename Tr::V *Z,
                                                const uint32_t *ops, int z_begin, int n, int k, int g, int lane) {
    const int per = 32 / g;            // z per round
    const int sub = lane & (g - 1);
    const int rs = n * g;              // words per round
    const unsigned full = 0xffffffffu;
    for (int z0 = 0; z0 < n; z0 += per) {
        const int zl = z0 + lane / g;
        typename Tr::Acc acc;
        acc.zero();
        if (zl < n) {
            const uint32_t *oz = ops + zl * g + sub;
            const int jfull = (k - sub + g - 1) / g;  // rounds in which this lane has an op
#pragma unroll 4
            for (int j = 0; j < jfull; ++j) {
                uint32_t op = __ldg(oz + j * rs);
                acc.fma(X[op & 0xffffu], Y[(op >> 16) & 0x7fffu], op & 0x80000000u);
            }
        }
        for (int off = g >> 1; off > 0; off >>= 1) acc.add_shfl(full, off);
        if (zl < n && sub == 0) Z[z_begin + zl] = acc.store();
    }
}

// One step for one site: whole rounds of the outputs with g lanes each, then
// the remaining outputs with g2 lanes each (fewer idle lanes in the last round).
template <class Tr>
__device__ __forceinline__ void small_step(const SmallPlan &P, const SmallStepDesc &d, typename Tr::V *R,
                                           int lane) {
    using V = typename Tr::V;
    const V *X = R + d.x_off;
    const V *Y = R + d.y_off;
    V *Z = R + d.z_off;
    small_step_part<Tr>(X, Y, Z, P.ops + d.op_off, 0, d.n_main, d.k, d.g, lane);
    if (d.n_main < d.n_z)
        small_step_part<Tr>(X, Y, Z, P.ops + d.op_off2, d.n_main, d.n_z - d.n_main, d.k, d.g2, lane);
    __syncwarp();
}

// Blocks (Sec. 2) for one site: Q, then f_P and/or f_N antisymmetric parts.
template <class Tr>
__device__ __forceinline__ void small_blocks(const SmallPlan &P, const int32_t *need, typename Tr::V *R, int lane) {
    using V = typename Tr::V;
    const int nxi = P.nxi;
    const V *S = R + P.s_off;
    V *Q = R + P.q_off;
    for (int e = lane; e < 3 * nxi * nxi; e += 32) {
        int c = e / (nxi * nxi), r = e % (nxi * nxi);
        Q[e] = diquark(S, nxi, nxi, P.n_g2, c, r / nxi, r % nxi);
    }
    __syncwarp();
    const int per_spin = P.npair * nxi;
    for (int b = 0; b < 2; ++b) {
        if (!need[b]) continue;
        V *F = R + P.blk_off[b];
        for (int e = lane; e < P.block_size; e += 32) {
            int dl = e / per_spin, r = e % per_spin;
            int pr = r / nxi, single = r % nxi;
            int i = c_pair_i[pr], j = c_pair_j[pr];
            V acc{0, 0};
            for (int c = 0; c < 3; ++c) {
                const V *Sr = S + (3 * dl + c) * nxi;
                if (b == 0) {  // proton: u pair (i, j) at slots 1, 2; d = single at slot 3
                    acc = cfma(Sr[i], Q[(c * nxi + j) * nxi + single], acc);
                    acc = cfms(Sr[j], Q[(c * nxi + i) * nxi + single], acc);
                } else {  // neutron: d pair (i, k=j) at slots 1, 3; u = single at slot 2
                    acc = cfma(Sr[i], Q[(c * nxi + single) * nxi + j], acc);
                    acc = cfms(Sr[j], Q[(c * nxi + single) * nxi + i], acc);
                }
            }
            F[e] = acc;
        }
    }
    __syncwarp();
}

// Phase table of one slab geometry: tab[site][mom] = exp(-2 pi i n.x / L).
__global__ void k_phase_table(FieldDesc F, MomDesc M, double2 *tab) {
    const int v3 = F.lx * F.ly * F.lz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v3 * M.n_mom; i += gridDim.x * blockDim.x) {
        int site = i / M.n_mom, q = i % M.n_mom;
        int x = site % F.lx, y = (site / F.lx) % F.ly, z = site / (F.lx * F.ly);
        tab[i] = mom_phase(M.mom[q], x, y, z, F.lx, F.ly, F.lz);
    }
}

// Shared-memory kernel, one warp per site (FP64 path).
template <class Tr>
__global__ void __launch_bounds__(1024, 1)
    k_small(const __grid_constant__ SmallBatch B, FieldDesc F, MomDesc M, const double2 *__restrict__ phase,
            double2 *partial_base) {
    using V = typename Tr::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    V *R = reinterpret_cast<V *>(smem_raw) + (int64_t)warp * B.site_stride;
    double2 *Cs = reinterpret_cast<double2 *>(reinterpret_cast<V *>(smem_raw) + (int64_t)T * B.site_stride);
    const int V3 = F.lx * F.ly * F.lz;
    const int tiles_per_slab = B.tiles_per_slab;
    int64_t tile;
    for (int li0; (li0 = next_item(B, tile)) >= 0;) {
        const int l_end = B.shared ? B.n_lists : li0 + 1;
        const SmallPlan &P0 = B.plan[li0];
        const int nxi = P0.nxi;
        const int64_t slab = tile / tiles_per_slab;
        const int tin = (int)(tile % tiles_per_slab);
        const int cfg = (int)(slab / F.n_t), t = F.t0 + (int)(slab % F.n_t);
        const int site = tin * T + warp;
        const bool live = site < V3;
        if (live) {
            const int64_t base = cfg * F.stride_cfg + t * F.stride_t + (int64_t)site * site_elems(F);
            // 1. propagator tile
            const int nent = nxi * nxi;
            for (int e = lane; e < nent; e += 32) R[P0.s_off + e] = Tr::from_d(load_prop(F, base, (e / nxi) * 12 + (e % nxi)));
            __syncwarp();
            // 2. blocks, once for every list of the item
            small_blocks<Tr>(P0, B.shared ? B.need_union : P0.need_blk, R, lane);
        }
        for (int li = li0; li < l_end; ++li) {
            const SmallPlan &P = B.plan[li];
            double2 *partial = partial_base + B.partial_off[li];
            if (live) {
                // 3. recursion
                for (int m = 0; m < P.n_steps; ++m) small_step<Tr>(P, P.step[m], R, lane);
                // 4. contraction with L, FP64
                const int g = P.fin_g, per = 32 / g, sub = lane & (g - 1);
                for (int c0 = 0; c0 < P.n_comp; c0 += per) {
                    int c = c0 + lane / g;
                    double re = 0.0, im = 0.0;
                    if (c < P.n_comp) {
                        for (int64_t e = P.fin_off[c] + sub; e < P.fin_off[c + 1]; e += g) {
                            double2 f = Tr::to_d(R[__ldg(P.fin_z + e)]);
                            double l = __ldg(P.fin_l + e);
                            re = __fma_rn(l, f.x, re);
                            im = __fma_rn(l, f.y, im);
                        }
                    }
                    for (int off = g >> 1; off > 0; off >>= 1) {
                        re += __shfl_xor_sync(0xffffffffu, re, off);
                        im += __shfl_xor_sync(0xffffffffu, im, off);
                    }
                    if (c < P.n_comp && sub == 0) Cs[warp * B.comp_stride + c] = make_double2(re, im);
                }
            } else {
                for (int c = lane; c < P.n_comp; c += 32) Cs[warp * B.comp_stride + c] = make_double2(0, 0);
            }
            __syncthreads();
            // tile partial: (1/N) sum over the T sites, in a fixed order, of phase * C
            const int site0 = tin * T;
            for (int o = threadIdx.x; o < M.n_mom * P.n_comp; o += blockDim.x) {
                int q = o / P.n_comp, c = o % P.n_comp;
                double re = 0.0, im = 0.0;
                for (int w = 0; w < T && site0 + w < V3; ++w) {
                    double2 ph = __ldg(phase + (int64_t)(site0 + w) * M.n_mom + q), cv = Cs[w * B.comp_stride + c];
                    re = __fma_rn(ph.x, cv.x, __fma_rn(-ph.y, cv.y, re));
                    im = __fma_rn(ph.x, cv.y, __fma_rn(ph.y, cv.x, im));
                }
                const double inv_norm = __ldg(P.comp_inv_norm + c);
                partial[tile * (int64_t)(M.n_mom * P.n_comp) + o] = make_double2(re * inv_norm, im * inv_norm);
            }
            if (li + 1 < l_end) __syncthreads();  // Cs is read before the next list writes it
        }
    }
}

}  // namespace mbc
