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
    int64_t op_off;   // warp-per-site layout [round][z][sub-lane]
    int64_t zop_off;  // lanes-are-sites layout: z-major, k ops per z
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
// puts the most expensive list first), handed out by an atomic counter.
constexpr int kMaxBatch = 8;
struct SmallBatch {
    int32_t n_lists;
    int32_t site_stride;      // warp-per-site kernel: entries of one site region (max over lists)
    int32_t comp_stride;      // warp-per-site kernel: components per site in the C area (max)
    int32_t tiles_per_slab;
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

// Ops of a step are stored as [round j][z][sub-lane]: in round j the g lanes
// of output z read ops j*g + sub, so a warp reads 32 consecutive words.
template <class Tr>
__device__ __forceinline__ void small_step(const SmallPlan &P, const SmallStepDesc &d, typename Tr::V *R,
                                           int lane) {
    using V = typename Tr::V;
    const V *X = R + d.x_off;
    const V *Y = R + d.y_off;
    V *Z = R + d.z_off;
    const uint32_t *ops = P.ops + d.op_off;
    const int g = d.g;                 // lanes per z (power of two)
    const int per = 32 / g;            // z per round
    const int sub = lane & (g - 1);
    const int64_t round_stride = (int64_t)d.n_z * g;
    const unsigned full = 0xffffffffu;
    for (int z0 = 0; z0 < d.n_z; z0 += per) {
        int z = z0 + lane / g;
        typename Tr::Acc acc;
        acc.zero();
        if (z < d.n_z) {
            const uint32_t *oz = ops + z * g + sub;
            const int rs = (int)round_stride;
            const int jfull = (d.k - sub + g - 1) / g;  // rounds in which this lane has an op
#pragma unroll 4
            for (int j = 0; j < jfull; ++j) {
                uint32_t op = __ldg(oz + j * rs);
                acc.fma(X[op & 0xffffu], Y[(op >> 16) & 0x7fffu], op & 0x80000000u);
            }
        }
        for (int off = g >> 1; off > 0; off >>= 1) acc.add_shfl(full, off);
        if (z < d.n_z && sub == 0) Z[z] = acc.store();
    }
    __syncwarp();
}

// Blocks (Sec. 2) for one site: Q, then f_P and/or f_N antisymmetric parts.
template <class Tr>
__device__ __forceinline__ void small_blocks(const SmallPlan &P, typename Tr::V *R, int lane) {
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
        if (!P.need_blk[b]) continue;
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
    for (int li; (li = next_item(B, tile)) >= 0;) {
        const SmallPlan &P = B.plan[li];
        double2 *partial = partial_base + B.partial_off[li];
        const int nxi = P.nxi;
        const int64_t slab = tile / tiles_per_slab;
        const int tin = (int)(tile % tiles_per_slab);
        const int cfg = (int)(slab / F.n_t), t = F.t0 + (int)(slab % F.n_t);
        const int site = tin * T + warp;
        const bool live = site < V3;
        if (live) {
            const int64_t base = cfg * F.stride_cfg + t * F.stride_t + (int64_t)site * site_elems(F);
            // 1. propagator tile
            const int nent = nxi * nxi;
            for (int e = lane; e < nent; e += 32) R[P.s_off + e] = Tr::from_d(load_prop(F, base, (e / nxi) * 12 + (e % nxi)));
            __syncwarp();
            // 2. blocks
            small_blocks<Tr>(P, R, lane);
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
    }
}

// ---- lanes-are-sites kernel (mixed path) -------------------------------------
// A CTA owns a tile of 32 sites, lane l of every warp works on site l; all
// per-site values are rows of 32 lanes in shared memory ([entry][lane], 8 B
// per lane), so every access of a warp is one conflict-free row. The warps
// split the output components of each step (warp-uniform op stream, loaded
// cooperatively and broadcast by shuffles); steps with fewer outputs than
// warps split each output's terms over several warps and combine the
// compensated partials in a fixed order.

// RN(d * 2^e) as FP32 from the bits of an FP64 value, integer operations only
// (GB300's FP64 pipe is 1/64 of FP32). Results below the FP32 normal range
// flush to zero; inputs here are scaled to |d| < 2.
__device__ __forceinline__ float f64_scaled_to_f32(double d, int e) {
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const uint32_t sign = hi & 0x80000000u;
    const int eb = (int)((hi >> 20) & 0x7ffu);
    const int ef = eb - 1023 + e + 127;
    if (eb == 0 || ef <= 0) return __int_as_float((int)sign);
    const uint32_t top = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1fffffffu;
    const uint32_t up = (rem > 0x10000000u) || (rem == 0x10000000u && (top & 1u));
    return __int_as_float((int)(sign | (((uint32_t)ef << 23) + top + up)));
}
__device__ __forceinline__ int f64_exponent(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d);
    const int eb = (int)((hi >> 20) & 0x7ffu);
    return eb == 0 ? -100000 : eb - 1023;
}
__device__ __forceinline__ float f32_scaled(float f, int e) {
    const uint32_t b = (uint32_t)__float_as_int(f);
    const int eb = (int)((b >> 23) & 0xffu);
    const int en = eb + e;
    if (eb == 0 || en <= 0) return __int_as_float((int)(b & 0x80000000u));
    return __int_as_float((int)((b & 0x807fffffu) | ((uint32_t)en << 23)));
}
__device__ __forceinline__ int f32_exponent(float f) {
    const int eb = (int)(((uint32_t)__float_as_int(f) >> 23) & 0xffu);
    return eb == 0 ? -100000 : eb - 127;
}

template <class Tr>
__global__ void __launch_bounds__(1024, 1)
    k_small_ls(const __grid_constant__ SmallBatch B, FieldDesc F, MomDesc M, const double2 *__restrict__ phase,
               double2 *partial_base) {
    using V = typename Tr::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *R = reinterpret_cast<V *>(smem_raw);  // [entry][32]
    __shared__ int sexp_s[32];
    const int NW = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int V3 = F.lx * F.ly * F.lz;
    const unsigned full = 0xffffffffu;
    const int tiles_per_slab = B.tiles_per_slab;
#define ROW(e) R[(int64_t)(e) * 32 + lane]

    int64_t tile;
    for (int li; (li = next_item(B, tile)) >= 0;) {  // next_item synchronises the CTA
        const SmallPlan &P = B.plan[li];
        double2 *partial = partial_base + B.partial_off[li];
        const int nxi = P.nxi, nent = nxi * nxi;
        const int64_t slab = tile / tiles_per_slab;
        const int tin = (int)(tile % tiles_per_slab);
        const int cfg = (int)(slab / F.n_t), t = F.t0 + (int)(slab % F.n_t);
        const int site0 = tin * 32;
        // 1. load and scale: one warp per site
        for (int s = warp; s < 32; s += NW) {
            const int site = site0 + s;
            const bool live = site < V3;
            const int64_t base = cfg * F.stride_cfg + t * F.stride_t + (int64_t)site * site_elems(F);
            // two passes over the tile (the second one hits L1): exponent, then values
            int emax = -100000;
            for (int e = lane; e < nent; e += 32) {
                const int idx = (e / nxi) * 12 + (e % nxi);
                if (!live) break;
                if (F.dtype == 0) {
                    const double2 v = __ldg(reinterpret_cast<const double2 *>(F.s) + base + idx);
                    emax = max(emax, max(f64_exponent(v.x), f64_exponent(v.y)));
                } else {
                    const float2 v = __ldg(reinterpret_cast<const float2 *>(F.s) + base + idx);
                    emax = max(emax, max(f32_exponent(v.x), f32_exponent(v.y)));
                }
            }
            for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(full, emax, off));
            const int se = emax == -100000 ? 0 : -emax;  // largest entry scaled into [1, 2)
            for (int e = lane; e < nent; e += 32) {
                const int idx = (e / nxi) * 12 + (e % nxi);
                float2 v = make_float2(0.f, 0.f);
                if (live) {
                    if (F.dtype == 0) {
                        const double2 dvv = __ldg(reinterpret_cast<const double2 *>(F.s) + base + idx);
                        v = make_float2(f64_scaled_to_f32(dvv.x, se), f64_scaled_to_f32(dvv.y, se));
                    } else {
                        const float2 fvv = __ldg(reinterpret_cast<const float2 *>(F.s) + base + idx);
                        v = make_float2(f32_scaled(fvv.x, se), f32_scaled(fvv.y, se));
                    }
                }
                R[(int64_t)(P.s_off + e) * 32 + s] = V{v.x, v.y};
            }
            if (lane == 0) sexp_s[s] = se;
        }
        __syncthreads();
        // 2. diquark and blocks (Sec. 2); lane = site
        for (int e = warp; e < 3 * nent; e += NW) {
            const int c = e / nent, r = e % nent, x2 = r / nxi, x3 = r % nxi;
            V acc{0, 0};
            for (int gg = 0; gg < P.n_g2; ++gg) {
                const int s2 = c_g2[gg][0], s3 = c_g2[gg][1], v = c_g2[gg][2];
                for (int q = 0; q < 2; ++q) {
                    const int c2 = c_eps[c][q][0], c3 = c_eps[c][q][1], sg = c_eps[c][q][2] * v;
                    const V a = ROW(P.s_off + (3 * s2 + c2) * nxi + x2), b = ROW(P.s_off + (3 * s3 + c3) * nxi + x3);
                    acc = sg > 0 ? cfma(a, b, acc) : cfms(a, b, acc);
                }
            }
            ROW(P.q_off + e) = acc;
        }
        __syncthreads();
        const int per_spin = P.npair * nxi;
        for (int b = 0; b < 2; ++b) {
            if (!P.need_blk[b]) continue;
            for (int e = warp; e < P.block_size; e += NW) {
                const int dl = e / per_spin, r = e % per_spin;
                const int pr = r / nxi, single = r % nxi;
                const int i = c_pair_i[pr], j = c_pair_j[pr];
                V acc{0, 0};
                for (int c = 0; c < 3; ++c) {
                    const int sr = P.s_off + (3 * dl + c) * nxi;
                    if (b == 0) {
                        acc = cfma(ROW(sr + i), ROW(P.q_off + (c * nxi + j) * nxi + single), acc);
                        acc = cfms(ROW(sr + j), ROW(P.q_off + (c * nxi + i) * nxi + single), acc);
                    } else {
                        acc = cfma(ROW(sr + i), ROW(P.q_off + (c * nxi + single) * nxi + j), acc);
                        acc = cfms(ROW(sr + j), ROW(P.q_off + (c * nxi + single) * nxi + i), acc);
                    }
                }
                ROW(P.blk_off[b] + e) = acc;
            }
        }
        __syncthreads();
        // 3. recursion
        for (int m = 0; m < P.n_steps; ++m) {
            const SmallStepDesc &d = P.step[m];
            const uint32_t *ops = P.zops + d.zop_off;
            const int split = d.n_z < NW ? NW / d.n_z : 1;  // CTA-uniform
            int64_t o_begin, o_end, zb;
            int part = -1;
            if (split <= 1) {
                zb = (int64_t)warp * d.n_z / NW;
                const int64_t ze = (int64_t)(warp + 1) * d.n_z / NW;
                o_begin = zb * d.k;
                o_end = ze * d.k;
            } else {
                const int u = warp;  // unit = (z, part)
                if (u < d.n_z * split) {
                    zb = u / split;
                    part = u % split;
                    o_begin = zb * d.k + (int64_t)part * d.k / split;
                    o_end = zb * d.k + (int64_t)(part + 1) * d.k / split;
                } else {
                    zb = 0;
                    o_begin = o_end = 0;
                }
            }
            typename Tr::Acc acc;
            acc.zero();
            // 32-bit lane pointers: row e of lane l sits at R[e * 32 + l]
            const V *Xl = R + (d.x_off << 5) + lane;
            const V *Yl = R + (d.y_off << 5) + lane;
            V *Zl = R + (d.z_off << 5) + lane;
            // output by output: each output's k terms are contiguous, loaded
            // 32 at a time and broadcast by shuffles; no per-term branch
            const int n_out = part < 0 ? (int)((o_end - o_begin) / d.k) : 1;
            const int len = part < 0 ? d.k : (int)(o_end - o_begin);
            const uint32_t *op_ptr = ops + o_begin;
            for (int zz = 0; zz < n_out; ++zz, op_ptr += len) {
                for (int b0 = 0; b0 < len; b0 += 32) {
                    const int nb = min(32, len - b0);
                    const uint32_t mine = lane < nb ? __ldg(op_ptr + b0 + lane) : 0u;
#pragma unroll 4
                    for (int q = 0; q < nb; ++q) {
                        const uint32_t op = __shfl_sync(full, mine, q);
                        acc.fma(Xl[(op & 0xffffu) << 5], Yl[((op >> 16) & 0x7fffu) << 5], op & 0x80000000u);
                    }
                }
                if (part < 0) {
                    Zl[((int)zb + zz) << 5] = acc.store();
                    acc.zero();
                }
            }
            if (split > 1) {
                if (part >= 0) {
                    ROW(P.part_off + 2 * warp) = V{acc.sr, acc.cr};
                    ROW(P.part_off + 2 * warp + 1) = V{acc.si, acc.ci};
                }
                __syncthreads();
                for (int zz = warp; zz < d.n_z; zz += NW) {
                    typename Tr::Acc a;
                    a.zero();
                    for (int pp = 0; pp < split; ++pp) {
                        const V r0 = ROW(P.part_off + 2 * (zz * split + pp));
                        const V r1 = ROW(P.part_off + 2 * (zz * split + pp) + 1);
                        a.add(r0.x, r0.y, r1.x, r1.y);
                    }
                    ROW(d.z_off + zz) = a.store();
                }
            }
            __syncthreads();
        }
        // 4. contraction with L in FP64, undo the scaling, phase, sum over the
        //    32 sites of the tile by a fixed xor tree
        const int site = site0 + lane;
        const bool live = site < V3;
        for (int c = warp; c < P.n_comp; c += NW) {
            const int ue = -__ldg(P.comp_deg + c) * sexp_s[lane];
            const double inv_norm = __ldg(P.comp_inv_norm + c);
            double re = 0.0, im = 0.0;
            for (int64_t e = P.fin_off[c]; e < P.fin_off[c + 1]; ++e) {
                const double2 f = Tr::to_d(ROW(__ldg(P.fin_z + e)));
                const double l = __ldg(P.fin_l + e);
                re = __fma_rn(l, f.x, re);
                im = __fma_rn(l, f.y, im);
            }
            re = live ? scalbn(re * inv_norm, ue) : 0.0;
            im = live ? scalbn(im * inv_norm, ue) : 0.0;
            for (int q = 0; q < M.n_mom; ++q) {
                const double2 ph = live ? __ldg(phase + (int64_t)site * M.n_mom + q) : make_double2(0, 0);
                double pr = __fma_rn(ph.x, re, -ph.y * im), pi = __fma_rn(ph.x, im, ph.y * re);
                for (int off = 16; off > 0; off >>= 1) {
                    pr += __shfl_xor_sync(full, pr, off);
                    pi += __shfl_xor_sync(full, pi, off);
                }
                if (lane == 0) partial[tile * (int64_t)(M.n_mom * P.n_comp) + q * P.n_comp + c] = make_double2(pr, pi);
            }
        }
    }
#undef ROW
}

}  // namespace mbc
