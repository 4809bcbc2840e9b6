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
    int64_t op_off;
};

struct SmallPlan {
    int32_t A, dim, nxi, n_g2, n_comp, n_steps;
    int32_t path0;
    int32_t need_blk[2], blk_off[2];
    int32_t s_off, q_off, fin_off_buf;  // entry offsets in the per-site region
    int32_t site_entries;               // per-site region size (entries)
    int32_t block_size, npair;
    int32_t fin_g;                      // lanes per component in the contraction
    SmallStepDesc step[16];
    const uint32_t *ops;                // packed: x | y << 16 | sign << 31
    const int64_t *fin_off;             // n_comp + 1
    const uint32_t *fin_z;
    const double *fin_l;                // integer L values
    double inv_norm;
};

struct FieldDesc {
    const void *s;        // u = d field
    int32_t dtype;        // 0: complex double, 1: complex float
    int32_t n_cfg, nt, lx, ly, lz;
    int64_t stride_cfg, stride_t;  // in complex elements
    int32_t t0, n_t;               // evaluated slices [t0, t0 + n_t)
};

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
    const int kk = (d.k + g - 1) / g;  // ops per lane
    const unsigned full = 0xffffffffu;
    for (int z0 = 0; z0 < d.n_z; z0 += per) {
        int z = z0 + lane / g;
        typename Tr::Acc acc;
        acc.zero();
        if (z < d.n_z) {
            const uint32_t *oz = ops + (int64_t)z * d.k;
            for (int j = 0; j < kk; ++j) {
                int jj = j * g + sub;
                if (jj < d.k) {
                    uint32_t op = __ldg(oz + jj);
                    acc.fma(X[op & 0xffffu], Y[(op >> 16) & 0x7fffu], op & 0x80000000u);
                }
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
                    acc = csub(acc, cmul(Sr[j], Q[(c * nxi + i) * nxi + single]));
                } else {  // neutron: d pair (i, k=j) at slots 1, 3; u = single at slot 2
                    acc = cfma(Sr[i], Q[(c * nxi + single) * nxi + j], acc);
                    acc = csub(acc, cmul(Sr[j], Q[(c * nxi + single) * nxi + i]));
                }
            }
            F[e] = acc;
        }
    }
    __syncwarp();
}

template <class Tr>
__global__ void __launch_bounds__(1024, 1)
    k_small(SmallPlan P, FieldDesc F, MomDesc M, double2 *partial, int64_t n_tiles, int tiles_per_slab) {
    using V = typename Tr::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    V *R = reinterpret_cast<V *>(smem_raw) + (int64_t)warp * P.site_entries;
    double2 *Cs = reinterpret_cast<double2 *>(reinterpret_cast<V *>(smem_raw) + (int64_t)T * P.site_entries);
    double2 *Ph = Cs + T * P.n_comp;  // [T][n_mom]
    const int V3 = F.lx * F.ly * F.lz;
    const int nxi = P.nxi;

    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t slab = tile / tiles_per_slab;
        const int tin = (int)(tile % tiles_per_slab);
        const int cfg = (int)(slab / F.n_t), t = F.t0 + (int)(slab % F.n_t);
        const int site = tin * T + warp;
        const bool live = site < V3;
        if (live) {
            const int64_t base = cfg * F.stride_cfg + t * F.stride_t + (int64_t)site * 144;
            // 1. propagator tile (+ exact power-of-two scaling for MIXED)
            double2 sv[5];
            double amax = 0.0;
            int nent = nxi * nxi;
            for (int q = 0; q < 5; ++q) {
                int e = lane + 32 * q;
                sv[q] = make_double2(0, 0);
                if (e < nent) {
                    sv[q] = load_prop(F, base, (e / nxi) * 12 + (e % nxi));
                    amax = fmax(amax, fmax(fabs(sv[q].x), fabs(sv[q].y)));
                }
            }
            int sexp = 0;
            if (sizeof(V) == sizeof(float2)) {
                for (int off = 16; off > 0; off >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, off));
                sexp = amax > 0.0 ? -ilogb(amax) : 0;
            }
            for (int q = 0; q < 5; ++q) {
                int e = lane + 32 * q;
                if (e < nent) R[P.s_off + e] = Tr::from_d(make_double2(scalbn(sv[q].x, sexp), scalbn(sv[q].y, sexp)));
            }
            __syncwarp();
            // 2. blocks
            small_blocks<Tr>(P, R, lane);
            // 3. recursion
            for (int m = 0; m < P.n_steps; ++m) small_step<Tr>(P, P.step[m], R, lane);
            // 4. contraction with L, FP64, undo the scaling
            const V *FA = R + P.fin_off_buf;
            const int g = P.fin_g, per = 32 / g, sub = lane & (g - 1);
            for (int c0 = 0; c0 < P.n_comp; c0 += per) {
                int c = c0 + lane / g;
                double re = 0.0, im = 0.0;
                if (c < P.n_comp) {
                    for (int64_t e = P.fin_off[c] + sub; e < P.fin_off[c + 1]; e += g) {
                        double2 f = Tr::to_d(FA[__ldg(P.fin_z + e)]);
                        double l = __ldg(P.fin_l + e);
                        re = __fma_rn(l, f.x, re);
                        im = __fma_rn(l, f.y, im);
                    }
                }
                for (int off = g >> 1; off > 0; off >>= 1) {
                    re += __shfl_xor_sync(0xffffffffu, re, off);
                    im += __shfl_xor_sync(0xffffffffu, im, off);
                }
                if (c < P.n_comp && sub == 0) {
                    int ue = -3 * P.A * sexp;
                    Cs[warp * P.n_comp + c] = make_double2(scalbn(re * P.inv_norm, ue), scalbn(im * P.inv_norm, ue));
                }
            }
            // phases of this site
            int x = site % F.lx, y = (site / F.lx) % F.ly, z = site / (F.lx * F.ly);
            for (int q = lane; q < M.n_mom; q += 32) Ph[warp * M.n_mom + q] = mom_phase(M.mom[q], x, y, z, F.lx, F.ly, F.lz);
        } else {
            for (int c = lane; c < P.n_comp; c += 32) Cs[warp * P.n_comp + c] = make_double2(0, 0);
            for (int q = lane; q < M.n_mom; q += 32) Ph[warp * M.n_mom + q] = make_double2(0, 0);
        }
        __syncthreads();
        // tile partial: sum over the T sites in a fixed order
        for (int o = threadIdx.x; o < M.n_mom * P.n_comp; o += blockDim.x) {
            int q = o / P.n_comp, c = o % P.n_comp;
            double re = 0.0, im = 0.0;
            for (int w = 0; w < T; ++w) {
                double2 ph = Ph[w * M.n_mom + q], cv = Cs[w * P.n_comp + c];
                re += ph.x * cv.x - ph.y * cv.y;
                im += ph.x * cv.y + ph.y * cv.x;
            }
            partial[tile * (int64_t)(M.n_mom * P.n_comp) + o] = make_double2(re, im);
        }
        __syncthreads();
    }
}

}  // namespace mbc
