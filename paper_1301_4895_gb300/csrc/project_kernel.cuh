// Momentum-projected blocks (Sec. 2: blocks carry a sink function s(x); here
// every baryon uses s(x) = exp(-2 pi i n.x / L)), then one recursion per
// (configuration, time slice, momentum) on the summed blocks.
//
//   k_project_blocks   per-site antisymmetric blocks in FP64, a chunk of
//                      entries at a time through shared memory, multiplied
//                      by the phase and summed over the 16 sites of a tile
//                      in a fixed order by one thread per (block, momentum,
//                      entry) -> tile partials, reduced over tiles by
//                      k_reduce_tiles (compensated, fixed order);
//   k_project_blocks_mx the same with FP32 products and compensated FP32
//                      sums (mixed precision), FP32 tile partials reduced by
//                      k_reduce_tiles_cols_mx;
//   k_load_proj_blocks copies the summed blocks of a wave of items into the
//                      [component][item] layout of the wave kernels (MIXED:
//                      exact power-of-two scaling per item);
//   k_write_items      writes each item's contracted components to out.
#pragma once

#include "large_kernel.cuh"

namespace mbc {

// Entries of a block chunk held in shared memory between the block pass and
// the phase-sum pass; the site index is padded to 17 so that the threads of
// the phase sum (consecutive entries) read distinct banks.
constexpr int kProjChunk = 128;
constexpr int kProjPad = 17;

// Shared memory of k_project_blocks for tiles of 16 sites.
inline size_t project_smem_bytes(int nrow, int nxi, int n_mom) {
    return sizeof(double2) * (16 * (size_t)tile_stride(nrow, nxi) + 16 * (size_t)diquark_stride(nxi) +
                              2 * (size_t)kProjChunk * kProjPad + 16 * (size_t)n_mom);
}

__global__ void __launch_bounds__(512) k_project_blocks(FieldDesc F, MomDesc M, const double2 *__restrict__ phase,
                                                        int nrow, int nxi, int n_g2, int block_size, int npair,
                                                        int need_p,
                                                        int need_n, int tiles_per_slab, int64_t n_tiles,
                                                        double2 *__restrict__ partial) {
    constexpr int NS = 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int sst = tile_stride(nrow, nxi), qst = diquark_stride(nxi);
    double2 *S = reinterpret_cast<double2 *>(smem_raw);  // [NS][sst]
    double2 *Q = S + NS * sst;                    // [NS][3*nxi*nxi]
    double2 *Fb = Q + NS * qst;                          // [2][kProjChunk][kProjPad]: block values of the chunk
    double2 *Ph = Fb + 2 * kProjChunk * kProjPad;        // [NS][n_mom]: the tile's phases
    const int sl = threadIdx.x % NS, slice = threadIdx.x / NS, nslice = blockDim.x / NS;
    const int nent = nrow * nxi, nq = nxi * nxi;
    const int v3 = F.lx * F.ly * F.lz;
    const int n_out = 2 * block_size;  // proton block, then neutron block
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t slab = tile / tiles_per_slab;
        const int tin = (int)(tile % tiles_per_slab);
        const int cfg = (int)(slab / F.n_t), t = F.t0 + (int)(slab % F.n_t);
        __syncthreads();  // shared memory of the previous tile is free
        for (int s = threadIdx.x >> 5; s < NS; s += blockDim.x >> 5) {
            const int lane = threadIdx.x & 31;
            const int site = tin * NS + s;
            const bool live = site < v3;
            const int64_t base = cfg * F.stride_cfg + t * F.stride_t + (int64_t)site * site_elems(F);
            for (int e = lane; e < nent; e += 32)
                S[s * sst + e] = live ? load_prop(F, base, tile_index(F, e, nxi)) : make_double2(0, 0);
        }
        for (int o = threadIdx.x; o < NS * M.n_mom; o += blockDim.x) {
            const int site = tin * NS + o / M.n_mom;
            Ph[o] = site < v3 ? __ldg(phase + (int64_t)site * M.n_mom + o % M.n_mom) : make_double2(0, 0);
        }
        __syncthreads();
        for (int e = slice; e < 3 * nq; e += nslice) {
            const int c = e / nq, r = e % nq;
            Q[sl * qst + e] = diquark(S + sl * sst, nxi, nxi, n_g2, c, r / nxi, r % nxi);
        }
        __syncthreads();
        const int site = tin * NS + sl;
        const bool live = site < v3;
        const double2 *Ss = S + sl * sst;
        const double2 *Qs = Q + sl * qst;
        const int per_spin = npair * nxi;
        for (int e0 = 0; e0 < block_size; e0 += kProjChunk) {
            // 1. block values of the chunk's entries for the tile's sites
            for (int el = slice; el < kProjChunk; el += nslice) {
                const int e = e0 + el;
                const bool ok = live && e < block_size;
                const int dl = e / per_spin, r = e % per_spin;
                const int pr = r / nxi, single = r % nxi;
                const int i = ok ? c_pair_i[pr] : 0, j = ok ? c_pair_j[pr] : 0;
                for (int b = 0; b < 2; ++b) {
                    double2 f = make_double2(0, 0);
                    if (ok && (b == 0 ? need_p : need_n)) {
                        for (int c = 0; c < 3; ++c) {
                            const double2 *Sr = Ss + (3 * dl + c) * nxi;
                            if (b == 0) {
                                f = cfma(Sr[i], Qs[(c * nxi + j) * nxi + single], f);
                                f = cfms(Sr[j], Qs[(c * nxi + i) * nxi + single], f);
                            } else {
                                f = cfma(Sr[i], Qs[(c * nxi + single) * nxi + j], f);
                                f = cfms(Sr[j], Qs[(c * nxi + single) * nxi + i], f);
                            }
                        }
                    }
                    Fb[(b * kProjChunk + el) * kProjPad + sl] = f;
                }
            }
            __syncthreads();
            // 2. phase-weighted sums over the tile's 16 sites in a fixed order,
            //    one (block, momentum, entry) per thread
            for (int o = threadIdx.x; o < 2 * M.n_mom * kProjChunk; o += blockDim.x) {
                const int el = o % kProjChunk, q = (o / kProjChunk) % M.n_mom, b = o / (kProjChunk * M.n_mom);
                const int e = e0 + el;
                if (e >= block_size) continue;
                const double2 *fv = Fb + (b * kProjChunk + el) * kProjPad;
                double re = 0.0, im = 0.0;
                for (int w = 0; w < NS; ++w) {
                    const double2 ph = Ph[w * M.n_mom + q], f = fv[w];
                    re = __fma_rn(ph.x, f.x, __fma_rn(-ph.y, f.y, re));
                    im = __fma_rn(ph.x, f.y, __fma_rn(ph.y, f.x, im));
                }
                partial[(tile * M.n_mom + q) * (int64_t)n_out + b * block_size + e] = make_double2(re, im);
            }
            __syncthreads();  // the chunk's values are consumed
        }
    }
}

// Shared memory of k_project_blocks_mx (FP32 values) for tiles of 16 sites.
inline size_t project_smem_bytes_mx(int nrow, int nxi, int n_mom) {
    return sizeof(float2) * (16 * (size_t)tile_stride(nrow, nxi) + 16 * (size_t)diquark_stride(nxi) +
                             2 * (size_t)kProjChunk * kProjPad + 16 * (size_t)n_mom);
}

// The same projection for the mixed path: the tile, the diquark and the
// blocks in FP32 products, the phase-weighted sum over the tile's 16 sites
// with compensated (two-word) FP32 accumulation in the same fixed order, the
// tile partial rounded once to FP32 for the reduction over tiles. The number of
// quark-index columns is a template parameter (6 or 12), so the decoding
// of an entry into (spin, pair, single) divides by constants.
template <int NXI>
__global__ void __launch_bounds__(512) k_project_blocks_mx(FieldDesc F, MomDesc M, const double2 *__restrict__ phase,
                                                           int nrow, int n_g2, int block_size, int need_p, int need_n,
                                                           int tiles_per_slab, int64_t n_tiles,
                                                           float2 *__restrict__ partial) {
    constexpr int NS = 16;
    constexpr int nxi = NXI, npair = NXI * (NXI - 1) / 2;
    using Acc = MixedTraits::Acc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int sst = tile_stride(nrow, nxi), qst = diquark_stride(nxi);
    float2 *S = reinterpret_cast<float2 *>(smem_raw);  // [NS][sst]
    float2 *Q = S + NS * sst;                   // [NS][3*nxi*nxi]
    float2 *Fb = Q + NS * qst;                         // [2][kProjChunk][kProjPad]
    float2 *Ph = Fb + 2 * kProjChunk * kProjPad;       // [NS][n_mom]
    const int sl = threadIdx.x % NS, slice = threadIdx.x / NS, nslice = blockDim.x / NS;
    const int nent = nrow * nxi, nq = nxi * nxi;
    const int v3 = F.lx * F.ly * F.lz;
    const int n_out = 2 * block_size;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t slab = tile / tiles_per_slab;
        const int tin = (int)(tile % tiles_per_slab);
        const int cfg = (int)(slab / F.n_t), t = F.t0 + (int)(slab % F.n_t);
        __syncthreads();  // shared memory of the previous tile is free
        for (int s = threadIdx.x >> 5; s < NS; s += blockDim.x >> 5) {
            const int lane = threadIdx.x & 31;
            const int site = tin * NS + s;
            const bool live = site < v3;
            const int64_t base = cfg * F.stride_cfg + t * F.stride_t + (int64_t)site * site_elems(F);
            for (int e = lane; e < nent; e += 32) {
                const double2 v = live ? load_prop(F, base, tile_index(F, e, nxi)) : make_double2(0, 0);
                S[s * sst + e] = make_float2((float)v.x, (float)v.y);
            }
        }
        for (int o = threadIdx.x; o < NS * M.n_mom; o += blockDim.x) {
            const int site = tin * NS + o / M.n_mom;
            const double2 p = site < v3 ? __ldg(phase + (int64_t)site * M.n_mom + o % M.n_mom) : make_double2(0, 0);
            Ph[o] = make_float2((float)p.x, (float)p.y);
        }
        __syncthreads();
        for (int e = slice; e < 3 * nq; e += nslice) {
            const int c = e / nq, r = e % nq;
            Q[sl * qst + e] = diquark(S + sl * sst, nxi, nxi, n_g2, c, r / nxi, r % nxi);
        }
        __syncthreads();
        const int site = tin * NS + sl;
        const bool live = site < v3;
        const float2 *Ss = S + sl * sst;
        const float2 *Qs = Q + sl * qst;
        const int per_spin = npair * nxi;
        for (int e0 = 0; e0 < block_size; e0 += kProjChunk) {
            for (int el = slice; el < kProjChunk; el += nslice) {
                const int e = e0 + el;
                const bool ok = live && e < block_size;
                const int dl = e / per_spin, r = e % per_spin;
                const int pr = r / nxi, single = r % nxi;
                const int i = ok ? c_pair_i[pr] : 0, j = ok ? c_pair_j[pr] : 0;
                for (int b = 0; b < 2; ++b) {
                    float2 f = make_float2(0.f, 0.f);
                    if (ok && (b == 0 ? need_p : need_n)) {
                        for (int c = 0; c < 3; ++c) {
                            const float2 *Sr = Ss + (3 * dl + c) * nxi;
                            if (b == 0) {
                                f = cfma(Sr[i], Qs[(c * nxi + j) * nxi + single], f);
                                f = cfms(Sr[j], Qs[(c * nxi + i) * nxi + single], f);
                            } else {
                                f = cfma(Sr[i], Qs[(c * nxi + single) * nxi + j], f);
                                f = cfms(Sr[j], Qs[(c * nxi + single) * nxi + i], f);
                            }
                        }
                    }
                    Fb[(b * kProjChunk + el) * kProjPad + sl] = f;
                }
            }
            __syncthreads();
            for (int o = threadIdx.x; o < 2 * M.n_mom * kProjChunk; o += blockDim.x) {
                const int el = o % kProjChunk, q = (o / kProjChunk) % M.n_mom, b = o / (kProjChunk * M.n_mom);
                const int e = e0 + el;
                if (e >= block_size) continue;
                const float2 *fv = Fb + (b * kProjChunk + el) * kProjPad;
                Acc acc;
                acc.zero();
                for (int w = 0; w < NS; ++w) acc.fma(Ph[w * M.n_mom + q], fv[w], 0u);
                partial[(tile * M.n_mom + q) * (int64_t)n_out + b * block_size + e] = acc.store();
            }
            __syncthreads();
        }
    }
}

// The reduction over tiles of the mixed projection: one thread per output
// (consecutive threads, consecutive outputs: coalesced) adds the slab's FP32
// tile partials in tile order with a packed Kahan step on (re, im); the sum
// goes out in FP64, Pf[slab][per_slab].
__global__ void __launch_bounds__(256) k_reduce_tiles_cols_mx(const float2 *__restrict__ partial, int64_t n_slabs,
                                                              int tiles_per_slab, int64_t per_slab,
                                                              double2 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_slabs * per_slab; o += stride) {
        const int64_t slab = o / per_slab, r = o % per_slab;
        const float2 *p = partial + slab * tiles_per_slab * per_slab + r;
        MixedTraits::Acc acc;
        acc.zero();
#pragma unroll 4
        for (int tl = 0; tl < tiles_per_slab; ++tl) {
            const float2 v = __ldg(p + (int64_t)tl * per_slab);
            f2_kahan(acc.s, acc.n, f2_pack(v.x, v.y));
        }
        out[o] = acc.value();
    }
}

// One warp per item of the wave: summed blocks -> wave layout. An item is
// (slab, group of n_k momenta); with n_k sink functions (Sec. 6) the sink
// index of the item's block is psi = n_k * alpha + k, and block entry
// (psi; pair, single) is entry (alpha; pair, single) of the block projected
// with momentum k of the group. Pf: [slab][momentum][P block, N block] with
// bs_site entries per block (one sink function).
template <class Tr>
__global__ void __launch_bounds__(256) k_load_proj_blocks(const double2 *__restrict__ Pf, int64_t n_items,
                                                          int64_t item0, int W, int bs_site, int per_spin, int n_k,
                                                          int n_mom, typename Tr::V *__restrict__ fP,
                                                          typename Tr::V *__restrict__ fN, int32_t *__restrict__ sexp) {
    const int lane = threadIdx.x & 31;
    const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (col >= W) return;
    const int64_t item = item0 + col;
    const bool live = item < n_items;
    const int n_groups = n_mom / n_k;
    const int64_t it = live ? item : 0;
    const int64_t slab = it / n_groups;
    const int q0 = (int)(it % n_groups) * n_k;
    const double2 *src = Pf + (slab * n_mom + q0) * 2 * (int64_t)bs_site;  // n_k consecutive momenta
    const int block_size = bs_site * n_k;
    int se = 0;
    if (sizeof(typename Tr::V) == sizeof(float2)) {
        double amax = 0.0;
        for (int e = lane; live && e < 2 * block_size; e += 32) {
            const double2 v = src[e];
            amax = fmax(amax, fmax(fabs(v.x), fabs(v.y)));
        }
        for (int off = 16; off > 0; off >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, off));
        se = amax > 0.0 ? -ilogb(amax) : 0;
    }
    for (int e = lane; e < block_size; e += 32) {
        const int psi = e / per_spin, r = e % per_spin;
        const int k = psi % n_k, alpha = psi / n_k;
        const double2 *s_k = src + (int64_t)k * 2 * bs_site + alpha * per_spin + r;
        const double2 p = live ? s_k[0] : make_double2(0, 0);
        const double2 n = live ? s_k[bs_site] : make_double2(0, 0);
        Tr::wave_st(fP, (int64_t)e * W + col, Tr::from_d(make_double2(scalbn(p.x, se), scalbn(p.y, se))));
        Tr::wave_st(fN, (int64_t)e * W + col, Tr::from_d(make_double2(scalbn(n.x, se), scalbn(n.y, se))));
    }
    if (lane == 0) sexp[col] = se;
}

// out[cfg][list][t - t0][mom][comp_stride] = C[comp][item] for the wave's items
// (n_mom: items per slab)
__global__ void k_write_items(const double2 *__restrict__ C, int64_t n_items, int64_t item0, int W, int n_comp,
                              int n_mom, int n_t, int list_idx, int n_lists, int comp_stride, double2 *out) {
    const int64_t total = (int64_t)n_comp * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / W), col = (int)(i % W);
        const int64_t item = item0 + col;
        if (item >= n_items) continue;
        const int64_t slab = item / n_mom;
        const int q = (int)(item % n_mom);
        const int cfg = (int)(slab / n_t), tt = (int)(slab % n_t);
        out[((((int64_t)cfg * n_lists + list_idx) * n_t + tt) * n_mom + q) * comp_stride + c] = C[i];
    }
}

}  // namespace mbc
