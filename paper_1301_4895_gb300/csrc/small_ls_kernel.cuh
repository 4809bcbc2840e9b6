// Shared-memory contraction kernel of the mixed path (lanes are sites). It
// shares the plan, batch and field descriptions of small_kernel.cuh and keeps
// its own source here, apart from the FP64 kernel.
#pragma once

#include "mixed_common.cuh"
#include "small_kernel.cuh"

namespace mbc {

// ---- lanes-are-sites kernel (mixed path) -------------------------------------
// A CTA owns a tile of 32 sites, lane l of every warp works on site l; all
// per-site values are rows of 32 lanes in shared memory ([entry][lane], 8 B
// per lane), so every access of a warp is one conflict-free row. The warps
// split the output components of each step; a warp's lanes decode 32
// operations at a time into the warp's records (the two row offsets, 8 B;
// an output's positive terms come first, so a ballot gives the batch's
// split into added and subtracted terms), which every lane then reads two
// at a time by broadcast; steps with fewer outputs than warps split each
// output's terms over several warps and combine the compensated partials in
// a fixed order. Shared memory: the site region and 64 partial rows of 32
// lanes, then the records (16 B per thread reserved, 8 B used).

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

// NXI > 0: every list of the batch has NXI quark index values (6 for the
// nonrelativistic operators), so the row-index arithmetic of the load,
// diquark and block phases divides by constants; NXI = 0 reads it from the plan.
template <class Tr, int NXI>
__global__ void __launch_bounds__(1024, 1)
    k_small_ls(const __grid_constant__ SmallBatch B, FieldDesc F, MomDesc M, const double2 *__restrict__ phase,
               double2 *partial_base) {
    using V = typename Tr::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *R = reinterpret_cast<V *>(smem_raw);  // [entry][32]
    __shared__ int sexp_s[32];
    const int NW = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // after the site region and the 64 partial rows: 32 operation records
    // (x and y row byte offsets, 8 B) per warp, read two at a time
    uint2 *rec = reinterpret_cast<uint2 *>(R + (int64_t)(B.site_stride + 64) * 32) + warp * 32;
    const uint4 *rec2 = reinterpret_cast<const uint4 *>(rec);
    const int V3 = F.lx * F.ly * F.lz;
    const unsigned full = 0xffffffffu;
    const int tiles_per_slab = B.tiles_per_slab;
#define ROW(e) R[(int64_t)(e) * 32 + lane]

    int64_t tile;
    for (int li0; (li0 = next_item(B, tile)) >= 0;) {  // next_item synchronises the CTA
        // a shared batch's item is a tile of every list: tile and blocks once
        const int l_end = B.shared ? B.n_lists : li0 + 1;
        const SmallPlan &P = B.plan[li0];
        const int32_t *need = B.shared ? B.need_union : P.need_blk;
        const int nxi = NXI > 0 ? NXI : P.nxi, nent = nxi * nxi;
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
        const int per_spin = (NXI > 0 ? NXI * (NXI - 1) / 2 : P.npair) * nxi;
        for (int b = 0; b < 2; ++b) {
            if (!need[b]) continue;
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
        for (int li = li0; li < l_end; ++li) {
            const SmallPlan &P = B.plan[li];
            double2 *partial = partial_base + B.partial_off[li];
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
                static_assert(sizeof(V) == 8, "a row of 32 lanes is 256 B");
                const char *Xb = reinterpret_cast<const char *>(R + (d.x_off << 5) + lane);
                const char *Yb = reinterpret_cast<const char *>(R + (d.y_off << 5) + lane);
                V *Zl = R + (d.z_off << 5) + lane;
                // output by output: each output's k terms are contiguous, decoded
                // 32 at a time into the warp's records; no per-term branch
                const int n_out = part < 0 ? (int)((o_end - o_begin) / d.k) : 1;
                const int len = part < 0 ? d.k : (int)(o_end - o_begin);
                const uint32_t *op_ptr = ops + o_begin;
                for (int zz = 0; zz < n_out; ++zz, op_ptr += len) {
                    for (int b0 = 0; b0 < len; b0 += 32) {
                        const int nb = min(32, len - b0);
                        // operands are byte offsets of 256 B rows, the sign is
                        // bit 0: decoded once per batch into the warp's records;
                        // an output's positive terms come first, so the batch's
                        // first npos terms are added and the rest subtracted
                        __syncwarp();
                        const uint32_t op = lane < nb ? __ldg(op_ptr + b0 + lane) : 0u;
                        if (lane < nb) rec[lane] = make_uint2(op & 0xff00u, op >> 16);
                        const int npos = nb - __popc(__ballot_sync(full, (op & 1u) != 0u));
                        __syncwarp();
#define LS_TERM(xo, yo, op_) acc.op_(*reinterpret_cast<const V *>(Xb + (xo)), *reinterpret_cast<const V *>(Yb + (yo)))
                        int q = 0;
#pragma unroll 2
                        for (; q + 1 < npos; q += 2) {
                            const uint4 r = rec2[q >> 1];
                            LS_TERM(r.x, r.y, add_prod);
                            LS_TERM(r.z, r.w, add_prod);
                        }
                        if (q < npos) {  // the last positive term, then possibly the first negative one
                            const uint4 r = rec2[q >> 1];
                            LS_TERM(r.x, r.y, add_prod);
                            if (q + 1 < nb) LS_TERM(r.z, r.w, sub_prod);
                            q += 2;
                        }
#pragma unroll 2
                        for (; q + 1 < nb; q += 2) {
                            const uint4 r = rec2[q >> 1];
                            LS_TERM(r.x, r.y, sub_prod);
                            LS_TERM(r.z, r.w, sub_prod);
                        }
                        if (q < nb) {
                            const uint2 r = rec[q];
                            LS_TERM(r.x, r.y, sub_prod);
                        }
#undef LS_TERM
                    }
                    if (part < 0) {
                        Zl[((int)zb + zz) << 5] = acc.store();
                        acc.zero();
                    }
                }
                if (split > 1) {
                    if (part >= 0) {
                        ROW(P.part_off + 2 * warp) = f2_unpack(acc.s);      // (sum re, sum im)
                        ROW(P.part_off + 2 * warp + 1) = f2_unpack(acc.n);  // their negated compensations
                    }
                    __syncthreads();
                    for (int zz = warp; zz < d.n_z; zz += NW) {
                        typename Tr::Acc a;
                        a.zero();
                        for (int pp = 0; pp < split; ++pp) {
                            const V r0 = ROW(P.part_off + 2 * (zz * split + pp));
                            const V r1 = ROW(P.part_off + 2 * (zz * split + pp) + 1);
                            a.add(r0.x, r1.x, r0.y, r1.y);
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
                    if (lane == 0)
                        partial[tile * (int64_t)(M.n_mom * P.n_comp) + q * P.n_comp + c] = make_double2(pr, pi);
                }
            }
            if (li + 1 < l_end) __syncthreads();  // the stages are read before the next list writes them
        }  // lists of the item
    }
#undef ROW
}

}  // namespace mbc
