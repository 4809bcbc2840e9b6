// Large-stage contraction kernels (relativistic nuclei: blocks of 3168
// components, stages up to millions of components per site, Sec. 7 P bound
// with D = 4). Stage buffers live in device scratch with the layout
// [component][wave site], so consecutive sites of one component are one
// coalesced row (mixed precision: sites in planar pairs, MixedTraits::wave_ld);
// a "wave" of W sites (a multiple of 64) is processed by the whole GPU one step
// at a time, and each step streams its term list once per wave. Lanes are
// sites; a warp walks the z-major list of its chunk with warp-uniform
// (x, y, sign) operands that the lanes load cooperatively and broadcast.
#pragma once

#include "async_copy.cuh"
#include "device_common.cuh"
#include "gen_ops.cuh"
#include "mixed_common.cuh"
#include "small_kernel.cuh"

namespace mbc {

struct WaveDesc {
    int64_t item0;         // first padded site item of the wave
    int32_t W;             // sites in the wave (multiple of 32)
    int32_t v3;            // sites per slab
    int32_t v3p;           // padded sites per slab (multiple of 32)
    int64_t n_items;       // total padded items
};

__device__ __forceinline__ bool item_site(const FieldDesc &F, const WaveDesc &wv, int64_t item, int &cfg, int &t,
                                          int &site) {
    if (item >= wv.n_items) return false;
    int64_t slab = item / wv.v3p;
    site = (int)(item % wv.v3p);
    cfg = (int)(slab / F.n_t);
    t = F.t0 + (int)(slab % F.n_t);
    return site < wv.v3;
}

// Per-site regions of the block kernels' shared memory are padded by one
// element: the 16 sites of a warp then read the same entry from 16 distinct
// banks (an unpadded 12 x 12 tile puts all of them in one bank).
__host__ __device__ constexpr int tile_stride(int nrow, int nxi) { return nrow * nxi + 1; }
__host__ __device__ constexpr int diquark_stride(int nxi) { return 3 * nxi * nxi + 1; }

// Blocks for NS sites per CTA (512 threads): thread = (site lane, entry
// slice). The tile of a site has nrow sink rows (3 x Dirac dimension) and nxi
// source columns (quark index over all sources, up to 24: two relativistic
// sources, Sec. 6); NS = 4 for 24 columns keeps the tiles and diquarks in
// shared memory.
constexpr int kTileLoads = 9;  // tile entries per lane: 12 x 24 / 32

template <class Tr, int NS>
__global__ void __launch_bounds__(512) k_large_blocks(FieldDesc F, WaveDesc wv, int nrow, int nxi, int n_g2,
                                                      int block_size, int npair, int need_p, int need_n,
                                                      typename Tr::V *fP, typename Tr::V *fN, int32_t *sexp_out) {
    using V = typename Tr::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int sst = tile_stride(nrow, nxi), qst = diquark_stride(nxi);
    V *S = reinterpret_cast<V *>(smem_raw);  // [NS][sst]: nrow*nxi entries each
    V *Q = S + NS * sst;                     // [NS][qst]: 3*nxi*nxi entries each
    const int sl = threadIdx.x % NS, slice = threadIdx.x / NS, nslice = blockDim.x / NS;
    const int w0 = blockIdx.x * NS;  // first site of this CTA within the wave
    const int nent = nrow * nxi, nq = nxi * nxi;
    // load + scale: one warp per site
    for (int s = threadIdx.x >> 5; s < NS; s += blockDim.x >> 5) {
        int lane = threadIdx.x & 31;
        int cfg, t, site;
        bool live = item_site(F, wv, wv.item0 + w0 + s, cfg, t, site);
        int64_t base = live ? cfg * F.stride_cfg + t * F.stride_t + (int64_t)site * site_elems(F) : 0;
        double2 sv[kTileLoads];
        double amax = 0.0;
#pragma unroll
        for (int q = 0; q < kTileLoads; ++q) {
            int e = lane + 32 * q;
            sv[q] = make_double2(0, 0);
            if (live && e < nent) {
                sv[q] = load_prop(F, base, tile_index(F, e, nxi));
                amax = fmax(amax, fmax(fabs(sv[q].x), fabs(sv[q].y)));
            }
        }
        int se = 0;
        if (sizeof(V) == sizeof(float2)) {
            for (int off = 16; off > 0; off >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, off));
            se = amax > 0.0 ? -ilogb(amax) : 0;
        }
#pragma unroll
        for (int q = 0; q < kTileLoads; ++q) {
            int e = lane + 32 * q;
            if (e < nent) S[s * sst + e] = Tr::from_d(make_double2(scalbn(sv[q].x, se), scalbn(sv[q].y, se)));
        }
        if (lane == 0) sexp_out[w0 + s] = se;
    }
    __syncthreads();
    for (int e = slice; e < 3 * nq; e += nslice) {
        int c = e / nq, r = e % nq;
        Q[sl * qst + e] = diquark(S + sl * sst, nxi, nxi, n_g2, c, r / nxi, r % nxi);
    }
    __syncthreads();
    const V *Ss = S + sl * sst;
    const V *Qs = Q + sl * qst;
    const int per_spin = npair * nxi;
    for (int b = 0; b < 2; ++b) {
        if (b == 0 ? !need_p : !need_n) continue;
        V *out = b == 0 ? fP : fN;
        for (int e = slice; e < block_size; e += nslice) {
            int dl = e / per_spin, r = e % per_spin;
            int pr = r / nxi, single = r % nxi;
            int i = c_pair_i[pr], j = c_pair_j[pr];
            V acc{0, 0};
            for (int c = 0; c < 3; ++c) {
                const V *Sr = Ss + (3 * dl + c) * nxi;
                if (b == 0) {
                    acc = cfma(Sr[i], Qs[(c * nxi + j) * nxi + single], acc);
                    acc = cfms(Sr[j], Qs[(c * nxi + i) * nxi + single], acc);
                } else {
                    acc = cfma(Sr[i], Qs[(c * nxi + single) * nxi + j], acc);
                    acc = cfms(Sr[j], Qs[(c * nxi + single) * nxi + i], acc);
                }
            }
            Tr::wave_st(out, (int64_t)e * wv.W + w0 + sl, acc);
        }
    }
}

// One recursion step (eq. recr_F) for a whole wave. Work item = (z chunk,
// 32-site group), site group fastest so that concurrent warps share list
// entries and nearby rows of X. LF: every warp regenerates the operations of
// its outputs (gen_ops.cuh), one per lane per 32, instead of reading opx /
// opy; on the FP64 pipe the integer work of one warp hides under the other
// warps' DFMAs (the mixed path shares it per CTA instead, k_large_step_gen).
template <class Tr, bool LF>
__global__ void __launch_bounds__(256) k_large_step(const uint32_t *__restrict__ opx, const uint16_t *__restrict__ opy,
                                                    GenStep gs, int64_t n_z, int64_t k, int64_t zchunk, int W,
                                                    int order, const typename Tr::V *__restrict__ X,
                                                    const typename Tr::V *__restrict__ Y, typename Tr::V *__restrict__ Z) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int ngroups = W >> 5;
    const int64_t nchunks = (n_z + zchunk - 1) / zchunk;
    const int wpb = blockDim.x >> 5;
    for (int64_t item = warp_global; item < nchunks * ngroups; item += nwarps) {
        // order 0: consecutive warps take the site groups of one chunk (they
        // share op words); order 1: the warps of a CTA take consecutive chunks
        // of one site group (they share rows of X and Y in L1)
        int64_t chunk;
        int group;
        if (order == 0 || nchunks % wpb != 0) {
            chunk = item / ngroups;
            group = (int)(item % ngroups);
        } else {
            const int64_t blk = item / wpb;
            group = (int)(blk % ngroups);
            chunk = (blk / ngroups) * wpb + item % wpb;
        }
        const int col = group * 32 + lane;
        const int64_t z_begin = chunk * zchunk;
        const int64_t z_end = min(n_z, z_begin + zchunk);
        const typename Tr::V *Xc = X + col;
        const typename Tr::V *Yc = Y + col;
        // output by output: its k terms are contiguous; 32 operand words are
        // loaded at once and broadcast, the loop body has no branch so the
        // gathers of several terms are in flight together
        for (int64_t z = z_begin; z < z_end; ++z) {
            typename Tr::Acc acc;
            acc.zero();
            const uint32_t *ox = LF ? nullptr : opx + z * k;
            const uint16_t *oy = LF ? nullptr : opy + z * k;
            uint32_t zkey[4];
            if (LF) g_key(gs, z, zkey);
            for (int64_t b0 = 0; b0 < k; b0 += 32) {
                const int nb = (int)min((int64_t)32, k - b0);
                uint32_t mx = 0, my = 0;
                if (lane < nb) {
                    if (LF) {
                        g_op(gs, zkey, b0 + lane, mx, my);
                    } else {
                        mx = __ldg(ox + b0 + lane);
                        my = __ldg(oy + b0 + lane);
                    }
                }
                // G terms' gathers are issued before their multiply-adds so that
                // several L2 round trips overlap (FP32: 4 terms, FP64: 2)
                constexpr int G = sizeof(typename Tr::V) == 8 ? 4 : 2;
                for (int t0 = 0; t0 < nb; t0 += G) {
                    typename Tr::V xv[G], yv[G];
                    uint32_t sg[G];
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const uint32_t x = __shfl_sync(0xffffffffu, mx, (t0 + g) & 31);
                        const uint32_t y = __shfl_sync(0xffffffffu, my, (t0 + g) & 31);
                        if (t0 + g < nb) {
                            xv[g] = __ldg(Xc + (int64_t)x * W);
                            yv[g] = __ldg(Yc + (int64_t)(y & 0x7fffu) * W);
                        }
                        sg[g] = (y & 0x8000u) << 16;
                    }
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        if (t0 + g < nb) acc.fma(xv[g], yv[g], sg[g]);
                }
            }
            Z[z * W + col] = acc.store();
        }
    }
}

// The mixed-precision step with two sites per lane: a warp covers 64
// consecutive sites of the wave, every gather is one 16 B load per lane
// (a 512 B row segment per warp), and both sites' products and compensated
// sums are packed FP32-pair instructions (PairAcc). The lanes decode 32
// operations at a time into per-warp shared-memory records (x, y, sign,
// sign), so a term costs one broadcast shared load, one multiply-add per
// operand address, two gathers and the arithmetic. W must be a multiple of 64.
__device__ __forceinline__ OpRec op_rec(uint32_t x, uint32_t y) {
    return OpRec{x, y & 0x7fffu, f2_sign_pair((y & 0x8000u) != 0)};
}

template <int G>
__device__ __forceinline__ void pair_terms(const OpRec *rec, int n, const unsigned char *Xc, const unsigned char *Yc,
                                           uint32_t row_bytes, PairAcc &acc) {
    int t = 0;
    for (; t + G <= n; t += G) {
        ulonglong2 xv[G], yv[G];
        uint64_t sg[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const OpRec r = rec[t + g];
            xv[g] = __ldg(reinterpret_cast<const ulonglong2 *>(Xc + (size_t)r.x * row_bytes));
            yv[g] = __ldg(reinterpret_cast<const ulonglong2 *>(Yc + (size_t)r.y * row_bytes));
            sg[g] = r.sg;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) acc.fma(xv[g], yv[g], sg[g]);
    }
    for (; t < n; ++t) {
        const OpRec r = rec[t];
        acc.fma(__ldg(reinterpret_cast<const ulonglong2 *>(Xc + (size_t)r.x * row_bytes)),
                __ldg(reinterpret_cast<const ulonglong2 *>(Yc + (size_t)r.y * row_bytes)), r.sg);
    }
}

template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS, WARPS == 8 ? 4 : 1)
    k_large_step_mx2(const uint32_t *__restrict__ opx, const uint16_t *__restrict__ opy, int64_t n_z, int64_t k,
                     int64_t zchunk, int W, int order, const float2 *__restrict__ X, const float2 *__restrict__ Y,
                     float2 *__restrict__ Z) {
    __shared__ OpRec recs[WARPS][32];
    const int lane = threadIdx.x & 31;
    OpRec *rec = recs[threadIdx.x >> 5];
    const int64_t warp_global = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * WARPS;
    const int ngroups = W >> 6;
    const int64_t nchunks = (n_z + zchunk - 1) / zchunk;
    const uint32_t row_bytes = (uint32_t)W * (uint32_t)sizeof(float2);
    for (int64_t item = warp_global; item < nchunks * ngroups; item += nwarps) {
        // order 0: consecutive warps take the site groups of one chunk (they
        // share operation words); order 1: the warps of a CTA take
        // consecutive chunks of one site group (they share rows of X and Y)
        int64_t chunk;
        int group;
        if (order == 0 || nchunks % WARPS != 0) {
            chunk = item / ngroups;
            group = (int)(item % ngroups);
        } else {
            const int64_t blk = item / WARPS;
            group = (int)(blk % ngroups);
            chunk = (blk / ngroups) * WARPS + item % WARPS;
        }
        const int col4 = group * 32 + lane;  // float4 column: sites 2 col4, 2 col4 + 1
        const unsigned char *Xc = reinterpret_cast<const unsigned char *>(reinterpret_cast<const float4 *>(X) + col4);
        const unsigned char *Yc = reinterpret_cast<const unsigned char *>(reinterpret_cast<const float4 *>(Y) + col4);
        const int64_t z_begin = chunk * zchunk;
        const int64_t z_end = min(n_z, z_begin + zchunk);
        for (int64_t z = z_begin; z < z_end; ++z) {
            PairAcc acc;
            acc.zero();
            const uint32_t *ox = opx + z * k;
            const uint16_t *oy = opy + z * k;
            for (int64_t b0 = 0; b0 < k; b0 += 32) {
                const int nb = (int)min((int64_t)32, k - b0);
                __syncwarp();  // the previous records are consumed
                if (lane < nb) rec[lane] = op_rec(__ldg(ox + b0 + lane), __ldg(oy + b0 + lane));
                __syncwarp();
                pair_terms<4>(rec, nb, Xc, Yc, row_bytes, acc);
            }
            reinterpret_cast<ulonglong2 *>(Z + z * W)[col4] = acc.store();
        }
    }
}

// The mixed step with one CTA of WARPS warps per SM, G gathers in flight per
// warp, and the terms of an output split over S warps (S = 1, 2, 4, ...,
// WARPS / 2): the CTA takes WARPS / S consecutive
// (output, 64-site group) pairs at a time, warp w works on pair w / S and
// its term range (w mod S) of k / S terms with a PairAcc (two sites per
// lane, as k_large_step_mx2). Each further warp of an output rounds its
// compensated partial sum to FP32 (the stored stage value is FP32 too) and
// passes it through its operation-record buffer; the output's first warp adds
// them to its own compensated sum in a fixed order (two-sum, the errors
// joining the compensation). No shared memory beyond the records: L1 keeps
// its room for the rows of X. Few outputs are in flight at once, so the rows
// they name stay in L2 even when their number per output is large; S = 1
// is k_large_step_mx2's order with one output per item. W must be a
// multiple of 64.
template <int WARPS, int G>
__global__ void __launch_bounds__(32 * WARPS, 1)
    k_large_step_split(const uint32_t *__restrict__ opx, const uint16_t *__restrict__ opy, int64_t n_z, int64_t k,
                       int S, int W, const float2 *__restrict__ X, const float2 *__restrict__ Y,
                       float2 *__restrict__ Z) {
    __shared__ OpRec recs[WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    OpRec *rec = recs[warp];
    const int opc = WARPS / S, oo = warp / S, seg = warp % S;
    const int ngroups = W >> 6;
    // outputs (z, site group) numbered with the group fastest; a CTA item is
    // WARPS / S consecutive ones (the measured-fastest order: a few outputs
    // across all site groups per CTA)
    const int64_t n_out = n_z * ngroups;
    const int64_t n_items = (n_out + opc - 1) / opc;
    const int64_t j0 = k * seg / S, j1 = k * (seg + 1) / S;
    const uint32_t row_bytes = (uint32_t)W * (uint32_t)sizeof(float2);
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int64_t o = item * opc + oo;
        const bool live = o < n_out;
        const int64_t z = live ? o / ngroups : 0;
        const int group = (int)(o % ngroups);
        const int col4 = group * 32 + lane;  // float4 column: sites 2 col4, 2 col4 + 1
        PairAcc acc;
        acc.zero();
        if (live) {
            const unsigned char *Xc =
                reinterpret_cast<const unsigned char *>(reinterpret_cast<const float4 *>(X) + col4);
            const unsigned char *Yc =
                reinterpret_cast<const unsigned char *>(reinterpret_cast<const float4 *>(Y) + col4);
            const uint32_t *ox = opx + z * k;
            const uint16_t *oy = opy + z * k;
            for (int64_t b0 = j0; b0 < j1; b0 += 32) {
                const int nb = (int)min((int64_t)32, j1 - b0);
                __syncwarp();  // the previous records are consumed
                if (lane < nb) rec[lane] = op_rec(__ldg(ox + b0 + lane), __ldg(oy + b0 + lane));
                __syncwarp();
                pair_terms<G>(rec, nb, Xc, Yc, row_bytes, acc);
            }
        }
        if (S == 1) {
            if (live) reinterpret_cast<ulonglong2 *>(Z + z * W)[col4] = acc.store();
            continue;
        }
        __syncthreads();  // every warp is done with its records
        ulonglong2 *mine = reinterpret_cast<ulonglong2 *>(recs[warp]);
        if (seg != 0) mine[lane] = acc.store();
        __syncthreads();
        if (seg == 0 && live) {
            for (int p = 1; p < S; ++p)
                acc.add(reinterpret_cast<const ulonglong2 *>(recs[warp + p])[lane], make_ulonglong2(0ull, 0ull));
            reinterpret_cast<ulonglong2 *>(Z + z * W)[col4] = acc.store();
        }
        __syncthreads();  // the partials are read before the next item's records overwrite them
    }
}

// The mixed step with the block rows staged in shared memory. The outputs
// of a stored step are cut, on the host, into runs of consecutive outputs
// whose operations name at most kYcRows distinct block rows f[y]; an
// operation's y is replaced by its row's slot in the run. A CTA takes
// (run, 64-site group) items: one thread copies the run's rows for the
// group (512 B each: 64 sites of FP32 complex in planar pairs) into shared
// memory with bulk asynchronous copies completing on an mbarrier, then the
// warps take the run's outputs, two sites per lane as in k_large_step_mx2,
// and per term gather only X[x] (a 512 B row segment) while f[y] is a
// conflict-free shared-memory read. Same terms in the same order with the
// same arithmetic as k_large_step_mx2: bitwise equal results. W must be a
// multiple of 64.
constexpr int kYcRows = 384;

template <int G>
__device__ __forceinline__ void yc_terms(const OpRec *rec, int n, const unsigned char *Xc, const unsigned char *Ys,
                                         uint32_t row_bytes, PairAcc &acc) {
    int t = 0;
    for (; t + G <= n; t += G) {
        ulonglong2 xv[G];
#pragma unroll
        for (int g = 0; g < G; ++g)
            xv[g] = __ldg(reinterpret_cast<const ulonglong2 *>(Xc + (size_t)rec[t + g].x * row_bytes));
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const OpRec r = rec[t + g];
            acc.fma(xv[g], *reinterpret_cast<const ulonglong2 *>(Ys + r.y), r.sg);
        }
    }
    for (; t < n; ++t) {
        const OpRec r = rec[t];
        acc.fma(__ldg(reinterpret_cast<const ulonglong2 *>(Xc + (size_t)r.x * row_bytes)),
                *reinterpret_cast<const ulonglong2 *>(Ys + r.y), r.sg);
    }
}

template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS, 1)
    k_large_step_yc(const uint32_t *__restrict__ opx, const uint16_t *__restrict__ oslot,
                    const uint32_t *__restrict__ run_z0, const uint32_t *__restrict__ run_y0,
                    const uint16_t *__restrict__ run_rows, int64_t n_runs, int64_t k, int W, uint32_t wait_limit,
                    const float2 *__restrict__ X, const float2 *__restrict__ Y, float2 *__restrict__ Z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *rows = smem_raw;                                      // [kYcRows][512 B]
    OpRec *recs = reinterpret_cast<OpRec *>(smem_raw + (size_t)kYcRows * 512);  // [WARPS][32]
    uint64_t *bar = reinterpret_cast<uint64_t *>(recs + WARPS * 32);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    OpRec *rec = recs + warp * 32;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    const int ngroups = W >> 6;
    const uint32_t row_bytes = (uint32_t)W * (uint32_t)sizeof(float2);
    uint32_t parity = 0;
    for (int64_t item = blockIdx.x; item < n_runs * ngroups; item += gridDim.x) {
        const int64_t r = item / ngroups;
        const int group = (int)(item % ngroups);
        if (threadIdx.x == 0) {
            const uint32_t y0 = __ldg(run_y0 + r), ny = __ldg(run_y0 + r + 1) - y0;
            fence_proxy_async_smem();  // the previous run's rows were read through the generic proxy
            mbar_arrive_expect_tx(bar, ny * 512u);
            const unsigned char *Yg = reinterpret_cast<const unsigned char *>(Y) + (size_t)group * 512;
            for (uint32_t i = 0; i < ny; ++i)
                bulk_copy_g2s(rows + (size_t)i * 512, Yg + (size_t)__ldg(run_rows + y0 + i) * row_bytes, 512u, bar);
        }
        const bool ok = mbar_wait_bounded(bar, parity, wait_limit);
        if (__syncthreads_or(!ok)) {
            // the status word is set; let copies in flight land, then leave
            mbar_wait_bounded(bar, parity, wait_limit);
            return;
        }
        parity ^= 1u;
        const int64_t z0 = __ldg(run_z0 + r), z1 = __ldg(run_z0 + r + 1);
        const unsigned char *Xc = reinterpret_cast<const unsigned char *>(X) + (size_t)group * 512 + lane * 16;
        const unsigned char *Ys = rows + lane * 16;
        for (int64_t z = z0 + warp; z < z1; z += WARPS) {
            PairAcc acc;
            acc.zero();
            const uint32_t *ox = opx + z * k;
            const uint16_t *os = oslot + z * k;
            for (int64_t b0 = 0; b0 < k; b0 += 32) {
                const int nb = (int)min((int64_t)32, k - b0);
                __syncwarp();  // the previous records are consumed
                if (lane < nb) {
                    const uint32_t sl = __ldg(os + b0 + lane);
                    rec[lane] = OpRec{__ldg(ox + b0 + lane), (sl & 0x7fffu) * 512u, f2_sign_pair((sl & 0x8000u) != 0)};
                }
                __syncwarp();
                yc_terms<4>(rec, nb, Xc, Ys, row_bytes, acc);
            }
            reinterpret_cast<ulonglong2 *>(Z + z * W)[group * 32 + lane] = acc.store();
        }
        __syncthreads();  // every warp has read the rows before the next copies overwrite them
    }
}

// A bounded wait that nothing completes: the wait runs out after `limit`
// polls, the status word records it and the kernel returns (the test of the
// timeout path; no copy is in flight).
__global__ void k_wait_timeout_check(uint32_t limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    mbar_wait_bounded(&bar, 0, limit);
}

// The mixed step with the operations regenerated once per CTA (the mixed
// path's choice for list-free lists). A CTA of 8 warps takes a z chunk and 8
// consecutive groups of 64 sites (two per lane, as k_large_step_mx2); for zb
// outputs at a time its 256 threads regenerate the outputs' operations once
// into shared memory, then every warp runs them on its sites exactly as the
// stored words would run (same order, same arithmetic), so the integer work
// is shared by the CTA's 512 sites (records as in k_large_step_mx2), and
// each warp keeps G gathers in flight. W must be a multiple of 64.
template <int G>
__global__ void __launch_bounds__(256, 3) k_large_step_gen(GenStep gs, int64_t n_z, int64_t k, int64_t zchunk, int zb,
                                                           int W, const float2 *__restrict__ X,
                                                           const float2 *__restrict__ Y, float2 *__restrict__ Z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OpRec *srec = reinterpret_cast<OpRec *>(smem_raw);  // [zb][k]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ngroups = W >> 6;
    const int nblk = (ngroups + 7) / 8;
    const uint32_t row_bytes = (uint32_t)W * (uint32_t)sizeof(float2);
    const int64_t nchunks = (n_z + zchunk - 1) / zchunk;
    for (int64_t item = blockIdx.x; item < nchunks * nblk; item += gridDim.x) {
        const int64_t chunk = item / nblk;
        const int group = (int)(item % nblk) * 8 + warp;
        const bool active = group < ngroups;
        const int col4 = (active ? group : 0) * 32 + lane;
        const unsigned char *Xc = reinterpret_cast<const unsigned char *>(reinterpret_cast<const float4 *>(X) + col4);
        const unsigned char *Yc = reinterpret_cast<const unsigned char *>(reinterpret_cast<const float4 *>(Y) + col4);
        const int64_t z_begin = chunk * zchunk;
        const int64_t z_end = min(n_z, z_begin + zchunk);
        for (int64_t zr = z_begin; zr < z_end; zr += zb) {
            const int nzr = (int)min((int64_t)zb, z_end - zr);
            __syncthreads();  // the previous round's operations are consumed
            for (int q = 0; q < nzr; ++q) {
                uint32_t zkey[4];
                g_key(gs, zr + q, zkey);
                for (int64_t j = threadIdx.x; j < k; j += blockDim.x) {
                    uint32_t ox, oy;
                    g_op(gs, zkey, j, ox, oy);
                    srec[q * k + j] = op_rec(ox, oy);
                }
            }
            __syncthreads();
            if (!active) continue;
            for (int q = 0; q < nzr; ++q) {
                PairAcc acc;
                acc.zero();
                pair_terms<G>(srec + q * k, (int)k, Xc, Yc, row_bytes, acc);  // k * 16 B fit shared memory
                reinterpret_cast<ulonglong2 *>(Z + (zr + q) * W)[col4] = acc.store();
            }
        }
    }
}

// Contraction with L (eq. C_final) in FP64: lanes = sites, warps = components.
template <class Tr>
__global__ void __launch_bounds__(256) k_large_contract(const int64_t *__restrict__ fin_off,
                                                        const uint32_t *__restrict__ fin_z,
                                                        const double *__restrict__ fin_l, int n_comp, int W,
                                                        const typename Tr::V *__restrict__ FA,
                                                        const int32_t *__restrict__ sexp, int degree,
                                                        double inv_norm, double2 *__restrict__ Cout) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int ngroups = W >> 5;
    for (int64_t item = warp_global; item < (int64_t)n_comp * ngroups; item += nwarps) {
        const int c = (int)(item / ngroups);
        const int col = (int)(item % ngroups) * 32 + lane;
        double re = 0.0, im = 0.0;
        for (int64_t e = fin_off[c]; e < fin_off[c + 1]; ++e) {
            double2 f = Tr::to_d(Tr::wave_ld(FA, (int64_t)__ldg(fin_z + e) * W + col));
            double l = __ldg(fin_l + e);
            re = __fma_rn(l, f.x, re);
            im = __fma_rn(l, f.y, im);
        }
        int ue = -degree * sexp[col];  // C is homogeneous of this degree in the scaled inputs
        Cout[(int64_t)c * W + col] = make_double2(scalbn(re * inv_norm, ue), scalbn(im * inv_norm, ue));
    }
}

// Momentum phases and the fixed-order sum over each 32-site group: one CTA
// per group, partial[tile][mom][comp].
__global__ void __launch_bounds__(256) k_large_sitesum(FieldDesc F, WaveDesc wv, MomDesc M, int n_comp,
                                                       const double2 *__restrict__ phase,
                                                       const double2 *__restrict__ C, double2 *__restrict__ partial) {
    __shared__ double2 ph[32 * kMaxMom];
    const int g = blockIdx.x;
    for (int i = threadIdx.x; i < 32 * M.n_mom; i += blockDim.x) {
        int s = i / M.n_mom, q = i % M.n_mom;
        int cfg, t, site;
        bool live = item_site(F, wv, wv.item0 + g * 32 + s, cfg, t, site);
        ph[i] = live ? __ldg(phase + (int64_t)site * M.n_mom + q) : make_double2(0, 0);
    }
    __syncthreads();
    const int64_t tile = (wv.item0 >> 5) + g;
    for (int o = threadIdx.x; o < M.n_mom * n_comp; o += blockDim.x) {
        int q = o / n_comp, c = o % n_comp;
        double re = 0.0, im = 0.0;
        for (int s = 0; s < 32; ++s) {
            double2 p = ph[s * M.n_mom + q], cv = C[(int64_t)c * wv.W + g * 32 + s];
            re = __fma_rn(p.x, cv.x, __fma_rn(-p.y, cv.y, re));
            im = __fma_rn(p.x, cv.y, __fma_rn(p.y, cv.x, im));
        }
        partial[tile * (int64_t)(M.n_mom * n_comp) + o] = make_double2(re, im);
    }
}

// Final reduction over the tiles of each slab: one warp per output, lanes
// take tiles lane, lane + 32, ... with Neumaier compensation, then a fixed
// xor tree combines the lanes' (sum, compensation) pairs - a fixed order, so
// results are bitwise reproducible. out[cfg][list][t - t0][mom][comp_stride].
__device__ __forceinline__ void neumaier(double &s, double &c, double v) {
    const double t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
}
__global__ void k_reduce_tiles(const double2 *__restrict__ partial, int64_t n_slabs, int tiles_per_slab, int n_mom,
                               int n_comp, int n_t, int list_idx, int n_lists, int comp_stride, double2 *out) {
    const int64_t per_slab = (int64_t)n_mom * n_comp;
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t o = wid; o < n_slabs * per_slab; o += nw) {
        const int64_t slab = o / per_slab;
        const int r = (int)(o % per_slab);
        double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
        for (int tl = lane; tl < tiles_per_slab; tl += 32) {
            const double2 v = partial[(slab * tiles_per_slab + tl) * per_slab + r];
            neumaier(sr, cr, v.x);
            neumaier(si, ci, v.y);
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double osr = __shfl_xor_sync(0xffffffffu, sr, off), ocr = __shfl_xor_sync(0xffffffffu, cr, off);
            const double osi = __shfl_xor_sync(0xffffffffu, si, off), oci = __shfl_xor_sync(0xffffffffu, ci, off);
            // both partners add in the same order, so they agree bit for bit
            double ar = lane & off ? osr : sr, br = lane & off ? sr : osr;
            double ai = lane & off ? osi : si, bi = lane & off ? si : osi;
            double ccr = cr + ocr, cci = ci + oci;
            sr = ar;
            cr = ccr;
            neumaier(sr, cr, br);
            si = ai;
            ci = cci;
            neumaier(si, ci, bi);
        }
        if (lane == 0) {
            const int cfg = (int)(slab / n_t), tt = (int)(slab % n_t);
            const int q = r / n_comp, c = r % n_comp;
            const int64_t oi = ((((int64_t)cfg * n_lists + list_idx) * n_t + tt) * n_mom + q) * comp_stride + c;
            out[oi] = make_double2(sr + cr, si + ci);
        }
    }
}

// The same reduction for slabs with many outputs (momentum-projected blocks:
// n_mom x 2 x block entries each, a few hundred tiles per slab): one thread
// per output adds the slab's tiles in a fixed order, tile tl into partial sum
// tl mod 4, then ((s0 + s1) + (s2 + s3)). Plain FP64 additions: GB300 issues
// few FP64 operations per clock, and with hundreds of thousands of outputs a
// compensated sum (six FP64 operations a term) costs more than the rest of
// the step; the error of this order is below (tiles/4 + 2) ulp of the sum of
// the magnitudes. Consecutive threads take consecutive outputs, so every load
// of a warp is one contiguous 512 B segment. out as in k_reduce_tiles.
__global__ void __launch_bounds__(256) k_reduce_tiles_cols(const double2 *__restrict__ partial, int64_t n_slabs,
                                                           int tiles_per_slab, int n_mom, int n_comp, int n_t,
                                                           int list_idx, int n_lists, int comp_stride,
                                                           double2 *out) {
    const int64_t per_slab = (int64_t)n_mom * n_comp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_slabs * per_slab; o += stride) {
        const int64_t slab = o / per_slab;
        const int r = (int)(o % per_slab);
        const double2 *p = partial + slab * tiles_per_slab * per_slab + r;
        double2 acc[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] = make_double2(0.0, 0.0);
        int tl = 0;
        for (; tl + 4 <= tiles_per_slab; tl += 4) {
            double2 v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = __ldg(p + (int64_t)(tl + j) * per_slab);
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = make_double2(acc[j].x + v[j].x, acc[j].y + v[j].y);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (tl + j < tiles_per_slab) {
                const double2 v = __ldg(p + (int64_t)(tl + j) * per_slab);
                acc[j] = make_double2(acc[j].x + v.x, acc[j].y + v.y);
            }
        const int cfg = (int)(slab / n_t), tt = (int)(slab % n_t);
        const int q = r / n_comp, c = r % n_comp;
        const int64_t oi = ((((int64_t)cfg * n_lists + list_idx) * n_t + tt) * n_mom + q) * comp_stride + c;
        out[oi] = make_double2((acc[0].x + acc[1].x) + (acc[2].x + acc[3].x),
                               (acc[0].y + acc[1].y) + (acc[2].y + acc[3].y));
    }
}

}  // namespace mbc
