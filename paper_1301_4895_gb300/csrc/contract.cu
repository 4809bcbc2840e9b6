// mbc_contract: device side of the recursive multibaryon contraction.
//
// Host responsibilities here: validate arguments, upload each term list once
// per device (cached on the list), pick the kernel regime and launch shape,
// own the device scratch (grown on demand, kept per device and stream), and
// enqueue everything on the caller's stream. All arithmetic of the path runs
// in the kernels of small_kernel.cuh / large_kernel.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <new>
#include <vector>

#include "large_kernel.cuh"
#include "mbc_internal.h"

#include <atomic>

namespace mbc {
// kernels launched by the contraction entry points since the library loaded
std::atomic<int64_t> g_kernel_launches{0};
inline void note_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace mbc
#include "probe.cuh"
#include "project_kernel.cuh"
#include "small_kernel.cuh"
#include "small_ls_kernel.cuh"

namespace mbc {

// After a synchronisation of stream: the kernels' latched status word, read
// and cleared (defined with mbc_sync_status).
mbc_status take_device_status(cudaStream_t stream);

#define MBC_CUDA_TRY(expr)                         \
    do {                                           \
        cudaError_t _e = (expr);                   \
        if (_e != cudaSuccess) {                   \
            (void)cudaGetLastError();              \
            return _e == cudaErrorMemoryAllocation ? MBC_ERR_OOM : MBC_ERR_CUDA; \
        }                                          \
    } while (0)

namespace {

constexpr int kSmemLimit = 227 * 1024;

int64_t binom64(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// Lanes per output component for a rectangular step (n_z outputs, k terms)
// in the warp-per-site kernel: minimise warp-instructions on the FP64 pipe,
// rounds * (ceil(k/g) * 4 DFMA + log2(g) * 2 DADD for the shuffle tree).
int pick_group(int64_t n_z, int64_t k, double c_op = 4.0, double c_level = 2.0) {
    int best = 1;
    double best_cost = 1e300;
    int lg = 0;
    for (int g = 1; g <= 32; g <<= 1, ++lg) {
        int64_t per = 32 / g;
        int64_t rounds = (n_z + per - 1) / per;
        int64_t kk = (k + g - 1) / g;
        double cost = (double)rounds * ((double)kk * c_op + lg * c_level);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = g;
        }
    }
    return best;
}

// Warp-per-site step layout: n_main outputs (whole rounds of 32 / g) with g
// lanes each and the remaining n_z - n_main with g2 lanes each, chosen by the
// same FP64 instruction cost as pick_group.
void split_groups(int64_t n_z, int64_t k, int32_t &g, int32_t &n_main, int32_t &g2) {
    auto cost = [&](int64_t n, int gg) {
        if (n <= 0) return 0.0;
        int lg = 0;
        while ((1 << lg) < gg) ++lg;
        const int64_t per = 32 / gg, rounds = (n + per - 1) / per, kk = (k + gg - 1) / gg;
        return (double)rounds * ((double)kk * 4.0 + lg * 2.0);
    };
    g = pick_group(n_z, k);
    n_main = (int32_t)n_z;
    g2 = g;
    double best = cost(n_z, g);
    for (int g1 = 1; g1 <= 32; g1 <<= 1) {
        const int64_t per = 32 / g1, nm = n_z / per * per;
        if (nm == n_z || nm == 0) continue;
        const int gt = pick_group(n_z - nm, k);
        const double c = cost(nm, g1) + cost(n_z - nm, gt);
        if (c < best - 1e-9) {
            best = c;
            g = g1;
            n_main = (int32_t)nm;
            g2 = gt;
        }
    }
}

struct Interval {
    int start, end;
    int64_t size, off;
};

// first-fit placement of buffers with lifetimes [start, end] (inclusive);
// the first n_fixed buffers keep the offsets they carry
void place(std::vector<Interval *> &bufs, size_t n_fixed = 0) {
    std::vector<Interval *> placed;
    for (size_t i = 0; i < n_fixed && i < bufs.size(); ++i) placed.push_back(bufs[i]);
    for (size_t i = n_fixed; i < bufs.size(); ++i) {
        Interval *b = bufs[i];
        std::vector<std::pair<int64_t, int64_t>> busy;
        for (Interval *p : placed)
            if (p->start <= b->end && b->start <= p->end) busy.push_back({p->off, p->off + p->size});
        std::sort(busy.begin(), busy.end());
        int64_t off = 0;
        for (auto &r : busy) {
            if (off + b->size <= r.first) break;
            off = std::max(off, r.second);
        }
        b->off = off;
        placed.push_back(b);
    }
}

}  // namespace

// Runs of consecutive outputs of a stored step whose operations name at most
// kYcRows distinct block rows (the mixed step that stages block rows in
// shared memory, k_large_step_yc): run r covers outputs [z0[r], z0[r+1]),
// its rows are rows[y0[r] .. y0[r+1]), and slot[z k + j] is the slot of
// operation j's row in its run, with the sign in bit 15.
struct YRuns {
    bool tried = false, ok = false;
    int64_t n_runs = 0;
    uint32_t *d_z0 = nullptr, *d_y0 = nullptr;
    uint16_t *d_rows = nullptr, *d_slot = nullptr;
};

struct DeviceCache {
    int device = -1;
    bool small_ok = false;
    bool ls_ok = false;      // the lanes-are-sites (mixed) kernel can take the list
    SmallPlan sp{};          // device pointers filled in
    int64_t site_entries = 0;
    uint32_t *d_small_ops = nullptr;
    uint32_t *d_small_zops = nullptr;
    // large path
    std::vector<uint32_t *> d_opx;
    std::vector<uint16_t *> d_opy;
    int64_t *d_fin_off = nullptr;
    uint32_t *d_fin_z = nullptr;
    double *d_fin_l = nullptr;
    std::vector<int64_t *> d_zrank;    // list-free steps: index tables
    std::vector<int32_t *> d_xmap;
    uint32_t *d_fin_zs = nullptr;      // small path: region offsets of the contracted entries
    double *d_comp_inv_norm = nullptr;
    int32_t *d_comp_deg = nullptr;
    int64_t max_stage = 0;
    std::vector<YRuns> yruns;          // per step, made on first mixed use
};

namespace {

void free_cache(DeviceCache *c) {
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (c->device >= 0) cudaSetDevice(c->device);
    cudaFree(c->d_small_ops);
    cudaFree(c->d_small_zops);
    for (auto p : c->d_opx) cudaFree(p);
    for (auto p : c->d_opy) cudaFree(p);
    for (auto p : c->d_zrank) cudaFree(p);
    for (auto p : c->d_xmap) cudaFree(p);
    for (auto &r : c->yruns) {
        cudaFree(r.d_z0);
        cudaFree(r.d_y0);
        cudaFree(r.d_rows);
        cudaFree(r.d_slot);
    }
    cudaFree(c->d_fin_off);
    cudaFree(c->d_fin_z);
    cudaFree(c->d_fin_l);
    cudaFree(c->d_fin_zs);
    cudaFree(c->d_comp_inv_norm);
    cudaFree(c->d_comp_deg);
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

template <class T>
mbc_status upload(T **dst, const T *src, size_t n) {
    *dst = nullptr;
    if (n == 0) return MBC_OK;
    MBC_CUDA_TRY(cudaMalloc((void **)dst, n * sizeof(T)));
    MBC_CUDA_TRY(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return MBC_OK;
}

// Nonzero entries of Gamma_2 (eq. def_g): 4 relativistic, 2 nonrelativistic.
inline int n_g2(const mbc_term_list *L) { return L->dim == 4 ? 4 : 2; }

// Build the small-kernel plan (shared-memory layout of one site) on the host.
// The shared-memory kernels hold square single-source tiles only.
// part_off receives, per nucleus of the list, the region offset of the stage
// its components are contracted from (blocks for a single baryon).
bool plan_small(const mbc_term_list *L, SmallPlan &P, int64_t &site_entries, std::vector<int> &part_off) {
    std::memset(&P, 0, sizeof(P));
    const int A = L->A;
    if (A > 16 || L->n_comp > kSmallMaxComp || L->n_comp < 1) return false;
    if (L->n_sources != 1) return false;
    for (const auto &s : L->steps)
        if (s.generated) return false;  // list-free lists run on the wave kernels
    P.A = A;
    P.dim = L->dim;
    P.nxi = L->nxi;
    P.n_g2 = n_g2(L);
    P.n_comp = L->n_comp;
    P.n_steps = A - 1;
    P.path0 = L->path[0];
    P.block_size = (int)L->block_size;
    P.npair = (int)binom64(L->nxi, 2);
    if (L->block_size >= 32768) return false;
    for (auto &s : L->steps)
        if (s.n_x >= 65536) return false;
    const int n_ph = 3 + A;  // phases: 0 load, 1 Q, 2 blocks, 3.. steps, 2 + A contraction
    Interval Sb{0, 2, (int64_t)L->nxi * L->nxi, 0}, Qb{1, 2, 3LL * L->nxi * L->nxi, 0};
    Interval blk[2];
    std::vector<Interval> stage((size_t)A + 1);
    // both blocks first, at fixed offsets [0, bs) and [bs, 2 bs), live to the
    // end: lists with the same tile shape then share one block computation
    // per site in a batch (blocks do not depend on the nucleus); the S tile,
    // the diquark and the stages are placed after them by first fit
    const int last_phase = 2 + A;
    std::vector<Interval *> order;
    for (int b = 0; b < 2; ++b) {
        P.need_blk[b] = L->need_block[b] ? 1 : 0;
        blk[b] = {2, last_phase, L->block_size, (int64_t)b * L->block_size};
        order.push_back(&blk[b]);
    }
    order.push_back(&Sb);
    order.push_back(&Qb);
    // a stage where a nucleus of the list ends stays live until the contraction
    std::vector<bool> contracted((size_t)A + 1, false);
    for (const auto &pt : L->parts) contracted[(size_t)pt.A] = true;
    for (int m = 1; m < A; ++m) {
        stage[(size_t)m + 1] = {3 + m - 1, contracted[(size_t)m + 1] ? last_phase : 3 + m,
                                L->steps[(size_t)m - 1].n_z, 0};
        order.push_back(&stage[(size_t)m + 1]);
    }
    (void)n_ph;
    place(order, 2);
    int64_t top = 0;
    for (auto *b : order) top = std::max(top, b->off + b->size);
    site_entries = (top + 1) & ~int64_t(1);
    P.site_entries = (int)site_entries;
    P.part_off = (int)site_entries;  // lanes-are-sites kernel: 64 partial rows after the site region
    P.s_off = (int)Sb.off;
    P.q_off = (int)Qb.off;
    for (int b = 0; b < 2; ++b) P.blk_off[b] = (int)blk[b].off;
    int64_t op_off = 0;
    for (int m = 1; m < A; ++m) {
        const Step &s = L->steps[(size_t)m - 1];
        SmallStepDesc &d = P.step[m - 1];
        d.n_z = (int)s.n_z;
        d.k = (int)s.k;
        split_groups(s.n_z, s.k, d.g, d.n_main, d.g2);
        d.x_off = m == 1 ? P.blk_off[L->path[0]] : (int)stage[(size_t)m].off;
        d.y_off = P.blk_off[s.baryon];
        d.z_off = (int)stage[(size_t)m + 1].off;
        d.op_off = op_off;
        op_off += s.n_z * s.k;
    }
    part_off.clear();
    for (const auto &pt : L->parts)
        part_off.push_back(pt.A == 1 ? P.blk_off[L->path[0]] : (int)stage[(size_t)pt.A].off);
    int64_t kmax = 1;
    for (int c = 0; c < L->n_comp; ++c) kmax = std::max(kmax, L->fin_off[(size_t)c + 1] - L->fin_off[(size_t)c]);
    P.fin_g = pick_group(L->n_comp, kmax);
    return true;
}

DeviceCache *get_cache(const mbc_term_list *Lc, int device, mbc_status &st) {
    mbc_term_list *L = const_cast<mbc_term_list *>(Lc);
    std::lock_guard<std::mutex> g(L->dev_mu);
    if ((int)L->dev.size() <= device) L->dev.resize((size_t)device + 1, nullptr);
    if (L->dev[(size_t)device]) {
        st = MBC_OK;
        return L->dev[(size_t)device];
    }
    DeviceCache *c = new (std::nothrow) DeviceCache();
    if (!c) {
        st = MBC_ERR_OOM;
        return nullptr;
    }
    c->device = device;
    st = MBC_OK;
    // contraction list
    std::vector<double> lval(L->fin_l.begin(), L->fin_l.end());
    if ((st = upload(&c->d_fin_off, L->fin_off.data(), L->fin_off.size())) != MBC_OK ||
        (st = upload(&c->d_fin_z, L->fin_z.data(), L->fin_z.size())) != MBC_OK ||
        (st = upload(&c->d_fin_l, lval.data(), lval.size())) != MBC_OK) {
        free_cache(c);
        return nullptr;
    }
    // small-kernel plan and packed ops
    std::vector<int> part_off;
    c->small_ok = !L->pauli_forbidden && plan_small(L, c->sp, c->site_entries, part_off);
    if (c->small_ok) {
        // contracted entries as offsets in the site region; per-component
        // normalisation and homogeneity degree of its nucleus
        std::vector<uint32_t> zs(L->fin_z.size());
        std::vector<double> inv((size_t)L->n_comp);
        std::vector<int32_t> deg((size_t)L->n_comp);
        for (size_t j = 0; j < L->parts.size(); ++j) {
            const auto &pt = L->parts[j];
            for (int cc = pt.c0; cc < pt.c1; ++cc) {
                inv[(size_t)cc] = 1.0 / pt.norm;
                deg[(size_t)cc] = 3 * pt.A;
                for (int64_t e = L->fin_off[(size_t)cc]; e < L->fin_off[(size_t)cc + 1]; ++e)
                    zs[(size_t)e] = L->fin_z[(size_t)e] + (uint32_t)part_off[j];
            }
        }
        if ((st = upload(&c->d_fin_zs, zs.data(), zs.size())) != MBC_OK ||
            (st = upload(&c->d_comp_inv_norm, inv.data(), inv.size())) != MBC_OK ||
            (st = upload(&c->d_comp_deg, deg.data(), deg.size())) != MBC_OK) {
            free_cache(c);
            return nullptr;
        }
        // per step and part (outputs [0, n_main) with g lanes, the rest with
        // g2): [round j][z][sub], padded to a whole number of rounds
        std::vector<uint32_t> packed;
        for (size_t m = 0; m < L->steps.size(); ++m) {
            const Step &s = L->steps[m];
            SmallStepDesc &d = c->sp.step[m];
            auto pack = [&](int64_t z_begin, int64_t n, int64_t g) {
                const int64_t off = (int64_t)packed.size(), kk = (s.k + g - 1) / g;
                packed.resize(packed.size() + (size_t)(kk * n * g), 0u);
                uint32_t *dst = packed.data() + off;
                for (int64_t zl = 0; zl < n; ++zl)
                    for (int64_t j = 0; j < s.k; ++j) {
                        const size_t i = (size_t)((z_begin + zl) * s.k + j);
                        const uint32_t op =
                            s.x[i] | ((uint32_t)(s.ys[i] & 0x7fffu) << 16) | ((uint32_t)(s.ys[i] >> 15) << 31);
                        dst[((j / g) * n + zl) * g + (j % g)] = op;
                    }
                return off;
            };
            d.op_off = pack(0, d.n_main, d.g);
            d.op_off2 = pack(d.n_main, s.n_z - d.n_main, d.g2);
        }
        if ((st = upload(&c->d_small_ops, packed.data(), packed.size())) != MBC_OK) {
            free_cache(c);
            return nullptr;
        }
        // lanes-are-sites layout: z-major, operands as byte offsets of their
        // 256 B shared-memory rows (x << 8 | sign in bit 0 | y << 24), which
        // needs every stage and block index below 256 (all nonrelativistic
        // lists); otherwise the mixed path takes the wave kernels. Each
        // output's terms are ordered positive first (stable), so the kernel
        // adds the first ones and subtracts the rest and its operation
        // records need no sign
        std::vector<uint32_t> zpk;
        c->ls_ok = true;
        for (size_t m = 0; m < L->steps.size(); ++m) {
            const Step &s = L->steps[m];
            c->sp.step[m].zop_off = (int64_t)zpk.size();
            for (int64_t z = 0; z < s.n_z; ++z)
                for (uint32_t want = 0; want < 2; ++want)
                    for (int64_t j = 0; j < s.k; ++j) {
                        const size_t i = (size_t)(z * s.k + j);
                        const uint32_t x = s.x[i], y = s.ys[i] & 0x7fffu, sg = (uint32_t)(s.ys[i] >> 15);
                        if (sg != want) continue;
                        if (x >= 256 || y >= 256) c->ls_ok = false;
                        zpk.push_back((x & 0xffu) << 8 | sg | (y & 0xffu) << 24);
                    }
        }
        if ((st = upload(&c->d_small_zops, zpk.data(), zpk.size())) != MBC_OK) {
            free_cache(c);
            return nullptr;
        }
        c->sp.zops = c->d_small_zops;
        c->sp.ops = c->d_small_ops;
        c->sp.fin_off = c->d_fin_off;
        c->sp.fin_z = c->d_fin_zs;
        c->sp.fin_l = c->d_fin_l;
        c->sp.comp_inv_norm = c->d_comp_inv_norm;
        c->sp.comp_deg = c->d_comp_deg;
    }
    // large-path op arrays
    c->d_opx.assign(L->steps.size(), nullptr);
    c->d_opy.assign(L->steps.size(), nullptr);
    c->d_zrank.assign(L->steps.size(), nullptr);
    c->d_xmap.assign(L->steps.size(), nullptr);
    for (size_t m = 0; m < L->steps.size(); ++m) {
        const Step &s = L->steps[m];
        c->max_stage = std::max(c->max_stage, s.n_z);
        if ((st = upload(&c->d_opx[m], s.x.data(), s.x.size())) != MBC_OK ||
            (st = upload(&c->d_opy[m], s.ys.data(), s.ys.size())) != MBC_OK ||
            (st = upload(&c->d_zrank[m], s.zrank.data(), s.zrank.size())) != MBC_OK ||
            (st = upload(&c->d_xmap[m], s.xmap.data(), s.xmap.size())) != MBC_OK) {
            free_cache(c);
            return nullptr;
        }
    }
    L->dev[(size_t)device] = c;
    return c;
}

// ---- scratch ---------------------------------------------------------------
struct Scratch {
    void *p = nullptr;
    size_t n = 0;
};
std::mutex g_scratch_mu;
std::map<std::pair<int, cudaStream_t>, Scratch> g_scratch;

mbc_status scratch_get(int device, cudaStream_t s, size_t bytes, void **out) {
    std::lock_guard<std::mutex> g(g_scratch_mu);
    Scratch &sc = g_scratch[{device, s}];
    if (sc.n < bytes) {
        if (sc.p) {
            cudaStreamSynchronize(s);
            cudaFree(sc.p);
            sc.p = nullptr;
            sc.n = 0;
        }
        size_t want = std::max(bytes, (size_t)(1 << 20));
        MBC_CUDA_TRY(cudaMalloc(&sc.p, want));
        sc.n = want;
    }
    *out = sc.p;
    return MBC_OK;
}

int g_const_dev_mask = 0;
std::mutex g_const_mu;

mbc_status ensure_constants(int device) {
    std::lock_guard<std::mutex> g(g_const_mu);
    if (device < 31 && (g_const_dev_mask >> device) & 1) return MBC_OK;
    uint8_t pi[276], pj[276];
    int r = 0;
    for (int j = 1; j < 24; ++j)
        for (int i = 0; i < j; ++i) {  // colex order: rank = i + j(j-1)/2
            pi[r] = (uint8_t)i;
            pj[r] = (uint8_t)j;
            ++r;
        }
    MBC_CUDA_TRY(cudaMemcpyToSymbol(c_pair_i, pi, sizeof(pi)));
    MBC_CUDA_TRY(cudaMemcpyToSymbol(c_pair_j, pj, sizeof(pj)));
    uint32_t bn[25][25];
    for (int n = 0; n < 25; ++n)
        for (int k = 0; k < 25; ++k) bn[n][k] = (uint32_t)binom64(n, k);
    MBC_CUDA_TRY(cudaMemcpyToSymbol(c_binom, bn, sizeof(bn)));
    if (device < 31) g_const_dev_mask |= 1 << device;
    return MBC_OK;
}

int sm_count(int device) {
    static std::mutex mu;
    static std::map<int, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(device);
    if (it != cache.end()) return it->second;
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
    if (n <= 0) n = 1;
    cache[device] = n;
    return n;
}

// cudaFuncSetAttribute / occupancy queries cost host time on every call;
// both are cached per (kernel, device, block size, shared memory)
mbc_status prepare_kernel(const void *kern, int device, int threads, size_t smem, int *per_sm) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int, size_t>, int> occ;
    static std::map<std::pair<const void *, int>, size_t> smem_set;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_tuple(kern, device, threads, smem);
    auto it = occ.find(key);
    if (it != occ.end()) {
        *per_sm = it->second;
        return MBC_OK;
    }
    size_t &have = smem_set[{kern, device}];
    if (smem > have) {
        MBC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        have = smem;
    }
    int n = 0;
    MBC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem));
    occ[key] = n;
    *per_sm = n;
    return MBC_OK;
}

// ---- launchers -------------------------------------------------------------

// Small-stage kernels. FP64: one warp per site (k_small). MIXED: 32 sites
// per CTA, lanes are sites (k_small_ls). Lists of this regime are contracted
// in batches of up to kMaxBatch by one persistent launch each.
struct SmallLaunch {
    bool ok = false;
    int T = 0;            // sites per tile
    int threads = 0;
    size_t smem = 0;
    int tiles_per_slab = 0;
};

// Launch shape of the shared-memory kernels for per-site buffers of
// site_stride entries and comp_stride components (host only).
SmallLaunch size_small_tiles(int32_t site_stride, int32_t comp_stride, const FieldDesc &F, const mbc_tune *tune,
                             bool mixed, int n_sm = 0) {
    SmallLaunch l;
    if (!mixed) {
        const int64_t per_site = site_stride * 16LL + 16LL * comp_stride;
        l.T = (int)std::min<int64_t>(32, kSmemLimit / per_site);
        if (tune && tune->sites_per_cta > 0) {
            l.T = std::min(l.T, tune->sites_per_cta);
        } else if (n_sm > 0) {
            // small lattices: fewer sites per CTA so that every SM gets a tile
            const int64_t sites = (int64_t)F.n_cfg * F.n_t * F.lx * F.ly * F.lz;
            l.T = (int)std::max<int64_t>(1, std::min<int64_t>(l.T, (sites + n_sm - 1) / n_sm));
        }
        l.threads = 32 * l.T;
        l.smem = (size_t)l.T * per_site;
    } else {
        l.T = 32;
        l.threads = (tune && tune->threads_per_cta > 0) ? tune->threads_per_cta : 1024;
        l.threads = std::max(64, std::min(1024, l.threads / 32 * 32));
        // rows of 32 lanes (site region + 64 partial rows), then 32 operation
        // records of 16 B per warp; fewer warps where the records do not fit
        const size_t rows = (size_t)(site_stride + 64) * 32 * sizeof(float2);
        while (l.threads > 256 && rows + (size_t)l.threads * 16 > (size_t)kSmemLimit - 2048) l.threads /= 2;
        l.threads = l.threads / 32 * 32;
        l.smem = rows + (size_t)l.threads * 16;
        if (l.smem > (size_t)kSmemLimit - 2048) return l;
    }
    if (l.T < 1) return l;
    const int v3 = F.lx * F.ly * F.lz;
    l.tiles_per_slab = (v3 + l.T - 1) / l.T;
    l.ok = true;
    return l;
}

SmallLaunch size_small_batch(const std::vector<const DeviceCache *> &cs, const FieldDesc &F, const mbc_tune *tune,
                             bool mixed, int32_t &site_stride, int32_t &comp_stride, int n_sm = 0) {
    site_stride = 0;
    comp_stride = 0;
    for (auto *c : cs) {
        site_stride = std::max(site_stride, (int32_t)c->site_entries);
        comp_stride = std::max(comp_stride, c->sp.n_comp);
    }
    return size_small_tiles(site_stride, comp_stride, F, tune, mixed, n_sm);
}

mbc_status launch_small_batch(const SmallBatch &B, const FieldDesc &F, const MomDesc &M, const SmallLaunch &l,
                              bool mixed, int device, cudaStream_t stream, const double2 *phase, double2 *partial,
                              bool timed) {
    bool nxi6 = true;
    for (int i = 0; i < B.n_lists; ++i) nxi6 = nxi6 && B.plan[i].nxi == 6;
    auto kern = !mixed ? k_small<FP64Traits> : nxi6 ? k_small_ls<MixedTraits, 6> : k_small_ls<MixedTraits, 0>;
    int per_sm = 0;
    mbc_status pst = prepare_kernel((const void *)kern, device, l.threads, l.smem, &per_sm);
    if (pst != MBC_OK) return pst;
    if (per_sm < 1) return MBC_ERR_UNSUPPORTED;
    int64_t grid = std::min<int64_t>(B.total_items, (int64_t)per_sm * sm_count(device));
    if (grid < 1) return MBC_OK;
    MBC_CUDA_TRY(cudaMemsetAsync(B.counter, 0, sizeof(unsigned long long), stream));
    if (timed) {
        TimedLaunch tl(stream);
        note_launch();
        kern<<<(unsigned)grid, l.threads, l.smem, stream>>>(B, F, M, phase, partial);
    } else {
        note_launch();
        kern<<<(unsigned)grid, l.threads, l.smem, stream>>>(B, F, M, phase, partial);
    }
    MBC_CUDA_TRY(cudaGetLastError());
    return MBC_OK;
}

// Site-operations (operations x sites) a wave needs at least.
constexpr int64_t kWaveSiteOps = 20000000000LL;

struct LargeSizes {
    int W;
    size_t blk_bytes, stage_bytes, c_bytes, sexp_bytes;
};

template <class Tr>
LargeSizes large_sizes(const mbc_term_list *L, const DeviceCache *c, const mbc_tune *tune, int64_t n_items) {
    using V = typename Tr::V;
    LargeSizes s{};
    int64_t per_site = (int64_t)sizeof(V) * (2 * L->block_size + 2 * std::max<int64_t>(c->max_stage, 1)) +
                       16LL * L->n_comp + 4;
    const int64_t budget = 8LL << 30;
    int64_t W = budget / per_site;
    // no wider than kWaveSiteOps site-operations need: narrow waves keep the
    // stage rows that concurrent outputs gather close together in L2
    // (measured on GB300: 8Be mixed 2,777 -> 3,251 correlators/s with 64
    // instead of 576 sites, FP64 318 -> 324), and waves of that much work
    // amortise their launches and small steps (4He (0,1,0,1), 8.5 M
    // operations: 52 K correlators/s with 64 sites, 132 K with 2,176). The
    // CTA-shared regeneration of list-free steps covers 512 sites per CTA
    // (8Be list-free mixed: 1,338 with 640 sites, 2,100 with 512).
    int64_t ops = 0;
    bool regen = false;
    for (const auto &st : L->steps) {
        ops += st.n_z * st.k;
        regen = regen || st.generated || (tune && tune->list_free == 1 && st.dense);
    }
    const bool regen_ctas = regen && sizeof(V) == sizeof(float2);
    W = std::min<int64_t>(W, std::max<int64_t>(regen_ctas ? 512 : 64,
                                               (kWaveSiteOps + ops - 1) / std::max<int64_t>(ops, 1)));
    if (regen_ctas && W >= 512) W = W / 512 * 512;  // whole CTAs of 8 site groups
    if (tune && tune->wave_sites > 0) W = tune->wave_sites;
    // multiples of 64 sites: the mixed step kernel covers 64 sites per warp
    W = std::max<int64_t>(64, std::min<int64_t>(W, 4096));
    W = std::min<int64_t>(W, (n_items + 63) / 64 * 64);
    W = std::max<int64_t>(64, W / 64 * 64);
    s.W = (int)W;
    s.blk_bytes = (size_t)(L->block_size * W) * sizeof(V);
    s.stage_bytes = (size_t)(std::max<int64_t>(c->max_stage, 1) * W) * sizeof(V);
    s.c_bytes = (size_t)L->n_comp * W * sizeof(double2);
    s.sexp_bytes = (size_t)W * sizeof(int32_t);
    return s;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Device description of step m (0-based) for regenerating its operations.
GenStep gen_step(const mbc_term_list *L, const DeviceCache *c, size_t m) {
    const Step &s = L->steps[m];
    GenStep g;
    std::memset(&g, 0, sizeof(g));
    g.b = s.baryon;
    g.bprev = L->path[0];
    g.x_block = m == 0;
    g.nxi = L->nxi;
    g.npair = (int)binom64(L->nxi, 2);
    g.dim = L->dim_snk;
    for (int i = 0; i < 4; ++i) {
        g.zk[i] = s.zk[i];
        g.xk[i] = s.xk[i];
        const int n = i < 2 ? L->dim_snk : L->nxi;
        g.zr[i] = binom64(n, s.zk[i]);
        g.xr[i] = binom64(n, s.xk[i]);
    }
    g.zrank = c->d_zrank[m];
    g.xmap = c->d_xmap[m];
    return g;
}

// Warps per CTA of k_large_step_yc (one CTA per SM: its staged rows take
// most of the shared memory) and the poll limit of its bounded waits
// (about a second).
constexpr int kYcWarps = 32;
constexpr uint32_t kWaitPolls = 1u << 24;
// Terms per output from which the mixed wave step keeps 8 gathers in flight
// per warp (20-warp CTAs) rather than 4 (32-warp CTAs).
constexpr int64_t kSplitWideTerms = 64;
// Terms per output from which a step of fewer items than SMs splits its
// outputs' terms over several warps.
constexpr int64_t kSplitFewTerms = 1024;

// The runs of step m for k_large_step_yc, cut on the host at the first mixed
// call that runs the step and uploaded with the list's device copy. A step
// takes the kernel only where staging pays: every output's rows fit one run,
// the staged rows are at most a fifth of the operations, and a run has on
// average at least four outputs per warp (with fewer, the warps of a run
// finish unevenly and the step measured slower than k_large_step_mx2).
// Returns nullptr otherwise.
const YRuns *yruns_for(const mbc_term_list *Lc, const DeviceCache *cc, size_t m) {
    mbc_term_list *L = const_cast<mbc_term_list *>(Lc);
    DeviceCache *c = const_cast<DeviceCache *>(cc);
    std::lock_guard<std::mutex> g(L->dev_mu);
    if (c->yruns.size() != L->steps.size()) c->yruns.assign(L->steps.size(), YRuns{});
    YRuns &R = c->yruns[m];
    if (R.tried) return R.ok ? &R : nullptr;
    R.tried = true;
    const Step &s = L->steps[m];
    if (s.generated || s.x.empty() || s.n_z < 1 || s.k < 1 || L->block_size > 32767) return nullptr;
    const int64_t nb = L->block_size;
    std::vector<int64_t> in_run((size_t)nb, -1), in_z((size_t)nb, -1);
    std::vector<uint16_t> slot_of((size_t)nb, 0);
    std::vector<uint32_t> z0{0}, y0{0};
    std::vector<uint16_t> rows;
    std::vector<uint16_t> slot((size_t)(s.n_z * s.k));
    int64_t run = 0, cur = 0;
    for (int64_t z = 0; z < s.n_z; ++z) {
        const uint16_t *ys = s.ys.data() + z * s.k;
        int64_t fresh = 0, distinct = 0;
        for (int64_t j = 0; j < s.k; ++j) {
            const int y = ys[j] & 0x7fff;
            if (in_z[(size_t)y] == z) continue;
            in_z[(size_t)y] = z;
            ++distinct;
            if (in_run[(size_t)y] != run) ++fresh;
        }
        if (distinct > kYcRows) return nullptr;
        if (cur + fresh > kYcRows) {  // close the run
            ++run;
            cur = 0;
            z0.push_back((uint32_t)z);
            y0.push_back((uint32_t)rows.size());
        }
        for (int64_t j = 0; j < s.k; ++j) {
            const int y = ys[j] & 0x7fff;
            if (in_run[(size_t)y] != run) {
                in_run[(size_t)y] = run;
                slot_of[(size_t)y] = (uint16_t)cur++;
                rows.push_back((uint16_t)y);
            }
            slot[(size_t)(z * s.k + j)] = (uint16_t)(slot_of[(size_t)y] | (ys[j] & 0x8000));
        }
    }
    z0.push_back((uint32_t)s.n_z);
    y0.push_back((uint32_t)rows.size());
    const int64_t n_runs = run + 1;
    const double ops = (double)s.n_z * (double)s.k;
    if ((double)rows.size() > 0.2 * ops || s.n_z < 4 * kYcWarps * n_runs) return nullptr;
    if (upload(&R.d_z0, z0.data(), z0.size()) != MBC_OK || upload(&R.d_y0, y0.data(), y0.size()) != MBC_OK ||
        upload(&R.d_rows, rows.data(), rows.size()) != MBC_OK || upload(&R.d_slot, slot.data(), slot.size()) != MBC_OK) {
        cudaFree(R.d_z0);
        cudaFree(R.d_y0);
        cudaFree(R.d_rows);
        cudaFree(R.d_slot);
        R = YRuns{};
        R.tried = true;
        (void)cudaGetLastError();
        return nullptr;
    }
    R.n_runs = n_runs;
    R.ok = true;
    return &R;
}

// One recursion step of a wave (k_large_step), reading the stored operations
// or regenerating them (list-free lists; dense steps on request).
template <class Tr>
mbc_status launch_step(const mbc_term_list *L, const DeviceCache *c, size_t m, const mbc_tune *tune, int W, int nsm,
                       const typename Tr::V *X, const typename Tr::V *Y, typename Tr::V *Z, cudaStream_t stream) {
    const Step &s = L->steps[m];
    const bool gen = s.generated || (tune && tune->list_free == 1 && s.dense);
    // FP32 arithmetic is too cheap to hide per-warp regeneration: the mixed
    // path regenerates once per CTA into shared memory
    if (gen && sizeof(typename Tr::V) == sizeof(float2)) {
        // CTA-shared regeneration: zb outputs' operations per round in shared memory
        const size_t per_z = (size_t)s.k * sizeof(OpRec);
        const int64_t nblk = (W / 64 + 7) / 8;
        const int64_t target = (int64_t)nsm * 3 * 8;
        int64_t nchunks = std::max<int64_t>(1, std::min<int64_t>(s.n_z, (target + nblk - 1) / nblk));
        // at most 16 outputs per item: the resident CTAs then cover a narrow
        // window of consecutive outputs (measured +3 % on 8Be, +2 % on 4He
        // (0,1,0,1) against one range per CTA)
        int64_t zchunk = std::min<int64_t>(16, (s.n_z + nchunks - 1) / nchunks);
        if (tune && tune->zchunk > 0) zchunk = tune->zchunk;
        nchunks = (s.n_z + zchunk - 1) / zchunk;
        const int zb = (int)std::max<int64_t>(1, std::min<int64_t>(zchunk, (int64_t)((64u << 10) / per_z)));
        const size_t smem = (size_t)zb * per_z + 16;
        // 6 gathers in flight per warp, 3 CTAs of 8 warps per SM (80
        // registers): measured on GB300 against 4 gathers, 4He (0,1,0,1)
        // list-free (24, 30 and 180 splits per output, no partial group)
        // 76.9 K -> 82.3 K correlators/s, 8Be list-free 2,099 -> 2,121; 8
        // gathers at 2 CTAs per SM and 4-warp CTAs (6 per SM, waves of 256
        // sites) measured slower
        int per_sm = 0;
        mbc_status pst = prepare_kernel((const void *)k_large_step_gen<6>, c->device, 256, smem, &per_sm);
        if (pst != MBC_OK) return pst;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(nchunks * nblk, (int64_t)nsm * std::max(per_sm, 1) * 4));
        {
            TimedLaunch tl(stream);
            note_launch();
            k_large_step_gen<6><<<(unsigned)grid, 256, smem, stream>>>(gen_step(L, c, m), s.n_z, s.k, zchunk, zb, W,
                                                                       reinterpret_cast<const float2 *>(X),
                                                                       reinterpret_cast<const float2 *>(Y),
                                                                       reinterpret_cast<float2 *>(Z));
        }
        MBC_CUDA_TRY(cudaGetLastError());
        return MBC_OK;
    }
    if constexpr (!std::is_same<Tr, FP64Traits>::value) {
        // mixed precision, stored operations: two sites per lane (W is a
        // multiple of 64; the planar pair layout of the wave buffers is this
        // kernel's).
        // wave_order (mixed): 0 (default): one CTA per SM takes consecutive
        // (output, 64-site group) pairs, group fastest, one warp per output
        // (k_large_step_split, S = 1): the outputs in flight are a few
        // hundred consecutive ones, whose rows of X stay in L2. Steps whose
        // outputs have at least kSplitWideTerms terms run 20-warp CTAs with 8
        // gathers in flight per warp (96 registers), the others 32-warp CTAs
        // with 4 (64 registers), where a group of 8 would leave a serial
        // tail of up to 7 terms; 2: 32 warps on every step, 6: 20 warps on
        // every step; 5: 32 warps with each output's terms split over S = 2
        // .. 16 warps (S grows with the splits per output) and the partial
        // sums combined in a fixed order (order 0 does this too on steps of
        // fewer items than SMs and at least kSplitFewTerms terms); 1: k_large_step_mx2 with 8-warp
        // CTAs on consecutive outputs of one site group; 3: 8-warp CTAs with
        // the site groups side by side; 4: the block rows of runs of outputs
        // staged in shared memory by bulk copies (k_large_step_yc, where the
        // runs qualify). Measured on GB300, mixed, sink-site correlators/s
        // (8Be with waves of 576 sites, before the narrower default waves):
        // 8Be 2,797 (0) / 2,517 (2) / 2,793 (6) / 2,086 (5) / 1,982 (1) /
        // 1,942 (4); 4He with all components 2,434 / 2,305 / 2,386 / 2,112 /
        // 2,033 / 1,871; 4He (0,1,0,1) 132.9 K / 132.7 K / 125.1 K / 127.4 K
        // / 104.8 K / 117 K. (24 warps x 6 gathers, 28 x 5 and 16 x 12 were
        // within 1 % of 20 x 8 on 8Be and up to 5 % slower on 4He; 6
        // gathers on the steps of 24 and 30 terms, which leave no tail,
        // measured -0.7 % to +2 %.)
        const int order = tune ? tune->wave_order : 0;
        if (order == 0 || order == 2 || order == 5 || order == 6) {
            const int ngroups = W / 64;
            // a step of fewer (output, site group) items than SMs with many
            // terms per output (8Be's last step: one output of 3,168 terms)
            // splits each output's terms over up to 16 warps of a 32-warp CTA
            // (8Be mixed 3,266 -> 3,308 correlators/s)
            const bool few = order == 0 && s.n_z * ngroups < (int64_t)nsm && s.k >= kSplitFewTerms;
            const bool wide = !few && (order == 6 || (order == 0 && s.k >= kSplitWideTerms));
            const int warps = wide ? 20 : 32;
            int S = 1;
            if (order == 5 || few)
                while (2 * S <= warps / 2 && (int64_t)(2 * S) * 32 <= s.k) S *= 2;
            const int opc = warps / S;
            const int64_t items = (s.n_z * (W / 64) + opc - 1) / opc;
            const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)nsm));
            {
                TimedLaunch tl(stream);
                note_launch();
                const uint32_t *ox = c->d_opx[m];
                const uint16_t *oy = c->d_opy[m];
                const float2 *Xf = reinterpret_cast<const float2 *>(X), *Yf = reinterpret_cast<const float2 *>(Y);
                float2 *Zf = reinterpret_cast<float2 *>(Z);
                if (wide)
                    k_large_step_split<20, 8><<<(unsigned)grid, 640, 0, stream>>>(ox, oy, s.n_z, s.k, S, W, Xf, Yf, Zf);
                else
                    k_large_step_split<32, 4><<<(unsigned)grid, 1024, 0, stream>>>(ox, oy, s.n_z, s.k, S, W, Xf, Yf, Zf);
            }
            MBC_CUDA_TRY(cudaGetLastError());
            return MBC_OK;
        }
        const YRuns *yr = order == 4 ? yruns_for(L, c, m) : nullptr;
        if (yr) {
            const size_t smem = (size_t)kYcRows * 512 + (size_t)kYcWarps * 32 * sizeof(OpRec) + 16;
            int per_sm = 0;
            mbc_status pst = prepare_kernel((const void *)k_large_step_yc<kYcWarps>, c->device, 32 * kYcWarps, smem,
                                            &per_sm);
            if (pst != MBC_OK) return pst;
            if (per_sm >= 1) {
                const int64_t items = yr->n_runs * (W / 64);
                const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)nsm * per_sm));
                {
                    TimedLaunch tl(stream);
                    note_launch();
                    k_large_step_yc<kYcWarps><<<(unsigned)grid, 32 * kYcWarps, smem, stream>>>(
                        c->d_opx[m], yr->d_slot, yr->d_z0, yr->d_y0, yr->d_rows, yr->n_runs, s.k, W, kWaitPolls,
                        reinterpret_cast<const float2 *>(X), reinterpret_cast<const float2 *>(Y),
                        reinterpret_cast<float2 *>(Z));
                }
                MBC_CUDA_TRY(cudaGetLastError());
                return MBC_OK;
            }
        }
        const int threads = 256;
        const int64_t ngroups = W / 64;
        // one output per warp item: the warps in flight then cover a few
        // hundred consecutive outputs, whose operations read a few rows of
        // the previous stage, and those stay in L2 (with items of many
        // outputs the window spans tens of thousands of outputs and the
        // gathers of X come from HBM: 4.9-6.0 TB/s on 8Be and 4He with all
        // components)
        int64_t zchunk = 1;
        if (tune && tune->zchunk > 0) zchunk = tune->zchunk;
        const int64_t items = ((s.n_z + zchunk - 1) / zchunk) * ngroups;
        const int wpb = threads / 32;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((items + wpb - 1) / wpb, (int64_t)nsm * 64 / wpb));
        {
            TimedLaunch tl(stream);
            note_launch();
            k_large_step_mx2<8><<<(unsigned)grid, threads, 0, stream>>>(
                    c->d_opx[m], c->d_opy[m], s.n_z, s.k, zchunk, W, order == 1 ? 1 : 0, reinterpret_cast<const float2 *>(X),
                    reinterpret_cast<const float2 *>(Y), reinterpret_cast<float2 *>(Z));
        }
        MBC_CUDA_TRY(cudaGetLastError());
        return MBC_OK;
    } else {
    const int threads = 256;
    const int64_t total_warps = (int64_t)nsm * 8 * (threads / 32);
    const int64_t ngroups = W / 32;
    int64_t zchunk = (s.n_z * ngroups + 8 * total_warps - 1) / (8 * total_warps);
    zchunk = std::max<int64_t>(1, std::min<int64_t>(zchunk, 256));
    if (tune && tune->zchunk > 0) zchunk = tune->zchunk;
    const int64_t items = ((s.n_z + zchunk - 1) / zchunk) * ngroups;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((items + 7) / 8, (int64_t)nsm * 8));
    const int order = tune ? tune->wave_order : 0;
    {
        TimedLaunch tl(stream);
        note_launch();
        if (gen)
            k_large_step<Tr, true><<<(unsigned)grid, threads, 0, stream>>>(nullptr, nullptr, gen_step(L, c, m), s.n_z,
                                                                           s.k, zchunk, W, order, X, Y, Z);
        else
            k_large_step<Tr, false><<<(unsigned)grid, threads, 0, stream>>>(c->d_opx[m], c->d_opy[m], GenStep{}, s.n_z,
                                                                            s.k, zchunk, W, order, X, Y, Z);
    }
    MBC_CUDA_TRY(cudaGetLastError());
    return MBC_OK;
    }
}

// Contraction with L (eq. C_final) of every nucleus of the list that ends at
// stage `stage` of the path, from that stage's buffer X ([component][W]);
// deg_per_baryon: homogeneity degree of C per baryon in the scaled inputs (3
// for propagator tiles, 1 for projected blocks).
template <class Tr>
mbc_status contract_parts(const mbc_term_list *L, const DeviceCache *c, int stage, const typename Tr::V *X, int W,
                          const int32_t *sexp, int deg_per_baryon, double2 *Cb, int nsm, cudaStream_t stream) {
    for (const auto &pt : L->parts) {
        if (pt.A != stage || pt.c1 <= pt.c0) continue;
        const int n = pt.c1 - pt.c0;
        const int64_t items = (int64_t)n * (W / 32);
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((items + 7) / 8, (int64_t)nsm * 8));
        note_launch();
        k_large_contract<Tr><<<(unsigned)grid, 256, 0, stream>>>(c->d_fin_off + pt.c0, c->d_fin_z, c->d_fin_l, n, W,
                                                                 X, sexp, deg_per_baryon * pt.A, 1.0 / pt.norm,
                                                                 Cb + (int64_t)pt.c0 * W);
        MBC_CUDA_TRY(cudaGetLastError());
    }
    return MBC_OK;
}

template <class Tr>
mbc_status run_large(const mbc_term_list *L, const DeviceCache *c, const FieldDesc &F, const MomDesc &M,
                     const mbc_tune *tune, int device, cudaStream_t stream, char *scratch, double2 *partial,
                     const LargeSizes &ls, int64_t n_items, int v3p, const double2 *phase) {
    using V = typename Tr::V;
    const int W = ls.W;
    char *p = scratch;
    V *fP = reinterpret_cast<V *>(p);
    p += align256(ls.blk_bytes);
    V *fN = reinterpret_cast<V *>(p);
    p += align256(ls.blk_bytes);
    V *buf[2];
    buf[0] = reinterpret_cast<V *>(p);
    p += align256(ls.stage_bytes);
    buf[1] = reinterpret_cast<V *>(p);
    p += align256(ls.stage_bytes);
    double2 *Cb = reinterpret_cast<double2 *>(p);
    p += align256(ls.c_bytes);
    int32_t *sexp = reinterpret_cast<int32_t *>(p);
    const int nsm = sm_count(device);
    const int nxi = L->nxi, nrow = 3 * L->dim;
    // sites per CTA of the block kernel: 16, or 4 for 24 source columns
    const int ns_blk = nxi > 12 ? 4 : 16;
    const void *blk_kern = ns_blk == 4 ? (const void *)k_large_blocks<Tr, 4> : (const void *)k_large_blocks<Tr, 16>;
    const size_t blk_smem = (size_t)ns_blk * (tile_stride(nrow, nxi) + diquark_stride(nxi)) * sizeof(V);
    {
        int per_sm = 0;
        mbc_status pst = prepare_kernel(blk_kern, device, 512, blk_smem, &per_sm);
        if (pst != MBC_OK) return pst;
        if (per_sm < 1) return MBC_ERR_UNSUPPORTED;
    }
    for (int64_t item0 = 0; item0 < n_items; item0 += W) {
        WaveDesc wv;
        wv.item0 = item0;
        wv.W = W;
        wv.v3 = F.lx * F.ly * F.lz;
        wv.v3p = v3p;
        wv.n_items = n_items;
        note_launch();
        if (ns_blk == 4)
            k_large_blocks<Tr, 4><<<W / 4, 512, blk_smem, stream>>>(F, wv, nrow, nxi, n_g2(L), (int)L->block_size,
                                                                    (int)binom64(nxi, 2), L->need_block[0],
                                                                    L->need_block[1], fP, fN, sexp);
        else
            k_large_blocks<Tr, 16><<<W / 16, 512, blk_smem, stream>>>(F, wv, nrow, nxi, n_g2(L), (int)L->block_size,
                                                                      (int)binom64(nxi, 2), L->need_block[0],
                                                                      L->need_block[1], fP, fN, sexp);
        MBC_CUDA_TRY(cudaGetLastError());
        const V *X = L->path[0] == MBC_PROTON ? fP : fN;
        mbc_status cst = contract_parts<Tr>(L, c, 1, X, W, sexp, 3, Cb, nsm, stream);
        if (cst != MBC_OK) return cst;
        for (size_t m = 0; m < L->steps.size(); ++m) {
            const Step &s = L->steps[m];
            V *Z = buf[(m + 1) & 1];
            const V *Y = s.baryon == MBC_PROTON ? fP : fN;
            if ((cst = launch_step<Tr>(L, c, m, tune, W, nsm, X, Y, Z, stream)) != MBC_OK) return cst;
            X = Z;
            if ((cst = contract_parts<Tr>(L, c, (int)m + 2, X, W, sexp, 3, Cb, nsm, stream)) != MBC_OK) return cst;
        }
        {
            int64_t groups = std::min<int64_t>(W, n_items - item0) / 32;
            note_launch();
            k_large_sitesum<<<(unsigned)groups, 256, 0, stream>>>(F, wv, M, L->n_comp, phase, Cb, partial);
            MBC_CUDA_TRY(cudaGetLastError());
        }
    }
    return MBC_OK;
}

// Momentum-projected blocks: per-site blocks summed over sites with the phase
// (FP64), then the recursion once per (slab, momentum group) item on the wave
// kernels; a group holds the n_sinks momenta of the list's sink functions.
template <class Tr>
mbc_status run_projected(const mbc_term_list *L, const DeviceCache *c, const FieldDesc &F, const MomDesc &M,
                         const mbc_tune *tune, int device, cudaStream_t stream, char *scratch, const double2 *phase,
                         int li, int n_lists, int comp_max, double2 *out, int64_t n_slabs, const LargeSizes &ls) {
    using V = typename Tr::V;
    const int nxi = L->nxi, nrow = 3 * L->dim, n_k = L->n_sinks;
    const int bs = (int)(L->block_size / n_k);  // one sink function: dirac_dim * C(nxi, 2) * nxi
    const int n_groups = M.n_mom / n_k;
    const int v3 = F.lx * F.ly * F.lz;
    const int tps = (v3 + 15) / 16;
    const int64_t n_tiles = n_slabs * tps;
    const int64_t n_out = 2LL * bs;
    char *p = scratch;
    double2 *partial = reinterpret_cast<double2 *>(p);
    p += align256((size_t)n_tiles * M.n_mom * n_out * sizeof(double2));
    double2 *Pf = reinterpret_cast<double2 *>(p);
    p += align256((size_t)n_slabs * M.n_mom * n_out * sizeof(double2));
    const int W = ls.W;
    V *fP = reinterpret_cast<V *>(p);
    p += align256(ls.blk_bytes);
    V *fN = reinterpret_cast<V *>(p);
    p += align256(ls.blk_bytes);
    V *buf[2];
    buf[0] = reinterpret_cast<V *>(p);
    p += align256(ls.stage_bytes);
    buf[1] = reinterpret_cast<V *>(p);
    p += align256(ls.stage_bytes);
    double2 *Cb = reinterpret_cast<double2 *>(p);
    p += align256(ls.c_bytes);
    int32_t *sexp = reinterpret_cast<int32_t *>(p);
    const int nsm = sm_count(device);
    // 1. blocks of every site, phase-weighted tile sums, reduction over tiles
    // FP64 blocks and sums for the FP64 path, FP32 products with compensated
    // FP32 sums for the mixed path
    const bool mx = sizeof(V) == sizeof(float2);
    if (mx && nxi != 6 && nxi != 12) return MBC_ERR_UNSUPPORTED;  // 3 x Dirac dimension x sources
    const void *pkern = !mx ? (const void *)k_project_blocks
                            : nxi == 6 ? (const void *)k_project_blocks_mx<6> : (const void *)k_project_blocks_mx<12>;
    const size_t smem = mx ? project_smem_bytes_mx(nrow, nxi, M.n_mom) : project_smem_bytes(nrow, nxi, M.n_mom);
    {
        int per_sm = 0;
        mbc_status pst = prepare_kernel(pkern, device, 512, smem, &per_sm);
        if (pst != MBC_OK) return pst;
    }
    {
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(n_tiles, (int64_t)nsm * 8));
        {
            TimedLaunch tl(stream);
            note_launch();
            float2 *partial_mx = reinterpret_cast<float2 *>(partial);  // the mixed path's FP32 partials
            if (mx && nxi == 6)
                k_project_blocks_mx<6><<<(unsigned)grid, 512, smem, stream>>>(
                    F, M, phase, nrow, n_g2(L), bs, L->need_block[0], L->need_block[1], tps, n_tiles, partial_mx);
            else if (mx)
                k_project_blocks_mx<12><<<(unsigned)grid, 512, smem, stream>>>(
                    F, M, phase, nrow, n_g2(L), bs, L->need_block[0], L->need_block[1], tps, n_tiles, partial_mx);
            else
                k_project_blocks<<<(unsigned)grid, 512, smem, stream>>>(F, M, phase, nrow, nxi, n_g2(L), bs,
                                                                        (int)binom64(nxi, 2), L->need_block[0],
                                                                        L->need_block[1], tps, n_tiles, partial);
        }
        MBC_CUDA_TRY(cudaGetLastError());
        // thousands of outputs per slab: one thread per output, coalesced
        const int64_t outs = n_slabs * M.n_mom * n_out;
        const unsigned rg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((outs + 255) / 256, (int64_t)nsm * 16));
        note_launch();
        if (mx)
            k_reduce_tiles_cols_mx<<<rg, 256, 0, stream>>>(reinterpret_cast<const float2 *>(partial), n_slabs, tps,
                                                           (int64_t)M.n_mom * n_out, Pf);
        else
            k_reduce_tiles_cols<<<rg, 256, 0, stream>>>(partial, n_slabs, tps, M.n_mom, (int)n_out, F.n_t, 0, 1,
                                                        (int)n_out, Pf);
        MBC_CUDA_TRY(cudaGetLastError());
    }
    // 2. recursion and contraction per item, a wave of W items at a time
    const int64_t n_items = n_slabs * n_groups;
    const int per_spin = (int)(binom64(nxi, 2) * nxi);
    for (int64_t item0 = 0; item0 < n_items; item0 += W) {
        note_launch();
        k_load_proj_blocks<Tr><<<(unsigned)((W + 7) / 8), 256, 0, stream>>>(Pf, n_items, item0, W, bs, per_spin, n_k,
                                                                            M.n_mom, fP, fN, sexp);
        MBC_CUDA_TRY(cudaGetLastError());
        const V *X = L->path[0] == MBC_PROTON ? fP : fN;
        mbc_status cst = contract_parts<Tr>(L, c, 1, X, W, sexp, 1, Cb, nsm, stream);
        if (cst != MBC_OK) return cst;
        for (size_t m = 0; m < L->steps.size(); ++m) {
            const Step &s = L->steps[m];
            V *Z = buf[(m + 1) & 1];
            const V *Y = s.baryon == MBC_PROTON ? fP : fN;
            if ((cst = launch_step<Tr>(L, c, m, tune, W, nsm, X, Y, Z, stream)) != MBC_OK) return cst;
            X = Z;
            if ((cst = contract_parts<Tr>(L, c, (int)m + 2, X, W, sexp, 1, Cb, nsm, stream)) != MBC_OK) return cst;
        }
        {
            const int64_t tot = (int64_t)L->n_comp * W;
            const unsigned g2 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 65535));
            note_launch();
            k_write_items<<<g2, 256, 0, stream>>>(Cb, n_items, item0, W, L->n_comp, n_groups, F.n_t, li, n_lists,
                                                  comp_max, out);
            MBC_CUDA_TRY(cudaGetLastError());
        }
    }
    return MBC_OK;
}

size_t projected_bytes(const mbc_term_list *L, const MomDesc &M, int v3, int64_t n_slabs, const LargeSizes &ls) {
    const int tps = (v3 + 15) / 16;
    const int64_t n_out = 2 * (L->block_size / L->n_sinks);
    return align256((size_t)n_slabs * tps * M.n_mom * n_out * sizeof(double2)) +
           align256((size_t)n_slabs * M.n_mom * n_out * sizeof(double2)) + 2 * align256(ls.blk_bytes) +
           2 * align256(ls.stage_bytes) + align256(ls.c_bytes) + align256(ls.sexp_bytes);
}

}  // namespace

void free_device_cache(mbc_term_list *list) {
    std::lock_guard<std::mutex> g(list->dev_mu);
    for (auto *c : list->dev) free_cache(c);
    list->dev.clear();
}

}  // namespace mbc

using namespace mbc;

namespace {

// Streams and events of the host-memory pipeline, kept per (device, caller
// stream) like the scratch: a copy stream and two compute streams whose
// contractions of consecutive chunks may overlap (the tail of one with the
// start of the next).
struct Pipe {
    cudaStream_t copy = nullptr, comp[2] = {nullptr, nullptr};
    cudaEvent_t start = nullptr, ready[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr},
                done[2] = {nullptr, nullptr};
};
std::mutex g_pipe_mu;
std::map<std::pair<int, cudaStream_t>, Pipe> g_pipes;

mbc_status get_pipe(int device, cudaStream_t s, Pipe **out) {
    std::lock_guard<std::mutex> g(g_pipe_mu);
    auto it = g_pipes.find({device, s});
    if (it != g_pipes.end()) {
        *out = &it->second;
        return MBC_OK;
    }
    Pipe p;
    bool ok = cudaStreamCreateWithFlags(&p.copy, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaStreamCreateWithFlags(&p.comp[b], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&p.ready[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p.used[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p.done[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return MBC_ERR_CUDA;  // the partial set leaks a few handles, the call fails cleanly
    *out = &(g_pipes[{device, s}] = p);
    return MBC_OK;
}

void release_pipes(int device) {
    std::lock_guard<std::mutex> g(g_pipe_mu);
    for (auto it = g_pipes.begin(); it != g_pipes.end();) {
        if (it->first.first != device) {
            ++it;
            continue;
        }
        Pipe &p = it->second;
        cudaStreamSynchronize(p.copy);
        cudaStreamDestroy(p.copy);
        cudaEventDestroy(p.start);
        for (int b = 0; b < 2; ++b) {
            cudaStreamSynchronize(p.comp[b]);
            cudaStreamDestroy(p.comp[b]);
            cudaEventDestroy(p.ready[b]);
            cudaEventDestroy(p.used[b]);
            cudaEventDestroy(p.done[b]);
        }
        it = g_pipes.erase(it);
    }
}

// Host-memory mode with the copies overlapped: the evaluated time slices go
// to the device in chunks through two staging buffers; the copy stream copies
// chunk i + 1 while a compute stream contracts chunk i (a device-memory call
// with the same lists and options), the two compute streams alternating so
// that consecutive chunks' kernels may overlap, and each chunk's results are
// copied back into their rows of out.
mbc_status contract_host_pipelined(const mbc_props *props, const mbc_term_list *const *lists, int32_t n_lists,
                                   const mbc_contract_opts *opts, void *out, cudaStream_t stream, int t0, int n_t,
                                   int64_t stride_cfg, int64_t stride_t, int64_t site_elems, int n_out_mom,
                                   int comp_max) {
    const size_t elem = props->dtype == MBC_C128 ? 16 : 8;
    const int64_t v3 = (int64_t)props->lx * props->ly * props->lz;
    const size_t slab_bytes = (size_t)v3 * site_elems * elem;
    const size_t total = (size_t)props->n_cfg * n_t * slab_bytes;
    int n_chunks = (int)std::min<size_t>(8, std::max<size_t>(2, total / ((size_t)64 << 20)));
    n_chunks = std::min(n_chunks, n_t);
    const int ct = (n_t + n_chunks - 1) / n_chunks;
    n_chunks = (n_t + ct - 1) / ct;
    const size_t buf_bytes = (size_t)props->n_cfg * ct * slab_bytes;
    const size_t row_out = (size_t)n_out_mom * comp_max * sizeof(double2);  // one (cfg, list, t)
    const size_t chunk_out = (size_t)props->n_cfg * n_lists * ct * row_out;
    int device = 0;
    MBC_CUDA_TRY(cudaGetDevice(&device));
    Pipe *pp = nullptr;
    mbc_status st = get_pipe(device, stream, &pp);
    if (st != MBC_OK) return st;
    const Pipe &P = *pp;
    // results gather on the device and go to the host in one copy at the end:
    // a copy into pageable host memory would hold the host thread until the
    // chunk is done and serialise the pipeline
    const size_t full_out = (size_t)props->n_cfg * n_lists * n_t * row_out;
    char *stage = nullptr;
    MBC_CUDA_TRY(cudaMallocAsync((void **)&stage, 2 * buf_bytes + 2 * align256(chunk_out) + align256(full_out), stream));
    char *buf[2] = {stage, stage + buf_bytes};
    char *cout[2] = {stage + 2 * buf_bytes, stage + 2 * buf_bytes + align256(chunk_out)};
    char *dout = stage + 2 * buf_bytes + 2 * align256(chunk_out);
    auto cuda_ok = [&](cudaError_t e) {
        if (e != cudaSuccess && st == MBC_OK) st = MBC_ERR_CUDA;
        return st == MBC_OK;
    };
    // every stream of the pipeline starts after the staging allocation
    if (cuda_ok(cudaEventRecord(P.start, stream)) && cuda_ok(cudaStreamWaitEvent(P.copy, P.start, 0)))
        for (int b = 0; b < 2; ++b) cuda_ok(cudaStreamWaitEvent(P.comp[b], P.start, 0));
    const char *host = reinterpret_cast<const char *>(props->s_u);
    char *hout = reinterpret_cast<char *>(out);
    for (int i = 0; i < n_chunks && st == MBC_OK; ++i) {
        const int b = i & 1;
        const int ta = t0 + i * ct, nc = std::min(ct, t0 + n_t - ta);
        if (i >= 2 && !cuda_ok(cudaStreamWaitEvent(P.copy, P.used[b], 0))) break;  // chunk i - 2 done with buf[b]
        for (int cfg = 0; cfg < props->n_cfg && st == MBC_OK; ++cfg) {
            const char *src = host + ((size_t)cfg * stride_cfg + (size_t)ta * stride_t) * elem;
            char *dst = buf[b] + (size_t)cfg * nc * slab_bytes;
            if (stride_t * (int64_t)elem == (int64_t)slab_bytes) {
                cuda_ok(cudaMemcpyAsync(dst, src, nc * slab_bytes, cudaMemcpyHostToDevice, P.copy));
            } else {
                for (int t = 0; t < nc && st == MBC_OK; ++t)
                    cuda_ok(cudaMemcpyAsync(dst + t * slab_bytes, src + (size_t)t * stride_t * elem, slab_bytes,
                                            cudaMemcpyHostToDevice, P.copy));
            }
        }
        if (st != MBC_OK || !cuda_ok(cudaEventRecord(P.ready[b], P.copy)) ||
            !cuda_ok(cudaStreamWaitEvent(P.comp[b], P.ready[b], 0)))
            break;
        mbc_props sub = *props;
        sub.s_u = sub.s_d = buf[b];
        sub.memory = MBC_MEM_DEVICE;
        sub.nt = nc;
        sub.stride_t = v3 * site_elems;
        sub.stride_cfg = (int64_t)nc * v3 * site_elems;
        mbc_contract_opts so = *opts;
        so.t0 = 0;
        so.t1 = nc;
        st = mbc_contract(&sub, lists, n_lists, &so, cout[b], P.comp[b]);
        if (st != MBC_OK || !cuda_ok(cudaEventRecord(P.used[b], P.comp[b]))) break;
        cuda_ok(cudaMemcpy2DAsync(dout + (size_t)(ta - t0) * row_out, (size_t)n_t * row_out, cout[b],
                                  (size_t)nc * row_out, (size_t)nc * row_out, (size_t)props->n_cfg * n_lists,
                                  cudaMemcpyDeviceToDevice, P.comp[b]));
    }
    // the caller's stream frees the staging after both compute streams and
    // the copy stream are done
    for (int b = 0; b < 2; ++b) {
        cudaEventRecord(P.done[b], P.comp[b]);
        cudaStreamWaitEvent(stream, P.done[b], 0);
    }
    cudaEventRecord(P.start, P.copy);
    cudaStreamWaitEvent(stream, P.start, 0);
    if (st == MBC_OK) cuda_ok(cudaMemcpyAsync(hout, dout, full_out, cudaMemcpyDeviceToHost, stream));
    cudaFreeAsync(stage, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess && st == MBC_OK) st = MBC_ERR_CUDA;
    if (st == MBC_OK) st = take_device_status(stream);  // synchronous call: report a latched timeout
    return st;
}

}  // namespace

extern "C" mbc_status mbc_contract(const mbc_props *props, const mbc_term_list *const *lists, int32_t n_lists,
                                   const mbc_contract_opts *opts, void *out, void *stream_v) {
    if (!props || !lists || n_lists < 1 || !opts || !out) return MBC_ERR_INVALID_ARG;
    if (!props->s_u || !props->s_d) return MBC_ERR_INVALID_ARG;
    if (props->s_u != props->s_d) return MBC_ERR_UNSUPPORTED;  // u = d fields only
    if (props->dtype != MBC_C128 && props->dtype != MBC_C64) return MBC_ERR_INVALID_ARG;
    if (props->memory != MBC_MEM_DEVICE && props->memory != MBC_MEM_HOST) return MBC_ERR_INVALID_ARG;
    if (props->n_cfg < 1 || props->nt < 1 || props->lx < 1 || props->ly < 1 || props->lz < 1) return MBC_ERR_INVALID_ARG;
    if (opts->precision != MBC_FP64 && opts->precision != MBC_MIXED) return MBC_ERR_INVALID_ARG;
    if (opts->n_mom < 1 || opts->n_mom > kMaxMom || !opts->mom) return MBC_ERR_INVALID_ARG;
    const int t0 = opts->t0, t1 = opts->t1 == 0 ? props->nt : opts->t1;
    if (t0 < 0 || t1 > props->nt || t1 <= t0) return MBC_ERR_INVALID_ARG;
    const int n_src = props->n_src == 0 ? 1 : props->n_src;
    if (n_src < 1 || n_src > 4) return MBC_ERR_INVALID_ARG;
    if (opts->sink_mode != MBC_SINK_POINT && opts->sink_mode != MBC_SINK_BLOCK_MOMENTUM) return MBC_ERR_INVALID_ARG;
    // sink functions per list: 1 for point sinks; with projected blocks every
    // list has the same n_k and the momenta come in groups of n_k (Sec. 6)
    const int n_k = lists[0] ? std::max(1, (int)lists[0]->n_sinks) : 1;
    for (int i = 0; i < n_lists; ++i) {
        if (!lists[i]) return MBC_ERR_INVALID_ARG;
        if (lists[i]->n_sources != n_src) return MBC_ERR_INVALID_ARG;  // list and field disagree
        // source tiles: up to 24 columns with point sinks (two relativistic
        // sources), 12 with momentum-projected blocks
        if (lists[i]->nxi > 24 || (lists[i]->nxi > 12 && opts->sink_mode != MBC_SINK_POINT))
            return MBC_ERR_UNSUPPORTED;
        if (lists[i]->n_sinks != n_k) return MBC_ERR_INVALID_ARG;
    }
    if (n_k > 1 && opts->sink_mode == MBC_SINK_POINT) return MBC_ERR_UNSUPPORTED;  // one sink point per site
    if (opts->n_mom % n_k != 0) return MBC_ERR_INVALID_ARG;
    const int n_out_mom = opts->n_mom / n_k;  // output momentum (group) index
    const int64_t v3 = (int64_t)props->lx * props->ly * props->lz;
    if (v3 > (1LL << 30)) return MBC_ERR_INVALID_ARG;
    const int64_t site_elems = 144LL * n_src;
    const int64_t stride_t = props->stride_t ? props->stride_t : v3 * site_elems;
    const int64_t stride_cfg = props->stride_cfg ? props->stride_cfg : stride_t * props->nt;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
    int device = 0;
    MBC_CUDA_TRY(cudaGetDevice(&device));
    mbc_status st = ensure_constants(device);
    if (st != MBC_OK) return st;

    int comp_max = 1;
    for (int i = 0; i < n_lists; ++i) comp_max = std::max(comp_max, (int)lists[i]->n_comp);
    const int n_t = t1 - t0;
    const size_t out_bytes = (size_t)props->n_cfg * n_lists * n_t * n_out_mom * comp_max * sizeof(double2);
    // overlapping copies pays once the field is large enough for chunks of
    // several MB; smaller fields are staged in one copy
    const size_t field_bytes = (size_t)props->n_cfg * n_t * v3 * site_elems * (props->dtype == MBC_C128 ? 16 : 8);
    if (props->memory == MBC_MEM_HOST && n_t >= 2 && field_bytes >= ((size_t)32 << 20))
        return contract_host_pipelined(props, lists, n_lists, opts, out, stream, t0, n_t, stride_cfg, stride_t,
                                       site_elems, n_out_mom, comp_max);

    // host-memory mode: stage the evaluated slices on the device
    const void *field = props->s_u;
    void *dev_out = out;
    const size_t elem = props->dtype == MBC_C128 ? 16 : 8;
    void *staging = nullptr;
    int64_t f_stride_cfg = stride_cfg, f_stride_t = stride_t, f_t_shift = 0;
    if (props->memory == MBC_MEM_HOST) {
        const size_t slab_bytes = (size_t)v3 * site_elems * elem;
        const size_t in_bytes = (size_t)props->n_cfg * n_t * slab_bytes;
        MBC_CUDA_TRY(cudaMallocAsync(&staging, in_bytes + out_bytes, stream));
        for (int cfg = 0; cfg < props->n_cfg; ++cfg) {
            const char *src = reinterpret_cast<const char *>(props->s_u) + ((size_t)cfg * stride_cfg + (size_t)t0 * stride_t) * elem;
            char *dst = reinterpret_cast<char *>(staging) + (size_t)cfg * n_t * slab_bytes;
            if (stride_t * (int64_t)elem == (int64_t)slab_bytes) {
                MBC_CUDA_TRY(cudaMemcpyAsync(dst, src, n_t * slab_bytes, cudaMemcpyHostToDevice, stream));
            } else {
                for (int t = 0; t < n_t; ++t)
                    MBC_CUDA_TRY(cudaMemcpyAsync(dst + t * slab_bytes, src + (size_t)t * stride_t * elem, slab_bytes,
                                                 cudaMemcpyHostToDevice, stream));
            }
        }
        field = staging;
        f_stride_t = v3 * site_elems;
        f_stride_cfg = f_stride_t * n_t;
        f_t_shift = t0;
        dev_out = reinterpret_cast<char *>(staging) + in_bytes;
    }

    FieldDesc F;
    F.s = field;
    F.dtype = props->dtype == MBC_C128 ? 0 : 1;
    F.n_cfg = props->n_cfg;
    F.nt = props->nt;
    F.lx = props->lx;
    F.ly = props->ly;
    F.lz = props->lz;
    F.stride_cfg = f_stride_cfg;
    F.stride_t = f_stride_t;
    F.t0 = (int)(t0 - f_t_shift);
    F.n_t = n_t;
    F.n_src = n_src;
    // with staging, slice t0 sits at index 0: shift the base instead
    MomDesc M;
    std::memset(&M, 0, sizeof(M));
    M.n_mom = opts->n_mom;
    for (int q = 0; q < opts->n_mom; ++q)
        for (int d = 0; d < 3; ++d) M.mom[q][d] = opts->mom[3 * q + d];

    cudaError_t ce = cudaMemsetAsync(dev_out, 0, out_bytes, stream);
    if (ce != cudaSuccess) return MBC_ERR_CUDA;
    const int64_t n_slabs = (int64_t)props->n_cfg * n_t;
    const bool mixed = opts->precision == MBC_MIXED;

    if (opts->sink_mode == MBC_SINK_BLOCK_MOMENTUM) {
        // every baryon's block projected to the momentum, one recursion per item
        const int64_t n_items_p = n_slabs * n_out_mom;
        std::vector<DeviceCache *> cs((size_t)n_lists, nullptr);
        std::vector<LargeSizes> lsz((size_t)n_lists);
        size_t need = 0;
        for (int li = 0; li < n_lists; ++li) {
            const mbc_term_list *L = lists[li];
            if (L->pauli_forbidden || L->n_comp == 0) continue;
            cs[(size_t)li] = get_cache(L, device, st);
            if (!cs[(size_t)li]) return st;
            lsz[(size_t)li] = mixed ? large_sizes<MixedTraits>(L, cs[(size_t)li], opts->tune, n_items_p)
                                    : large_sizes<FP64Traits>(L, cs[(size_t)li], opts->tune, n_items_p);
            need = std::max(need, projected_bytes(L, M, (int)v3, n_slabs, lsz[(size_t)li]));
        }
        const size_t phase_bytes_p = align256((size_t)v3 * M.n_mom * sizeof(double2));
        void *scr_p = nullptr;
        if ((st = scratch_get(device, stream, phase_bytes_p + need, &scr_p)) != MBC_OK) return st;
        double2 *phase_p = reinterpret_cast<double2 *>(scr_p);
        unsigned pg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((v3 * M.n_mom + 255) / 256, 4096));
        note_launch();
        k_phase_table<<<pg, 256, 0, stream>>>(F, M, phase_p);
        MBC_CUDA_TRY(cudaGetLastError());
        for (int li = 0; li < n_lists; ++li) {
            if (!cs[(size_t)li]) continue;
            char *rest_p = reinterpret_cast<char *>(scr_p) + phase_bytes_p;
            st = mixed ? run_projected<MixedTraits>(lists[li], cs[(size_t)li], F, M, opts->tune, device, stream,
                                                    rest_p, phase_p, li, n_lists, comp_max,
                                                    reinterpret_cast<double2 *>(dev_out), n_slabs, lsz[(size_t)li])
                       : run_projected<FP64Traits>(lists[li], cs[(size_t)li], F, M, opts->tune, device, stream, rest_p,
                                                   phase_p, li, n_lists, comp_max,
                                                   reinterpret_cast<double2 *>(dev_out), n_slabs, lsz[(size_t)li]);
            if (st != MBC_OK) return st;
        }
    } else {
    // plan every list: regime and scratch bytes; small-regime lists go into
    // batches (most operations per site first) contracted by one launch each
    const int v3p = (int)((v3 + 31) / 32 * 32);
    const int64_t n_items = n_slabs * v3p;
    const int regime = opts->tune ? opts->tune->regime : 0;
    std::vector<DeviceCache *> caches((size_t)n_lists, nullptr);
    std::vector<int> small_ids, large_ids;
    for (int li = 0; li < n_lists; ++li) {
        const mbc_term_list *L = lists[li];
        if (L->pauli_forbidden || L->n_comp == 0) continue;  // identically zero
        caches[(size_t)li] = get_cache(L, device, st);
        if (!caches[(size_t)li]) return st;
        bool small = caches[(size_t)li]->small_ok && (!mixed || caches[(size_t)li]->ls_ok) && regime != 2;
        if (small) {  // the list alone must fit the shared-memory kernel
            int32_t ss, cs;
            small = size_small_batch({caches[(size_t)li]}, F, opts->tune, mixed, ss, cs).ok;
        }
        if (regime == 1 && !small) return MBC_ERR_UNSUPPORTED;
        (small ? small_ids : large_ids).push_back(li);
    }
    std::stable_sort(small_ids.begin(), small_ids.end(), [&](int a, int b) {
        return lists[a]->stats.n_ops_total > lists[b]->stats.n_ops_total;
    });
    struct BatchRun {
        std::vector<int> ids;
        SmallLaunch sl;
        SmallBatch B;
        size_t part_bytes = 0;
    };
    std::vector<BatchRun> batches;
    for (size_t i = 0; i < small_ids.size();) {
        // grow the batch while the combined shared-memory footprint still fits
        BatchRun br;
        std::vector<const DeviceCache *> cs;
        while (i < small_ids.size() && (int)br.ids.size() < kMaxBatch) {
            std::vector<const DeviceCache *> trial = cs;
            trial.push_back(caches[(size_t)small_ids[i]]);
            int32_t ss, cc;
            SmallLaunch l = size_small_batch(trial, F, opts->tune, mixed, ss, cc);
            if (!l.ok && !br.ids.empty()) break;
            cs = trial;
            br.ids.push_back(small_ids[i]);
            ++i;
        }
        std::memset(&br.B, 0, sizeof(br.B));
        br.sl = size_small_batch(cs, F, opts->tune, mixed, br.B.site_stride, br.B.comp_stride, sm_count(device));
        br.B.n_lists = (int)br.ids.size();
        br.B.tiles_per_slab = br.sl.tiles_per_slab;
        int64_t items = 0, poff = 0;
        for (int j = 0; j < br.B.n_lists; ++j) {
            const DeviceCache *c = caches[(size_t)br.ids[(size_t)j]];
            br.B.plan[j] = c->sp;
            br.B.item_base[j] = items;
            br.B.partial_off[j] = poff;
            const int64_t tiles = n_slabs * br.sl.tiles_per_slab;
            items += tiles;
            poff += tiles * M.n_mom * c->sp.n_comp;
        }
        br.B.item_base[br.B.n_lists] = items;
        br.B.total_items = items;
        // lists with the same tile shape and S / diquark / block offsets share
        // one tile load and block computation per site: items become tiles
        bool share = br.B.n_lists > 1;
        for (int j = 1; j < br.B.n_lists && share; ++j) {
            const SmallPlan &a = br.B.plan[0], &b = br.B.plan[j];
            share = a.nxi == b.nxi && a.dim == b.dim && a.n_g2 == b.n_g2 && a.block_size == b.block_size &&
                    a.npair == b.npair && a.s_off == b.s_off && a.q_off == b.q_off && a.blk_off[0] == b.blk_off[0] &&
                    a.blk_off[1] == b.blk_off[1];
        }
        if (share) {
            br.B.shared = 1;
            for (int j = 0; j < br.B.n_lists; ++j)
                for (int b = 0; b < 2; ++b) br.B.need_union[b] |= br.B.plan[j].need_blk[b];
            br.B.total_items = n_slabs * br.sl.tiles_per_slab;
        }
        br.part_bytes = (size_t)poff * sizeof(double2);
        batches.push_back(br);
    }
    size_t small_bytes = 0;
    for (auto &br : batches) small_bytes += 256 + align256(br.part_bytes);
    size_t large_bytes = 0;
    std::vector<LargeSizes> lsz((size_t)n_lists);
    for (int li : large_ids) {
        const mbc_term_list *L = lists[li];
        DeviceCache *c = caches[(size_t)li];
        lsz[(size_t)li] = mixed ? large_sizes<MixedTraits>(L, c, opts->tune, n_items)
                                : large_sizes<FP64Traits>(L, c, opts->tune, n_items);
        const LargeSizes &ls = lsz[(size_t)li];
        const size_t pbytes = (size_t)(n_items / 32) * M.n_mom * L->n_comp * sizeof(double2);
        large_bytes = std::max(large_bytes, align256(pbytes) + 2 * align256(ls.blk_bytes) +
                                                2 * align256(ls.stage_bytes) + align256(ls.c_bytes) +
                                                align256(ls.sexp_bytes));
    }
    const size_t phase_bytes = align256((size_t)v3 * M.n_mom * sizeof(double2));
    void *scr = nullptr;
    if ((st = scratch_get(device, stream, phase_bytes + small_bytes + large_bytes, &scr)) != MBC_OK) return st;
    double2 *phase = reinterpret_cast<double2 *>(scr);
    {
        unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((v3 * M.n_mom + 255) / 256, 4096));
        note_launch();
        k_phase_table<<<grid, 256, 0, stream>>>(F, M, phase);
        MBC_CUDA_TRY(cudaGetLastError());
    }
    char *cur = reinterpret_cast<char *>(scr) + phase_bytes;
    auto reduce = [&](int li, const double2 *partial, int tiles_per_slab) -> mbc_status {
        const mbc_term_list *L = lists[li];
        int64_t outs = n_slabs * M.n_mom * L->n_comp;
        unsigned grid = (unsigned)std::min<int64_t>((outs + 7) / 8, 65535);
        note_launch();
        k_reduce_tiles<<<std::max(grid, 1u), 256, 0, stream>>>(partial, n_slabs, tiles_per_slab, M.n_mom, L->n_comp,
                                                              n_t, li, n_lists, comp_max,
                                                              reinterpret_cast<double2 *>(dev_out));
        MBC_CUDA_TRY(cudaGetLastError());
        return MBC_OK;
    };
    for (auto &br : batches) {
        br.B.counter = reinterpret_cast<unsigned long long *>(cur);
        double2 *partial = reinterpret_cast<double2 *>(cur + 256);
        cur += 256 + align256(br.part_bytes);
        if ((st = launch_small_batch(br.B, F, M, br.sl, mixed, device, stream, phase, partial, true)) != MBC_OK)
            return st;
        for (int j = 0; j < br.B.n_lists; ++j)
            if ((st = reduce(br.ids[(size_t)j], partial + br.B.partial_off[j], br.sl.tiles_per_slab)) != MBC_OK)
                return st;
    }
    for (int li : large_ids) {
        const mbc_term_list *L = lists[li];
        double2 *partial = reinterpret_cast<double2 *>(cur);
        const size_t pbytes = (size_t)(n_items / 32) * M.n_mom * L->n_comp * sizeof(double2);
        char *bufs = cur + align256(pbytes);
        st = mixed ? run_large<MixedTraits>(L, caches[(size_t)li], F, M, opts->tune, device, stream, bufs, partial,
                                            lsz[(size_t)li], n_items, v3p, phase)
                   : run_large<FP64Traits>(L, caches[(size_t)li], F, M, opts->tune, device, stream, bufs, partial,
                                           lsz[(size_t)li], n_items, v3p, phase);
        if (st != MBC_OK) return st;
        if ((st = reduce(li, partial, v3p / 32)) != MBC_OK) return st;
    }

    }  // point sinks

    if (props->memory == MBC_MEM_HOST) {
        MBC_CUDA_TRY(cudaMemcpyAsync(out, dev_out, out_bytes, cudaMemcpyDeviceToHost, stream));
        MBC_CUDA_TRY(cudaFreeAsync(staging, stream));
        MBC_CUDA_TRY(cudaStreamSynchronize(stream));
        return take_device_status(stream);  // synchronous call: report a latched timeout
    }
    return MBC_OK;
}

extern "C" mbc_status mbc_sync_status(void *stream_v) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return MBC_ERR_CUDA;
    }
    return mbc::take_device_status(stream);
}

namespace mbc {
// After a synchronisation of stream: the kernels' latched status word (a
// bounded wait that ran out), read and cleared; MBC_ERR_TIMEOUT if set.
mbc_status take_device_status(cudaStream_t stream) {
    unsigned int word = 0;
    if (cudaMemcpyFromSymbolAsync(&word, g_device_status, sizeof(word), 0, cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return MBC_ERR_CUDA;
    }
    if (word) {
        const unsigned int zero = 0;
        if (cudaMemcpyToSymbolAsync(g_device_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            (void)cudaGetLastError();
            return MBC_ERR_CUDA;
        }
        return MBC_ERR_TIMEOUT;
    }
    return MBC_OK;
}
}  // namespace mbc

extern "C" mbc_status mbc_check_wait_timeout(uint32_t polls, void *stream_v) {
    if (polls < 1 || polls > (1u << 20)) return MBC_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
    k_wait_timeout_check<<<1, 32, 0, stream>>>(polls);
    MBC_CUDA_TRY(cudaGetLastError());
    return MBC_OK;
}

extern "C" void mbc_release_scratch(void) {
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return;
    {
        std::lock_guard<std::mutex> g(g_scratch_mu);
        for (auto it = g_scratch.begin(); it != g_scratch.end();) {
            if (it->first.first == device) {
                cudaStreamSynchronize(it->first.second);
                cudaFree(it->second.p);
                it = g_scratch.erase(it);
            } else {
                ++it;
            }
        }
    }
    release_pipes(device);  // after the scratch of its compute streams
}

extern "C" void mbc_timing_enable(int32_t on) {
    TimingState &t = timing();
    std::lock_guard<std::mutex> g(t.mu);
    t.on = on != 0;
}

extern "C" mbc_status mbc_timing_read(double *ms, int64_t *launches) {
    if (!ms || !launches) return MBC_ERR_INVALID_ARG;
    TimingState &t = timing();
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    {
        std::lock_guard<std::mutex> g(t.mu);
        ev.swap(t.ev);
    }
    double tot = 0.0;
    mbc_status st = MBC_OK;
    for (auto &e : ev) {
        float f = 0.f;
        if (cudaEventSynchronize(e.second) != cudaSuccess || cudaEventElapsedTime(&f, e.first, e.second) != cudaSuccess) {
            (void)cudaGetLastError();
            st = MBC_ERR_CUDA;
        }
        tot += f;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    *ms = tot;
    *launches = (int64_t)ev.size();
    return st;
}

extern "C" mbc_status mbc_fma_probe(int32_t precision, double *flops) {
    if (!flops || (precision != MBC_FP64 && precision != MBC_MIXED)) return MBC_ERR_INVALID_ARG;
    int device = 0;
    MBC_CUDA_TRY(cudaGetDevice(&device));
    const int nsm = sm_count(device);
    const int threads = 256;
    // one full wave: every SM runs as many probe blocks as fit at once
    int per_sm = 0;
    if (precision == MBC_FP64)
        MBC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe64, threads, 0));
    else
        MBC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe32, threads, 0));
    const int blocks = nsm * std::max(1, per_sm);
    // tens of milliseconds per launch (clocks settle, launch cost vanishes)
    const int iters = precision == MBC_FP64 ? 2048 : 65536;
    void *buf = nullptr;
    MBC_CUDA_TRY(cudaMalloc(&buf, (size_t)threads * blocks * sizeof(double)));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a);
        if (precision == MBC_FP64)
            k_fma_probe64<<<blocks, threads>>>((double *)buf, iters);
        else
            k_fma_probe32<<<blocks, threads>>>((float *)buf, iters);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0) best = std::min(best, ms);
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    if (e != cudaSuccess) return MBC_ERR_CUDA;
    const double fmas = precision == MBC_FP64 ? probe64_fmas(iters) : probe32_fmas(iters);
    *flops = 2.0 * fmas * (double)threads * blocks / (best * 1e-3);
    return MBC_OK;
}

// ---- contraction without allocation ------------------------------------------
// Callers that must not allocate device memory in steady state (services
// whose device memory is reserved up front by their own pool, so that a
// cudaMalloc would fail or fragment it; real-time loops, where cudaMalloc and
// cudaFree may synchronise the device) use mbc_contract_noalloc. Its scratch - the momentum phase table and the
// per-tile partial sums of the FP64 shared-memory kernel - lives in one
// static device array of kStaticScratchBytes, which every GPU that loads the
// library holds until the process exits.
namespace {
constexpr size_t kStaticScratchBytes = (size_t)8 << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
std::mutex g_static_mu;
std::map<int, void *> g_static_addr;  // device ordinal -> device address of g_static_scratch

// The host-side name of g_static_scratch is only a stand-in: the device
// address comes from cudaGetSymbolAddress, once per device, with that device
// current.
mbc_status static_scratch_address(int device, void **ptr) {
    std::lock_guard<std::mutex> g(g_static_mu);
    auto it = g_static_addr.find(device);
    if (it != g_static_addr.end()) {
        *ptr = it->second;
        return MBC_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
        (void)cudaGetLastError();
        return MBC_ERR_CUDA;
    }
    g_static_addr[device] = p;
    *ptr = p;
    return MBC_OK;
}

DeviceCache *find_cache(const mbc_term_list *Lc, int device) {
    mbc_term_list *L = const_cast<mbc_term_list *>(Lc);
    std::lock_guard<std::mutex> g(L->dev_mu);
    return device < (int)L->dev.size() ? L->dev[(size_t)device] : nullptr;
}
}  // namespace

extern "C" mbc_status mbc_contract_noalloc(const mbc_props *props, const mbc_term_list *list,
                                           const mbc_contract_opts *opts, void *out, void *stream_v) {
    // ---- host-only checks: nothing below touches the device before they pass
    if (!props || !list || !opts || !out || !props->s_u || !props->s_d) return MBC_ERR_INVALID_ARG;
    if (props->s_u != props->s_d) return MBC_ERR_UNSUPPORTED;
    if (list->n_sources != 1 || list->n_sinks != 1) return MBC_ERR_UNSUPPORTED;
    if (props->n_src > 1) return MBC_ERR_UNSUPPORTED;
    if (props->memory != MBC_MEM_DEVICE || opts->precision != MBC_FP64) return MBC_ERR_UNSUPPORTED;
    if (opts->sink_mode != MBC_SINK_POINT) return MBC_ERR_UNSUPPORTED;
    if (props->dtype != MBC_C128 && props->dtype != MBC_C64) return MBC_ERR_INVALID_ARG;
    if (props->n_cfg < 1 || props->nt < 1 || props->lx < 1 || props->ly < 1 || props->lz < 1) return MBC_ERR_INVALID_ARG;
    if (opts->n_mom < 1 || opts->n_mom > kMaxMom || !opts->mom) return MBC_ERR_INVALID_ARG;
    const int t0 = opts->t0, t1 = opts->t1 == 0 ? props->nt : opts->t1;
    if (t0 < 0 || t1 > props->nt || t1 <= t0) return MBC_ERR_INVALID_ARG;
    const int64_t v3 = (int64_t)props->lx * props->ly * props->lz;
    if (v3 > (1LL << 30)) return MBC_ERR_INVALID_ARG;
    const int n_t = t1 - t0;
    const int64_t n_slabs = (int64_t)props->n_cfg * n_t;
    const int comp_max = std::max(1, (int)list->n_comp);
    const size_t out_bytes = (size_t)n_slabs * opts->n_mom * comp_max * sizeof(double2);
    const int64_t stride_t = props->stride_t ? props->stride_t : v3 * 144;
    FieldDesc F;
    F.s = props->s_u;
    F.dtype = props->dtype == MBC_C128 ? 0 : 1;
    F.n_cfg = props->n_cfg;
    F.nt = props->nt;
    F.lx = props->lx;
    F.ly = props->ly;
    F.lz = props->lz;
    F.stride_t = stride_t;
    F.stride_cfg = props->stride_cfg ? props->stride_cfg : stride_t * props->nt;
    F.t0 = t0;
    F.n_t = n_t;
    F.n_src = 1;
    SmallPlan hp;
    int64_t site_entries = 0;
    const bool zero = list->pauli_forbidden || list->n_comp == 0;
    size_t phase_bytes = 0, part_bytes = 0;
    SmallLaunch l;
    if (!zero) {
        std::vector<int> part_off;
        if (!plan_small(list, hp, site_entries, part_off)) return MBC_ERR_UNSUPPORTED;  // relativistic lists: no static variant
        // the launch shape the kernel will run with, and from it the bytes
        // of the tile partials (one sizing, used for the check and the launch)
        l = size_small_tiles((int32_t)site_entries, hp.n_comp, F, opts->tune, false);
        if (!l.ok) return MBC_ERR_UNSUPPORTED;
        const int64_t tiles = n_slabs * l.tiles_per_slab;
        phase_bytes = align256((size_t)v3 * opts->n_mom * sizeof(double2));
        part_bytes = (size_t)tiles * opts->n_mom * hp.n_comp * sizeof(double2);
        if (phase_bytes + 256 + part_bytes > kStaticScratchBytes) return MBC_ERR_UNSUPPORTED;  // beyond 8 MiB
    }
    // ---- device work: no allocation from here on
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
    int device = 0;
    MBC_CUDA_TRY(cudaGetDevice(&device));
    if (zero) {
        MBC_CUDA_TRY(cudaMemsetAsync(out, 0, out_bytes, stream));
        return MBC_OK;
    }
    DeviceCache *c = find_cache(list, device);
    if (!c || !c->small_ok) return MBC_ERR_INVALID_ARG;  // the list's device copy must exist already
    if (c->site_entries != site_entries || c->sp.n_comp != hp.n_comp) return MBC_ERR_INVALID_ARG;
    void *scr = nullptr;
    mbc_status st = static_scratch_address(device, &scr);
    if (st != MBC_OK) return st;
    if ((st = ensure_constants(device)) != MBC_OK) return st;
    MomDesc M;
    std::memset(&M, 0, sizeof(M));
    M.n_mom = opts->n_mom;
    for (int q = 0; q < opts->n_mom; ++q)
        for (int dd = 0; dd < 3; ++dd) M.mom[q][dd] = opts->mom[3 * q + dd];
    double2 *phase = reinterpret_cast<double2 *>(scr);
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(scr) + phase_bytes);
    double2 *partial = reinterpret_cast<double2 *>(reinterpret_cast<char *>(scr) + phase_bytes + 256);
    // every phase-table entry and every tile partial is written before it is
    // read; the work counter is set to zero below
    unsigned pgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((v3 * M.n_mom + 255) / 256, 4096));
    note_launch();
    k_phase_table<<<pgrid, 256, 0, stream>>>(F, M, phase);
    MBC_CUDA_TRY(cudaGetLastError());
    SmallBatch B;
    std::memset(&B, 0, sizeof(B));
    B.site_stride = (int32_t)site_entries;
    B.comp_stride = hp.n_comp;
    B.n_lists = 1;
    B.tiles_per_slab = l.tiles_per_slab;
    B.total_items = n_slabs * l.tiles_per_slab;
    B.item_base[1] = B.total_items;
    B.counter = counter;
    B.plan[0] = c->sp;
    if ((st = launch_small_batch(B, F, M, l, false, device, stream, phase, partial, false)) != MBC_OK) return st;
    const int64_t outs = n_slabs * M.n_mom * list->n_comp;
    const unsigned rgrid = (unsigned)std::min<int64_t>((outs + 7) / 8, 65535);
    note_launch();
    k_reduce_tiles<<<std::max(rgrid, 1u), 256, 0, stream>>>(partial, n_slabs, B.tiles_per_slab, M.n_mom,
                                                            list->n_comp, n_t, 0, 1, comp_max,
                                                            reinterpret_cast<double2 *>(out));
    MBC_CUDA_TRY(cudaGetLastError());
    return MBC_OK;
}

extern "C" int64_t mbc_kernel_launches(void) { return mbc::g_kernel_launches.load(std::memory_order_relaxed); }
