// Internal layout of a term list, shared by the host builder and the CUDA
// contraction. Not part of the public ABI (include/mbc.h).
#pragma once

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/mbc.h"

namespace mbc {

// One step F^(m) -> F^(m+1) of the F_- recursion (Sec. 4 eq. recr_F).
// Output components z (compact index at stage m+1) each have exactly
// k operations (all splits of a needed key, Sec. 3/7), stored z-major:
// op j of z at z * k + j. x indexes stage m (for m = 1 it is the block
// index of the first baryon), y the block of the added baryon, and the sign
// sgn(x|y) of eq. antis_product_2 sits in bit 15 of ys.
struct Step {
    int baryon = 0;          // MBC_PROTON or MBC_NEUTRON
    int64_t n_x = 0;         // size of the input stage (block size for m = 1)
    int64_t n_z = 0;         // size of the output stage
    int64_t k = 0;           // operations per output component
    bool dense = false;      // both stages hold their whole index space: the
                             // compact index is the dense rank (Sec. 3 tuples)
    bool generated = false;  // list-free: no op arrays, the kernels regenerate
                             // every split of an output from its key
    std::vector<uint32_t> x; // n_z * k (empty when generated)
    std::vector<uint16_t> ys;
    // generated steps: dense rank of each output (empty when the output stage
    // is dense) and compact index of each dense rank of the input stage
    // (empty when the input stage is dense or is the first baryon's block)
    std::vector<int64_t> zrank;
    std::vector<int32_t> xmap;
    int32_t zk[4] = {0, 0, 0, 0}, xk[4] = {0, 0, 0, 0};  // set sizes (dp, dn, u, d)
};

struct DeviceCache;  // defined by the CUDA side

}  // namespace mbc

struct mbc_term_list {
    int A = 0, n_p = 0, n_n = 0, dim = 4, n_sources = 1, n_sinks = 1;
    int dim_snk = 4, dim_src = 4;  // baryon index values at the sink / source (Sec. 6 psi / chi)
    int8_t path[MBC_MAX_A] = {0};
    bool pauli_forbidden = false;
    int nxi = 12;             // quark index values: 3 * dim * n_sources
    int64_t block_size = 0;   // dim_snk * C(nxi, 2) * nxi
    bool need_block[2] = {false, false};
    std::vector<mbc::Step> steps;        // A - 1 steps
    int64_t final_size = 0;              // components of F^(A) kept
    int32_t n_comp = 0;
    std::vector<int8_t> comp_snk, comp_src;     // n_comp * A
    // contraction with L (eq. C_final): entries of component c at
    // [fin_off[c], fin_off[c+1]): F^(A) index and L value (an integer for a
    // single component, a weighted sum for a projection, Sec. 5)
    std::vector<int64_t> fin_off;
    std::vector<uint32_t> fin_z;
    std::vector<double> fin_l;
    double norm = 1.0;
    // nuclei of the list (one, or several on one path, Sec. 7): components
    // [c0, c1) belong to the nucleus of the first A baryons of the path and
    // are contracted at stage A with normalisation (n_P! n_N!)^2
    struct Part {
        int32_t n_p, n_n, A;
        int32_t c0, c1;
        double norm;
    };
    std::vector<Part> parts;
    mbc_list_stats stats{};
    // device copies, one per device ordinal, created on first use
    std::mutex dev_mu;
    std::vector<mbc::DeviceCache *> dev;
};

namespace mbc {
// Implemented by the CUDA side; releases the device copies of a list.
void free_device_cache(mbc_term_list *list);
}  // namespace mbc
