/*
 * mbc.h - C ABI of libmbc: recursive multibaryon correlation functions on
 * one GB300 (sm_103a).
 *
 * Method: Guenther, Toth, Varnhorst, "A recursive approach to determine
 * correlation functions in multibaryon systems" (arXiv:1301.4895).
 *
 * Two calls make up the path:
 *
 *   mbc_build_term_list  - host only, once per nucleus: the G tensors
 *                          (Sec. 2 eq. def_g), the symbolic tensor L by the
 *                          bullet recursion (Sec. 4 eq. recr_L, Sec. 7
 *                          eqs. rec_L_P / rec_L_N), the components of
 *                          interest (Sec. 4-5), backward pruning into the
 *                          operation lists Lambda^(m) (Sec. 3, Fig. 1).
 *   mbc_contract         - on the GPU, per (configuration, time slice, sink
 *                          site): the baryon blocks (Sec. 2, blocks
 *                          equation, with the sink function a delta at the
 *                          site), the F_- recursion over the lists (Sec. 4
 *                          eq. recr_F), the contraction with L (eq.
 *                          C_final) and the sum over sink sites with a
 *                          momentum phase.
 *
 * Beyond one nucleus at a point sink: momentum-projected blocks (Sec. 2 sink
 * functions, mbc_contract_opts.sink_mode), spin projections (Sec. 5,
 * MBC_SPIN_PROJECTED), several quark sources and sink functions (Sec. 6,
 * n_sources / n_sinks), several nuclei on one recursion path (Sec. 7,
 * mbc_build_combined) and lists without operation arrays (Sec. 3,
 * list_free). Term lists can be written to and read from files.
 *
 * Conventions (the paper leaves them open; every choice below changes at
 * most a global sign, identically for every component):
 *   - spinor-colour index xi = 3 * spin + colour, 0..11;
 *   - Euclidean Dirac representation, C = gamma_2 gamma_4, so that
 *     C gamma_5 has entries (0,1) = -1, (1,0) = +1, (2,3) = -1, (3,2) = +1;
 *   - relativistic operators Gamma_1 = 1, Gamma_2 = C gamma_5; nonrelativistic
 *     Gamma_1 = P_nr, Gamma_2 = C gamma_5 P_nr, P_nr = (1 + gamma_4) / 2
 *     (Sec. 7), which keeps spins 0 and 1 only;
 *   - proton (u, u, d), neutron (d, u, d) (Sec. 7); the same G at sink and
 *     source;
 *   - spin components are written protons first, then neutrons, each
 *     species as an ascending set (the antisymmetric tuples of Sec. 3);
 *   - C = (1 / (n_P! n_N!)^2) sum F_-^(A) L^(A) for the antisymmetric
 *     components produced by the bullet recursion (eq. C_final; the paper's
 *     normalisation also carries n_u! n_d!, which belongs to a different
 *     block convention - the Wick definition decides);
 *   - momentum phase exp(-2 pi i (n_x x / L_x + n_y y / L_y + n_z z / L_z)).
 *
 * Errors: every call returns an mbc_status; nothing throws across the ABI.
 * Thread safety: term lists are immutable after construction and may be
 * shared between threads; one mbc_contract call at a time per stream.
 */
#ifndef MBC_H
#define MBC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MBC_OK = 0,
    MBC_ERR_INVALID_ARG = 1,     /* malformed spec, pointer or size          */
    MBC_ERR_PAULI_FORBIDDEN = 2, /* nucleus/component vanishes identically  */
    MBC_ERR_OOM = 3,             /* host or device allocation failed         */
    MBC_ERR_CUDA = 4,            /* a CUDA runtime call failed               */
    MBC_ERR_TIMEOUT = 5,         /* a bounded device wait gave up            */
    MBC_ERR_UNSUPPORTED = 6      /* valid request outside what is built      */
} mbc_status;

/* Human-readable name of a status; static storage, never NULL. */
const char *mbc_status_string(mbc_status s);

/* ------------------------------------------------------------------------
 * Term lists (host, once per nucleus)
 * ---------------------------------------------------------------------- */

enum { MBC_SPIN_ALL = 0, MBC_SPIN_LISTED = 1, MBC_SPIN_PROJECTED = 2 };
enum { MBC_PROTON = 0, MBC_NEUTRON = 1 };

/*
 * Operator specification (Sec. 7).
 *   n_p, n_n     number of protons and neutrons, A = n_p + n_n, 1 <= A <= 16.
 *   dirac_dim    4 = relativistic (Gamma_1 = 1, Gamma_2 = C gamma_5),
 *                2 = nonrelativistic (Gamma_1 = P_nr, Gamma_2 = C gamma_5 P_nr).
 *   n_sources    number of mutually orthogonal quark sources N_s (Sec. 6):
 *                source baryon indices become spin x source, chi = N_s alpha + s,
 *                quark indices spinor-colour x source, xi = N_s kappa + s, and
 *                G carries the source deltas (eq. G_tilde); 3 dirac_dim N_s
 *                must not exceed 24. Stages whose index space exceeds 2^27
 *                (two relativistic sources) are pruned with sorted index
 *                lists instead of dense marks. Contraction kernels take
 *                3 dirac_dim N_s <= 24 with point sinks and <= 12 with
 *                momentum-projected blocks (see mbc_props.n_src).
 *   n_sinks      number of sink functions N_k for the sink baryon indices
 *                psi = N_k alpha + k (Sec. 6); 0 or 1 = one sink. N_k > 1
 *                lists contract with momentum-projected blocks, one momentum
 *                per sink function (mbc_contract_opts.sink_mode).
 *   spin_mode    MBC_SPIN_ALL: every independent component, i.e. every pair
 *                (sink spin set, source spin set) (Sec. 4); the output
 *                component index is snk_index * n_sets + src_index with the
 *                sets ordered as by mbc_term_list_components.
 *                MBC_SPIN_LISTED: the n_spin_sel pairs given by snk_spins and
 *                src_spins (each n_spin_sel * A int8 values, protons first;
 *                within a species any order, the antisymmetry sign is
 *                applied) (Sec. 5, Sec. 8 delta projection).
 *                MBC_SPIN_PROJECTED: n_proj outputs, each a projection
 *                C_M = sum_t w_t C(snk_t; src_t) of Sec. 5: the n_spin_sel
 *                terms give snk_spins / src_spins (A entries each, protons
 *                first, any order within a species: the antisymmetry sign is
 *                applied, repeated spins make the term vanish), term_proj[t]
 *                (the output it belongs to) and term_coef[t] (a real weight).
 *                The builder folds each projection into one modified list
 *                L_M, so only the components it needs are computed.
 *   path         NULL, or path_len == A entries MBC_PROTON / MBC_NEUTRON: the
 *                order in which baryons are added (Sec. 7). NULL selects the
 *                paper's rule: the more numerous species first, neutrons
 *                first on a tie.
 *   list_free    0: every step keeps its operation arrays. 1: no step
 *                stores operation arrays; the contraction kernels regenerate
 *                every split of an output component from its key (Sec. 3
 *                tuples, the split order of the stored lists). A step whose
 *                stages are dense (every component of the index space is
 *                needed, e.g. all stages of 8Be and of nonrelativistic 4He)
 *                needs nothing else; otherwise two index tables stand in for
 *                the arrays (dense rank of each output, compact index of each
 *                dense input rank), e.g. 4He relativistic, all components:
 *                3.19 GB of arrays become about 100 MB of tables. Such lists
 *                run on the wave kernels only.
 * The spec is read during the call only; the caller keeps ownership.
 */
typedef struct {
    int32_t n_p, n_n;
    int32_t dirac_dim;
    int32_t n_sources;
    int32_t spin_mode;
    int32_t n_spin_sel;
    const int8_t *snk_spins;
    const int8_t *src_spins;
    int32_t path_len;
    const int8_t *path;
    int32_t n_proj;
    const int32_t *term_proj;
    const double *term_coef;
    int32_t n_sinks;
    int32_t list_free;
} mbc_op_spec;

typedef struct mbc_term_list mbc_term_list; /* opaque, library-owned */

#define MBC_MAX_A 16

/* Statistics of a term list (Sec. 3 eqs. gen_P / gen_Q, Sec. 7 P, Q_P, Q_N;
 * N_Lambda as in Tables 1-6). */
typedef struct {
    int32_t A;
    int32_t n_steps;                     /* A - 1                            */
    int8_t path[MBC_MAX_A];              /* baryon added at each stage       */
    int64_t n_ops_total;                 /* N_Lambda                         */
    int64_t n_ops[MBC_MAX_A];            /* ops of step m -> m+1, index m-1  */
    int64_t ops_per_z[MBC_MAX_A];        /* splits per output component      */
    int64_t stage_size[MBC_MAX_A];       /* needed components of stage m     */
    int64_t stage_bound[MBC_MAX_A];      /* P(n_P, n_N) upper bound          */
    int64_t q_bound[MBC_MAX_A];          /* Q_P / Q_N upper bound of step m  */
    int64_t block_size;                  /* antisymmetric block components   */
    int32_t n_comp;                      /* output components per site       */
    int64_t n_l_total;                   /* nonzero L entries, all components */
    double norm;                         /* (n_P! n_N!)^2 of the largest nucleus */
    int32_t n_parts;                     /* nuclei in the list (mbc_build_combined) */
    uint32_t dense_mask;                 /* bit m-1: step m -> m+1 has dense stages */
    int64_t op_bytes;                    /* host bytes of the operation arrays (or of
                                            the index tables of a list-free list) */
} mbc_list_stats;

/*
 * Build the term list for one nucleus (host only; no device involvement).
 * On MBC_OK or MBC_ERR_PAULI_FORBIDDEN, *out receives a list the caller
 * frees with mbc_free_term_list; a Pauli-forbidden list holds no
 * operations and every component it yields is exactly zero (e.g. more
 * than dirac_dim baryons of one species, Sec. 6 on the 12-quark limit).
 * On any other status *out is set to NULL.
 */
mbc_status mbc_build_term_list(const mbc_op_spec *spec, mbc_term_list **out);

/*
 * Build one term list for n_specs nuclei on one recursion path (Sec. 7: the
 * stages of the largest nucleus pass through every smaller nucleus whose
 * baryons are the first ones added, and its components are contracted at
 * that stage with its own L; only the union of the needed components is
 * computed). The specs share dirac_dim, n_sources and n_sinks; the largest
 * nucleus fixes the path (its path field, else the paper's rule); every
 * other spec must have (n_p, n_n) equal to the counts of the first
 * n_p + n_n path entries, and a path field, if given, equal to that prefix.
 * Each spec keeps its own spin_mode and selections. The outputs are the
 * specs' components in the order given, spec after spec (mbc_term_list_part
 * gives the ranges); mbc_term_list_components pads the labels of a smaller
 * nucleus with -1 up to the largest A. With n_specs = 1 this is
 * mbc_build_term_list. Errors as mbc_build_term_list; a spec off the path,
 * with other operators, or (n_specs > 1) a Pauli-forbidden largest nucleus
 * gives MBC_ERR_INVALID_ARG.
 */
mbc_status mbc_build_combined(const mbc_op_spec *specs, int32_t n_specs, mbc_term_list **out);

/* One nucleus of a list: its baryon counts and output components [c0, c1). */
typedef struct {
    int32_t n_p, n_n;
    int32_t c0, c1;
} mbc_list_part;

/* Part j (0 <= j < stats.n_parts) of a list into *part (caller-owned). */
mbc_status mbc_term_list_part(const mbc_term_list *list, int32_t j, mbc_list_part *part);

/*
 * Term lists on disk (no counterpart in the paper: a cache so that ranks and
 * runs load a large list instead of rebuilding it). mbc_save_term_list
 * writes every field of the list to path (overwritten); mbc_load_term_list
 * reads such a file into a new list the caller frees with
 * mbc_free_term_list. A file from another format version or build layout,
 * a truncated or inconsistent file, or an I/O error gives
 * MBC_ERR_INVALID_ARG (nothing is returned); a Pauli-forbidden list loads
 * with MBC_ERR_PAULI_FORBIDDEN, as it was built. Host only.
 */
mbc_status mbc_save_term_list(const mbc_term_list *list, const char *path);
mbc_status mbc_load_term_list(const char *path, mbc_term_list **out);

/* Fill *st (caller-owned). */
mbc_status mbc_term_list_stats(const mbc_term_list *list, mbc_list_stats *st);

/* Spin labels of the output components: snk and src each receive
 * n_comp * A int8 values (caller-owned), protons first; -1 for the outputs
 * of MBC_SPIN_PROJECTED lists. */
mbc_status mbc_term_list_components(const mbc_term_list *list, int8_t *snk, int8_t *src);

/* Number of nonzero L entries of output component c (N_L, Tables 4-6). */
int64_t mbc_term_list_n_l(const mbc_term_list *list, int32_t c);

/* Release a list and its cached device copies (NULL is a no-op). Must not
 * race with an mbc_contract call still using the list. */
void mbc_free_term_list(mbc_term_list *list);

/* ------------------------------------------------------------------------
 * Contraction (GPU)
 * ---------------------------------------------------------------------- */

enum { MBC_C128 = 0, MBC_C64 = 1 };              /* propagator storage */
enum { MBC_FP64 = 0, MBC_MIXED = 1 };            /* arithmetic          */
enum { MBC_MEM_DEVICE = 0, MBC_MEM_HOST = 1 };   /* where s_u/s_d/out live */
enum { MBC_SINK_POINT = 0, MBC_SINK_BLOCK_MOMENTUM = 1 };  /* sink function   */

/*
 * Propagator fields, layout [cfg][t][z][y][x][(source)][row 12][col 12] complex,
 * row = sink spinor-colour index, col = source index, re/im interleaved.
 *   s_u, s_d     u and d fields (may be the same pointer: u = d).
 *   dtype        MBC_C128 (complex double) or MBC_C64 (complex float).
 *   memory       MBC_MEM_DEVICE: s_u, s_d and out are device pointers.
 *                MBC_MEM_HOST: they are host pointers (pinned memory gives
 *                overlap); the library copies slabs in and results out on
 *                the given stream and returns after the results are in out.
 *   stride_cfg, stride_t  element strides (in complex numbers) between
 *                configurations and time slices; 0 selects the dense values.
 *   n_src        quark sources (Sec. 6); 0 means 1. A site then holds n_src
 *                consecutive 12 x 12 matrices, [source][row][col], one per
 *                source, and every list must have been built with
 *                n_sources = n_src (else MBC_ERR_INVALID_ARG). The source
 *                quark index of the lists is xi = n_src * kappa + s for
 *                column kappa of source s. Contraction kernels take
 *                3 * dirac_dim * n_src <= 24 source columns with point
 *                sinks (two relativistic sources: 12 x 24 tiles) and <= 12
 *                with momentum-projected blocks (MBC_ERR_UNSUPPORTED
 *                otherwise); the allocation-free entry point takes n_src = 1
 *                only.
 */
typedef struct {
    const void *s_u;
    const void *s_d;
    int32_t dtype;
    int32_t memory;
    int32_t n_cfg, nt, lx, ly, lz;
    int64_t stride_cfg, stride_t;
    int32_t n_src;
} mbc_props;

/* Launch tuning; zero fields select the library's choice. */
typedef struct {
    int32_t sites_per_cta;      /* FP64 small-stage kernel: sites per CTA      */
    int32_t threads_per_cta;    /* mixed small-stage kernel: threads per CTA   */
    int32_t wave_sites;         /* large-stage kernels: sites in flight (0: the
                                   narrowest multiple of 64 that gives a wave at
                                   least 2e10 site-operations, within an 8 GB
                                   scratch budget; mixed list-free lists at least
                                   512, in multiples of 512)                      */
    int32_t regime;             /* 0 auto, 1 force small-stage, 2 force large  */
    int32_t zchunk;             /* large-stage step kernel: outputs per warp item
                                   (mixed default 1)                            */
    int32_t wave_order;         /* large-stage step kernels on stored lists. FP64:
                                   0 site groups of a chunk side by side, 1 a CTA's
                                   warps on consecutive chunks of one site group.
                                   Mixed: 0 one CTA per SM on consecutive (output,
                                   site group) pairs, one warp per output: 20 warps
                                   with 8 gathers in flight each on steps of at least
                                   64 terms per output, 32 warps with 4 on the others,
                                   an output's terms split over up to 16 warps on steps
                                   of fewer items than SMs and at least 1024 terms;
                                   2 32 warps on every step; 6 20 warps on every step;
                                   5 32 warps with an output's terms split over
                                   several warps; 1 8-warp CTAs on consecutive
                                   outputs of one site group; 3 8-warp CTAs with the
                                   site groups side by side; 4 block rows of runs of
                                   outputs staged in shared memory by bulk copies
                                   (where the runs qualify)                       */
    int32_t list_free;          /* large-stage step kernel: 0 regenerate the splits of
                                   list-free lists, read the arrays of the others;
                                   1 also regenerate the dense steps of lists with
                                   arrays                                           */
} mbc_tune;

/*
 * Options.
 *   precision    MBC_FP64: FP64 products and sums throughout.
 *                MBC_MIXED: per-site power-of-two input scaling, FP32 complex
 *                products with compensated (two-sum) float-float
 *                accumulation of every component, FP64 for the contraction
 *                with L and for the site/momentum sum.
 *   n_mom, mom   n_mom >= 1 momenta, mom[3 * i + {0, 1, 2}] = (n_x, n_y, n_z)
 *                integers (host pointer, read during the call).
 *   t0, t1       time slices [t0, t1) are evaluated; t1 == 0 means nt.
 *   tune         NULL or launch tuning.
 *   sink_mode    MBC_SINK_POINT: the correlator of all baryons at one sink
 *                point, summed over sites with the momentum phase.
 *                MBC_SINK_BLOCK_MOMENTUM: every baryon's block is projected to
 *                the momentum first, f_B = sum_x exp(-2 pi i n.x / L) f_B(x)
 *                (Sec. 2 sink function s(x)), and the recursion runs once
 *                per (configuration, time slice, momentum) on those blocks.
 *                The blocks and their site sums are FP64 in the FP64 path;
 *                the mixed path forms them with FP32 products, sums each
 *                16-site tile with compensated FP32 accumulation, rounds the
 *                tile sum once to FP32 and adds the tiles with compensated
 *                FP32 accumulation, the result in FP64. Lists built
 *                with n_sinks = N_k > 1 (Sec. 6 sink functions s_1 .. s_N_k)
 *                take the momenta in groups of N_k (n_mom a multiple of N_k,
 *                all lists of the call with the same N_k): sink function k
 *                of group g is momentum g N_k + k, the block of sink index
 *                psi = N_k alpha + k is the spin-alpha block projected with
 *                it, and the recursion runs once per (configuration, time
 *                slice, group). MBC_SINK_POINT takes N_k = 1 only
 *                (MBC_ERR_UNSUPPORTED).
 */
typedef struct {
    int32_t precision;
    int32_t n_mom;
    const int32_t *mom;
    int32_t t0, t1;
    const mbc_tune *tune;
    int32_t sink_mode;
} mbc_contract_opts;

/*
 * Evaluate the correlators of n_lists nuclei.
 * out: complex128 [n_cfg][n_lists][t1 - t0][n_mom / N_k][n_comp_max], where
 * n_comp_max is the largest n_comp of the lists; unused tail entries are
 * zero. With memory == MBC_MEM_DEVICE the call is asynchronous on stream
 * (a cudaStream_t; NULL = legacy default stream) and out is written in a
 * fixed reduction order (bitwise reproducible). Device scratch is owned by
 * the library, grown on demand and reused across calls; the first call per
 * list uploads it to the current device and caches it there.
 * Returns MBC_ERR_INVALID_ARG for bad sizes/pointers, MBC_ERR_OOM when
 * device memory cannot be had, MBC_ERR_CUDA for a failed CUDA call.
 */
mbc_status mbc_contract(const mbc_props *props, const mbc_term_list *const *lists, int32_t n_lists,
                        const mbc_contract_opts *opts, void *out, void *stream);

/*
 * mbc_contract without any device allocation. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc in steady
 * state - services whose device memory is reserved up front by their own
 * pool (a cudaMalloc would fail or fragment it), or real-time loops whose
 * latency budget forbids allocator calls (cudaMalloc and cudaFree may
 * synchronise the device).
 *
 * Same arguments and output layout as mbc_contract with n_lists = 1:
 * out is complex128 [n_cfg][1][t1 - t0][n_mom][max(1, n_comp)], device
 * memory owned by the caller, written completely on each call.
 * Supported: MBC_FP64, MBC_MEM_DEVICE, MBC_SINK_POINT, and lists that take the
 * shared-memory kernel (the nonrelativistic nuclei); anything else returns
 * MBC_ERR_UNSUPPORTED before touching the device.
 *
 * Scratch: one static device array of 8 MiB (MBC_NOALLOC_SCRATCH_BYTES)
 * inside the library, which every GPU that loads the library holds until the
 * process exits. The momentum phase table (16 * L_x L_y L_z * n_mom bytes,
 * rounded up to 256) plus the tile partials (16 * n_mom * n_comp bytes per
 * tile of up to 32 sites) must fit; a larger request returns
 * MBC_ERR_UNSUPPORTED before any device work.
 *
 * Preconditions and behaviour:
 *   - the list must already have its device copy on the current device,
 *     made by an earlier mbc_contract call with that list (that call may
 *     allocate; do it during set-up); otherwise MBC_ERR_INVALID_ARG;
 *   - the first call on a device looks up the device address of the static
 *     array (cudaGetSymbolAddress, once per device, with that device current)
 *     and loads the kernel constants; make that first call before any stream
 *     capture begins;
 *   - no cudaMalloc, cudaFree or other allocating routine is called;
 *   - every call shares the one array and leaves the last call's contents in
 *     it. The one word that must start at zero (the work counter of the
 *     persistent kernel) is zeroed by each call on its stream; every other
 *     entry is written before it is read. Calls that overlap on the GPU - on
 *     different streams, or from several host threads - race on the array and
 *     give wrong results: serialise them.
 */
#define MBC_NOALLOC_SCRATCH_BYTES (8u << 20)
mbc_status mbc_contract_noalloc(const mbc_props *props, const mbc_term_list *list, const mbc_contract_opts *opts,
                                void *out, void *stream);

/*
 * Wait for the stream and report the kernels' deferred device-side status:
 * MBC_ERR_TIMEOUT when a bounded wait of a kernel ran out since the last
 * report (the kernel then stopped without finishing its work, so the
 * results of the calls in between are not valid; the status is cleared by
 * this report and the context stays usable), MBC_ERR_CUDA for a failed CUDA
 * call, MBC_OK otherwise. The kernels' waits are on asynchronous copies
 * into shared memory and give up after about a second of polling. A
 * mbc_contract call with props->memory = MBC_MEM_HOST synchronises before it
 * returns and reports (and clears) the same status itself; calls on device
 * memory are asynchronous and leave it to this function.
 */
mbc_status mbc_sync_status(void *stream);

/*
 * Test of the timeout path (no counterpart in the paper): launches on stream
 * one CTA that waits, with the library's bounded wait, on a barrier nothing
 * completes, giving up after polls polls (1 .. 2^20). The next
 * mbc_sync_status on that stream then returns MBC_ERR_TIMEOUT. No copy is in
 * flight and nothing faults. MBC_ERR_INVALID_ARG for polls out of range.
 */
mbc_status mbc_check_wait_timeout(uint32_t polls, void *stream);

/* Release the library's device scratch on the current device. */
void mbc_release_scratch(void);

/*
 * Kernel timing for benchmarks. While enabled, every launch of the
 * contraction kernels (the shared-memory kernel, or the per-step wave
 * kernels) is bracketed by CUDA events recorded on its launch stream.
 * mbc_timing_read waits for those events and returns the summed device time
 * in milliseconds and the number of bracketed launches since the previous
 * read (or since enabling), then forgets them. Off by default; the flag is
 * process-wide.
 */
void mbc_timing_enable(int32_t on);
mbc_status mbc_timing_read(double *ms, int64_t *launches);

/* Kernels launched by the library's contraction entry points since it was
 * loaded (cumulative, all devices and streams; the FMA probe excluded), for
 * counting the launches of a timed region. No counterpart in the paper. */
int64_t mbc_kernel_launches(void);

/*
 * Arithmetic peak probe: fills every SM of the current device (one wave at
 * the occupancy limit) with independent FMA work and writes the achieved
 * flop/s (2 flops per FMA) to *flops. MBC_FP64: complex multiply-accumulate
 * on FP64 registers (the operand pattern of the contraction kernels; chains
 * that reuse one multiplier register read back lower on this pipe).
 * MBC_MIXED: packed FP32-pair FMA chains. Synchronous; used as the measured
 * denominator of the ALU roofline. No counterpart in the paper.
 */
mbc_status mbc_fma_probe(int32_t precision, double *flops);

/* Library version string, static storage. */
const char *mbc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MBC_H */
