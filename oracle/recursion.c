/*
 * O3: the recursive method written out plainly (CPU oracle).
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the CPU
 * baseline legs of bench.py may load this library. It shares no code, table
 * or helper with the product library.
 *
 * Steps, in the paper's order:
 *   1. antisymmetric components of G_P and G_N (Sec. 3, Sec. 4): the signed
 *      sum over the orderings of the same-flavour slots of one baryon;
 *   2. L^(A) by the bullet recursion L^(m+1) = L^(m) . G_{B_{m+1}}
 *      (eq. recr_L, eqs. rec_L_P / rec_L_N), the product of eq.
 *      antis_product_2 with sgn(x|y) of Sec. 3;
 *   3. the components of interest: for every requested (sink set, source
 *      set) pair, the keys (sink set, U, D) with L(source set; U, D) != 0
 *      (Sec. 4-5; a single component is the delta projection of Sec. 8);
 *   4. backward pruning (Sec. 3, Fig. 1): the components of stage m needed
 *      by some split of a needed component of stage m+1; every split of a
 *      needed component is one operation (Sec. 7: N_Lambda);
 *   5. per site: the blocks f_B (Sec. 2, blocks equation with s(x) = delta
 *      at the site), their antisymmetric components, the recursion
 *      F^(m+1) = F^(m) . f_{B_{m+1}} (eq. recr_F) over the needed keys, and
 *      the contraction of eq. C_final. Normalisation: 1 / (n_P! n_N!)^2 for
 *      the antisymmetric-component conventions used here (the paper's
 *      factor also carries n_u! n_d!, which belongs to a different block
 *      convention; the Wick definition decides, see the tests).
 *
 * Alongside every value the same recursion runs on magnitudes
 * (|G||S||S||S| for blocks, |X||Y| per product, |F||L| in the contraction):
 * that is the scale "sum |terms|" used for the error bounds.
 *
 * Keys are 32-bit: bits 0-3 proton spin set, 4-7 neutron spin set, 8-19 the
 * set of u indices, 20-31 the set of d indices (one quark source). Built
 * with O3_WIDE the keys are 64-bit for two relativistic quark sources
 * (Sec. 6: 24 quark index values, 8 source baryon index values): bits 0-7
 * and 8-15 the spin sets, 16-39 the u set, 40-63 the d set; the blocks then
 * take 12 x 24 propagator tiles (sink rows x source columns) and the
 * pruning collects keys in sorted arrays instead of a bitmap over all keys.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef O3_WIDE
typedef uint64_t key_t32;
#define NQ 24  /* quark index values */
#define NSP 8  /* source baryon index values */
#define KEY(dp, dn, u, d) \
    ((uint64_t)(dp) | ((uint64_t)(dn) << 8) | ((uint64_t)(u) << 16) | ((uint64_t)(d) << 40))
#define KDP(k) ((uint32_t)((k) & 0xFFu))
#define KDN(k) ((uint32_t)(((k) >> 8) & 0xFFu))
#define KU(k) ((uint32_t)(((k) >> 16) & 0xFFFFFFu))
#define KD(k) ((uint32_t)(((k) >> 40) & 0xFFFFFFu))
#else
typedef uint32_t key_t32;
#define NQ 12
#define NSP 4
#define KEY(dp, dn, u, d) ((uint32_t)(dp) | ((uint32_t)(dn) << 4) | ((uint32_t)(u) << 8) | ((uint32_t)(d) << 20))
#define KDP(k) ((k) & 0xFu)
#define KDN(k) (((k) >> 4) & 0xFu)
#define KU(k) (((k) >> 8) & 0xFFFu)
#define KD(k) (((k) >> 20) & 0xFFFu)
#endif
#define NBLK ((int64_t)4 * NQ * NQ * NQ) /* block entries: sink spin x three source indices */

typedef struct { key_t32 key; int64_t val; } kv_t;

typedef struct {
    int A, n_p, n_n, dim;
    int8_t path[16];          /* 0 = proton, 1 = neutron, in recursion order */
    int n_req;
    uint8_t *req_dp, *req_dn; /* sink spin sets per request (bitmasks) */
    /* L(source set) slice per request */
    int64_t *req_off;         /* n_req + 1 */
    key_t32 *req_key;         /* (U, D) with sink spin sets of the request */
    int64_t *req_lval;
    /* needed keys per stage (sorted), stage 1..A at index 0..A-1 */
    int64_t n_need[16];
    key_t32 *need[16];
    int64_t ops[16];          /* ops of step m -> m+1 at index m-1 */
    int8_t G[NSP * NQ * NQ * NQ]; /* source tensor: L (eq. def_L) */
    int8_t Gs[4 * 12 * 12 * 12];  /* sink tensor: the blocks (eq. def_f) */
    double norm;
} o3_plan;

static int popc(uint32_t x) { return __builtin_popcount(x); }

/* sgn(x|y) for one group: (-1)^{#(i in x, j in y, i > j)} */
static int sgn_group(uint32_t x, uint32_t y) {
    int n = 0;
    for (int j = 0; j < NQ; ++j)
        if (y & (1u << j)) n += popc(x >> (j + 1));
    return (n & 1) ? -1 : 1;
}

static int sgn_key(key_t32 x, key_t32 y) {
    return sgn_group(KDP(x), KDP(y)) * sgn_group(KDN(x), KDN(y)) * sgn_group(KU(x), KU(y)) *
           sgn_group(KD(x), KD(y));
}

static int disjoint(key_t32 x, key_t32 y) {
    return (KDP(x) & KDP(y)) == 0 && (KDN(x) & KDN(y)) == 0 && (KU(x) & KU(y)) == 0 &&
           (KD(x) & KD(y)) == 0;
}

static int cmp_kv(const void *a, const void *b) {
    key_t32 x = ((const kv_t *)a)->key, y = ((const kv_t *)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}
static int cmp_key(const void *a, const void *b) {
    key_t32 x = *(const key_t32 *)a, y = *(const key_t32 *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* sort by key, add equal keys, drop zeros; returns new length */
static int64_t reduce_kv(kv_t *v, int64_t n) {
    qsort(v, (size_t)n, sizeof(kv_t), cmp_kv);
    int64_t w = 0;
    for (int64_t i = 0; i < n;) {
        int64_t j = i;
        int64_t s = 0;
        while (j < n && v[j].key == v[i].key) s += v[j++].val;
        if (s != 0) { v[w].key = v[i].key; v[w].val = s; ++w; }
        i = j;
    }
    return w;
}

static int64_t sorted_unique(key_t32 *k, int64_t n) {
    qsort(k, (size_t)n, sizeof(key_t32), cmp_key);
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i)
        if (w == 0 || k[w - 1] != k[i]) k[w++] = k[i];
    return w;
}

static int64_t find_key(const key_t32 *k, int64_t n, key_t32 x) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (k[mid] == x) return mid;
        if (k[mid] < x) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Antisymmetric components of G for baryon b (0 = P, 1 = N) (Sec. 3-4). */
static int64_t g_minus(const o3_plan *p, int b, kv_t *out) {
    int64_t n = 0;
    const int8_t *G = p->G;
#define GV(a, i, j, k) ((int64_t)G[(((a) * NQ + (i)) * NQ + (j)) * NQ + (k)])
    for (int a = 0; a < NSP; ++a)
        for (int i = 0; i < NQ; ++i)
            for (int j = 0; j < NQ; ++j)
                for (int k = 0; k < NQ; ++k) {
                    int64_t v;
                    key_t32 key;
                    if (b == 0) { /* proton (u,u,d): u pair slots 1,2 */
                        if (!(i < j)) continue;
                        v = GV(a, i, j, k) - GV(a, j, i, k);
                        key = KEY(1u << a, 0, (1u << i) | (1u << j), 1u << k);
                    } else { /* neutron (d,u,d): d pair slots 1,3 */
                        if (!(i < k)) continue;
                        v = GV(a, i, j, k) - GV(a, k, j, i);
                        key = KEY(0, 1u << a, 1u << j, (1u << i) | (1u << k));
                    }
                    if (v != 0) { out[n].key = key; out[n].val = v; ++n; }
                }
#undef GV
    return n;
}

/* all splits y of z for adding baryon b: calls back with (x, y-key, sign) */
typedef void (*split_cb)(void *ctx, key_t32 x, key_t32 y, int sgn);

static int bits_of(uint32_t m, int *pos) {
    int n = 0;
    for (int i = 0; i < NQ; ++i) if (m & (1u << i)) pos[n++] = i;
    return n;
}

static int64_t for_splits(key_t32 z, int b, split_cb cb, void *ctx) {
    int dpos[NQ], upos[NQ], qpos[NQ];
    uint32_t dset = b == 0 ? KDP(z) : KDN(z);
    int nd = bits_of(dset, dpos), nu = bits_of(KU(z), upos), nq = bits_of(KD(z), qpos);
    int64_t cnt = 0;
    for (int a = 0; a < nd; ++a) {
        uint32_t yd = 1u << dpos[a];
        if (b == 0) {
            for (int i = 0; i < nu; ++i)
                for (int j = i + 1; j < nu; ++j)
                    for (int k = 0; k < nq; ++k) {
                        key_t32 y = KEY(yd, 0, (1u << upos[i]) | (1u << upos[j]), 1u << qpos[k]);
                        key_t32 x = KEY(KDP(z) & ~KDP(y), KDN(z), KU(z) & ~KU(y), KD(z) & ~KD(y));
                        if (cb) cb(ctx, x, y, sgn_key(x, y));
                        ++cnt;
                    }
        } else {
            for (int j = 0; j < nu; ++j)
                for (int i = 0; i < nq; ++i)
                    for (int k = i + 1; k < nq; ++k) {
                        key_t32 y = KEY(0, yd, 1u << upos[j], (1u << qpos[i]) | (1u << qpos[k]));
                        key_t32 x = KEY(KDP(z), KDN(z) & ~KDN(y), KU(z) & ~KU(y), KD(z) & ~KD(y));
                        if (cb) cb(ctx, x, y, sgn_key(x, y));
                        ++cnt;
                    }
        }
    }
    return cnt;
}

typedef struct { key_t32 *buf; int64_t n, cap; } keyvec;
static void kv_push_cb(void *ctx, key_t32 x, key_t32 y, int s) {
    (void)y; (void)s;
    keyvec *v = (keyvec *)ctx;
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 1024;
        v->buf = (key_t32 *)realloc(v->buf, (size_t)v->cap * sizeof(key_t32));
    }
    v->buf[v->n++] = x;
}

#ifndef O3_WIDE
static void mark_cb(void *ctx, key_t32 x, key_t32 y, int s) {
    (void)y; (void)s;
    uint64_t *bm = (uint64_t *)ctx;
    __atomic_fetch_or(&bm[x >> 6], (uint64_t)1 << (x & 63), __ATOMIC_RELAXED);
}
#endif

static double factorial(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

void o3_free(o3_plan *p) {
    if (!p) return;
    free(p->req_dp); free(p->req_dn); free(p->req_off); free(p->req_key); free(p->req_lval);
    for (int m = 0; m < 16; ++m) free(p->need[m]);
    free(p);
}

/*
 * Build the symbolic part. G: dense int8 G(alpha; xi1, xi2, xi3), 4x12x12x12.
 * path: A entries (0 = P, 1 = N). req_snk / req_src: n_req rows of A spins,
 * protons first then neutrons, each group sorted ascending.
 * Returns 0 on success, 1 on invalid input.
 */
int o3_plan_build(int n_p, int n_n, int dim, const int8_t *path, const int8_t *G, int n_req,
                  const int8_t *req_snk, const int8_t *req_src, o3_plan **out) {
    int A = n_p + n_n;
    if (A < 1 || A > 16 || n_p < 0 || n_n < 0) return 1;
    o3_plan *p = (o3_plan *)calloc(1, sizeof(o3_plan));
    p->A = A; p->n_p = n_p; p->n_n = n_n; p->dim = dim; p->n_req = n_req;
    memcpy(p->path, path, (size_t)A);
    memcpy(p->G, G, sizeof(p->G));
#ifndef O3_WIDE
    memcpy(p->Gs, G, sizeof(p->Gs)); /* one source: the same tensor at the sink */
#endif
    p->norm = factorial(n_p) * factorial(n_n);
    p->norm *= p->norm;

    /* 1-2: L by the bullet recursion over the antisymmetric G components */
    kv_t *gm[2];
    int64_t ngm[2];
    for (int b = 0; b < 2; ++b) {
        gm[b] = (kv_t *)malloc(sizeof(kv_t) * NSP * NQ * NQ * NQ);
        ngm[b] = g_minus(p, b, gm[b]);
    }
    int64_t nL = ngm[path[0]];
    kv_t *L = (kv_t *)malloc(sizeof(kv_t) * (size_t)(nL ? nL : 1));
    memcpy(L, gm[path[0]], sizeof(kv_t) * (size_t)nL);
    for (int m = 1; m < A; ++m) {
        int b = path[m];
        int64_t cap = nL * ngm[b] + 1, n = 0;
        kv_t *Z = (kv_t *)malloc(sizeof(kv_t) * (size_t)cap);
        for (int64_t i = 0; i < nL; ++i)
            for (int64_t j = 0; j < ngm[b]; ++j)
                if (disjoint(L[i].key, gm[b][j].key)) {
                    Z[n].key = L[i].key | gm[b][j].key;
                    Z[n].val = L[i].val * gm[b][j].val * sgn_key(L[i].key, gm[b][j].key);
                    ++n;
                }
        n = reduce_kv(Z, n);
        free(L);
        L = Z;
        nL = n;
    }
    free(gm[0]); free(gm[1]);

    /* 3: requested components and the needed final keys */
    p->req_dp = (uint8_t *)calloc((size_t)n_req + 1, 1);
    p->req_dn = (uint8_t *)calloc((size_t)n_req + 1, 1);
    p->req_off = (int64_t *)calloc((size_t)n_req + 1, sizeof(int64_t));
    keyvec fin = {0, 0, 0};
    int64_t tot = 0;
    key_t32 *tmpk = (key_t32 *)malloc(sizeof(key_t32) * (size_t)(nL + 1));
    int64_t *tmpv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nL + 1));
    p->req_key = NULL; p->req_lval = NULL;
    for (int r = 0; r < n_req; ++r) {
        uint32_t sp = 0, sn = 0, ap = 0, an = 0;
        for (int k = 0; k < n_p; ++k) { sp |= 1u << req_snk[r * A + k]; ap |= 1u << req_src[r * A + k]; }
        for (int k = 0; k < n_n; ++k) { sn |= 1u << req_snk[r * A + n_p + k]; an |= 1u << req_src[r * A + n_p + k]; }
        if (popc(sp) != n_p || popc(sn) != n_n || popc(ap) != n_p || popc(an) != n_n) { o3_free(p); free(L); return 1; }
        p->req_dp[r] = (uint8_t)sp; p->req_dn[r] = (uint8_t)sn;
        int64_t c = 0;
        for (int64_t i = 0; i < nL; ++i)
            if (KDP(L[i].key) == ap && KDN(L[i].key) == an) {
                tmpk[c] = KEY(sp, sn, KU(L[i].key), KD(L[i].key));
                tmpv[c] = L[i].val;
                ++c;
            }
        p->req_key = (key_t32 *)realloc(p->req_key, sizeof(key_t32) * (size_t)(tot + c + 1));
        p->req_lval = (int64_t *)realloc(p->req_lval, sizeof(int64_t) * (size_t)(tot + c + 1));
        memcpy(p->req_key + tot, tmpk, sizeof(key_t32) * (size_t)c);
        memcpy(p->req_lval + tot, tmpv, sizeof(int64_t) * (size_t)c);
        for (int64_t i = 0; i < c; ++i) kv_push_cb(&fin, tmpk[i], 0, 0);
        tot += c;
        p->req_off[r + 1] = tot;
    }
    free(tmpk); free(tmpv); free(L);
    fin.n = sorted_unique(fin.buf, fin.n);
    p->need[A - 1] = fin.buf;
    p->n_need[A - 1] = fin.n;

#ifdef O3_WIDE
    /* 4: backward pruning: the x of every split of a needed key of stage m+1,
     * sorted and made unique, are the needed keys of stage m; every split of
     * a needed key is one operation */
    for (int m = A - 1; m >= 1; --m) {
        keyvec xs = {0, 0, 0};
        int64_t ops = 0;
        for (int64_t i = 0; i < p->n_need[m]; ++i) ops += for_splits(p->need[m][i], path[m], kv_push_cb, &xs);
        p->ops[m - 1] = ops;
        p->n_need[m - 1] = sorted_unique(xs.buf, xs.n);
        p->need[m - 1] = xs.buf ? xs.buf : (key_t32 *)malloc(sizeof(key_t32));
    }
#else
    /* 4: backward pruning: a bitmap over all 2^32 keys marks the needed
     * components of stage m; every split of a needed key is one operation */
    uint64_t *bm = (uint64_t *)calloc((size_t)1 << 26, sizeof(uint64_t));
    for (int m = A - 1; m >= 1; --m) {
        int64_t ops = 0;
        const key_t32 *zs = p->need[m];
        const int b = path[m];
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : ops)
        for (int64_t i = 0; i < p->n_need[m]; ++i)
            ops += for_splits(zs[i], b, mark_cb, bm);
        p->ops[m - 1] = ops;
        int64_t cnt = 0;
        for (int64_t w = 0; w < ((int64_t)1 << 26); ++w) cnt += __builtin_popcountll(bm[w]);
        key_t32 *keys = (key_t32 *)malloc(sizeof(key_t32) * (size_t)(cnt + 1));
        int64_t n = 0;
        for (int64_t w = 0; w < ((int64_t)1 << 26); ++w) {
            uint64_t v = bm[w];
            while (v) {
                keys[n++] = (key_t32)(w * 64 + __builtin_ctzll(v));
                v &= v - 1;
            }
            bm[w] = 0;
        }
        p->need[m - 1] = keys;
        p->n_need[m - 1] = n;
    }
    free(bm);
#endif
    *out = p;
    return 0;
}

/* Replace the sink tensor used for the blocks (default: the source tensor).
 * With several quark sources (Sec. 6) the sink keeps G(alpha; sink spinor-
 * colour indices) while L is built from G~ over the source indices. */
void o3_plan_set_sink(o3_plan *p, const int8_t *Gs) { memcpy(p->Gs, Gs, sizeof(p->Gs)); }

int64_t o3_n_ops(const o3_plan *p, int64_t *per_step, int64_t *stage_sizes) {
    int64_t t = 0;
    for (int m = 0; m + 1 < p->A; ++m) { if (per_step) per_step[m] = p->ops[m]; t += p->ops[m]; }
    for (int m = 0; m < p->A; ++m) if (stage_sizes) stage_sizes[m] = p->n_need[m];
    return t;
}

/* Needed keys of stage m (1-based), ascending; returns their number and
 * copies them to out when out is not NULL. */
int64_t o3_stage_keys(const o3_plan *p, int m, key_t32 *out) {
    if (m < 1 || m > p->A) return -1;
    if (out) memcpy(out, p->need[m - 1], sizeof(key_t32) * (size_t)p->n_need[m - 1]);
    return p->n_need[m - 1];
}

int64_t o3_req_nl(const o3_plan *p, int r) { return p->req_off[r + 1] - p->req_off[r]; }
double o3_norm(const o3_plan *p) { return p->norm; }

/* ---- numeric part ---------------------------------------------------- */

typedef struct { double re, im; } cplx;
static cplx cmul(cplx a, cplx b) { cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static double cabs2(cplx a) { return sqrt(a.re * a.re + a.im * a.im); }

typedef struct {
    const o3_plan *p;
    int nb;                 /* sites in the batch */
    const cplx *X; const double *Xm;   /* stage m: [need][nb] */
    const cplx *Y; const double *Ym;   /* block of the added baryon: [site][NBLK] */
    int64_t nX;
    const key_t32 *kX;
    cplx *acc; double *accm;           /* [nb] */
} eval_ctx;

static int64_t block_index(key_t32 y, int b) {
    int pos[NQ];
    uint32_t dset = b == 0 ? KDP(y) : KDN(y);
    int a = __builtin_ctz(dset);
    if (b == 0) {
        bits_of(KU(y), pos);
        int i = pos[0], j = pos[1], k = __builtin_ctz(KD(y));
        return ((int64_t)(a * NQ + i) * NQ + j) * NQ + k;
    } else {
        bits_of(KD(y), pos);
        int i = pos[0], k = pos[1], j = __builtin_ctz(KU(y));
        return ((int64_t)(a * NQ + i) * NQ + j) * NQ + k;
    }
}

static void eval_cb(void *vctx, key_t32 x, key_t32 y, int sgn) {
    eval_ctx *c = (eval_ctx *)vctx;
    int64_t ix = find_key(c->kX, c->nX, x);
    if (ix < 0) return; /* cannot happen: every x of a needed z is needed */
    int64_t iy = block_index(y, (KDP(y) != 0) ? 0 : 1);
    const cplx *xv = c->X + ix * c->nb;
    const double *xm = c->Xm + ix * c->nb;
    const int64_t NBk = NBLK;
    for (int s = 0; s < c->nb; ++s) {
        cplx t = cmul(xv[s], c->Y[s * NBk + iy]);
        c->acc[s].re += sgn * t.re;
        c->acc[s].im += sgn * t.im;
        c->accm[s] += xm[s] * c->Ym[s * NBk + iy];
    }
}

/* 5a: raw blocks f(delta; xi1, xi2, xi3) = sum G(delta; xi') S S S of nb
 * sites and their antisymmetric components for P and N; fm[b], fmm[b] are
 * [site][NBLK] (values and magnitudes), allocated here. S: [site][12][NQ]
 * (sink row xi', source column xi). */
static void blocks_batch(const o3_plan *p, int nb, const cplx *S, cplx *fm[2], double *fmm[2]) {
    const int64_t NB = NBLK;
    cplx *fraw = (cplx *)calloc((size_t)(NB * nb), sizeof(cplx));
    double *fmag = (double *)calloc((size_t)(NB * nb), sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < nb; ++s) {
        const cplx *Ss = S + (int64_t)s * 12 * NQ;
        for (int a = 0; a < 4; ++a)
            for (int p1 = 0; p1 < 12; ++p1)
                for (int p2 = 0; p2 < 12; ++p2)
                    for (int p3 = 0; p3 < 12; ++p3) {
                        int g = p->Gs[((a * 12 + p1) * 12 + p2) * 12 + p3];
                        if (!g) continue;
                        for (int i = 0; i < NQ; ++i)
                            for (int j = 0; j < NQ; ++j)
                                for (int k = 0; k < NQ; ++k) {
                                    int64_t idx = ((int64_t)(a * NQ + i) * NQ + j) * NQ + k;
                                    cplx t = cmul(cmul(Ss[p1 * NQ + i], Ss[p2 * NQ + j]), Ss[p3 * NQ + k]);
                                    fraw[s * NB + idx].re += g * t.re;
                                    fraw[s * NB + idx].im += g * t.im;
                                    fmag[s * NB + idx] += abs(g) * cabs2(Ss[p1 * NQ + i]) *
                                                          cabs2(Ss[p2 * NQ + j]) * cabs2(Ss[p3 * NQ + k]);
                                }
                    }
    }
    for (int b = 0; b < 2; ++b) {
        fm[b] = (cplx *)calloc((size_t)(NB * nb), sizeof(cplx));
        fmm[b] = (double *)calloc((size_t)(NB * nb), sizeof(double));
    }
#pragma omp parallel for schedule(static)
    for (int s = 0; s < nb; ++s)
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < NQ; ++i)
                for (int j = 0; j < NQ; ++j)
                    for (int k = 0; k < NQ; ++k) {
                        int64_t idx = ((int64_t)(a * NQ + i) * NQ + j) * NQ + k;
                        int64_t sw_p = ((int64_t)(a * NQ + j) * NQ + i) * NQ + k; /* f(a; j, i, k) */
                        int64_t sw_n = ((int64_t)(a * NQ + k) * NQ + j) * NQ + i; /* f(a; k, j, i) */
                        const int64_t o = s * NB;
                        if (i < j) {
                            fm[0][o + idx].re = fraw[o + idx].re - fraw[o + sw_p].re;
                            fm[0][o + idx].im = fraw[o + idx].im - fraw[o + sw_p].im;
                            fmm[0][o + idx] = fmag[o + idx] + fmag[o + sw_p];
                        }
                        if (i < k) {
                            fm[1][o + idx].re = fraw[o + idx].re - fraw[o + sw_n].re;
                            fm[1][o + idx].im = fraw[o + idx].im - fraw[o + sw_n].im;
                            fmm[1][o + idx] = fmag[o + idx] + fmag[o + sw_n];
                        }
                    }
    free(fraw);
    free(fmag);
}

/* 5b-5d for nb items whose blocks are given ([item][NBLK]); results to
 * out/scale rows o0 .. o0 + nb - 1. */
static void recursion_batch(const o3_plan *p, int nb, cplx *const fm[2], double *const fmm[2], int64_t o0,
                            double *out, double *scale) {
    const int A = p->A;
    const int64_t NB = NBLK;
    /* 5b: F^(1) = f_{B1} on the needed keys of stage 1 */
    int b0 = p->path[0];
    cplx *X = (cplx *)calloc((size_t)(p->n_need[0] * nb), sizeof(cplx));
    double *Xm = (double *)calloc((size_t)(p->n_need[0] * nb), sizeof(double));
    for (int64_t i = 0; i < p->n_need[0]; ++i) {
        int64_t iy = block_index(p->need[0][i], b0);
        for (int s = 0; s < nb; ++s) { X[i * nb + s] = fm[b0][s * NB + iy]; Xm[i * nb + s] = fmm[b0][s * NB + iy]; }
    }
    /* 5c: F^(m+1)[z] = sum over splits sgn(x|y) F^(m)[x] f[y] */
    for (int m = 1; m < A; ++m) {
        int b = p->path[m];
        int64_t nz = p->n_need[m];
        cplx *Z = (cplx *)calloc((size_t)(nz * nb), sizeof(cplx));
        double *Zm = (double *)calloc((size_t)(nz * nb), sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < nz; ++i) {
            eval_ctx c;
            c.p = p; c.nb = nb; c.X = X; c.Xm = Xm; c.Y = fm[b]; c.Ym = fmm[b];
            c.nX = p->n_need[m - 1]; c.kX = p->need[m - 1];
            c.acc = Z + i * nb; c.accm = Zm + i * nb;
            for_splits(p->need[m][i], b, eval_cb, &c);
        }
        free(X); free(Xm);
        X = Z; Xm = Zm;
    }
    /* 5d: C(r) = (1/N) sum F^(A)[(sink set, U, D)] L(source set; U, D) */
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < p->n_req; ++r)
        for (int s = 0; s < nb; ++s) {
            double re = 0, im = 0, mg = 0;
            for (int64_t e = p->req_off[r]; e < p->req_off[r + 1]; ++e) {
                int64_t iz = find_key(p->need[A - 1], p->n_need[A - 1], p->req_key[e]);
                double l = (double)p->req_lval[e];
                re += X[iz * nb + s].re * l;
                im += X[iz * nb + s].im * l;
                mg += Xm[iz * nb + s] * fabs(l);
            }
            int64_t o = (o0 + s) * p->n_req + r;
            out[2 * o] = re / p->norm;
            out[2 * o + 1] = im / p->norm;
            if (scale) scale[o] = mg / p->norm;
        }
    free(X); free(Xm);
}

/*
 * Evaluate the plan on n_sites sites. S: [site][12][NQ] complex (re, im
 * interleaved), u = d. out: [site][n_req] complex; scale: [site][n_req]
 * (the magnitude recursion). batch: sites evaluated together.
 */
int o3_eval(const o3_plan *p, int64_t n_sites, const double *S_in, double *out, double *scale, int batch) {
    if (batch < 1) batch = 1;
    for (int64_t s0 = 0; s0 < n_sites; s0 += batch) {
        int nb = (int)((n_sites - s0) < batch ? (n_sites - s0) : batch);
        cplx *fm[2]; double *fmm[2];
        blocks_batch(p, nb, (const cplx *)S_in + s0 * 12 * NQ, fm, fmm);
        recursion_batch(p, nb, fm, fmm, s0, out, scale);
        for (int b = 0; b < 2; ++b) { free(fm[b]); free(fmm[b]); }
    }
    return 0;
}

/* Antisymmetric block components of n_sites sites (Sec. 2, Sec. 4):
 * out_fm[b]: [site][4][NQ][NQ][NQ] complex (re, im interleaved), out_mag[b]
 * the magnitudes, for b = 0 (proton) and 1 (neutron); entries that are not
 * independent components are zero. */
int o3_blocks(const o3_plan *p, int64_t n_sites, const double *S_in, double *fm_p, double *fm_n, double *mag_p,
              double *mag_n) {
    const int64_t NB = NBLK;
    cplx *fm[2]; double *fmm[2];
    blocks_batch(p, (int)n_sites, (const cplx *)S_in, fm, fmm);
    memcpy(fm_p, fm[0], sizeof(cplx) * (size_t)(NB * n_sites));
    memcpy(fm_n, fm[1], sizeof(cplx) * (size_t)(NB * n_sites));
    memcpy(mag_p, fmm[0], sizeof(double) * (size_t)(NB * n_sites));
    memcpy(mag_n, fmm[1], sizeof(double) * (size_t)(NB * n_sites));
    for (int b = 0; b < 2; ++b) { free(fm[b]); free(fmm[b]); }
    return 0;
}

/* The recursion and contraction (eq. recr_F, eq. C_final) for n_items sets of
 * given blocks, e.g. blocks summed over sink sites with a momentum phase
 * (Sec. 2). Layouts as o3_blocks; out: [item][n_req] complex, scale:
 * [item][n_req] (the magnitude recursion run on the given magnitudes). */
int o3_eval_blocks(const o3_plan *p, int64_t n_items, const double *fm_p, const double *fm_n, const double *mag_p,
                   const double *mag_n, double *out, double *scale) {
    cplx *fm[2] = {(cplx *)fm_p, (cplx *)fm_n};
    double *fmm[2] = {(double *)mag_p, (double *)mag_n};
    recursion_batch(p, (int)n_items, fm, fmm, 0, out, scale);
    return 0;
}
