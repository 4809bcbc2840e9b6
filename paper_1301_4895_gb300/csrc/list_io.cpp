// Term lists on disk: a built list written once and loaded by every rank or
// run that needs the same nucleus and selection, instead of rebuilding it
// (the builder takes about a minute for 8Be's 448,496,928 operations).
//
// Format: the bytes "MBCL", a version, the sizes of the stats record and of
// the index types (so a file from another build is refused), then every
// field of the list in a fixed order, vectors as a uint64 length followed by
// their elements. Little-endian hosts only (x86-64 and AArch64 both are).
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "mbc_internal.h"

namespace {

constexpr char kMagic[4] = {'M', 'B', 'C', 'L'};
constexpr uint32_t kVersion = 1;

struct Writer {
    FILE *f;
    bool ok = true;
    void bytes(const void *p, size_t n) {
        if (ok && n && std::fwrite(p, 1, n, f) != n) ok = false;
    }
    template <class T>
    void pod(const T &v) {
        static_assert(std::is_trivially_copyable<T>::value, "plain data only");
        bytes(&v, sizeof(T));
    }
    template <class T>
    void vec(const std::vector<T> &v) {
        pod<uint64_t>(v.size());
        bytes(v.data(), v.size() * sizeof(T));
    }
};

struct Reader {
    FILE *f;
    uint64_t left;  // bytes of the file not read yet
    bool ok = true;
    void bytes(void *p, size_t n) {
        if (ok && n > left) ok = false;
        if (ok && n && std::fread(p, 1, n, f) != n) ok = false;
        if (ok) left -= n;
    }
    template <class T>
    void pod(T &v) {
        bytes(&v, sizeof(T));
    }
    // a length is checked against the bytes left before anything is
    // allocated, so a damaged length field cannot request a huge vector
    template <class T>
    void vec(std::vector<T> &v) {
        uint64_t n = 0;
        pod(n);
        if (!ok || n > left / sizeof(T)) {
            ok = false;
            return;
        }
        v.resize((size_t)n);
        bytes(v.data(), (size_t)n * sizeof(T));
    }
};

// size of an open file, or -1
int64_t file_size(FILE *f) {
    if (std::fseek(f, 0, SEEK_END) != 0) return -1;
    const long n = std::ftell(f);
    if (n < 0 || std::fseek(f, 0, SEEK_SET) != 0) return -1;
    return (int64_t)n;
}

template <class IO, class L>
void fields(IO &io, L &list) {
    io.pod(list.A);
    io.pod(list.n_p);
    io.pod(list.n_n);
    io.pod(list.dim);
    io.pod(list.n_sources);
    io.pod(list.n_sinks);
    io.pod(list.dim_snk);
    io.pod(list.dim_src);
    io.pod(list.path);
    io.pod(list.pauli_forbidden);
    io.pod(list.nxi);
    io.pod(list.block_size);
    io.pod(list.need_block);
    io.pod(list.final_size);
    io.pod(list.n_comp);
    io.vec(list.comp_snk);
    io.vec(list.comp_src);
    io.vec(list.fin_off);
    io.vec(list.fin_z);
    io.vec(list.fin_l);
    io.pod(list.norm);
    io.vec(list.parts);
    io.pod(list.stats);
}

template <class IO, class S>
void step_fields(IO &io, S &s) {
    io.pod(s.baryon);
    io.pod(s.n_x);
    io.pod(s.n_z);
    io.pod(s.k);
    io.pod(s.dense);
    io.pod(s.generated);
    io.pod(s.zk);
    io.pod(s.xk);
    io.vec(s.x);
    io.vec(s.ys);
    io.vec(s.zrank);
    io.vec(s.xmap);
}

void header(Writer &w) {
    w.bytes(kMagic, 4);
    w.pod(kVersion);
    w.pod<uint32_t>((uint32_t)sizeof(mbc_list_stats));
    w.pod<uint32_t>((uint32_t)sizeof(mbc_term_list::Part));
}

bool header_ok(Reader &r) {
    char m[4];
    uint32_t v = 0, ss = 0, ps = 0;
    r.bytes(m, 4);
    r.pod(v);
    r.pod(ss);
    r.pod(ps);
    return r.ok && std::memcmp(m, kMagic, 4) == 0 && v == kVersion && ss == sizeof(mbc_list_stats) &&
           ps == sizeof(mbc_term_list::Part);
}

int64_t binom_i(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// Every index the kernels will use must lie inside its buffer: a list read
// from a file is checked entry by entry before it can reach a device.
bool indices_ok(const mbc_term_list &L) {
    if (L.nxi < 1 || L.nxi > 24 || L.dim_snk < 1 || L.dim_snk > 16 || L.dim < 1 || L.dim > 4) return false;
    if (L.block_size != (int64_t)L.dim_snk * binom_i(L.nxi, 2) * L.nxi) return false;
    if (L.pauli_forbidden) return true;
    int64_t n_prev = L.block_size;
    std::vector<int64_t> stage_size(1, L.block_size);  // stage 1: the first baryon's block
    for (const auto &s : L.steps) {
        if (s.baryon != MBC_PROTON && s.baryon != MBC_NEUTRON) return false;
        if (s.n_x != n_prev || s.n_z < 0 || s.k < 0 || s.n_z > ((int64_t)1 << 32)) return false;
        if (s.generated) {
            int64_t zs = binom_i(L.dim_snk, s.zk[0]) * binom_i(L.dim_snk, s.zk[1]) * binom_i(L.nxi, s.zk[2]) *
                         binom_i(L.nxi, s.zk[3]);
            int64_t xs = binom_i(L.dim_snk, s.xk[0]) * binom_i(L.dim_snk, s.xk[1]) * binom_i(L.nxi, s.xk[2]) *
                         binom_i(L.nxi, s.xk[3]);
            if (s.zrank.empty() ? s.n_z != zs : (int64_t)s.zrank.size() != s.n_z) return false;
            for (int64_t r : s.zrank)
                if (r < 0 || r >= zs) return false;
            if (!s.xmap.empty()) {
                if ((int64_t)s.xmap.size() != xs) return false;
                for (int32_t v : s.xmap)
                    if (v < -1 || v >= s.n_x) return false;
            } else if (&s != &L.steps[0] && xs != s.n_x) {
                return false;
            }
        } else {
            if ((int64_t)s.x.size() != s.n_z * s.k || s.ys.size() != s.x.size()) return false;
            for (uint32_t v : s.x)
                if ((int64_t)v >= s.n_x) return false;
            for (uint16_t v : s.ys)
                if ((int64_t)(v & 0x7fffu) >= L.block_size) return false;
        }
        n_prev = s.n_z;
        stage_size.push_back(s.n_z);
    }
    for (const auto &pt : L.parts) {
        if (pt.A < 1 || pt.A > L.A || pt.c0 < 0 || pt.c1 < pt.c0 || pt.c1 > L.n_comp) return false;
        for (int c = pt.c0; c < pt.c1; ++c)
            for (int64_t e = L.fin_off[(size_t)c]; e < L.fin_off[(size_t)c + 1]; ++e)
                if (e < 0 || e >= (int64_t)L.fin_z.size() || (int64_t)L.fin_z[(size_t)e] >= stage_size[(size_t)pt.A - 1])
                    return false;
    }
    return !L.parts.empty() || L.n_comp == 0;
}

}  // namespace

extern "C" {

mbc_status mbc_save_term_list(const mbc_term_list *list, const char *path) {
    if (!list || !path) return MBC_ERR_INVALID_ARG;
    FILE *f = std::fopen(path, "wb");
    if (!f) return MBC_ERR_INVALID_ARG;
    Writer w{f};
    header(w);
    fields(w, *list);
    w.pod<uint64_t>(list->steps.size());
    for (const auto &s : list->steps) step_fields(w, s);
    const bool closed = std::fclose(f) == 0;
    return w.ok && closed ? MBC_OK : MBC_ERR_INVALID_ARG;
}

mbc_status mbc_load_term_list(const char *path, mbc_term_list **out) {
    if (!out) return MBC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!path) return MBC_ERR_INVALID_ARG;
    FILE *f = std::fopen(path, "rb");
    if (!f) return MBC_ERR_INVALID_ARG;
    mbc_term_list *L = new (std::nothrow) mbc_term_list();
    if (!L) {
        std::fclose(f);
        return MBC_ERR_OOM;
    }
    const int64_t size = file_size(f);
    if (size < 0) {
        std::fclose(f);
        delete L;
        return MBC_ERR_INVALID_ARG;
    }
    Reader r{f, (uint64_t)size};
    mbc_status st = MBC_OK;
    try {
        if (!header_ok(r)) {
            st = MBC_ERR_INVALID_ARG;
        } else {
            fields(r, *L);
            uint64_t n_steps = 0;
            r.pod(n_steps);
            if (!r.ok || n_steps > MBC_MAX_A) {
                st = MBC_ERR_INVALID_ARG;
            } else {
                L->steps.resize((size_t)n_steps);
                for (auto &s : L->steps) step_fields(r, s);
            }
            // consistency of what the kernels index with
            const bool sane = r.ok && L->A >= 1 && L->A <= MBC_MAX_A &&
                              ((int)L->steps.size() == L->A - 1 || (L->pauli_forbidden && L->steps.empty())) &&
                              L->n_comp >= 0 && L->fin_off.size() == (size_t)L->n_comp + 1 &&
                              L->fin_off.back() == (int64_t)L->fin_z.size() && L->fin_z.size() == L->fin_l.size() &&
                              L->comp_snk.size() == (size_t)L->n_comp * L->A;
            if (st == MBC_OK && !sane) st = MBC_ERR_INVALID_ARG;
            if (st == MBC_OK && !indices_ok(*L)) st = MBC_ERR_INVALID_ARG;
        }
    } catch (const std::bad_alloc &) {
        st = MBC_ERR_OOM;
    }
    std::fclose(f);
    if (st != MBC_OK) {
        delete L;
        return st;
    }
    *out = L;
    return L->pauli_forbidden ? MBC_ERR_PAULI_FORBIDDEN : MBC_OK;
}

}  // extern "C"
