// Device helpers shared by the contraction kernels: complex storage types,
// FP64 and compensated float-float accumulators, sign flips without
// arithmetic, and the baryon-block formulas.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace mbc {

// ---- precision traits ------------------------------------------------------

struct FP64Traits {
    using V = double2;  // stored stage value
    struct Acc {
        double re, im;
        __device__ __forceinline__ void zero() { re = 0.0; im = 0.0; }
        // acc += (sign) * x * y  - four DFMA, the sign flips x by bit ops
        __device__ __forceinline__ void fma(double2 x, double2 y, uint32_t neg) {
            double xr = __hiloint2double(__double2hiint(x.x) ^ (int)neg, __double2loint(x.x));
            double xi = __hiloint2double(__double2hiint(x.y) ^ (int)neg, __double2loint(x.y));
            re = __fma_rn(xr, y.x, re);
            re = __fma_rn(-xi, y.y, re);
            im = __fma_rn(xr, y.y, im);
            im = __fma_rn(xi, y.x, im);
        }
        __device__ __forceinline__ void add_shfl(unsigned mask, int off) {
            re += __shfl_xor_sync(mask, re, off);
            im += __shfl_xor_sync(mask, im, off);
        }
        __device__ __forceinline__ double2 value() const { return make_double2(re, im); }
        __device__ __forceinline__ V store() const { return make_double2(re, im); }
    };
    __device__ __forceinline__ static double2 to_d(V v) { return v; }
    __device__ __forceinline__ static V from_d(double2 v) { return v; }
    // entry idx of a wave buffer ([component][site], plain)
    __device__ __forceinline__ static V wave_ld(const V *p, int64_t idx) { return p[idx]; }
    __device__ __forceinline__ static void wave_st(V *p, int64_t idx, V v) { p[idx] = v; }
};

// float-float (two-sum) accumulation of FP32 complex products
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// ---- packed FP32 pairs --------------------------------------------------------
// A 64-bit register pair holds two FP32 values and one f32x2 instruction
// (sm_100 and later) works on both lanes, each rounded to nearest exactly as
// the scalar instruction would round it: half the issue slots for the same
// arithmetic.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_neg(uint64_t a) { return a ^ 0x8000000080000000ull; }

// Kahan step on two lanes at once: s += p, c collects the rounding lost
// (value = s - c), the scalar sequence y = p - c, t = s + y,
// c = (t - s) - y, s = t.
__device__ __forceinline__ void f2_kahan(uint64_t &s, uint64_t &c, uint64_t p) {
    const uint64_t y = f2_sub(p, c);
    const uint64_t t = f2_add(s, y);
    c = f2_sub(f2_sub(t, s), y);
    s = t;
}

struct MixedTraits {
    using V = float2;
    // Kahan-compensated FP32 accumulation of FP32 complex products: value =
    // s - c, where c carries the rounding lost by the running sum s; the
    // real and imaginary parts share packed instructions.
    struct Acc {
        uint64_t s, c;  // (re, im) pairs
        __device__ __forceinline__ void zero() { s = c = 0ull; }
        __device__ __forceinline__ void fma(float2 x, float2 y, uint32_t neg) {
            float xr = __int_as_float(__float_as_int(x.x) ^ (int)neg);
            float xi = __int_as_float(__float_as_int(x.y) ^ (int)neg);
            f2_kahan(s, c, f2_pack(__fmaf_rn(xr, y.x, -__fmul_rn(xi, y.y)), __fmaf_rn(xr, y.y, __fmul_rn(xi, y.x))));
        }
        // combine with another accumulator (s2 - c2): two-sum of the sums
        __device__ __forceinline__ void add(float s2r, float c2r, float s2i, float c2i) {
            float2 sv = f2_unpack(s), cv = f2_unpack(c);
            float sr, er, si, ei;
            two_sum(sv.x, s2r, sr, er);
            two_sum(sv.y, s2i, si, ei);
            s = f2_pack(sr, si);
            c = f2_pack(__fsub_rn(__fadd_rn(cv.x, c2r), er), __fsub_rn(__fadd_rn(cv.y, c2i), ei));
        }
        __device__ __forceinline__ void add_shfl(unsigned mask, int off) {
            float2 sv = f2_unpack(s), cv = f2_unpack(c);
            float a = __shfl_xor_sync(mask, sv.x, off), b = __shfl_xor_sync(mask, cv.x, off);
            float d = __shfl_xor_sync(mask, sv.y, off), e = __shfl_xor_sync(mask, cv.y, off);
            add(a, b, d, e);
        }
        __device__ __forceinline__ double2 value() const {
            float2 sv = f2_unpack(s), cv = f2_unpack(c);
            return make_double2((double)sv.x - (double)cv.x, (double)sv.y - (double)cv.y);
        }
        __device__ __forceinline__ V store() const { return f2_unpack(f2_sub(s, c)); }
    };
    __device__ __forceinline__ static double2 to_d(V v) { return make_double2(v.x, v.y); }
    __device__ __forceinline__ static V from_d(double2 v) { return make_float2((float)v.x, (float)v.y); }
    // Wave buffers ([component][site], rows of an even number of sites) keep
    // each pair of sites (2j, 2j + 1) planar in 16 B: (re 2j, re 2j+1,
    // im 2j, im 2j+1), so the two-sites-per-lane kernels load a real pair and
    // an imaginary pair ready for packed arithmetic.
    __device__ __forceinline__ static int64_t wave_word(int64_t idx) { return (idx & ~(int64_t)1) * 2 + (idx & 1); }
    __device__ __forceinline__ static V wave_ld(const V *p, int64_t idx) {
        const float *f = reinterpret_cast<const float *>(p) + wave_word(idx);
        return make_float2(f[0], f[2]);
    }
    __device__ __forceinline__ static void wave_st(V *p, int64_t idx, V v) {
        float *f = reinterpret_cast<float *>(p) + wave_word(idx);
        f[0] = v.x;
        f[2] = v.y;
    }
};

// Two sites' accumulators side by side (the wave kernels' two sites per
// lane): lane 0 of every pair is the first site, lane 1 the second, so the
// complex products of both sites are packed instructions too. The
// operation's sign enters as a pair (sg, sg) of +-1 in the first Kahan
// step (an exact multiply), and the compensation is kept negated (n = -c):
// the same roundings as MixedTraits::Acc, bit for bit. Operands and results
// are 16 B of a planar wave buffer (MixedTraits::wave_ld).
struct PairAcc {
    uint64_t sr, si, nr, ni;  // sums and negated compensations, (site 0, site 1)
    __device__ __forceinline__ void zero() { sr = si = nr = ni = 0ull; }
    __device__ __forceinline__ static void step(uint64_t &s, uint64_t &n, uint64_t p, uint64_t sg) {
        const uint64_t y = f2_fma(p, sg, n);  // sg p - c
        const uint64_t t = f2_add(s, y);
        n = f2_sub(y, f2_sub(t, s));  // -((t - s) - y)
        s = t;
    }
    // x, y: (real pair, imaginary pair) of the two sites
    __device__ __forceinline__ void fma(ulonglong2 x, ulonglong2 y, uint64_t sg) {
        const uint64_t pr = f2_fma(x.x, y.x, f2_neg(f2_mul(x.y, y.y)));  // xr yr - xi yi
        const uint64_t pi = f2_fma(x.x, y.y, f2_mul(x.y, y.x));           // xr yi + xi yr
        step(sr, nr, pr, sg);
        step(si, ni, pi, sg);
    }
    __device__ __forceinline__ ulonglong2 store() const {
        return make_ulonglong2(f2_add(sr, nr), f2_add(si, ni));
    }
};

// plain complex helpers in the storage type (block construction)
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(__fma_rn(a.x, b.x, -a.y * b.y), __fma_rn(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, -a.y * b.y), __fmaf_rn(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    return make_double2(__fma_rn(a.x, b.x, __fma_rn(-a.y, b.y, c.x)), __fma_rn(a.x, b.y, __fma_rn(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
    return make_float2(__fmaf_rn(a.x, b.x, __fmaf_rn(-a.y, b.y, c.x)), __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, c.y)));
}
// c - a * b with fused multiply-adds only
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {
    return make_double2(__fma_rn(-a.x, b.x, __fma_rn(a.y, b.y, c.x)), __fma_rn(-a.x, b.y, __fma_rn(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 c) {
    return make_float2(__fmaf_rn(-a.x, b.x, __fmaf_rn(a.y, b.y, c.x)), __fmaf_rn(-a.x, b.y, __fmaf_rn(-a.y, b.x, c.y)));
}

// ---- the G tensor (eq. def_g) in factorised form -----------------------------
// Gamma_2 = C gamma_5 entries (s2, s3, value); the nonrelativistic form keeps
// the first two. Gamma_1 is diagonal with unit entries for spins < dim.
__constant__ int c_g2[4][3] = {{0, 1, -1}, {1, 0, 1}, {2, 3, -1}, {3, 2, 1}};
// epsilon: for colour c of slot 1, the two (c2, c3, sign) completions
__constant__ int c_eps[3][2][3] = {{{1, 2, 1}, {2, 1, -1}}, {{2, 0, 1}, {0, 2, -1}}, {{0, 1, 1}, {1, 0, -1}}};
// colex pair decoding for up to 12 values: pair rank -> (i < j)
__constant__ uint8_t c_pair_i[66];
__constant__ uint8_t c_pair_j[66];

// Diquark Q[c][xi2][xi3] = sum_{Gamma_2, eps} v eps S[3 s2 + c2][xi2] S[3 s3 + c3][xi3]
// (the slot-2/slot-3 part of a block, Sec. 2). S is an nxi x nxi tile.
template <class V>
__device__ __forceinline__ V diquark(const V *S, int ld, int nxi, int n_g2, int c, int x2, int x3) {
    V acc{0, 0};
    for (int g = 0; g < n_g2; ++g) {
        int s2 = c_g2[g][0], s3 = c_g2[g][1], v = c_g2[g][2];
        for (int e = 0; e < 2; ++e) {
            int c2 = c_eps[c][e][0], c3 = c_eps[c][e][1], sg = c_eps[c][e][2] * v;
            const V a = S[(3 * s2 + c2) * ld + x2], b = S[(3 * s3 + c3) * ld + x3];
            acc = sg > 0 ? cfma(a, b, acc) : cfms(a, b, acc);
        }
    }
    return acc;
}

}  // namespace mbc
