// Mixed-precision helpers: packed FP32-pair arithmetic (f32x2), compensated
// FP32 accumulation of FP32 complex products, decoded operation records, and
// the FP32 storage type of the mixed path with its wave-buffer layout.
#pragma once

#include "device_common.cuh"

namespace mbc {

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

// Kahan step on two lanes at once with the compensation kept negated
// (n = -c): the scalar sequence y = p - c, t = s + y, c = (t - s) - y, s = t
// becomes y = p + n, t = s + y, n = y - (t - s), rounding for rounding the
// same, since negation is exact.
__device__ __forceinline__ void f2_kahan(uint64_t &s, uint64_t &n, uint64_t p) {
    const uint64_t y = f2_add(p, n);
    const uint64_t t = f2_add(s, y);
    n = f2_sub(y, f2_sub(t, s));
    s = t;
}
// The same step adding sg * p for a sign pair sg = (+-1, +-1): the multiply
// is exact, so y = fma(p, sg, n) is the scalar y of the signed term.
__device__ __forceinline__ void f2_kahan_signed(uint64_t &s, uint64_t &n, uint64_t p, uint64_t sg) {
    const uint64_t y = f2_fma(p, sg, n);
    const uint64_t t = f2_add(s, y);
    n = f2_sub(y, f2_sub(t, s));
    s = t;
}
// (+1, +1) or (-1, -1) as a packed pair
__device__ __forceinline__ uint64_t f2_sign_pair(bool negative) {
    const float v = negative ? -1.f : 1.f;
    return f2_pack(v, v);
}

// An operation decoded for broadcast from shared memory: the two operand
// offsets and the sign as a (+-1, +-1) pair, 16 B, one load.
struct __align__(16) OpRec {
    uint32_t x, y;
    uint64_t sg;
};

struct MixedTraits {
    using V = float2;
    // Kahan-compensated FP32 accumulation of FP32 complex products: value =
    // s + n, where n = -c carries the rounding lost by the running sum s; the
    // real and imaginary parts share packed instructions.
    struct Acc {
        uint64_t s, n;  // (re, im) pairs
        __device__ __forceinline__ void zero() { s = n = 0ull; }
        __device__ __forceinline__ static uint64_t prod(float xr, float xi, float2 y) {
            return f2_pack(__fmaf_rn(xr, y.x, -__fmul_rn(xi, y.y)), __fmaf_rn(xr, y.y, __fmul_rn(xi, y.x)));
        }
        // acc += (sign) x y, the sign flipping x by bit operations
        __device__ __forceinline__ void fma(float2 x, float2 y, uint32_t neg) {
            float xr = __int_as_float(__float_as_int(x.x) ^ (int)neg);
            float xi = __int_as_float(__float_as_int(x.y) ^ (int)neg);
            f2_kahan(s, n, prod(xr, xi, y));
        }
        // acc += sg x y with the sign as a pair (OpRec::sg), folded into the
        // Kahan step; the same result as fma()
        __device__ __forceinline__ void fma_sg(float2 x, float2 y, uint64_t sg) {
            f2_kahan_signed(s, n, prod(x.x, x.y, y), sg);
        }
        // acc += x y and acc -= x y: the Kahan step's first sum is p + n
        // and n - p, rounded as fma_sg's fma(p, +-1, n)
        __device__ __forceinline__ void add_prod(float2 x, float2 y) { f2_kahan(s, n, prod(x.x, x.y, y)); }
        __device__ __forceinline__ void sub_prod(float2 x, float2 y) {
            const uint64_t p = prod(x.x, x.y, y);
            const uint64_t yv = f2_sub(n, p);
            const uint64_t t = f2_add(s, yv);
            n = f2_sub(yv, f2_sub(t, s));
            s = t;
        }
        // combine with another accumulator (s2 + n2): two-sum of the sums
        __device__ __forceinline__ void add(float s2r, float n2r, float s2i, float n2i) {
            float2 sv = f2_unpack(s), nv = f2_unpack(n);
            float sr, er, si, ei;
            two_sum(sv.x, s2r, sr, er);
            two_sum(sv.y, s2i, si, ei);
            s = f2_pack(sr, si);
            n = f2_pack(__fadd_rn(er, __fadd_rn(nv.x, n2r)), __fadd_rn(ei, __fadd_rn(nv.y, n2i)));
        }
        __device__ __forceinline__ void add_shfl(unsigned mask, int off) {
            float2 sv = f2_unpack(s), nv = f2_unpack(n);
            float a = __shfl_xor_sync(mask, sv.x, off), b = __shfl_xor_sync(mask, nv.x, off);
            float d = __shfl_xor_sync(mask, sv.y, off), e = __shfl_xor_sync(mask, nv.y, off);
            add(a, b, d, e);
        }
        __device__ __forceinline__ double2 value() const {
            float2 sv = f2_unpack(s), nv = f2_unpack(n);
            return make_double2((double)sv.x + (double)nv.x, (double)sv.y + (double)nv.y);
        }
        __device__ __forceinline__ V store() const { return f2_unpack(f2_add(s, n)); }
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
    // x, y: (real pair, imaginary pair) of the two sites
    __device__ __forceinline__ void fma(ulonglong2 x, ulonglong2 y, uint64_t sg) {
        const uint64_t pr = f2_fma(x.x, y.x, f2_neg(f2_mul(x.y, y.y)));  // xr yr - xi yi
        const uint64_t pi = f2_fma(x.x, y.y, f2_mul(x.y, y.x));           // xr yi + xi yr
        f2_kahan_signed(sr, nr, pr, sg);
        f2_kahan_signed(si, ni, pi, sg);
    }
    __device__ __forceinline__ ulonglong2 store() const {
        return make_ulonglong2(f2_add(sr, nr), f2_add(si, ni));
    }
    // add another accumulator (t = its sums, u = its negated compensations):
    // two-sum of the sums, the rounding error joins the compensations
    __device__ __forceinline__ void add(ulonglong2 t, ulonglong2 u) {
        const uint64_t r = f2_add(sr, t.x), br = f2_sub(r, sr);
        const uint64_t er = f2_add(f2_sub(sr, f2_sub(r, br)), f2_sub(t.x, br));
        const uint64_t i = f2_add(si, t.y), bi = f2_sub(i, si);
        const uint64_t ei = f2_add(f2_sub(si, f2_sub(i, bi)), f2_sub(t.y, bi));
        sr = r;
        si = i;
        nr = f2_add(er, f2_add(nr, u.x));
        ni = f2_add(ei, f2_add(ni, u.y));
    }
};

}  // namespace mbc
