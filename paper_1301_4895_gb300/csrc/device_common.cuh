// Device helpers shared by the contraction kernels: the FP64 storage type and
// accumulator, sign flips without arithmetic, complex helpers and the
// baryon-block formulas. The mixed-precision types live in mixed_common.cuh.
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
// colex pair decoding for up to 24 quark index values (two relativistic
// sources): pair rank -> (i < j)
__constant__ uint8_t c_pair_i[276];
__constant__ uint8_t c_pair_j[276];

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
