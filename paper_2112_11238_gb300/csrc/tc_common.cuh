// tc_common.cuh -- pieces shared by the tensor-core kernels: the split forms,
// index maps, loading and splitting of operand chunks, and the
// swizzled (64-byte) K-major shared-memory layout the tcgen05 descriptors
// describe.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "ptx.cuh"

namespace kron {

template <int F>
struct FT;
template <>
struct FT<kTF32x3> {
    static constexpr int KIND = 0, PIECES = 2, ELEM = 4, NPROD = 3, FMT = 2, MMA_K = 8;
};
template <>
struct FT<kBF16x3> {
    static constexpr int KIND = 1, PIECES = 2, ELEM = 2, NPROD = 3, FMT = 1, MMA_K = 16;
};
template <>
struct FT<kBF16x6> {
    static constexpr int KIND = 1, PIECES = 3, ELEM = 2, NPROD = 6, FMT = 1, MMA_K = 16;
};

template <>
struct FT<kFX32> {
    static constexpr int KIND = 1, PIECES = 4, ELEM = 2, NPROD = 10, FMT = 1, MMA_K = 16;
};
// 29-bit fixed point in three FP16 digit slices (kind::f16, both operands f16)
template <>
struct FT<kFX32H> {
    static constexpr int KIND = 1, PIECES = 3, ELEM = 2, NPROD = 6, FMT = 0, MMA_K = 16;
};
template <int F>
__host__ __device__ constexpr bool is_fx_f() { return F == kFX32 || F == kFX32H; }

// Tensor-memory accumulator regions per accumulator set: the split forms keep
// hi*hi (region 0) apart from the cross products (region 1); the fixed-point
// form keeps level 0 (exact: integer-valued sums below 2^24) apart from
// levels 1..3 (region 1; with balanced digits its partial sums have no
// preferred sign, so the truncation of the FP32 accumulation does not
// accumulate a bias).
template <int F>
struct Regions {
    static constexpr int N = 2;
};

// Products (piece of A, piece of B), smallest magnitude first.
template <int F>
__device__ __forceinline__ void prod_pieces(int i, int &pa, int &pb) {
    if constexpr (F == kFX32) {
        // levels 3 and 2, then level 1, then level 0
        const int ta[10] = {3, 2, 1, 0, 2, 1, 0, 1, 0, 0};
        const int tb[10] = {0, 1, 2, 3, 0, 1, 2, 0, 1, 0};
        pa = ta[i];
        pb = tb[i];
    } else if constexpr (FT<F>::PIECES == 2) {
        // lo*hi, hi*lo, hi*hi
        pa = (i == 0) ? 1 : 0;
        pb = (i == 1) ? 1 : 0;
    } else {
        // three pieces (BF16x6, and the FX32H digits: levels 2, 1, 0):
        // (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
        const int ta[6] = {2, 1, 0, 1, 0, 0};
        const int tb[6] = {0, 1, 2, 0, 1, 0};
        pa = ta[i];
        pb = tb[i];
    }
}

// Region of product i and whether it is the first product written there.
template <int F>
__device__ __forceinline__ int region_of(int i) {
    return (i == FT<F>::NPROD - 1) ? 0 : 1;
}
template <int F>
__device__ __forceinline__ bool first_in_region(int i) {
    return i == 0 || i == FT<F>::NPROD - 1;
}

constexpr int kRowBytes = 64;       // bytes of one K-major row per K-block (64-byte swizzle)
constexpr int kChunks = kRowBytes / 16;  // 16-byte chunks per row
constexpr int kBM = 128;            // rows per tile (MMA M)

__host__ __device__ __forceinline__ int64_t imap(const IdxMap &m, int64_t x) {
    if (m.R0 == 0) return x * m.s0;
    return (x % m.R0) * m.s0 + (x / m.R0) * m.s1;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void to_hl(float x, float &h, float &l) {
    h = x;
    l = 0.f;
}
__device__ __forceinline__ void to_hl(double x, float &h, float &l) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}

// Loads CH consecutive-k values of one row (zero outside the tensor).  VEC:
// the CH values are contiguous and 16-byte aligned whenever fully in range.
// COH: coherent L2 loads (ld.global.cg) for data written earlier in the same
// launch by other CTAs; otherwise read-only loads (ld.global.nc).
template <bool COH, typename T>
__device__ __forceinline__ T ldx(const T *p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

template <int F, typename Tin, bool COH = false>
__device__ __forceinline__ void load_chunk(const Tin *__restrict__ src, int64_t ro, const IdxMap &km,
                                           int64_t k0, int64_t K, bool vec, Tin (&v)[16 / FT<F>::ELEM]) {
    constexpr int CH = 16 / FT<F>::ELEM;
    if (vec && ro >= 0 && k0 + CH <= K) {
        const uint4 *q = reinterpret_cast<const uint4 *>(src + ro + k0);
        constexpr int NV = CH * (int)sizeof(Tin) / 16;
        uint4 w[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) w[i] = ldx<COH>(q + i);
#pragma unroll
        for (int i = 0; i < NV; ++i) *reinterpret_cast<uint4 *>(&v[i * (16 / sizeof(Tin))]) = w[i];
        return;
    }
#pragma unroll
    for (int e = 0; e < CH; ++e) {
        const int64_t k = k0 + e;
        v[e] = (ro >= 0 && k < K) ? ldx<COH>(src + ro + imap(km, k)) : Tin(0);
    }
}

// Splits CH values into the form's pieces, one 16-byte chunk per piece.
template <int F, typename Tin>
__device__ __forceinline__ void split_pack(const Tin (&v)[16 / FT<F>::ELEM], uint4 (&out)[FT<F>::PIECES]) {
    constexpr int CH = 16 / FT<F>::ELEM;
    // FP32 input has no low part (l = 0): its residuals skip the addition
    constexpr bool LO = sizeof(Tin) == 8;
    float h[CH], l[CH];
#pragma unroll
    for (int e = 0; e < CH; ++e) to_hl(v[e], h[e], l[e]);
    if constexpr (F == kTF32x3) {
        uint32_t a0[4], a1[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            a0[e] = to_tf32(h[e]);
            float r = h[e] - __uint_as_float(a0[e]);
            if constexpr (LO) r += l[e];
            a1[e] = to_tf32(r);
        }
        out[0] = make_uint4(a0[0], a0[1], a0[2], a0[3]);
        out[1] = make_uint4(a1[0], a1[1], a1[2], a1[3]);
    } else {
        // two values at a time: one paired round-to-nearest conversion per
        // piece gives the bf16x2 word directly (element e in the low half)
        uint32_t w[FT<F>::PIECES][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const __nv_bfloat162 b0 = __floats2bfloat162_rn(h[e], h[e + 1]);
            const float2 f0 = __bfloat1622float2(b0);
            float r0 = h[e] - f0.x, r1 = h[e + 1] - f0.y;
            if constexpr (LO) {
                r0 += l[e];
                r1 += l[e + 1];
            }
            const __nv_bfloat162 b1 = __floats2bfloat162_rn(r0, r1);
            w[0][e / 2] = *reinterpret_cast<const uint32_t *>(&b0);
            w[1][e / 2] = *reinterpret_cast<const uint32_t *>(&b1);
            if constexpr (FT<F>::PIECES == 3) {
                const float2 f1 = __bfloat1622float2(b1);
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(r0 - f1.x, r1 - f1.y);
                w[2][e / 2] = *reinterpret_cast<const uint32_t *>(&b2);
            }
        }
#pragma unroll
        for (int p = 0; p < FT<F>::PIECES; ++p) out[p] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    }
}

// 32-bit fixed-point values -> four balanced base-256 digits each,
// x = d0 2^24 + d1 2^16 + d2 2^8 + d3 with d1..d3 in [-128, 127] and
// d0 in [-128, 128]; slice t = d_t * 2^(-8t), exact in bf16.  Balanced
// digits make the slice products left out (levels 4 and up) average to zero
// instead of always pulling the same way.
// Digits without a carry chain: y = x + 0x808080 has the unsigned bytes
// d1 + 128, d2 + 128, d3 + 128 and y >> 24 = d0.  Each digit becomes a float
// exactly through the 2^23 exponent trick (one OR, one FMA), and the high
// halves of two floats are packed into one bf16x2 word with a byte permute.
// mul: a power of two the values are scaled by first (their left shift),
// folded into the digit offset's addition as one multiply-add.
__device__ __forceinline__ void fx_pack(const int32_t (&v)[8], uint4 (&out)[4], int mul = 1) {
    uint32_t w[4][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        float f[4][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long y64 = (long long)v[e + h] * mul + 0x808080ll;
            const uint32_t y = (uint32_t)y64;
            const int d0 = (int)(y64 >> 24);
            f[0][h] = __int_as_float(0x4B400000 + d0) - 12582912.0f;
            f[1][h] = fmaf(__uint_as_float(0x4B000000u | ((y >> 16) & 0xFFu)), 0.00390625f, -32768.5f);
            f[2][h] = fmaf(__uint_as_float(0x4B000000u | ((y >> 8) & 0xFFu)), 1.52587890625e-05f, -128.001953125f);
            f[3][h] = fmaf(__uint_as_float(0x4B000000u | (y & 0xFFu)), 5.9604644775390625e-08f, -0.50000762939453125f);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
            w[t][e / 2] = __byte_perm(__float_as_uint(f[t][0]), __float_as_uint(f[t][1]), 0x7632);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) out[t] = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

// 29-bit fixed-point values (|x| < 2^29) -> three balanced digits each,
// x = d0 2^22 + d1 2^11 + d2 with d1, d2 in [-1024, 1023] and d0 in
// [-128, 128]; slice t is d0 2^8, d1 2^-3, d2 2^-14: all exact and in the
// normal FP16 range (|slice| in [2^-14, 2^15]), and x = 2^14 (sum of slices).
// Digits without a carry chain: y = x + 0x200400 holds d1 + 1024 and
// d2 + 1024 in its 11-bit fields and y >> 22 = d0 (no overflow below 2^29);
// each digit becomes a float exactly through the 2^23 exponent trick, and
// pairs are rounded to f16x2, exact for these values.
__device__ __forceinline__ void fx_pack3(const int32_t (&v)[8], uint4 (&out)[3], int mul = 1) {
    uint32_t w[3][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        float f[3][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int y = v[e + h] * mul + 0x200400;
            f[0][h] = fmaf(__int_as_float(0x4B400000 + (y >> 22)), 256.0f, -3221225472.0f);
            f[1][h] = fmaf(__uint_as_float(0x4B000000u | (((uint32_t)y >> 11) & 0x7FFu)), 0.125f, -1048704.0f);
            f[2][h] = fmaf(__uint_as_float(0x4B000000u | ((uint32_t)y & 0x7FFu)), 6.103515625e-05f,
                           -512.0625f);
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const __half2 hh = __floats2half2_rn(f[t][0], f[t][1]);
            w[t][e / 2] = *reinterpret_cast<const uint32_t *>(&hh);
        }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) out[t] = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

// Digits of the fixed-point form F.
template <int F>
__device__ __forceinline__ void fx_pack_f(const int32_t (&v)[8], uint4 (&out)[FT<F>::PIECES], int mul = 1) {
    if constexpr (F == kFX32H) fx_pack3(v, out, mul);
    else fx_pack(v, out, mul);
}

template <int F, typename Tin>
__device__ __forceinline__ void load_split(const Tin *__restrict__ src, int64_t ro, const IdxMap &km,
                                           int64_t k0, int64_t K, uint4 (&out)[FT<F>::PIECES]) {
    Tin v[16 / FT<F>::ELEM];
    load_chunk<F, Tin>(src, ro, km, k0, K, false, v);
    split_pack<F, Tin>(v, out);
}

// Byte offset of 16-byte chunk `ch` of row `row` in a K-major tile with the
// 64-byte swizzle: rows 64 bytes apart, chunk index XOR-ed with bits 1..2 of
// the row (address bits 4..5 ^= bits 7..8), tile base 1024-byte aligned.
__device__ __forceinline__ uint32_t swz(int row, int ch) {
    return (uint32_t)row * kRowBytes + ((uint32_t)(ch ^ ((row >> 1) & 3)) << 4);
}

// Stores 16 consecutive output columns of one row: C[ro + colC(c0 + e)],
// e < cmax.  The accumulate flag is tested once (no speculative loads of C
// when it is off); unit-stride aligned rows use 16-byte stores.
template <typename To>
__device__ __forceinline__ void store_row16(void *C, int64_t ro, const IdxMap &colC, int64_t c0, int cmax,
                                            const float (&v)[16], bool acc) {
    To *base = static_cast<To *>(C) + ro;
    if (colC.R0 != 0) {
#pragma unroll
        for (int e = 0; e < 16; ++e)
            if (e < cmax) {
                To *d = base + imap(colC, c0 + e);
                *d = acc ? (To)(*d + (To)v[e]) : (To)v[e];
            }
        return;
    }
    const int64_t cs = colC.s0;
    To *cp = base + c0 * cs;
    if (acc) {
#pragma unroll
        for (int e = 0; e < 16; ++e)
            if (e < cmax) cp[e * cs] += (To)v[e];
        return;
    }
    if (cs == 1 && cmax == 16 && (reinterpret_cast<uintptr_t>(cp) & 15) == 0) {
        if constexpr (sizeof(To) == 4) {
#pragma unroll
            for (int e = 0; e < 16; e += 4)
                *reinterpret_cast<float4 *>(cp + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        } else {
#pragma unroll
            for (int e = 0; e < 16; e += 2)
                *reinterpret_cast<double2 *>(cp + e) = make_double2((double)v[e], (double)v[e + 1]);
        }
        return;
    }
#pragma unroll
    for (int e = 0; e < 16; ++e)
        if (e < cmax) cp[e * cs] = (To)v[e];
}

}  // namespace kron
