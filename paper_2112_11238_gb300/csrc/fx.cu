// fx.cu -- helpers of the fixed-point forms (KRON_PREC_FX32, _FX32H): the
// sliced image of op(L) with one power-of-two scale per row, and the
// conversion of a floating-point tensor into fixed point with one scale.
//
// Fixed point with b magnitude bits (b = 31 for FX32, 29 for FX32H): a tensor
// X with scale e holds the values X * 2^(e - b), |X| <= 2^b - 1, so
// |value| < 2^e.  A row c of op(L) is held as Y = round(L[c, :] * 2^(b - f_c))
// with 2^(f_c - 1) <= max_k |L[c, k]| < 2^f_c.  Both are cut into digit slices
// (fx_pack / fx_pack3, tc_common.cuh).
#include <algorithm>
#include <climits>

#include "tc_common.cuh"

namespace kron {

namespace {

// Exponent f with |x| < 2^f for the largest |x| of a set (0 for an all-zero set).
__device__ __forceinline__ int exp_bound(double mx) {
    int f = 0;
    if (mx > 0.0) frexp(mx, &f);
    return f;
}

__device__ __forceinline__ int32_t to_fixed(double v, int f, int bits) {
    const double lim = ldexp(1.0, bits) - 1.0;
    double y = rint(ldexp(v, bits - f));
    y = fmax(-lim, fmin(lim, y));
    return (int32_t)y;
}

// One warp per row of op(L): row exponent and |row| sum (bound on the output
// growth).  The largest row sum goes to *g through an atomic maximum on the
// bits of a non-negative double.
template <typename T>
__global__ void fx_rows_kernel(const T *__restrict__ B, IdxMap colB, IdxMap kB, int64_t N, int64_t K, int *f,
                               unsigned long long *g) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (row >= N) return;
    const int64_t ro = imap(colB, row);
    double mx = 0.0, sum = 0.0;
    for (int64_t k = lane; k < K; k += 32) {
        const double v = fabs((double)B[ro + imap(kB, k)]);
        mx = fmax(mx, v);
        sum += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if (lane == 0) {
        f[row] = exp_bound(mx);
        atomicMax(g, (unsigned long long)__double_as_longlong(sum));
    }
}

// Image items (nt, kb, row, chunk): eight consecutive k of one row of op(L),
// fixed point with the row's exponent, cut into the slices of form F.
template <typename T, int F>
__global__ void fx_image_kernel(const T *__restrict__ B, IdxMap colB, IdxMap kB, int64_t N, int64_t K, int BN,
                                int64_t KB, int64_t NT, const int *__restrict__ f, uint8_t *img) {
    constexpr int bits = (F == kFX32H) ? 29 : 31;
    constexpr int BK = kRowBytes / 2;
    const int64_t total = NT * KB * BN * kChunks;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(idx % kChunks);
        int64_t rest = idx / kChunks;
        const int row = (int)(rest % BN);
        rest /= BN;
        const int64_t kb = rest % KB;
        const int64_t nt = rest / KB;
        const int64_t c = nt * BN + row;
        int32_t x[8];
        const int fc = c < N ? f[c] : 0;
        const int64_t ro = c < N ? imap(colB, c) : 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int64_t k = kb * BK + ch * 8 + e;
            x[e] = (c < N && k < K) ? to_fixed((double)B[ro + imap(kB, k)], fc, bits) : 0;
        }
        constexpr int NP = FT<F>::PIECES;
        uint4 out[NP];
        fx_pack_f<F>(x, out);
        uint8_t *base = img + (size_t)((nt * KB + kb) * NP) * BN * kRowBytes;
        const uint32_t off = swz(row, ch);
#pragma unroll
        for (int q = 0; q < NP; ++q) *reinterpret_cast<uint4 *>(base + (size_t)q * BN * kRowBytes + off) = out[q];
    }
}

// Smallest e with |v| < 2^e for a normal nonzero v (INT_MIN for zero and
// subnormal values, which the fixed point rounds to zero anyway); integer
// operations only.
__device__ __forceinline__ int ebound(double v) {
    const int E = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
    return E ? E - 1022 : INT_MIN;
}
__device__ __forceinline__ int ebound(float v) {
    const int E = (int)((__float_as_uint(v) >> 23) & 0xFF);
    return E ? E - 126 : INT_MIN;
}

// round(v * 2^(bits - e)) from the bits of v, for |v| < 2^e (integer only),
// clamped to 2^bits - 1.
__device__ __forceinline__ int32_t fixed_bits(double v, int e, int bits) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) return 0;
    const unsigned long long mant = (1ull << 52) | (b & ((1ull << 52) - 1));
    const int r = e + 1075 - bits - E;  // right shift, >= 53 - bits when |v| < 2^e
    unsigned long long x = 0;
    if (r < 64) x = r > 0 ? (mant + (1ull << (r - 1))) >> r : mant << (-r);
    const unsigned long long lim = (1ull << bits) - 1;
    if (x > lim) x = lim;
    return (b >> 63) ? -(int32_t)x : (int32_t)x;
}
__device__ __forceinline__ int32_t fixed_bits(float v, int e, int bits) {
    const uint32_t b = __float_as_uint(v);
    const int E = (int)((b >> 23) & 0xFF);
    if (E == 0) return 0;
    const unsigned long long mant = (1u << 23) | (b & ((1u << 23) - 1));
    const int r = e + 150 - bits - E;
    unsigned long long x = 0;
    if (r < 64) x = r > 0 ? (mant + (1ull << (r - 1))) >> r : mant << (-r);
    const unsigned long long lim = (1ull << bits) - 1;
    if (x > lim) x = lim;
    return (b >> 31) ? -(int32_t)x : (int32_t)x;
}

template <typename T>
__global__ void fx_maxabs_kernel(const T *__restrict__ src, int64_t n, int *emax) {
    int m = INT_MIN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, ebound(src[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m != INT_MIN) atomicMax(emax, m);
}

template <typename T>
__global__ void fx_convert_kernel(const T *__restrict__ src, int64_t n, const int *emax, int32_t *X, FxScale *s,
                                  int bits) {
    const int e = (*emax < -100000) ? 0 : *emax;  // all-zero tensor: any scale
    unsigned m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = fixed_bits(src[i], e, bits);
        X[i] = x;
        m = max(m, (unsigned)(x < 0 ? -x : x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&s->maxabs, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) s->e = e;
}

}  // namespace

cudaError_t fx_reset(FxScale *s, cudaStream_t st) {
    return cudaMemsetAsync(&s->maxabs, 0, sizeof(unsigned), st);
}

cudaError_t fx_build_bimage(int form, const Contraction &c, void *img, int *f, unsigned long long *g,
                            cudaStream_t st) {
    return fx_build_bimage_bn(form, c, img, f, g, tc_tile_n(form, c.N), st);
}

cudaError_t fx_build_bimage_bn(int form, const Contraction &c, void *img, int *f, unsigned long long *g, int bn,
                               cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(g, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const unsigned rows_blocks = (unsigned)((c.N + 7) / 8);
    if (c.B_f64)
        fx_rows_kernel<double><<<rows_blocks, 256, 0, st>>>(static_cast<const double *>(c.B), c.colB, c.kB, c.N, c.K, f, g);
    else
        fx_rows_kernel<float><<<rows_blocks, 256, 0, st>>>(static_cast<const float *>(c.B), c.colB, c.kB, c.N, c.K, f, g);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nt = (c.N + bn - 1) / bn;
    const int64_t kb = (c.K + kRowBytes / 2 - 1) / (kRowBytes / 2);
    const int64_t total = nt * kb * bn * kChunks;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
    auto *out = static_cast<uint8_t *>(img);
    const bool h = form == kFX32H;
    if (c.B_f64 && h)
        fx_image_kernel<double, kFX32H><<<blocks, 256, 0, st>>>(static_cast<const double *>(c.B), c.colB, c.kB, c.N,
                                                                c.K, bn, kb, nt, f, out);
    else if (c.B_f64)
        fx_image_kernel<double, kFX32><<<blocks, 256, 0, st>>>(static_cast<const double *>(c.B), c.colB, c.kB, c.N,
                                                               c.K, bn, kb, nt, f, out);
    else if (h)
        fx_image_kernel<float, kFX32H><<<blocks, 256, 0, st>>>(static_cast<const float *>(c.B), c.colB, c.kB, c.N,
                                                               c.K, bn, kb, nt, f, out);
    else
        fx_image_kernel<float, kFX32><<<blocks, 256, 0, st>>>(static_cast<const float *>(c.B), c.colB, c.kB, c.N,
                                                              c.K, bn, kb, nt, f, out);
    return cudaGetLastError();
}

cudaError_t fx_from_float(int form, const void *src, bool src64, int64_t count, int32_t *X, FxScale *s,
                          unsigned long long *scratch, cudaStream_t st) {
    const int bits = fx_bits(form);
    int *emax = reinterpret_cast<int *>(scratch);
    cudaError_t e = cudaMemsetAsync(emax, 0x80, sizeof(int), st);  // 0x80808080: below every bound
    if (e == cudaSuccess) e = fx_reset(s, st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152 * 8));
    if (src64) {
        fx_maxabs_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double *>(src), count, emax);
        fx_convert_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double *>(src), count, emax, X, s, bits);
    } else {
        fx_maxabs_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(src), count, emax);
        fx_convert_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(src), count, emax, X, s, bits);
    }
    return cudaGetLastError();
}

}  // namespace kron
