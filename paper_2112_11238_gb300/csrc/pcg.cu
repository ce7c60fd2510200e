// pcg.cu -- preconditioned conjugate gradients for a linear system whose
// matrix is a Kronecker sum, M = M_d (+) ... (+) M_1, with an ADI-type
// Kronecker-product preconditioner P = P_d (x) ... (x) P_1 (Section 3.4,
// Eqs. (prec), (preconnd); the semilinear example of Section 4.5):
//   M v  = vec(sum_mu V x_mu M_mu)             (Eq. (actkron), kron_kronsumv)
//   P^{-1} v = vec(V x_1 P_1^{-1} ... x_d P_d^{-1})   (kron_itucker)
// The vector operations and the dot products (FP64, fixed summation order:
// per-block partial sums, then one block sums them in order) are kernels of
// this file; the host loop reads two scalars per iteration.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace kron {

namespace {

constexpr int kDotBlocks = 304;  // 2 x the SM count of the target
constexpr int kDotThreads = 256;

template <typename T>
__device__ __forceinline__ double ld(const void *p, int64_t i) {
    return (double)static_cast<const T *>(p)[i];
}

// partial[b] = sum over block b's elements of x[i] * y[i]
template <typename T>
__global__ void dot_partial_kernel(const void *x, const void *y, int64_t n, double *partial) {
    __shared__ double sm[kDotThreads];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(ld<T>(x, i), ld<T>(y, i), s);
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void dot_final_kernel(const double *partial, int nb, double *out) {
    __shared__ double sm[kDotThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

// y = a * x + b * y (a, b from device scalars: a = sa[0] / sa[1] when sa,
// sign applied), all of type T.
template <typename T>
__global__ void axpby_kernel(int64_t n, double a, const double *num, const double *den, const void *x, double b,
                             const double *bnum, const double *bden, void *y) {
    double aa = a, bb = b;
    if (num) aa *= *num / *den;
    if (bnum) bb *= *bnum / *bden;
    T *yy = static_cast<T *>(y);
    const T *xx = static_cast<const T *>(x);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        yy[i] = (T)(aa * (double)xx[i] + (bb == 0.0 ? 0.0 : bb * (double)yy[i]));
}

unsigned grid_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
}

}  // namespace

cudaError_t pcg_dot(const void *x, const void *y, bool f64, int64_t n, double *partial, double *out,
                    cudaStream_t st) {
    if (f64) dot_partial_kernel<double><<<kDotBlocks, kDotThreads, 0, st>>>(x, y, n, partial);
    else dot_partial_kernel<float><<<kDotBlocks, kDotThreads, 0, st>>>(x, y, n, partial);
    dot_final_kernel<<<1, kDotThreads, 0, st>>>(partial, kDotBlocks, out);
    return cudaGetLastError();
}

// y = a (num/den) x + b (bnum/bden) y; null num/bnum: plain a / b.
cudaError_t pcg_axpby(bool f64, int64_t n, double a, const double *num, const double *den, const void *x, double b,
                      const double *bnum, const double *bden, void *y, cudaStream_t st) {
    if (f64) axpby_kernel<double><<<grid_for(n), 256, 0, st>>>(n, a, num, den, x, b, bnum, bden, y);
    else axpby_kernel<float><<<grid_for(n), 256, 0, st>>>(n, a, num, den, x, b, bnum, bden, y);
    return cudaGetLastError();
}

size_t pcg_partial_doubles() { return kDotBlocks; }

}  // namespace kron
