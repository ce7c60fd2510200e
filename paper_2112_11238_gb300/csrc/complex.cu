// complex.cu -- the real form of a complex mu-mode product's matrix.
//
// A complex tensor is held as interleaved (real, imaginary) pairs.  Over that
// real view a complex mu-mode product S^(mu) = G X^(mu) (Eq. (mmp) over C) is
// one real contraction of twice the length: the contracted index runs over
// (c, k) with c the real / imaginary part of X, the output index over
// (c', j), and the real 2n x 2m matrix is, per (j, k),
//     [ Re G[j,k]  -Im G[j,k] ]     rows (c' = 0, 1), columns (c = 0, 1),
//     [ Im G[j,k]   Re G[j,k] ]
// so that Re S = Re G Re X - Im G Im X and Im S = Im G Re X + Re G Im X.
// Interleaved as the tensor: row c' + 2j, column c + 2k.
#include <algorithm>

#include "internal.h"

namespace kron {

namespace {

// G = op(L): L[j + ldL k] (trans = 0) or L[k + ldL j] (trans = 1), complex
// elements; conj negates the imaginary part (trans = 1, conj = 1: L^*).
template <typename T>
__global__ void cexpand_kernel(const T *__restrict__ L, int64_t ldL, int64_t n, int64_t m, int trans, int conj,
                               T *__restrict__ M) {
    const int64_t rows = 2 * n, total = 4 * n * m;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t jh = idx % rows, kh = idx / rows;
        const int64_t j = jh >> 1, k = kh >> 1;
        const int cp = (int)(jh & 1), c = (int)(kh & 1);
        const int64_t e = trans ? k + ldL * j : j + ldL * k;
        const T gr = L[2 * e];
        const T gi = conj ? -L[2 * e + 1] : L[2 * e + 1];
        M[idx] = (cp == c) ? gr : (cp == 1 ? gi : -gi);
    }
}

}  // namespace

cudaError_t complex_expand(const void *L, bool f64, int64_t ldL, int64_t n, int64_t m, bool trans, bool conj,
                           void *M, cudaStream_t st) {
    const int64_t total = 4 * n * m;
    if (total == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
    if (f64)
        cexpand_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double *>(L), ldL, n, m, trans, conj,
                                                       static_cast<double *>(M));
    else
        cexpand_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(L), ldL, n, m, trans, conj,
                                                      static_cast<float *>(M));
    return cudaGetLastError();
}

}  // namespace kron
