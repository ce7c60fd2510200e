// spectral.cu -- transform matrices of a Hermite--Laguerre--Fourier (HLF)
// pseudospectral decomposition (the paper's HLF experiment): the
// Gauss--Hermite and generalized Gauss--Laguerre rules (host, FP64), the
// normalized and scaled Hermite and generalized Laguerre functions at given
// points, and the real trigonometric resampling matrix (device, FP64).  The
// decomposition itself is then two Tucker operators (Eq. (tensinterp)).
//
// Quadrature (Golub--Welsch): the nodes of the m-point Gauss rule of a
// weight are the eigenvalues of its Jacobi matrix, the symmetric tridiagonal
// matrix of the three-term recurrence of the orthonormal polynomials; they
// come from the implicit QL iteration with Wilkinson's shift.  With the
// orthonormal *functions* phi_i = p_i sqrt(weight), the weight of node x_k
// for integrating a product of two such functions is 1 / sum_i phi_i(x_k)^2
// (the reciprocal Christoffel function), which neither overflows nor
// underflows.
//
// Functions: the orthonormal recurrences, carried as a mantissa q_i times
// 2^ex with the common factor exp(-y^2/2) (Hermite) or y^(alpha/2) exp(-y/2)
// (Laguerre) applied through logarithms at the end, so that neither the
// factor (which underflows far out) nor the mantissa (which then grows)
// leaves the double range.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace kron {

namespace {

constexpr double kLn2 = 0.69314718055994530942;
constexpr double kPi = 3.14159265358979323846;

// value = q * 2^ex * exp(lbase)
__host__ __device__ inline double scaled_value(double q, int ex, double lbase) {
    if (q == 0.0) return 0.0;
    return copysign(exp(log(fabs(q)) + ex * kLn2 + lbase), q);
}

__host__ __device__ inline void rescale(double &q0, double &q1, int &ex) {
    if (fabs(q1) > 0x1p500) {
        q0 *= 0x1p-500;
        q1 *= 0x1p-500;
        ex += 500;
    }
}

// Normalized scaled Hermite functions H_i(x) = sqrt(beta) h_i(beta x),
// h_i the orthonormal Hermite functions of L^2(R) (physicists' polynomials
// times exp(-y^2/2), normalized): h_0 = pi^(-1/4) exp(-y^2/2),
// h_1 = sqrt(2) y h_0, h_i = sqrt(2/i) y h_{i-1} - sqrt((i-1)/i) h_{i-2}.
template <typename Emit>
__host__ __device__ inline void hermite_seq(int64_t m, double beta, double x, Emit &&emit) {
    const double y = beta * x;
    const double lbase = -0.5 * y * y + 0.5 * log(beta) - 0.25 * log(kPi);
    double q0 = 1.0, q1 = sqrt(2.0) * y;
    int ex = 0;
    emit((int64_t)0, scaled_value(q0, ex, lbase));
    if (m > 1) emit((int64_t)1, scaled_value(q1, ex, lbase));
    for (int64_t i = 2; i < m; ++i) {
        const double q2 = sqrt(2.0 / (double)i) * y * q1 - sqrt((double)(i - 1) / (double)i) * q0;
        q0 = q1;
        q1 = q2;
        rescale(q0, q1, ex);
        emit(i, scaled_value(q1, ex, lbase));
    }
}

// Normalized scaled generalized Laguerre functions
// L_i(x) = sqrt(beta) l_i(beta x), l_i the orthonormal functions of
// L^2(R+): l_i(y) = sqrt(i! / Gamma(i + alpha + 1)) L_i^alpha(y) y^(alpha/2)
// exp(-y/2) (i = 0, 1, ...); recurrence
// sqrt(i (i + alpha)) l_i = (2i - 1 + alpha - y) l_{i-1}
//                           - sqrt((i - 1)(i - 1 + alpha)) l_{i-2}.
template <typename Emit>
__host__ __device__ inline void laguerre_seq(int64_t m, double alpha, double beta, double x, Emit &&emit) {
    const double y = beta * x;
    double lbase = -0.5 * y + 0.5 * log(beta) - 0.5 * lgamma(alpha + 1.0);
    if (alpha != 0.0) lbase += 0.5 * alpha * log(y);  // y = 0, alpha > 0: the functions vanish
    double q0 = 1.0, q1 = (alpha + 1.0 - y) / sqrt(alpha + 1.0);
    int ex = 0;
    emit((int64_t)0, scaled_value(q0, ex, lbase));
    if (m > 1) emit((int64_t)1, scaled_value(q1, ex, lbase));
    for (int64_t i = 2; i < m; ++i) {
        const double di = (double)i;
        const double q2 = ((2.0 * di - 1.0 + alpha - y) * q1 - sqrt((di - 1.0) * (di - 1.0 + alpha)) * q0) /
                          sqrt(di * (di + alpha));
        q0 = q1;
        q1 = q2;
        rescale(q0, q1, ex);
        emit(i, scaled_value(q1, ex, lbase));
    }
}

// Eigenvalues of the symmetric tridiagonal matrix with diagonal d[0..n-1]
// and off-diagonal e[0..n-2] (e[i] couples i and i+1), by the implicit QL
// iteration with Wilkinson's shift (one Givens sweep per iteration from the
// bottom of the unreduced block up to its top).  d is overwritten with the
// eigenvalues in ascending order.  False if an eigenvalue needs more than 60
// iterations.
bool tridiag_eigenvalues(std::vector<double> &d, std::vector<double> e) {
    const int64_t n = (int64_t)d.size();
    e.resize((size_t)n, 0.0);
    if (n > 0) e[(size_t)n - 1] = 0.0;
    for (int64_t l = 0; l < n; ++l) {
        int it = 0;
        while (true) {
            // end of the unreduced block that starts at l
            int64_t mm = l;
            for (; mm < n - 1; ++mm) {
                const double dd = fabs(d[mm]) + fabs(d[mm + 1]);
                if (fabs(e[mm]) <= 0x1p-53 * dd) break;
            }
            if (mm == l) break;
            if (++it > 60) return false;
            // Wilkinson shift from the leading 2x2 block
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            bool deflated = false;
            for (int64_t i = mm - 1; i >= l; --i) {
                const double f = s * e[i], b = c * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {  // the sweep splits the block: restart on the smaller one
                    d[i + 1] -= p;
                    e[mm] = 0.0;
                    deflated = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
            }
            if (deflated) continue;
            d[l] -= p;
            e[l] = g;
            e[mm] = 0.0;
        }
    }
    std::sort(d.begin(), d.end());
    return true;
}

// Receivers of the function values phi_i(x): a sum of squares (weights) or
// a matrix entry.
struct SumSq {
    double *ss;
    __host__ __device__ void operator()(int64_t, double v) const { *ss += v * v; }
};
struct Store {
    double *F;
    int64_t ldF, l;
    int trans;
    __host__ __device__ void operator()(int64_t i, double v) const { F[trans ? i + ldF * l : l + ldF * i] = v; }
};

__global__ void hermite_kernel(int64_t m, double beta, const double *__restrict__ x, int64_t n, double *F,
                               int64_t ldF, int trans) {
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        hermite_seq(m, beta, x[l], Store{F, ldF, l, trans});
}

__global__ void laguerre_kernel(int64_t m, double alpha, double beta, const double *__restrict__ x, int64_t n,
                                double *F, int64_t ldF, int trans) {
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        laguerre_seq(m, alpha, beta, x[l], Store{F, ldF, l, trans});
}

// F[l, j] = D(l/n - j/m): the trigonometric interpolant of period 1 through
// m equispaced samples at j/m, evaluated at l/n, with
// D(s) = (1/m) (1 + 2 sum_{k=1}^{(m-1)/2} cos(2 pi k s) + [m even] cos(pi m s)),
// the even-m Nyquist term split symmetrically (real interpolant).
__global__ void fourier_kernel(int64_t m, int64_t n, double *F, int64_t ldF) {
    const int64_t total = m * n;
    const int64_t K = (m - 1) / 2;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = t % n, j = t / n;
        // s = l/n - j/m as (l m - j n) / (n m); cos(2 pi k s) = cospi(2 k s)
        const double s = (double)(l * m - j * n) / (double)(n * m);
        double acc = 1.0;
        for (int64_t k = 1; k <= K; ++k) acc += 2.0 * cospi(2.0 * (double)k * s);
        if (m % 2 == 0) acc += cospi((double)m * s);
        F[l + ldF * j] = acc / (double)m;
    }
}

unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 127) / 128, 152 * 8)); }

}  // namespace

}  // namespace kron

using namespace kron;

extern "C" {

kron_status kron_gauss_hermite(int64_t m, double beta, double *x, double *w) {
    if (m < 1 || !(beta > 0.0) || !x || !w) return KRON_ERR_INVALID_ARG;
    // Jacobi matrix of the orthonormal Hermite polynomials (weight exp(-y^2)):
    // zero diagonal, off-diagonal sqrt(i / 2)
    std::vector<double> d((size_t)m, 0.0), e((size_t)m, 0.0);
    for (int64_t i = 1; i < m; ++i) e[(size_t)i - 1] = sqrt(0.5 * (double)i);
    if (!tridiag_eigenvalues(d, e)) return KRON_ERR_NUMERIC;
    for (int64_t k = 0; k < m; ++k) {
        const double xk = d[(size_t)k] / beta;
        double ss = 0.0;
        hermite_seq(m, beta, xk, SumSq{&ss});
        x[k] = xk;
        w[k] = 1.0 / ss;
    }
    return KRON_OK;
}

kron_status kron_gauss_laguerre(int64_t m, double alpha, double beta, double *x, double *w) {
    if (m < 1 || !(alpha > -1.0) || !(beta > 0.0) || !x || !w) return KRON_ERR_INVALID_ARG;
    // Jacobi matrix of the orthonormal generalized Laguerre polynomials
    // (weight y^alpha exp(-y)): diagonal 2i + alpha + 1, off-diagonal
    // sqrt(i (i + alpha))
    std::vector<double> d((size_t)m), e((size_t)m, 0.0);
    for (int64_t i = 0; i < m; ++i) d[(size_t)i] = 2.0 * (double)i + alpha + 1.0;
    for (int64_t i = 1; i < m; ++i) e[(size_t)i - 1] = sqrt((double)i * ((double)i + alpha));
    if (!tridiag_eigenvalues(d, e)) return KRON_ERR_NUMERIC;
    for (int64_t k = 0; k < m; ++k) {
        const double xk = d[(size_t)k] / beta;
        double ss = 0.0;
        laguerre_seq(m, alpha, beta, xk, SumSq{&ss});
        x[k] = xk;
        w[k] = 1.0 / ss;
    }
    return KRON_OK;
}

kron_status kron_hermite_functions(int64_t m, double beta, const double *x, int64_t n, double *F, int64_t ldF,
                                   int trans, kron_stream_t stream) {
    if (m < 1 || n < 0 || !(beta > 0.0) || (n > 0 && (!x || !F)) || (trans != 0 && trans != 1))
        return KRON_ERR_INVALID_ARG;
    if (trans ? ldF < m : ldF < std::max<int64_t>(n, 1)) return KRON_ERR_INVALID_ARG;
    if (n == 0) return KRON_OK;
    hermite_kernel<<<blocks_for(n), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(m, beta, x, n, F, ldF, trans);
    return cudaGetLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

kron_status kron_laguerre_functions(int64_t m, double alpha, double beta, const double *x, int64_t n, double *F,
                                    int64_t ldF, int trans, kron_stream_t stream) {
    if (m < 1 || n < 0 || !(alpha > -1.0) || !(beta > 0.0) || (n > 0 && (!x || !F)) || (trans != 0 && trans != 1))
        return KRON_ERR_INVALID_ARG;
    if (trans ? ldF < m : ldF < std::max<int64_t>(n, 1)) return KRON_ERR_INVALID_ARG;
    if (n == 0) return KRON_OK;
    laguerre_kernel<<<blocks_for(n), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(m, alpha, beta, x, n, F, ldF,
                                                                                        trans);
    return cudaGetLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

kron_status kron_fourier_resample(int64_t m, int64_t n, double *F, int64_t ldF, kron_stream_t stream) {
    if (m < 1 || n < 1 || !F || ldF < n) return KRON_ERR_INVALID_ARG;
    fourier_kernel<<<blocks_for(m * n), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(m, n, F, ldF);
    return cudaGetLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

}  // extern "C"
