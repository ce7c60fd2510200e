// expm.cu -- E = exp(tau A) in FP64 on the GPU (Section 3.3: the small
// matrix exponentials exp(tau A_mu) of Eq. (exptucker)).
//
// Method: scaling and squaring with the [13/13] Pade approximant (Higham,
// "The scaling and squaring method for the matrix exponential revisited",
// SIAM J. Matrix Anal. Appl. 26 (2005)):
//   s = max(0, ceil(log2(||tau A||_1 / theta_13))),  B = tau A / 2^s,
//   U = B [B6 (b13 B6 + b11 B4 + b9 B2) + b7 B6 + b5 B4 + b3 B2 + b1 I],
//   V =    B6 (b12 B6 + b10 B4 + b8 B2) + b6 B6 + b4 B4 + b2 B2 + b0 I,
//   (V - U) X = (V + U),  E = X^(2^s).
// The linear system is solved by Gauss-Jordan elimination with partial
// pivoting on [V-U | V+U | I] (giving X and (V-U)^{-1}), then one step of
// iterative refinement with the FP64 residual R = (V+U) - (V-U) X:
// X <- X + (V-U)^{-1} R.
//
// Everything runs in ONE cooperative launch (one block per SM) whose phases
// are separated by a grid barrier with a bounded wait; FP64 GEMMs are split
// into 16 x 16 tiles spread over the blocks.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "internal.h"
#include "ptx.cuh"

namespace kron {

namespace {

constexpr int kT = 16;          // GEMM tile
constexpr int kThreadsE = 256;  // = kT * kT

struct ExpmDev {
    int n;
    const double *A;
    int64_t ldA;
    double tau;
    double *E;
    double *w;           // workspace base (doubles)
    unsigned *bar;       // [0] count, [1] generation
    unsigned long long *norm_bits;
    double b[14];
    double theta;
};

__device__ bool grid_sync(unsigned *bar) {
    __syncthreads();
    __shared__ int failed;
    if (threadIdx.x == 0) {
        failed = 0;
        volatile unsigned *vgen = bar + 1;
        const unsigned my_gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            while (*vgen == my_gen) {
                if (device_error_set() || globaltimer_ns() - t0 > kWaitLimitNs) {
                    latch_error(kErrTimeout);
                    failed = 1;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return failed == 0;
}

// C = alpha * A * B + beta * C0 (+ gamma * I), all n x n with ld n.  C0 may
// alias C; A and B must not.  Tiles are spread over the grid.
__device__ void gemm(int n, double alpha, const double *A, const double *B, double beta,
                     const double *C0, double gamma, double *C) {
    __shared__ double As[kT][kT + 1], Bs[kT][kT + 1];
    const int tiles = (n + kT - 1) / kT;
    const int tr = threadIdx.x % kT, tc = threadIdx.x / kT;
    for (int t = blockIdx.x; t < tiles * tiles; t += gridDim.x) {
        const int i0 = (t % tiles) * kT, j0 = (t / tiles) * kT;
        double acc = 0.0;
        for (int k0 = 0; k0 < n; k0 += kT) {
            const int ia = i0 + tr, ka = k0 + tc;
            As[tc][tr] = (ia < n && ka < n) ? A[ia + (int64_t)n * ka] : 0.0;
            const int kb = k0 + tr, jb = j0 + tc;
            Bs[tc][tr] = (kb < n && jb < n) ? B[kb + (int64_t)n * jb] : 0.0;
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kT; ++k) acc = fma(As[k][tr], Bs[tc][k], acc);
            __syncthreads();
        }
        const int i = i0 + tr, j = j0 + tc;
        if (i < n && j < n) {
            const int64_t o = i + (int64_t)n * j;
            double v = alpha * acc;
            if (beta != 0.0) v += beta * C0[o];
            if (i == j) v += gamma;
            C[o] = v;
        }
    }
}

// Y = sum_k c_k X_k (+ g I), elementwise over the grid.
__device__ void lincomb(int n, double *Y, double c1, const double *X1, double c2, const double *X2,
                        double c3, const double *X3, double g) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (X1) v += c1 * X1[e];
        if (X2) v += c2 * X2[e];
        if (X3) v += c3 * X3[e];
        if (e % n == e / n) v += g;
        Y[e] = v;
    }
}

__global__ void __launch_bounds__(kThreadsE) expm_kernel(const ExpmDev p) {
    const int n = p.n;
    const int64_t nn = (int64_t)n * n;
    double *B = p.w, *B2 = B + nn, *B4 = B2 + nn, *B6 = B4 + nn, *T1 = B6 + nn, *T2 = T1 + nn;
    double *U = T2 + nn, *V = U + nn, *Q0 = V + nn, *P0 = Q0 + nn, *X = P0 + nn, *R = X + nn;
    double *G = R + nn;  // augmented [Q | P | I]: n x 3n, ld n
    __shared__ double colk[1024];
    __shared__ double red_v[kThreadsE];
    __shared__ int red_i[kThreadsE];

    // ---- ||tau A||_1
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        double s = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s += fabs(p.tau * p.A[i + p.ldA * j]);
        red_v[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red_v[threadIdx.x] += red_v[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicMax(p.norm_bits, (unsigned long long)__double_as_longlong(red_v[0]));
        __syncthreads();
    }
    if (!grid_sync(p.bar)) return;
    const double nrm = __longlong_as_double((long long)*(volatile unsigned long long *)p.norm_bits);
    if (!isfinite(nrm)) {  // non-finite input
        if (blockIdx.x == 0 && threadIdx.x == 0) latch_error(kErrNumeric);
        return;
    }
    int s = 0;
    if (nrm > p.theta) s = (int)ceil(log2(nrm / p.theta));
    const double scale = ldexp(p.tau, -s);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x)
        B[e] = scale * p.A[(e % n) + p.ldA * (e / n)];
    if (!grid_sync(p.bar)) return;
    gemm(n, 1.0, B, B, 0.0, nullptr, 0.0, B2);
    if (!grid_sync(p.bar)) return;
    gemm(n, 1.0, B2, B2, 0.0, nullptr, 0.0, B4);
    if (!grid_sync(p.bar)) return;
    gemm(n, 1.0, B4, B2, 0.0, nullptr, 0.0, B6);
    if (!grid_sync(p.bar)) return;
    const double *b = p.b;
    // T1 = b13 B6 + b11 B4 + b9 B2 ; T2 = b12 B6 + b10 B4 + b8 B2
    lincomb(n, T1, b[13], B6, b[11], B4, b[9], B2, 0.0);
    lincomb(n, T2, b[12], B6, b[10], B4, b[8], B2, 0.0);
    if (!grid_sync(p.bar)) return;
    // U' = B6 T1 + b7 B6 + b5 B4 + b3 B2 + b1 I  (into R as scratch first)
    lincomb(n, R, b[7], B6, b[5], B4, b[3], B2, b[1]);
    lincomb(n, X, b[6], B6, b[4], B4, b[2], B2, b[0]);
    if (!grid_sync(p.bar)) return;
    gemm(n, 1.0, B6, T1, 1.0, R, 0.0, R);
    gemm(n, 1.0, B6, T2, 1.0, X, 0.0, V);
    if (!grid_sync(p.bar)) return;
    gemm(n, 1.0, B, R, 0.0, nullptr, 0.0, U);
    if (!grid_sync(p.bar)) return;
    // Q0 = V - U, P0 = V + U, augmented G = [Q0 | P0 | I]
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double q = V[e] - U[e], pp = V[e] + U[e];
        Q0[e] = q;
        P0[e] = pp;
        G[e] = q;
        G[nn + e] = pp;
        G[2 * nn + e] = (e % n == e / n) ? 1.0 : 0.0;
    }
    if (!grid_sync(p.bar)) return;
    // ---- Gauss-Jordan with partial pivoting.  Column j of G is owned by
    // block (j % gridDim.x); at step k every block reads column k (final
    // after the previous barrier), finds the pivot, and updates only its own
    // columns j > k.
    for (int k = 0; k < n; ++k) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = G[i + (int64_t)n * k];
        __syncthreads();
        double best = -1.0;
        int bi = k;
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            const double a = fabs(colk[i]);
            if (a > best) { best = a; bi = i; }
        }
        red_v[threadIdx.x] = best;
        red_i[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                const double ov = red_v[threadIdx.x + o];
                const int oi = red_i[threadIdx.x + o];
                if (ov > red_v[threadIdx.x] || (ov == red_v[threadIdx.x] && oi < red_i[threadIdx.x])) {
                    red_v[threadIdx.x] = ov;
                    red_i[threadIdx.x] = oi;
                }
            }
            __syncthreads();
        }
        const int piv = red_i[0];
        const double pv = colk[piv];
        // multipliers after the swap of rows k and piv
        __syncthreads();
        if (threadIdx.x == 0) {
            const double t = colk[k];
            colk[k] = colk[piv];
            colk[piv] = t;
        }
        __syncthreads();
        const double inv = 1.0 / pv;
        for (int j = blockIdx.x; j < 3 * n; j += gridDim.x) {
            if (j <= k) continue;
            double *col = G + (int64_t)n * j;
            // swap rows k and piv of this column
            __syncthreads();
            double rk = 0.0;
            if (threadIdx.x == 0) {
                const double t = col[k];
                col[k] = col[piv];
                col[piv] = t;
            }
            __syncthreads();
            rk = col[k] * inv;
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x)
                col[i] = (i == k) ? rk : fma(-colk[i], rk, col[i]);
            __syncthreads();
        }
        if (!grid_sync(p.bar)) return;
    }
    double *Xs = G + nn, *Qi = G + 2 * nn;
    // ---- one refinement step: R = P0 - Q0 Xs ; X = Xs + Qi R
    gemm(n, -1.0, Q0, Xs, 1.0, P0, 0.0, R);
    if (!grid_sync(p.bar)) return;
    gemm(n, 1.0, Qi, R, 1.0, Xs, 0.0, X);
    if (!grid_sync(p.bar)) return;
    // ---- squaring: ping-pong between X and T1, last one into E
    double *cur = X;
    for (int r = 0; r < s; ++r) {
        double *dst = (r == s - 1) ? p.E : (cur == X ? T1 : X);
        gemm(n, 1.0, cur, cur, 0.0, nullptr, 0.0, dst);
        if (!grid_sync(p.bar)) return;
        cur = dst;
    }
    if (s == 0) {
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
             e += (int64_t)gridDim.x * blockDim.x)
            p.E[e] = X[e];
    }
}

// [13/13] Pade numerator coefficients, b13 = 1, from the closed form
// c_j = (2m - j)! m! / ((2m)! j! (m - j)!) through c_{j-1} = c_j (2m-j+1) j / (m-j+1).
void pade13(double *b) {
    const int m = 13;
    unsigned long long c[14];
    c[13] = 1;
    for (int j = 13; j >= 1; --j) c[j - 1] = c[j] * (unsigned long long)(2 * m - j + 1) * j / (m - j + 1);
    for (int j = 0; j <= 13; ++j) b[j] = (double)c[j];
}

}  // namespace

cudaError_t expm_error_word(unsigned int *out, bool clear) { return read_error_word(out, clear); }

size_t expm_workspace_bytes(int64_t n) {
    // 13 n x n matrices + the n x 3n augmented matrix + barrier/norm words
    return (size_t)(16 * n * n) * sizeof(double) + 256;
}

cudaError_t expm_pade13(int64_t n, const double *A, int64_t ldA, double tau, double *E, void *ws,
                        cudaStream_t st) {
    ExpmDev p{};
    p.n = (int)n;
    p.A = A;
    p.ldA = ldA;
    p.tau = tau;
    p.E = E;
    auto *base = static_cast<uint8_t *>(ws);
    p.bar = reinterpret_cast<unsigned *>(base);
    p.norm_bits = reinterpret_cast<unsigned long long *>(base + 64);
    p.w = reinterpret_cast<double *>(base + 256);
    pade13(p.b);
    p.theta = 5.371920351148152;  // theta_13 of Higham (2005), Table 2.3
    cudaError_t e = cudaMemsetAsync(base, 0, 256, st);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expm_kernel, kThreadsE, 0);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, sms * std::min(per_sm, 1));
    void *args[] = {&p};
    return cudaLaunchCooperativeKernel((void *)expm_kernel, dim3(blocks), dim3(kThreadsE), args, 0, st);
}

}  // namespace kron
