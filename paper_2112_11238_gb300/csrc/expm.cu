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
// Several exponentials (one per mode) run in ONE cooperative launch (one
// block per SM): the blocks are split into one group per matrix, and each
// group's phases are separated by its own barrier with a bounded wait.  FP64
// GEMMs are split into 16 x 16 tiles spread over the group.  The elimination
// goes by panels of kNB columns: every block of the group factors the panel
// in shared memory (the same pivots everywhere), then updates the columns it
// owns, one warp per column -- one barrier per panel instead of per column.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.h"
#include "ptx.cuh"

namespace kron {

namespace {

constexpr int kT = 16;          // GEMM tile
constexpr int kThreadsE = 256;  // = kT * kT
constexpr int kNB = 16;         // Gauss-Jordan panel width
constexpr int kWarpsE = kThreadsE / 32;

// Tile maps: one byte per 16 x 16 tile of an n x n matrix, nonzero when the
// tile may hold a nonzero (kFlagMats maps of kMaxTiles^2 bytes per problem).
constexpr int kMaxTiles = 64;  // n <= 1024
constexpr int kFlagMats = 8;
constexpr size_t kFlagBytes = (size_t)kFlagMats * kMaxTiles * kMaxTiles;

struct ExpmProb {
    int n;
    const double *A;
    int64_t ldA;
    double *E;
    double *w;           // workspace base (doubles)
    unsigned *bar;       // [0] count, [1] generation
    unsigned long long *norm_bits;
    unsigned char *flags;  // kFlagMats tile maps
};

struct ExpmDev {
    int count;
    ExpmProb p[KRON_MAX_D];
    double tau;
    double b[14];
    double theta;
};

// Barrier of the gs blocks of one group (bounded wait).
__device__ bool grid_sync(unsigned *bar, int gs) {
    __syncthreads();
    __shared__ int failed;
    if (threadIdx.x == 0) {
        failed = 0;
        volatile unsigned *vgen = bar + 1;
        const unsigned my_gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == (unsigned)gs - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            while (*vgen == my_gen) {
                if (timeout_latched() || globaltimer_ns() - t0 > kWaitLimitNs) {
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
// alias C; A and B must not.  Tiles are spread over the group (block lb of gs).
// fa / fb: tile maps of A and B (null: dense); a K-step whose A or B tile is
// all zero is skipped (it adds exact zeros: the polynomial of the banded
// stepper matrices is banded).  fc: the map of C to write (null: none).
__device__ void gemm(int n, double alpha, const double *A, const double *B, double beta,
                     const double *C0, double gamma, double *C, int lb, int gs,
                     const unsigned char *fa = nullptr, const unsigned char *fb = nullptr,
                     unsigned char *fc = nullptr) {
    __shared__ double As[kT][kT + 1], Bs[kT][kT + 1];
    const int tiles = (n + kT - 1) / kT;
    const int tr = threadIdx.x % kT, tc = threadIdx.x / kT;
    for (int t = lb; t < tiles * tiles; t += gs) {
        const int i0 = (t % tiles) * kT, j0 = (t / tiles) * kT;
        const int ti = t % tiles, tj = t / tiles;
        double acc = 0.0;
        for (int k0 = 0; k0 < n; k0 += kT) {
            const int tk = k0 / kT;
            // the same decision in every thread of the block (same bytes)
            if (fa && (__ldcg(fa + ti + kMaxTiles * tk) == 0 || __ldcg(fb + tk + kMaxTiles * tj) == 0)) continue;
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
        double v = 0.0;
        if (i < n && j < n) {
            const int64_t o = i + (int64_t)n * j;
            v = alpha * acc;
            if (beta != 0.0) v += beta * C0[o];
            if (i == j) v += gamma;
            C[o] = v;
        }
        if (fc) {
            const int nz = __syncthreads_or(v != 0.0);
            if (threadIdx.x == 0) fc[ti + kMaxTiles * tj] = nz ? 1 : 0;
        }
    }
}

// Tile map of a combination of matrices: a tile may be nonzero where any
// of theirs may, and on the diagonal when an identity term is added.
__device__ void flag_union(int n, unsigned char *f, const unsigned char *f1, const unsigned char *f2,
                           const unsigned char *f3, bool diag, int lb, int gs) {
    const int tiles = (n + kT - 1) / kT;
    for (int t = lb * blockDim.x + threadIdx.x; t < tiles * tiles; t += gs * blockDim.x) {
        const int ti = t % tiles, tj = t / tiles, o = ti + kMaxTiles * tj;
        f[o] = (f1[o] | f2[o] | f3[o] | (diag && ti == tj)) ? 1 : 0;
    }
}

// Y = sum_k c_k X_k (+ g I), elementwise over the group.
__device__ void lincomb(int n, double *Y, double c1, const double *X1, double c2, const double *X2,
                        double c3, const double *X3, double g, int lb, int gs) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = (int64_t)lb * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gs * blockDim.x) {
        double v = 0.0;
        if (X1) v += c1 * X1[e];
        if (X2) v += c2 * X2[e];
        if (X3) v += c3 * X3[e];
        if (e % n == e / n) v += g;
        Y[e] = v;
    }
}

// Gauss-Jordan elimination with partial pivoting on the n x ncols matrix G
// (ld n, ncols >= n), by panels of kNB columns (see the file comment).  smem
// holds the panel (kNB x n) and one n-column buffer per warp.  A zero pivot
// (singular matrix) latches kErrNumeric.
__device__ bool gauss_jordan(int n, int ncols, double *G, unsigned *bar, int lb, int gs, double *smem) {
    double *pan = smem;
    double *cb = smem + (size_t)kNB * n + (size_t)(threadIdx.x >> 5) * n;
    __shared__ int pivs[kNB];
    __shared__ double invs[kNB], rr[kNB], rv[kWarpsE];
    __shared__ int ri[kWarpsE];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int k0 = 0; k0 < n; k0 += kNB) {
        const int kw = min(kNB, n - k0);
        for (int e = tid; e < kw * n; e += blockDim.x) pan[e] = G[(int64_t)n * k0 + e];
        __syncthreads();
        for (int kk = 0; kk < kw; ++kk) {
            const int k = k0 + kk;
            const double *pc = pan + (size_t)kk * n;
            // pivot: largest |entry| in rows k.., lowest row on ties
            double best = -1.0;
            int bi = k;
            for (int i = k + tid; i < n; i += blockDim.x) {
                const double a = fabs(pc[i]);
                if (a > best) {
                    best = a;
                    bi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (lane == 0) {
                rv[wid] = best;
                ri[wid] = bi;
            }
            __syncthreads();
            if (tid == 0) {
                double b = rv[0];
                int i0 = ri[0];
                for (int w = 1; w < kWarpsE; ++w)
                    if (rv[w] > b || (rv[w] == b && ri[w] < i0)) {
                        b = rv[w];
                        i0 = ri[w];
                    }
                pivs[kk] = i0;
                if (!(b > 0.0) && lb == 0) latch_error(kErrNumeric);
            }
            __syncthreads();
            const int piv = pivs[kk];
            if (tid >= kk && tid < kw && piv != k) {
                double *c = pan + (size_t)tid * n;
                const double t = c[k];
                c[k] = c[piv];
                c[piv] = t;
            }
            __syncthreads();
            const double inv = 1.0 / pc[k];
            if (tid == 0) invs[kk] = inv;
            if (tid > kk && tid < kw) rr[tid] = pan[(size_t)tid * n + k] * inv;
            __syncthreads();
            for (int i = tid; i < n; i += blockDim.x) {
                const double m = pc[i];
                for (int c = kk + 1; c < kw; ++c) {
                    double *pcol = pan + (size_t)c * n;
                    pcol[i] = (i == k) ? rr[c] : fma(-m, rr[c], pcol[i]);
                }
            }
            __syncthreads();
        }
        // the columns right of the panel, one warp per column
        for (int j = k0 + kw + lb * kWarpsE + wid; j < ncols; j += gs * kWarpsE) {
            double *col = G + (int64_t)n * j;
            for (int i = lane; i < n; i += 32) cb[i] = col[i];
            __syncwarp();
            for (int kk = 0; kk < kw; ++kk) {
                const int k = k0 + kk, piv = pivs[kk];
                if (lane == 0 && piv != k) {
                    const double t = cb[k];
                    cb[k] = cb[piv];
                    cb[piv] = t;
                }
                __syncwarp();
                const double r = cb[k] * invs[kk];
                __syncwarp();
                const double *m = pan + (size_t)kk * n;
                for (int i = lane; i < n; i += 32) cb[i] = (i == k) ? r : fma(-m[i], r, cb[i]);
                __syncwarp();
            }
            for (int i = lane; i < n; i += 32) col[i] = cb[i];
            __syncwarp();
        }
        if (!grid_sync(bar, gs)) return false;
    }
    return true;
}

__global__ void __launch_bounds__(kThreadsE) expm_kernel(const __grid_constant__ ExpmDev d) {
    extern __shared__ double esm[];
    const int gs = gridDim.x / d.count;  // blocks per matrix
    const int g = blockIdx.x / gs, lb = blockIdx.x % gs;
    if (g >= d.count) return;  // spare blocks take part in nothing
    const ExpmProb &p = d.p[g];
    const int n = p.n;
    const int64_t nn = (int64_t)n * n;
    double *B = p.w, *B2 = B + nn, *B4 = B2 + nn, *B6 = B4 + nn, *T1 = B6 + nn, *T2 = T1 + nn;
    double *U = T2 + nn, *V = U + nn, *Q0 = V + nn, *P0 = Q0 + nn, *X = P0 + nn, *R = X + nn;
    double *G = R + nn;  // augmented [Q | P | I]: n x 3n, ld n
    __shared__ double red_v[kThreadsE];
    const int tiles = (n + kT - 1) / kT;
    unsigned char *fB = p.flags, *fB2 = fB + kMaxTiles * kMaxTiles, *fB4 = fB2 + kMaxTiles * kMaxTiles,
                  *fB6 = fB4 + kMaxTiles * kMaxTiles, *fT = fB6 + kMaxTiles * kMaxTiles,
                  *fR = fT + kMaxTiles * kMaxTiles;
    for (int t = lb * blockDim.x + threadIdx.x; t < tiles * tiles; t += gs * blockDim.x)
        fB[(t % tiles) + kMaxTiles * (t / tiles)] = 0;

    // ---- ||tau A||_1
    for (int j = lb; j < n; j += gs) {
        double s = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s += fabs(d.tau * p.A[i + p.ldA * j]);
        red_v[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red_v[threadIdx.x] += red_v[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicMax(p.norm_bits, (unsigned long long)__double_as_longlong(red_v[0]));
        __syncthreads();
    }
    if (!grid_sync(p.bar, gs)) return;
    const double nrm = __longlong_as_double((long long)*(volatile unsigned long long *)p.norm_bits);
    if (!isfinite(nrm)) {  // non-finite input
        if (lb == 0 && threadIdx.x == 0) latch_error(kErrNumeric);
        return;
    }
    int s = 0;
    if (nrm > d.theta) s = (int)ceil(log2(nrm / d.theta));
    const double scale = ldexp(d.tau, -s);
    for (int64_t e = (int64_t)lb * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gs * blockDim.x) {
        const double v = scale * p.A[(e % n) + p.ldA * (e / n)];
        B[e] = v;
        if (v != 0.0) fB[(int)((e % n) / kT) + kMaxTiles * (int)((e / n) / kT)] = 1;
    }
    if (!grid_sync(p.bar, gs)) return;
    // the polynomial's products skip the all-zero tiles of their operands
    gemm(n, 1.0, B, B, 0.0, nullptr, 0.0, B2, lb, gs, fB, fB, fB2);
    if (!grid_sync(p.bar, gs)) return;
    gemm(n, 1.0, B2, B2, 0.0, nullptr, 0.0, B4, lb, gs, fB2, fB2, fB4);
    if (!grid_sync(p.bar, gs)) return;
    gemm(n, 1.0, B4, B2, 0.0, nullptr, 0.0, B6, lb, gs, fB4, fB2, fB6);
    if (!grid_sync(p.bar, gs)) return;
    const double *b = d.b;
    // T1 = b13 B6 + b11 B4 + b9 B2 ; T2 = b12 B6 + b10 B4 + b8 B2
    lincomb(n, T1, b[13], B6, b[11], B4, b[9], B2, 0.0, lb, gs);
    lincomb(n, T2, b[12], B6, b[10], B4, b[8], B2, 0.0, lb, gs);
    // U' = B6 T1 + b7 B6 + b5 B4 + b3 B2 + b1 I  (into R as scratch first)
    lincomb(n, R, b[7], B6, b[5], B4, b[3], B2, b[1], lb, gs);
    lincomb(n, X, b[6], B6, b[4], B4, b[2], B2, b[0], lb, gs);
    flag_union(n, fT, fB6, fB4, fB2, false, lb, gs);  // the map of T1 and of T2
    if (!grid_sync(p.bar, gs)) return;
    gemm(n, 1.0, B6, T1, 1.0, R, 0.0, R, lb, gs, fB6, fT, fR);
    gemm(n, 1.0, B6, T2, 1.0, X, 0.0, V, lb, gs, fB6, fT, nullptr);
    if (!grid_sync(p.bar, gs)) return;
    gemm(n, 1.0, B, R, 0.0, nullptr, 0.0, U, lb, gs, fB, fR, nullptr);
    if (!grid_sync(p.bar, gs)) return;
    // Q0 = V - U, P0 = V + U, augmented G = [Q0 | P0 | I]
    for (int64_t e = (int64_t)lb * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gs * blockDim.x) {
        const double q = V[e] - U[e], pp = V[e] + U[e];
        Q0[e] = q;
        P0[e] = pp;
        G[e] = q;
        G[nn + e] = pp;
        G[2 * nn + e] = (e % n == e / n) ? 1.0 : 0.0;
    }
    if (!grid_sync(p.bar, gs)) return;
    if (!gauss_jordan(n, 3 * n, G, p.bar, lb, gs, esm)) return;
    double *Xs = G + nn, *Qi = G + 2 * nn;
    // ---- one refinement step: R = P0 - Q0 Xs ; X = Xs + Qi R
    gemm(n, -1.0, Q0, Xs, 1.0, P0, 0.0, R, lb, gs);
    if (!grid_sync(p.bar, gs)) return;
    gemm(n, 1.0, Qi, R, 1.0, Xs, 0.0, X, lb, gs);
    if (!grid_sync(p.bar, gs)) return;
    // ---- squaring: ping-pong between X and T1, last one into E
    double *cur = X;
    for (int r = 0; r < s; ++r) {
        double *dst = (r == s - 1) ? p.E : (cur == X ? T1 : X);
        gemm(n, 1.0, cur, cur, 0.0, nullptr, 0.0, dst, lb, gs);
        if (!grid_sync(p.bar, gs)) return;
        cur = dst;
    }
    if (s == 0) {
        for (int64_t e = (int64_t)lb * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gs * blockDim.x)
            p.E[e] = X[e];
    }
}

struct InvProb {
    int n;
    const void *P;
    int64_t ldP;
    double *G;      // n x 2n: [P | I] -> [I | P^{-1}]
    unsigned *bar;  // [0] count, [1] generation
};

struct InvDev {
    int count, p64;
    InvProb p[KRON_MAX_D];
};

// P^{-1} of several matrices (one group of blocks each), Gauss-Jordan with
// partial pivoting on [P | I] in FP64.
__global__ void __launch_bounds__(kThreadsE) inv_kernel(const __grid_constant__ InvDev d) {
    extern __shared__ double esm[];
    const int gs = gridDim.x / d.count;
    const int g = blockIdx.x / gs, lb = blockIdx.x % gs;
    if (g >= d.count) return;
    const InvProb &p = d.p[g];
    const int n = p.n;
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = (int64_t)lb * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gs * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        const int64_t src = i + p.ldP * j;
        p.G[e] = d.p64 ? static_cast<const double *>(p.P)[src] : (double)static_cast<const float *>(p.P)[src];
        p.G[nn + e] = (i == j) ? 1.0 : 0.0;
    }
    if (!grid_sync(p.bar, gs)) return;
    gauss_jordan(n, 2 * n, p.G, p.bar, lb, gs, esm);
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

cudaError_t expm_error_word(unsigned int *out, bool clear, cudaStream_t st) { return read_error_word(out, clear, st); }

size_t expm_workspace_bytes(int64_t n) {
    // 13 n x n matrices + the n x 3n augmented matrix + barrier/norm words +
    // the tile maps
    return (size_t)(16 * n * n) * sizeof(double) + 256 + kFlagBytes;
}

cudaError_t expm_pade13_batch(int count, const int64_t *n, const double *const *A, const int64_t *ldA, double tau,
                              double *const *E, void *const *ws, cudaStream_t st) {
    if (count < 1 || count > KRON_MAX_D) return cudaErrorInvalidValue;
    ExpmDev d{};
    d.count = count;
    d.tau = tau;
    pade13(d.b);
    d.theta = 5.371920351148152;  // theta_13 of Higham (2005), Table 2.3
    int64_t nmax = 1;
    for (int i = 0; i < count; ++i) {
        ExpmProb &p = d.p[i];
        p.n = (int)n[i];
        p.A = A[i];
        p.ldA = ldA[i];
        p.E = E[i];
        auto *base = static_cast<uint8_t *>(ws[i]);
        p.bar = reinterpret_cast<unsigned *>(base);
        p.norm_bits = reinterpret_cast<unsigned long long *>(base + 64);
        p.w = reinterpret_cast<double *>(base + 256);
        p.flags = base + 256 + (size_t)(16 * n[i] * n[i]) * sizeof(double);
        nmax = std::max(nmax, n[i]);
        cudaError_t e = cudaMemsetAsync(base, 0, 256, st);
        if (e != cudaSuccess) return e;
    }
    const size_t smem = (size_t)(kNB + kWarpsE) * nmax * sizeof(double);
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(expm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)((kNB + kWarpsE) * 1024 * sizeof(double)));
    });
    if (attr != cudaSuccess) return attr;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expm_kernel, kThreadsE, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int blocks = std::max(count, sms);  // one block per SM, whole groups
    void *args[] = {&d};
    return cudaLaunchCooperativeKernel((void *)expm_kernel, dim3(blocks), dim3(kThreadsE), args, smem, st);
}

cudaError_t expm_pade13(int64_t n, const double *A, int64_t ldA, double tau, double *E, void *ws,
                        cudaStream_t st) {
    return expm_pade13_batch(1, &n, &A, &ldA, tau, &E, &ws, st);
}

size_t inv_workspace_bytes(int64_t n) { return (size_t)(2 * n * n) * sizeof(double) + 256; }

double *inv_result(int64_t n, void *ws) {
    return reinterpret_cast<double *>(static_cast<uint8_t *>(ws) + 256) + n * n;
}

cudaError_t inv_gj_batch(int count, const int64_t *n, const void *const *P, const int64_t *ldP, bool p64,
                         void *const *ws, cudaStream_t st) {
    if (count < 1 || count > KRON_MAX_D) return cudaErrorInvalidValue;
    InvDev d{};
    d.count = count;
    d.p64 = p64 ? 1 : 0;
    int64_t nmax = 1;
    for (int i = 0; i < count; ++i) {
        InvProb &p = d.p[i];
        p.n = (int)n[i];
        p.P = P[i];
        p.ldP = ldP[i];
        auto *base = static_cast<uint8_t *>(ws[i]);
        p.bar = reinterpret_cast<unsigned *>(base);
        p.G = reinterpret_cast<double *>(base + 256);
        nmax = std::max(nmax, n[i]);
        cudaError_t e = cudaMemsetAsync(base, 0, 256, st);
        if (e != cudaSuccess) return e;
    }
    const size_t smem = (size_t)(kNB + kWarpsE) * nmax * sizeof(double);
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)((kNB + kWarpsE) * 1024 * sizeof(double)));
    });
    if (attr != cudaSuccess) return attr;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, inv_kernel, kThreadsE, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int blocks = std::max(count, sms);
    void *args[] = {&d};
    return cudaLaunchCooperativeKernel((void *)inv_kernel, dim3(blocks), dim3(kThreadsE), args, smem, st);
}

}  // namespace kron
