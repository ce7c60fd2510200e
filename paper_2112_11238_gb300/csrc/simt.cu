// simt.cu -- FP64 / FP32 contractions on the CUDA cores (fused multiply-add).
//
// The plain-precision path of the library: the same strided contraction
//     C[r, c] = sum_k A[r, k] * B[k, c]
// as the tensor-core path, with every operand read through its index map (no
// permute).  64 x 64 output tile per 256-thread block, 4 x 4 outputs per
// thread, K staged through shared memory 16 at a time.  Loads are coalesced
// along whichever of (row, k) is contiguous in memory; each output is one
// FMA chain in ascending k.
#include <algorithm>

#include "internal.h"

namespace kron {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ int64_t imap(const IdxMap &m, int64_t x) {
    if (m.R0 == 0) return x * m.s0;
    return (x % m.R0) * m.s0 + (x / m.R0) * m.s1;
}

template <typename Tc>
__device__ __forceinline__ Tc ldv(const void *p, bool f64, int64_t off) {
    if (f64) return (Tc)__ldg(static_cast<const double *>(p) + off);
    return (Tc)__ldg(static_cast<const float *>(p) + off);
}

struct SimtDev {
    int64_t M, N, K;
    const void *A;
    IdxMap rowA, kA;
    const void *B;
    IdxMap colB, kB;
    void *C;
    IdxMap rowC, colC;
    int a64, b64, c64, acc, akc, bkc;
    int64_t kchunk;     // contracted indices per blockIdx.z (split-K), else K
    int64_t czstride;   // element offset of C per blockIdx.z
    int avec, cvec;     // small kernel: FP32 rows of A / C contiguous and 16-byte aligned
};

template <typename Tc>
__global__ void __launch_bounds__(NT) simt_gemm_kernel(const SimtDev p) {
    __shared__ Tc As[BK][BM + 1];
    __shared__ Tc Bs[BK][BN + 1];
    __shared__ int64_t ra[BM], cb[BN], rc[BM], cc[BN];
    const int t = threadIdx.x;
    const int64_t tiles_m = (p.M + BM - 1) / BM;
    const int64_t r0 = ((int64_t)blockIdx.x % tiles_m) * BM, c0 = ((int64_t)blockIdx.x / tiles_m) * BN;
    if (t < BM) {
        const int64_t r = r0 + t;
        ra[t] = r < p.M ? imap(p.rowA, r) : -1;
        rc[t] = r < p.M ? imap(p.rowC, r) : -1;
    } else if (t < BM + BN) {
        const int64_t c = c0 + (t - BM);
        cb[t - BM] = c < p.N ? imap(p.colB, c) : -1;
        cc[t - BM] = c < p.N ? imap(p.colC, c) : -1;
    }
    __syncthreads();
    const int tr = t & 15, tc = t >> 4;
    Tc acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (Tc)0;

    const int64_t kbeg = (int64_t)blockIdx.z * p.kchunk;
    const int64_t kend = min(p.K, kbeg + p.kchunk);
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int e = 0; e < (BM * BK) / NT; ++e) {
            const int idx = t + e * NT;
            int r, k;
            if (p.akc) { k = idx % BK; r = idx / BK; }
            else { r = idx % BM; k = idx / BM; }
            const int64_t kg = k0 + k;
            Tc v = (Tc)0;
            if (ra[r] >= 0 && kg < kend) v = ldv<Tc>(p.A, p.a64, ra[r] + imap(p.kA, kg));
            As[k][r] = v;
        }
#pragma unroll
        for (int e = 0; e < (BN * BK) / NT; ++e) {
            const int idx = t + e * NT;
            int c, k;
            if (p.bkc) { k = idx % BK; c = idx / BK; }
            else { c = idx % BN; k = idx / BN; }
            const int64_t kg = k0 + k;
            Tc v = (Tc)0;
            if (cb[c] >= 0 && kg < kend) v = ldv<Tc>(p.B, p.b64, cb[c] + imap(p.kB, kg));
            Bs[k][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            Tc av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[k][tr + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tc + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int c = tc + 16 * b;
        if (cc[c] < 0) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int r = tr + 16 * a;
            if (rc[r] < 0) continue;
            const int64_t off = (int64_t)blockIdx.z * p.czstride + rc[r] + cc[c];
            if (p.c64) {
                double *d = static_cast<double *>(p.C) + off;
                *d = p.acc ? *d + (double)acc[a][b] : (double)acc[a][b];
            } else {
                float *d = static_cast<float *>(p.C) + off;
                *d = p.acc ? (float)((Tc)*d + acc[a][b]) : (float)acc[a][b];
            }
        }
    }
}

bool kcontig(const IdxMap &k) { return k.s0 == 1 && k.R0 != 1; }

// Fixed-order sum of split-K partials: C[r, c] (+)= sum_z P[z][r + M c].
template <typename Tc>
__global__ void simt_reduce_kernel(const Tc *__restrict__ P, int64_t splits, int64_t M, int64_t N,
                                   void *C, IdxMap rowC, IdxMap colC, int c64, int acc) {
    const int64_t total = M * N;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        Tc s = (Tc)0;
        for (int64_t z = 0; z < splits; ++z) s += P[z * total + idx];
        const int64_t r = idx % M, c = idx / M;
        const int64_t off = imap(rowC, r) + imap(colC, c);
        if (c64) {
            double *d = static_cast<double *>(C) + off;
            *d = acc ? *d + (double)s : (double)s;
        } else {
            float *d = static_cast<float *>(C) + off;
            *d = acc ? (float)((Tc)*d + s) : (float)s;
        }
    }
}

int64_t splitk_chunk(int64_t M, int64_t N, int64_t K) {
    const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    int64_t splits = std::max<int64_t>(1, (4 * 152 + tiles - 1) / tiles);
    int64_t chunk = (K + splits - 1) / splits;
    chunk = std::max<int64_t>(BK, (chunk + BK - 1) / BK * BK);
    return chunk;
}

SimtDev make_simt(const Contraction &c) {
    SimtDev d{};
    d.M = c.M; d.N = c.N; d.K = c.K;
    d.A = c.A; d.rowA = c.rowA; d.kA = c.kA;
    d.B = c.B; d.colB = c.colB; d.kB = c.kB;
    d.C = c.C; d.rowC = c.rowC; d.colC = c.colC;
    d.a64 = c.A_f64; d.b64 = c.B_f64; d.c64 = c.C_f64; d.acc = c.accumulate;
    d.akc = kcontig(c.kA);
    d.bkc = kcontig(c.kB);
    d.kchunk = std::max<int64_t>(c.K, 1);
    d.czstride = 0;
    return d;
}

// Contractions with a short contracted index and few outputs per row (the
// small modes of a high-order tensor, such as the 20 x 20 factors of a 20^6
// tensor), where a 64 x 64 output tile would be mostly empty: one thread
// per row, op(L) (K x N, zero-padded to NM columns) in shared memory, the
// row's K values read once each (eight loads in flight) and its N outputs
// accumulated in registers, in ascending k.  Rows of consecutive threads are consecutive fibres, so
// the loads along k are coalesced whenever the fibres are contiguous.
constexpr int kSmallK = 64;

template <typename Tc, int NM>
__global__ void __launch_bounds__(256) simt_small_kernel(const SimtDev p) {
    __shared__ Tc sB[kSmallK * NM];
    for (int idx = threadIdx.x; idx < kSmallK * NM; idx += blockDim.x) {
        const int k = idx / NM, j = idx % NM;
        sB[idx] = (k < p.K && j < p.N) ? ldv<Tc>(p.B, p.b64, imap(p.colB, j) + imap(p.kB, k)) : Tc(0);
    }
    __syncthreads();
    const int K = (int)p.K, N = (int)p.N;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < p.M; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ra = imap(p.rowA, r), rc = imap(p.rowC, r);
        Tc acc[NM];
#pragma unroll
        for (int j = 0; j < NM; ++j) acc[j] = Tc(0);
        // eight loads in flight, then their products (rows of sB past K are
        // zero and the values past K are zero: fma(0, 0, acc) = acc)
        for (int k0 = 0; k0 < K; k0 += 8) {
            Tc av[8];
            if (sizeof(Tc) == 4 && p.avec) {
                // a contiguous, aligned FP32 row (K a multiple of 4): 16-byte loads
                const float4 *q = reinterpret_cast<const float4 *>(static_cast<const float *>(p.A) + ra + k0);
                const float4 v0 = __ldg(q);
                const float4 v1 = (k0 + 4 < K) ? __ldg(q + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
                av[0] = v0.x; av[1] = v0.y; av[2] = v0.z; av[3] = v0.w;
                av[4] = v1.x; av[5] = v1.y; av[6] = v1.z; av[7] = v1.w;
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) av[u] = (k0 + u < K) ? ldv<Tc>(p.A, p.a64, ra + imap(p.kA, k0 + u)) : Tc(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const Tc *b = sB + (k0 + u) * NM;
#pragma unroll
                for (int j = 0; j < NM; ++j) acc[j] = fma(av[u], b[j], acc[j]);
            }
        }
        if (sizeof(Tc) == 4 && p.cvec) {
            // a contiguous, aligned FP32 output row (N a multiple of 4)
            float4 *q = reinterpret_cast<float4 *>(static_cast<float *>(p.C) + rc);
#pragma unroll
            for (int j = 0; j < NM; j += 4)
                if (j < N) q[j / 4] = make_float4((float)acc[j], (float)acc[j + 1], (float)acc[j + 2], (float)acc[j + 3]);
            continue;
        }
#pragma unroll
        for (int j = 0; j < NM; ++j) {
            if (j >= N) break;
            const int64_t o = rc + imap(p.colC, j);
            if (p.c64) {
                double *q = static_cast<double *>(p.C) + o;
                *q = p.acc ? *q + (double)acc[j] : (double)acc[j];
            } else {
                float *q = static_cast<float *>(p.C) + o;
                *q = p.acc ? (float)(*q + acc[j]) : (float)acc[j];
            }
        }
    }
}

template <typename Tc, int NM>
cudaError_t launch_small(const SimtDev &d, cudaStream_t st) {
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((d.M + 255) / 256, 152 * 8));
    simt_small_kernel<Tc, NM><<<(unsigned)blocks, 256, 0, st>>>(d);
    return cudaGetLastError();
}

}  // namespace

bool simt_small_fits(bool f64, int64_t K, int64_t N) { return K >= 1 && K <= kSmallK && N >= 1 && N <= (f64 ? 32 : 64); }

cudaError_t simt_contract_small(bool f64, const Contraction &c, cudaStream_t st) {
    if (c.M == 0 || c.N == 0) return cudaSuccess;
    if (!simt_small_fits(f64, c.K, c.N)) return cudaErrorInvalidValue;
    SimtDev d = make_simt(c);
    const bool abase = (reinterpret_cast<uintptr_t>(c.A) & 15) == 0, cbase = (reinterpret_cast<uintptr_t>(c.C) & 15) == 0;
    d.avec = (!f64 && !c.A_f64 && abase && c.kA.R0 == 0 && c.kA.s0 == 1 && c.rowA.R0 == 0 && c.rowA.s0 % 4 == 0 &&
              c.K % 4 == 0) ? 1 : 0;
    d.cvec = (!f64 && !c.C_f64 && cbase && !c.accumulate && c.colC.R0 == 0 && c.colC.s0 == 1 && c.rowC.R0 == 0 &&
              c.rowC.s0 % 4 == 0 && c.N % 4 == 0) ? 1 : 0;
    if (f64) {
        if (c.N <= 8) return launch_small<double, 8>(d, st);
        if (c.N <= 16) return launch_small<double, 16>(d, st);
        if (c.N <= 24) return launch_small<double, 24>(d, st);
        return launch_small<double, 32>(d, st);
    }
    if (c.N <= 8) return launch_small<float, 8>(d, st);
    if (c.N <= 16) return launch_small<float, 16>(d, st);
    if (c.N <= 24) return launch_small<float, 24>(d, st);
    if (c.N <= 32) return launch_small<float, 32>(d, st);
    if (c.N <= 48) return launch_small<float, 48>(d, st);
    return launch_small<float, 64>(d, st);
}

size_t simt_splitk_partial_bytes(bool f64, int64_t M, int64_t N, int64_t K) {
    const int64_t chunk = splitk_chunk(M, N, K);
    const int64_t splits = (K + chunk - 1) / chunk;
    return (size_t)std::max<int64_t>(splits, 1) * M * N * (f64 ? 8 : 4);
}

cudaError_t simt_contract_splitk(bool f64, const Contraction &c, void *partial, cudaStream_t st) {
    if (c.M == 0 || c.N == 0) return cudaSuccess;
    SimtDev d = make_simt(c);
    d.kchunk = splitk_chunk(c.M, c.N, c.K);
    const int64_t splits = std::max<int64_t>(1, (c.K + d.kchunk - 1) / d.kchunk);
    d.C = partial;
    d.c64 = f64;
    d.acc = 0;
    d.rowC = IdxMap{0, 1, 0};
    d.colC = IdxMap{0, c.M, 0};
    d.czstride = c.M * c.N;
    const int64_t tiles = ((c.M + BM - 1) / BM) * ((c.N + BN - 1) / BN);
    if (tiles > 0x7fffffff || splits > 65535) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)tiles, 1, (unsigned)splits);
    if (f64) simt_gemm_kernel<double><<<grid, NT, 0, st>>>(d);
    else simt_gemm_kernel<float><<<grid, NT, 0, st>>>(d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = c.M * c.N;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096));
    if (f64)
        simt_reduce_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(
            static_cast<const double *>(partial), splits, c.M, c.N, c.C, c.rowC, c.colC, c.C_f64, c.accumulate);
    else
        simt_reduce_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(
            static_cast<const float *>(partial), splits, c.M, c.N, c.C, c.rowC, c.colC, c.C_f64, c.accumulate);
    return cudaGetLastError();
}

cudaError_t simt_contract(bool f64, const Contraction &c, cudaStream_t st) {
    if (c.M == 0 || c.N == 0) return cudaSuccess;
    SimtDev d = make_simt(c);
    const int64_t tiles = ((c.M + BM - 1) / BM) * ((c.N + BN - 1) / BN);
    if (tiles > 0x7fffffff) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)tiles);
    if (f64) simt_gemm_kernel<double><<<grid, NT, 0, st>>>(d);
    else simt_gemm_kernel<float><<<grid, NT, 0, st>>>(d);
    return cudaGetLastError();
}

}  // namespace kron
