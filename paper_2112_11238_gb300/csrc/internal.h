// internal.h -- host-side interfaces between the C ABI layer and the kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/kron.h"

namespace kron {

// A 2-level index map used for rows, columns and the contracted index of
// every contraction in the library: index x -> (x % R0) * s0 + (x / R0) * s1.
// R0 == 0 means "no split": x -> x * s0.
struct IdxMap {
    int64_t R0 = 0;
    int64_t s0 = 0;
    int64_t s1 = 0;
};

// Strided generic contraction
//     C[r, c] = sum_k A[r, k] * B[k, c]
// with A[r, k] at A.ptr + rowA(r) + kA(k), B[k, c] at B.ptr + colB(c) + kB(k),
// C[r, c] at C.ptr + rowC(r) + colC(c).  Every mu-mode product, every
// step of the Tucker chain and the dL contraction of the adjoint is one of
// these with suitable maps (no permute is ever formed).
struct Contraction {
    int64_t M = 0, N = 0, K = 0;
    const void *A = nullptr;
    bool A_f64 = false;
    IdxMap rowA, kA;
    const void *B = nullptr;
    bool B_f64 = false;
    IdxMap colB, kB;
    void *C = nullptr;
    bool C_f64 = false;
    IdxMap rowC, colC;
    // C = acc (+ C if accumulate)
    bool accumulate = false;
};

// The split-precision forms of the tensor-core path.
enum TcForm { kTF32x3 = 0, kBF16x3 = 1, kBF16x6 = 2, kFX32 = 3, kFX32H = 4 };

inline int form_of(kron_prec p) {
    switch (p) {
        case KRON_PREC_3XTF32: return kTF32x3;
        case KRON_PREC_BF16X3: return kBF16x3;
        case KRON_PREC_BF16X6: return kBF16x6;
        case KRON_PREC_FX32: return kFX32;
        case KRON_PREC_FX32H: return kFX32H;
        default: return -1;
    }
}
inline bool is_fx(kron_prec p) { return p == KRON_PREC_FX32 || p == KRON_PREC_FX32H; }
inline bool is_split(kron_prec p) { return form_of(p) >= 0 && !is_fx(p); }
inline bool is_fx_form(int form) { return form == kFX32 || form == kFX32H; }
// Magnitude bits of a fixed-point form's integers: |X| < 2^bits.
inline int fx_bits(int form) { return form == kFX32H ? 29 : 31; }

// Scale word of a 32-bit fixed-point tensor: value = X * 2^(e - 31), and the
// largest |X| stored (maintained with atomicMax by the kernel that writes X).
struct FxScale {
    int e;
    unsigned maxabs;
};

// ---- tensor-core path (tc.cu) ----
// Bytes of the pre-split, pre-swizzled image of an (N x K) B operand.
size_t tc_bimage_bytes(int form, int64_t N, int64_t K);
// the same for an explicit N-tile width bn
size_t tc_bimage_bytes_bn(int form, int64_t N, int64_t K, int bn);
// N-tile width the tensor-core kernels use for a given N (at most cap).
int tc_tile_n(int form, int64_t N);
int tc_tile_n_cap(int form, int64_t N, int cap);
// Writes the image of B (given as a Contraction's B side: colB/kB maps over
// N x K) into `img` (device, tc_bimage_bytes long).
cudaError_t tc_build_bimage(int form, const Contraction &c, void *img, cudaStream_t st);
// the same image for N-tiles of width bn (tc_bimage_bytes_bn long)
cudaError_t tc_build_bimage_bn(int form, const Contraction &c, void *img, int bn, cudaStream_t st);
// The images of count (<= KRON_MAX_D) contractions' B operands in one launch,
// image j with N-tile bns[j] into imgs[j]; the same bytes as
// tc_build_bimage_bn builds for each.
cudaError_t tc_build_bimages(int form, int count, const Contraction *cs, void *const *imgs, const int *bns,
                             cudaStream_t st);
// C = A * B with the B operand from an image made by tc_build_bimage.
cudaError_t tc_contract_bimage(int form, const Contraction &c, const void *img, cudaStream_t st);
// Split-K contraction with both operands converted on load (the adjoint's
// dL); partial sums go to `partial` (FP32, splits * M * N), then reduced in a
// fixed order into C.  Returns the number of splits used via *splits.
size_t tc_splitk_partial_bytes(int64_t M, int64_t N, int64_t K);
cudaError_t tc_contract_splitk(int form, const Contraction &c, float *partial, cudaStream_t st);

// ---- persistent tensor-core path (tcp.cu) ----
// One contraction (B from an image made by tc_build_bimage).
cudaError_t tcp_contract(int form, const Contraction &c, const void *img, cudaStream_t st);
// One fixed-point contraction (FX32): A 32-bit fixed point (scale fxA), B
// from an image made by fx_build_bimage (row exponents fxF, row-sum bound
// fxG); C 32-bit fixed point with scale fxC, or values when fxC is null.
// reset_next: a scale word that the launch clears once the launches before it
// are complete (the output scale of the next fixed-point product; launches are
// programmatic dependent launches, so no memset may sit between them).
cudaError_t tcp_contract_fx(int form, const Contraction &c, const void *img, const FxScale *fxA, const int *fxF,
                            const unsigned long long *fxG, FxScale *fxC, cudaStream_t st,
                            FxScale *reset_next = nullptr);

// ---- fixed-point helpers (fx.cu) ----
// Image of op(L) for the FX32 form (same layout as tc_build_bimage, four
// slices), per-row exponents f[N] and the row-sum bound *g (zeroed here).
cudaError_t fx_build_bimage(int form, const Contraction &c, void *img, int *f, unsigned long long *g, cudaStream_t st);
// the same image for N-tiles of width bn (the tail tiles of tcp_contract_fx_tail)
cudaError_t fx_build_bimage_bn(int form, const Contraction &c, void *img, int *f, unsigned long long *g, int bn,
                               cudaStream_t st);
// tcp_contract_fx with the last, partial round of tiles split into tiles of
// half the width (second image img_half, tiles of width tc_tile_n / 2), so
// that it takes about half a tile's time; one launch.  Falls back to
// tcp_contract_fx when the split does not apply.
cudaError_t tcp_contract_fx_tail(int form, const Contraction &c, const void *img, const void *img_half, const FxScale *fxA,
                                 const int *fxF, const unsigned long long *fxG, FxScale *fxC, FxScale *reset_next,
                                 cudaStream_t st);
// Dense FP64/FP32 tensor of `count` elements -> 32-bit fixed point X with
// one scale (written to *s); `scratch` is 8 bytes of device memory.
cudaError_t fx_from_float(int form, const void *src, bool src64, int64_t count, int32_t *X, FxScale *s,
                          unsigned long long *scratch, cudaStream_t st);
// Zeroes the running maximum of a scale word before a kernel fills it.
cudaError_t fx_reset(FxScale *s, cudaStream_t st);
// A table of contractions run by one persistent launch; a job may wait for
// an earlier one (dep = its index) whose output it reads.
struct TcpJobs {
    int form = 0;
    std::vector<uint8_t> host;  // packed device job records
    int total_tiles = 0;
    int bn_max = 16;
    int nkb_max = 1;
    // launch configuration chosen by a caller (0: the built-in rule):
    // pipeline stages and accumulator sets per tile
    int stages = 0, nacc = 0;
    std::vector<int> tile_job;  // job of every tile (uploaded for tables above 8 jobs)
};
size_t tcp_job_bytes();
void tcp_jobs_begin(TcpJobs &jobs, int form);
// bn: N-tile width of the job (that of its image; 0: tc_tile_n).
int tcp_jobs_add(TcpJobs &jobs, const Contraction &c, const void *img, int dep, int bn = 0);
size_t tcp_jobs_table_bytes(const TcpJobs &jobs);
// `table`: device copy of jobs.host and `tile_job` of jobs.tile_job (both
// needed above 8 jobs); `done`: one int per job plus one of device scratch
// (zeroed by the call).
cudaError_t tcp_jobs_run(const TcpJobs &jobs, const void *table, int *done, cudaStream_t st,
                         const int *tile_job = nullptr);

// ---- fused groups of small modes (tcg.cu) ----
// Modes a .. a+g-1 (g <= 3) of a column-major tensor X[P, m_0, .., m_{g-1}, Q]
// mapped to n_0 .. n_{g-1} in one launch, applied in that order; img[t]: the
// image of op(L_t) made by tc_build_bimage_bn with N-tiles of kTcgBN columns.
// Every m, n <= 32; the split forms.
constexpr int kTcgBN = 32;
struct GroupSpec {
    int g = 0;
    int64_t P = 1, Q = 1;
    int64_t m[3] = {1, 1, 1}, n[3] = {1, 1, 1};
    const void *img[3] = {nullptr, nullptr, nullptr};
    // the FP32 CUDA-core variant reads op(L_t) itself: L_t, its leading
    // dimension, op = L^T (trans), FP64 storage (l64)
    const void *L[3] = {nullptr, nullptr, nullptr};
    int64_t ldL[3] = {0, 0, 0};
    bool trans = false, l64 = false;
};
bool tcg_fits(int form, const GroupSpec &gs);
cudaError_t tcg_run(int form, const GroupSpec &gs, const float *src, void *dst, bool dst64, cudaStream_t st);
// The same fused group in FP32 on the CUDA cores (fused multiply-add, each
// output one ascending sum over k).
bool tcf_fits(const GroupSpec &gs);
cudaError_t tcf_run(const GroupSpec &gs, const float *src, void *dst, bool dst64, cudaStream_t st);

// ---- CUDA-core path (simt.cu) ----
// FP64 (f64 = true) or FP32 fused multiply-add.
cudaError_t simt_contract(bool f64, const Contraction &c, cudaStream_t st);
// Short contracted index and few outputs per row (K <= 64, N <= 64 in FP32,
// <= 32 in FP64): one thread per row of C, op(L) in shared memory.  Rows of
// the contraction must be the tensor's fibres (the tensor-core layout).
bool simt_small_fits(bool f64, int64_t K, int64_t N);
cudaError_t simt_contract_small(bool f64, const Contraction &c, cudaStream_t st);

// The real 2n x 2m matrix of a complex mu-mode product with G = op(L)
// (complex.cu): L complex (interleaved, FP64 or FP32 parts), ldL in complex
// elements; op = L, L^T (trans) or conj of either (conj).  M column-major,
// ld 2n, same part type as L.
cudaError_t complex_expand(const void *L, bool f64, int64_t ldL, int64_t n, int64_t m, bool trans, bool conj,
                           void *M, cudaStream_t st);
// Split-K variant for a long contracted index (the adjoint's dL): partials
// (FP64 or FP32, splits * M * N) summed in a fixed order into C.
size_t simt_splitk_partial_bytes(bool f64, int64_t M, int64_t N, int64_t K);
cudaError_t simt_contract_splitk(bool f64, const Contraction &c, void *partial, cudaStream_t st);

// ---- FP64 dense helpers (expm.cu) ----
size_t expm_workspace_bytes(int64_t n);
cudaError_t expm_pade13(int64_t n, const double *A, int64_t ldA, double tau, double *E, void *ws,
                        cudaStream_t st);
// count exponentials in one launch (disjoint block groups); ws[i] of
// expm_workspace_bytes(n[i]) bytes each
cudaError_t expm_pade13_batch(int count, const int64_t *n, const double *const *A, const int64_t *ldA, double tau,
                              double *const *E, void *const *ws, cudaStream_t st);
// P^{-1} of count matrices (FP64 Gauss-Jordan, one launch): ws[i] of
// inv_workspace_bytes(n[i]) bytes each; the inverse (n x n, ld n, FP64) is
// at inv_result(n[i], ws[i]).  P is FP64 (p64) or FP32 with leading dim ldP.
size_t inv_workspace_bytes(int64_t n);
// PCG vector kernels (pcg.cu): FP64 dot products in a fixed order, scaled updates
cudaError_t pcg_dot(const void *x, const void *y, bool f64, int64_t n, double *partial, double *out, cudaStream_t st);
cudaError_t pcg_axpby(bool f64, int64_t n, double a, const double *num, const double *den, const void *x, double b,
                      const double *bnum, const double *bden, void *y, cudaStream_t st);
size_t pcg_partial_doubles();
double *inv_result(int64_t n, void *ws);
cudaError_t inv_gj_batch(int count, const int64_t *n, const void *const *P, const int64_t *ldP, bool p64,
                         void *const *ws, cudaStream_t st);

// Device error words of the translation units whose kernels latch errors
// (bounded waits, non-finite input): stream-ordered read, optional clear.
cudaError_t tc_error_word(unsigned int *out, bool clear, cudaStream_t st);
cudaError_t tcp_error_word(unsigned int *out, bool clear, cudaStream_t st);
cudaError_t expm_error_word(unsigned int *out, bool clear, cudaStream_t st);

// Test hook of the in-launch job dependencies of the persistent kernel
// (tcp.cu): with hold != 0 every dependency wants one more finished tile
// than its job has, so the wait can only end by its time limit, which is
// limit_ns (0: the default kWaitLimitNs).  Applies to launches made after
// the call, on every device.
void tcp_debug_dependency_timeout(int hold, unsigned long long limit_ns);

}  // namespace kron
