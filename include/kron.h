/*
 * kron.h -- C ABI of libkron, a GB300 (sm_103a) library for mu-mode products
 * and Tucker operators (Caliari, Cassini, Zivcovich, "A mu-mode BLAS approach
 * for multidimensional tensor-structured problems", arXiv 2112.11238).
 *
 * Conventions shared by every call
 * --------------------------------
 *  * Tensors are dense and column-major: T in R^{m_1 x ... x m_d} stores
 *    T(j_1, ..., j_d) (0-based) at j_1 + m_1 (j_2 + m_2 (j_3 + ...)), the vec
 *    ordering of the paper's Appendix A.  d is 1..KRON_MAX_D.
 *  * A matrix L_mu of size n_mu x m_mu is column-major with leading dimension
 *    ldL >= n_mu: element (i, j) at L[i + ldL * j].  With trans = 1 the call
 *    uses L^T instead, L then being m_mu x n_mu with ldL >= m_mu.
 *  * Every tensor/matrix pointer is a DEVICE pointer owned by the caller.
 *    Shape arrays and arrays of pointers live in HOST memory.  Element type is
 *    given by kron_dtype (double or float) and is the same for all tensors and
 *    matrices of a call, except where a call says otherwise.
 *  * Calls are asynchronous and ordered on the given CUDA stream (0 = legacy
 *    default stream).  No call synchronises the device; the calls that
 *    must read a result on the host (kron_get_device_error,
 *    kron_kronsum_pcg, kron_batched_bind) wait for their stream only.  The
 *    library allocates no device memory in any compute call: scratch comes from the caller's workspace `ws`
 *    (`ws_bytes` long, 256-byte aligned), whose required size the matching
 *    *_workspace_size call reports.  Plans are host-only objects.
 *  * Output tensors must not overlap inputs or the workspace (except where a
 *    call states an in-place update).
 *  * Errors: invalid host-side arguments are reported synchronously by the
 *    returned status and nothing is launched.  Errors detected by a kernel
 *    (a bounded wait that timed out) are latched in a per-device error word
 *    read by kron_get_device_error.  No C++ exception crosses this ABI.
 *  * Effective FLOPs of a Tucker operator are the algorithmic
 *    sum_mu 2 n_mu m_mu prod(other current sizes), independent of precision.
 */
#ifndef KRON_H
#define KRON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define KRON_API __attribute__((visibility("default")))
#else
#define KRON_API
#endif

/* CUDA stream handle; identical to cudaStream_t. */
typedef struct CUstream_st *kron_stream_t;

#define KRON_MAX_D 6

typedef enum kron_status {
    KRON_OK = 0,
    KRON_ERR_INVALID_ARG = 1, /* bad size, null pointer, bad enum, ld too small */
    KRON_ERR_UNSUPPORTED = 2, /* valid but not provided (e.g. a size above a limit) */
    KRON_ERR_ALIGNMENT = 3,   /* a pointer is not aligned to its element size / 256 B workspace */
    KRON_ERR_WORKSPACE = 4,   /* ws_bytes smaller than the reported requirement */
    KRON_ERR_CUDA = 5,        /* a CUDA runtime call failed (launch error, ...) */
    KRON_ERR_TIMEOUT = 6,     /* a kernel's bounded wait ran out (device error word) */
    KRON_ERR_NUMERIC = 7      /* non-finite input where a finite one is required */
} kron_status;

typedef enum kron_dtype { KRON_F64 = 0, KRON_F32 = 1 } kron_dtype;

/*
 * Arithmetic used for the contractions.
 *  KRON_PREC_FP64   : FP64 fused multiply-add on CUDA cores, FP64 intermediates.
 *  KRON_PREC_FP32   : FP32 fused multiply-add on CUDA cores, FP32 intermediates.
 *  KRON_PREC_3XTF32 : tensor cores (tcgen05 kind::tf32); each operand split
 *                     x = x_hi + x_lo into two TF32 pieces (round to nearest),
 *                     three products lo*hi + hi*lo + hi*hi accumulated in FP32.
 *  KRON_PREC_BF16X3 : tensor cores (tcgen05 kind::f16, bf16 operands); two
 *                     bf16 pieces per operand, three products, FP32 accumulate.
 *  KRON_PREC_BF16X6 : three bf16 pieces per operand, the six products with
 *                     piece-index sum <= 2, FP32 accumulate.
 *  KRON_PREC_FX32   : error-free slicing in the manner of Ozaki et al. (Numer.
 *                     Algorithms 59, 2012): the tensor is held as 32-bit fixed
 *                     point with one power-of-two scale per tensor, every row
 *                     of L as 32-bit fixed point with its own scale; both are
 *                     cut into four balanced base-256 digits stored exactly as
 *                     bf16 (so the products left out average to zero), and
 *                     the ten slice products down to 2^-24 are accumulated in
 *                     two tensor-memory accumulators, the leading one exactly
 *                     (integer-valued sums below 2^24), then combined in
 *                     64-bit integer arithmetic.  About 31 significant bits
 *                     per stored value and per product, for contraction
 *                     lengths up to 256; intermediates are 32-bit fixed point.
 *                     Supported by kron_mump, kron_tucker, kron_kronsumv,
 *                     kron_itucker and the stepper (not by the adjoint).
 *  KRON_PREC_FX32H  : the same scheme with 29-bit fixed point cut into three
 *                     balanced digits of 8, 11 and 11 bits stored exactly as
 *                     FP16 slices d0 2^8, d1 2^-3, d2 2^-14 (all in the normal
 *                     FP16 range), and the six slice products with digit
 *                     index sum <= 2 (tcgen05 kind::f16 with f16 operands):
 *                     6 products instead of 10, about 26 significant bits per
 *                     product.  Same calls as KRON_PREC_FX32.
 * Split forms keep intermediates in FP32.  Inputs stored as double are split
 * from their double value.
 */
typedef enum kron_prec {
    KRON_PREC_FP64 = 0,
    KRON_PREC_FP32 = 1,
    KRON_PREC_3XTF32 = 2,
    KRON_PREC_BF16X3 = 3,
    KRON_PREC_BF16X6 = 4,
    KRON_PREC_FX32 = 5,
    KRON_PREC_FX32H = 6
} kron_prec;

/* Plan flags. */
#define KRON_PLAN_TRANS_L 0x1u     /* use L_mu^T for every mode (cf. the paper's cttucker) */
#define KRON_PLAN_NATURAL_ORDER 0x2u /* apply modes in order 1..d instead of the cost-minimising order */
#define KRON_PLAN_UNFUSED 0x4u     /* split forms: every mode product its own launch (no fused groups) */

typedef struct kron_plan_s *kron_plan;

KRON_API const char *kron_status_string(kron_status s);

/* Library version as major * 10000 + minor * 100 + patch. */
KRON_API int kron_version(void);

/*
 * Reads, and with clear != 0 resets, the device error word of the current
 * device: the OR of the words of every kernel file that latches errors
 * (bit 0: a bounded wait inside a kernel timed out -- the mbarrier phases of
 * the tensor-core pipelines, the in-launch job dependencies of the persistent
 * kernel, the grid barriers of the exponential; bit 1: non-finite input or a
 * zero pivot).  The read is ordered on `stream` and waits for that stream
 * only (work queued on other streams is not waited for); *code receives the
 * word.  Returns KRON_ERR_TIMEOUT if bit 0 is set, KRON_ERR_NUMERIC if bit 1
 * is, KRON_OK otherwise.  A latched bit stays until cleared (it does not
 * change how later launches run); the results of the launches that latched it
 * are not to be trusted.
 */
KRON_API kron_status kron_get_device_error(kron_stream_t stream, int *code, int clear);

/*
 * Test hook for the timeout path (the paper has no counterpart).  With
 * hold != 0, every in-launch job dependency of the persistent tensor-core
 * kernel (the batched Tucker operators) waits for one finished tile more than
 * its job has, so the wait ends only at its time limit, `limit_ms`
 * milliseconds (0: the default of 2 s; at most 10 s): the kernel then latches
 * the timeout bit (see kron_get_device_error), carries on with the tile and
 * returns normally, and the context stays usable.  hold = 0 restores normal
 * operation.  Affects launches made after the call, on every device; not for
 * production use.  KRON_ERR_INVALID_ARG for a negative or larger limit.
 */
KRON_API kron_status kron_debug_dependency_timeout(int hold, double limit_ms);

/* ------------------------------------------------------------------------ */
/* mu-mode product: Definition "mu-mode product", Eq. (mmp)                  */
/* ------------------------------------------------------------------------ */
/*
 * S = T x_mu op(L):  S^{(mu)} = op(L) T^{(mu)}, i.e. op(L) (n x m_mu) applied
 * to every mu-fibre of T.  mu is 0-based (0 <= mu < d).  T has sizes
 * m[0..d-1]; S has the same sizes with n in position mu.  The unfolding is
 * never formed: for mu > 0 the call runs a strided batched contraction over
 * the slabs T(:, :, q), for mu == 0 a plain GEMM.  n >= 1, all m >= 1.
 */
KRON_API kron_status kron_mump_workspace_size(int d, const int64_t *m, int mu, int64_t n,
                                     kron_dtype dtype, kron_prec prec, size_t *bytes);
KRON_API kron_status kron_mump(int d, const int64_t *m, int mu, int64_t n, const void *T,
                      const void *L, int64_t ldL, int transL, void *S,
                      kron_dtype dtype, kron_prec prec, void *ws, size_t ws_bytes,
                      kron_stream_t stream);

/*
 * The same product as kron_mump for the split forms (3XTF32, BF16X3, BF16X6),
 * for callers that cannot provide device memory: a host application whose
 * own pool holds all of the device memory, or a latency-critical loop that
 * must not call cudaMalloc (an allocation can synchronise the device).  The
 * paper has no counterpart; this is a deployment variant of kron_mump.
 * No workspace is passed and nothing is allocated: the scratch (the split
 * image of op(L)) lives in a 1 MiB array compiled into the library, which
 * every GPU that loads the library holds until the process exits.  Sizes whose
 * image exceeds 1 MiB return KRON_ERR_WORKSPACE (n and m_mu up to 256 always
 * fit).  The first call on a device, and the first one after a device reset,
 * looks up the array's device address (host code cannot use the array's name
 * as one); make that call before any stream capture.  All calls on a device
 * share the array: calls whose execution overlaps on the GPU (other streams,
 * other host threads) race and give wrong results; calls ordered on one
 * stream are safe.  Other precisions return KRON_ERR_UNSUPPORTED.
 */
KRON_API kron_status kron_mump_noalloc(int d, const int64_t *m, int mu, int64_t n, const void *T,
                                       const void *L, int64_t ldL, int transL, void *S,
                                       kron_dtype dtype, kron_prec prec, kron_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Tucker operator: Definition "Tucker operator", Eq. (tuckerop)             */
/* ------------------------------------------------------------------------ */
/*
 * A plan fixes d, the sizes m (input) and n (output), the storage dtype, the
 * precision and the flags; it chooses the order in which the d mu-mode
 * products run (the result is independent of the order, Section 2) so as to
 * minimise the flop count, unless KRON_PLAN_NATURAL_ORDER is given.
 * With the split forms, up to three small modes (m_mu, n_mu <= 32) applied one
 * after the other on neighbouring indices mu, mu + 1, .. run as one fused
 * launch that keeps the intermediates on chip (the first group's input must
 * then be FP32); KRON_PLAN_UNFUSED runs every product as its own launch.
 */
KRON_API kron_status kron_plan_create(kron_plan *plan, int d, const int64_t *m, const int64_t *n,
                             kron_dtype dtype, kron_prec prec, unsigned flags);
KRON_API kron_status kron_plan_destroy(kron_plan plan);
/* Workspace of kron_tucker for this plan. */
KRON_API kron_status kron_plan_workspace_size(kron_plan plan, size_t *bytes);
/* The 0-based mode order the plan applies (d entries). */
KRON_API kron_status kron_plan_order(kron_plan plan, int *order);
/*
 * How kron_tucker runs the chain of this plan: *count launches of mode
 * products, sizes[i] (up to d host entries) the number of mode products the
 * i-th runs, in the plan's order: 1 for a product of its own, 2 or 3 for a
 * fused group of small modes whose intermediates stay on chip.  The paper has
 * no counterpart (its products each go through memory).  Host-only.
 */
KRON_API kron_status kron_plan_launches(kron_plan plan, int *sizes, int *count);
/* Algorithmic FLOPs of one Tucker operator of this plan (see header comment). */
KRON_API double kron_plan_flops(kron_plan plan);

/*
 * S = T x_1 op(L_1) x_2 ... x_d op(L_d)   (Eq. (tuckerop); Eq. (nestedmumode)
 * element-wise; vec(S) = (L_d (x) ... (x) L_1) vec(T), Lemma "krontomu").
 * L[mu] / ldL[mu]: host arrays of d device pointers / leading dimensions.
 */
KRON_API kron_status kron_tucker(kron_plan plan, const void *T, const void *const *L,
                        const int64_t *ldL, void *S, void *ws, size_t ws_bytes,
                        kron_stream_t stream);

/*
 * Adjoint of the Tucker operator, for S = T x_1 L_1 ... x_d L_d (the plan must
 * not carry KRON_PLAN_TRANS_L).  Given the cotangent dS (sizes n):
 *   dT = dS x_1 L_1^T ... x_d L_d^T   (Appendix A, property 5, transposed
 *                                      Kronecker form of Lemma "krontomu");
 *   dL_mu = G_{mu+1}^{(mu)} (X_mu^{(mu)})^T  (from Eq. (mmp)), where
 *   X_mu = T x_1 L_1 ... x_{mu-1} L_{mu-1} and G_{mu+1} = dS pulled back
 *   through the modes after mu.  X_mu is recomputed from T, not stored.
 * dT (sizes m) may be NULL; dL[mu] (n_mu x m_mu, ld n_mu) may be NULL per mode
 * (dL itself may be NULL).  The contraction order is fixed (modes 1..d), so
 * results are deterministic.
 */
KRON_API kron_status kron_adjoint_workspace_size(kron_plan plan, size_t *bytes);
KRON_API kron_status kron_tucker_adjoint(kron_plan plan, const void *T, const void *const *L,
                                const int64_t *ldL, const void *dS, void *dT,
                                void *const *dL, void *ws, size_t ws_bytes,
                                kron_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Complex Tucker operator: Eq. (tuckerop) over C; conjugate transposes as   */
/* in the remark after Eq. (tensinterp) (the paper's cttucker)               */
/* ------------------------------------------------------------------------ */
/*
 * S = T x_1 op(L_1) x_2 ... x_d op(L_d) for complex T, L_mu and S, with
 *   op(L) = L     (L is n_mu x m_mu)          plan without KRON_PLAN_TRANS_L,
 *   op(L) = L^T   (L is m_mu x n_mu)          plan with KRON_PLAN_TRANS_L, conj = 0,
 *   op(L) = L^*   (conjugate transpose)       plan with KRON_PLAN_TRANS_L, conj = 1,
 * the last being the paper's cttucker: the evaluation of a pseudospectral
 * decomposition at the quadrature points with Phi_mu = Psi_mu^* without
 * forming Phi_mu.  conj = 1 without KRON_PLAN_TRANS_L gives op(L) = conj(L).
 * Storage: complex values as interleaved (real, imaginary) pairs of the
 * plan's dtype (KRON_F64: complex double, KRON_F32: complex float);
 * tensors column-major with the plan's sizes m (T) and n (S) counted in
 * complex elements; ldL[mu] in complex elements.  Pointers aligned to one
 * complex element.  Each complex mu-mode product runs as one real
 * contraction of twice the length over the (real, imaginary) view of the
 * tensor, with the real 2n_mu x 2m_mu matrix [[Re G, -Im G], [Im G, Re G]]
 * (G = op(L_mu), entries interleaved as the tensor's) built in the
 * workspace.  Precisions: KRON_PREC_FP64, FP32, 3XTF32, BF16X3, BF16X6
 * (the fixed-point forms return KRON_ERR_UNSUPPORTED).  T and S must not
 * alias.
 */
KRON_API kron_status kron_ctucker_workspace_size(kron_plan plan, size_t *bytes);
KRON_API kron_status kron_ctucker(kron_plan plan, const void *T, const void *const *L, const int64_t *ldL,
                                  int conj, void *S, void *ws, size_t ws_bytes, kron_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Hermite--Laguerre--Fourier transform matrices (the HLF decomposition of   */
/* the paper's pseudospectral example; used through Eq. (tensinterp))        */
/* ------------------------------------------------------------------------ */
/*
 * Quadrature rules (host arrays x, w of length m; FP64; host computation):
 *   kron_gauss_hermite: nodes x_k = xi_k / beta of the m-point Gauss rule of
 *     the weight exp(-y^2), and the weights w_k with which
 *     sum_k w_k f(x_k) H_i(x_k) approximates the coefficient of f on the
 *     normalized scaled Hermite function H_i (exact when f H_i is a
 *     product of two such functions of total degree < 2m);
 *   kron_gauss_laguerre: the same for the generalized Laguerre weight
 *     y^alpha exp(-y) (alpha > -1) and the functions L_i below.
 * Nodes by Golub--Welsch (eigenvalues of the Jacobi matrix, implicit QL),
 * weights w_k = 1 / sum_{i<m} phi_i(x_k)^2 (reciprocal Christoffel function
 * of the orthonormal functions).  KRON_ERR_NUMERIC if the iteration fails to
 * converge.
 *
 * Function matrices (device, FP64; x device array of n points):
 *   H_i(x) = sqrt(beta / (sqrt(pi) 2^i i!)) H_i^phys(beta x) exp(-beta^2 x^2 / 2),
 *   L_i(x) = sqrt(beta i! / Gamma(i + alpha + 1)) L_i^alpha(beta x)
 *            (beta x)^(alpha / 2) exp(-beta x / 2)     (x >= 0),
 * i = 0 .. m-1 (the paper's i_mu - 1), orthonormal in L^2(R) / L^2(R+).
 * trans = 0: F[l + ldF i] = phi_i(x_l) (n x m, the evaluation matrix Phi);
 * trans = 1: F[i + ldF l] (m x n, the transform matrix Psi when x are the
 * nodes).  Stream-ordered; overflow-free for any m (scaled recurrences).
 *
 * kron_fourier_resample: the real n x m matrix F[l, j] of the trigonometric
 * interpolation of m equispaced samples of a period (at j/m) evaluated at
 * the n equispaced points l/n (the even-m Nyquist term split symmetrically),
 * i.e. the resampling of an FFT-based interpolation, as a matrix for a
 * mu-mode product.
 */
KRON_API kron_status kron_gauss_hermite(int64_t m, double beta, double *x, double *w);
KRON_API kron_status kron_gauss_laguerre(int64_t m, double alpha, double beta, double *x, double *w);
KRON_API kron_status kron_hermite_functions(int64_t m, double beta, const double *x, int64_t n, double *F,
                                            int64_t ldF, int trans, kron_stream_t stream);
KRON_API kron_status kron_laguerre_functions(int64_t m, double alpha, double beta, const double *x, int64_t n,
                                             double *F, int64_t ldF, int trans, kron_stream_t stream);
KRON_API kron_status kron_fourier_resample(int64_t m, int64_t n, double *F, int64_t ldF, kron_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Action of a Kronecker sum: Section 2, Eq. (actkron)                       */
/* ------------------------------------------------------------------------ */
/*
 * S = sum_mu V x_mu op(L_mu), i.e. vec(S) = (L_d (+) ... (+) L_1) vec(V)
 * (Eq. (actkron); Appendix A for the Kronecker sum), without forming the
 * Kronecker sum.  The plan must be square (m == n); its precision and the
 * flag KRON_PLAN_TRANS_L apply as for kron_tucker.  The d mu-mode products
 * all read V; the first writes S and the others accumulate into it, in mode
 * order 1..d (results are deterministic).  V and S must not alias.
 */
KRON_API kron_status kron_kronsumv_workspace_size(kron_plan plan, size_t *bytes);
KRON_API kron_status kron_kronsumv(kron_plan plan, const void *V, const void *const *L, const int64_t *ldL,
                                   void *S, void *ws, size_t ws_bytes, kron_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Inverse Tucker operator (preconditioner): Section 3.4, Eqs. (prec),       */
/* (preconnd)                                                                */
/* ------------------------------------------------------------------------ */
/*
 * S = V x_1 op(P_1)^{-1} x_2 ... x_d op(P_d)^{-1}, i.e.
 * vec(S) = (op(P_d) (x) ... (x) op(P_1))^{-1} vec(V)  (Eq. (preconnd) with
 * Lemma "krontomu"; op as set by KRON_PLAN_TRANS_L).  The plan must be square
 * (m == n, every n_mu <= 1024); P_mu are device matrices of the plan's dtype
 * with leading dimensions ldP[mu].  The P_mu are inverted in FP64 on the GPU
 * (Gauss-Jordan with partial pivoting, one launch for all modes); the chain
 * of inverses runs in the plan's precision; then `refine` (0..8) steps of
 * iterative refinement: R = V - S x_1 op(P_1) ... x_d op(P_d) in FP64 and
 * S += R x_1 op(P_1)^{-1} ... x_d op(P_d)^{-1} in the plan's precision.
 * A zero pivot (singular P_mu) sets KRON_ERR_NUMERIC in the device error word
 * (kron_get_device_error).  V and S must not alias.
 */
KRON_API kron_status kron_itucker_workspace_size(kron_plan plan, int refine, size_t *bytes);
KRON_API kron_status kron_itucker(kron_plan plan, const void *V, const void *const *P, const int64_t *ldP,
                                  int refine, void *S, void *ws, size_t ws_bytes, kron_stream_t stream);

/*
 * Preconditioned conjugate gradients for M x = b with the Kronecker-sum
 * matrix M = M_d (+) ... (+) M_1 (symmetric positive definite) and the
 * ADI-type preconditioner P = P_d (x) ... (x) P_1 (Section 3.4, Eq. (prec);
 * Section 4.5): M v by kron_kronsumv, P^{-1} v by kron_itucker (no
 * refinement).  P == NULL runs plain CG.  X holds the initial guess on entry
 * and the solution on return; B and X (sizes n, the plan's dtype) must not
 * alias.  Stops when ||b - M x||_2 <= tol ||b||_2 or after maxit iterations;
 * *iters and *relres (host pointers, may be NULL) receive the iteration count
 * and ||b - M x|| / ||b|| of the returned x (recurrence residual).  Dot
 * products are FP64 with a fixed summation order.  Unlike the other calls,
 * this one synchronises `stream` once per iteration (it reads the residual
 * norm on the host).  The plan's precision applies to the products (FP64 for
 * a solve to FP64 accuracy).
 */
KRON_API kron_status kron_kronsum_pcg_workspace_size(kron_plan plan, int precondition, size_t *bytes);
KRON_API kron_status kron_kronsum_pcg(kron_plan plan, const void *const *M, const int64_t *ldM,
                                      const void *const *P, const int64_t *ldP, const void *B, void *X,
                                      double tol, int maxit, int *iters, double *relres, void *ws,
                                      size_t ws_bytes, kron_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Exponential of a Kronecker sum: Section 3.3, Eqs. (expmat), (exptucker)   */
/* ------------------------------------------------------------------------ */
/*
 * E = exp(tau A) for a dense n x n FP64 matrix (device, ld ldA >= n), E dense
 * n x n (ld n), by scaling and squaring with the [13/13] Pade approximant
 * (Higham, SIAM J. Matrix Anal. Appl. 26, 2005), all in FP64 on the GPU; the
 * Pade linear system is solved by Gauss-Jordan elimination with partial
 * pivoting followed by one step of iterative refinement with an FP64
 * residual.  1 <= n <= 1024.
 */
KRON_API kron_status kron_expm_workspace_size(int64_t n, size_t *bytes);
KRON_API kron_status kron_expm(int64_t n, const double *A, int64_t ldA, double tau, double *E,
                      void *ws, size_t ws_bytes, kron_stream_t stream);

/*
 * nsteps steps of u <- exp(tau (A_d (+) ... (+) A_1)) u, i.e. in tensor form
 * U <- U x_1 E_1 x_2 ... x_d E_d with E_mu = exp(tau A_mu) (Eq. (exptucker)).
 * The plan must be square (m == n) and unflagged; U (sizes n) is updated in
 * place, stored with the plan's dtype.  A[mu] are FP64 device matrices with
 * leading dimensions ldA[mu].  The E_mu are computed once per call by
 * kron_expm (FP64); the steps use the plan's precision, split forms keeping
 * the state in FP32 between steps and converting back at the end.  Over many
 * chained steps the FP32-accumulating forms (3XTF32, BF16X3, BF16X6) drift by
 * about 1e-6 per step (9e-5 / 3e-5 after 100 steps at 256^3); the fixed-point
 * forms FX32H and FX32 stay within 2e-6 (1.4e-7 / 6.8e-8).
 * kron_expkronsum_apply does the same with given E_mu (FP64, ld ldE[mu]).
 */
KRON_API kron_status kron_expkronsum_workspace_size(kron_plan plan, size_t *bytes);
KRON_API kron_status kron_expkronsum_step(kron_plan plan, const double *const *A, const int64_t *ldA,
                                 double tau, int nsteps, void *U, void *ws, size_t ws_bytes,
                                 kron_stream_t stream);
KRON_API kron_status kron_expkronsum_apply(kron_plan plan, const double *const *E, const int64_t *ldE,
                                  int nsteps, void *U, void *ws, size_t ws_bytes,
                                  kron_stream_t stream);

/*
 * kron_expkronsum_step for a state held in host memory (an addition for
 * callers whose data lives on the host; the paper's operation is the one
 * above).  U_in: host, sizes n, the plan's dtype, column-major; it is copied
 * into the device buffer U_dev (same size, the caller's), the steps run on
 * U_dev as in kron_expkronsum_step, and the result is copied to U_out (host;
 * may be U_in).  The copy to the device runs on a stream of the library's
 * own (one per device), forked from `stream` after its earlier work and
 * joined back before the state is first read, so it overlaps the
 * exponentials and the images of E when U_in is page-locked; from pageable
 * memory the copy is not asynchronous.  The call only enqueues: U_out is
 * complete, and U_in and U_dev may be reused, once `stream` has completed.
 * Errors: KRON_ERR_INVALID_ARG for null pointers, KRON_ERR_ALIGNMENT for an
 * unaligned U_dev, otherwise those of kron_expkronsum_step.
 */
KRON_API kron_status kron_expkronsum_step_host(kron_plan plan, const double *const *A,
                                      const int64_t *ldA, double tau, int nsteps,
                                      const void *U_in, void *U_out, void *U_dev, void *ws,
                                      size_t ws_bytes, kron_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batched Tucker operators (Section 3.2, Eq. (tensinterp); Section 4.3)     */
/* ------------------------------------------------------------------------ */
/*
 * Many independent Tucker operators of possibly different sizes (same d,
 * dtype, precision) in one persistent kernel launch.  The plan fixes the
 * shapes; bind uploads the pointer tables of one set of operands into the
 * workspace; run launches the work (one L-splitting launch and one persistent
 * launch), so a bound run can be captured in a CUDA graph and replayed.
 *   m, n     : host arrays batch*d (row b holds the sizes of problem b).
 *   T[b]     : input of problem b;  S[b]: output;  L[b*d + mu]: L_mu of b,
 *              dense with ld n (no transpose).
 * Split precisions only (3XTF32, BF16X3, BF16X6).  1 <= batch <= 65536.
 */
typedef struct kron_batched_plan_s *kron_batched_plan;
KRON_API kron_status kron_batched_plan_create(kron_batched_plan *plan, int batch, int d,
                                     const int64_t *m, const int64_t *n, kron_dtype dtype,
                                     kron_prec prec, unsigned flags);
KRON_API kron_status kron_batched_plan_destroy(kron_batched_plan plan);
KRON_API kron_status kron_batched_workspace_size(kron_batched_plan plan, size_t *bytes);
KRON_API double kron_batched_flops(kron_batched_plan plan);
KRON_API kron_status kron_batched_bind(kron_batched_plan plan, const void *const *T,
                              const void *const *L, void *const *S, void *ws,
                              size_t ws_bytes, kron_stream_t stream);
KRON_API kron_status kron_batched_run(kron_batched_plan plan, void *ws, size_t ws_bytes,
                             kron_stream_t stream);

/*
 * Autotuning of a bound plan (the paper has no counterpart; Section 3.2 and
 * Section 4.3 give the workload).  Times candidate launch configurations of
 * the persistent kernel on the bound operands -- N-tile width cap 32, 64 or
 * 128 (64 at most for BF16X6), 2 pipeline stages or as many as fit, 1, 2 or
 * as many accumulator sets per tile as tensor memory allows -- each on three
 * runs after a warm-up, keeps the fastest for later kron_batched_run calls
 * and re-binds the tables into the workspace.  The runs overwrite the bound
 * outputs S.  If the environment variable KRON_AUTOTUNE_CACHE names a file,
 * the choice is looked up there first, keyed by the GPU's name, d, batch, a
 * hash of the shapes, dtype and precision (*from_cache = 1 and nothing is
 * timed), and otherwise appended to it as one JSON object per line.  The
 * tile width and the stage count do not change the arithmetic; the number of
 * accumulator sets changes the order of the FP32 sums, so results may differ
 * in the last bits.  Synchronises `stream` (it reads the timings).
 * kron_batched_tuning reports the configuration in use (0: built-in rule).
 */
KRON_API kron_status kron_batched_autotune(kron_batched_plan plan, void *ws, size_t ws_bytes, kron_stream_t stream,
                                           int *from_cache);
KRON_API kron_status kron_batched_tuning(kron_batched_plan plan, int *bn_cap, int *stages, int *nacc);

/*
 * One-shot form of the above (Section 3.2, Eq. (tensinterp)): plans, binds
 * and runs in one call, S[b] = T[b] x_1 L[b][0] ... x_d L[b][d-1] for every
 * problem b.  m, n: host arrays batch*d as for kron_batched_plan_create;
 * T, S: host arrays of batch device pointers; L: host array of batch host
 * arrays of d device pointers (L[b][mu] dense, ld n).  The workspace (size
 * from kron_tucker_batched_workspace_size) receives the job tables, copied
 * from pageable host memory on `stream` (the copy has read them when the call
 * returns); no device or pinned memory is allocated.  Each call rebuilds the
 * plan on the host, so for repeated runs of the same shapes (and for stream
 * capture) use the plan / bind / run calls.  Same precisions and limits.
 */
KRON_API kron_status kron_tucker_batched_workspace_size(int batch, int d, const int64_t *m, const int64_t *n,
                                                        kron_dtype dtype, kron_prec prec, size_t *bytes);
KRON_API kron_status kron_tucker_batched(int batch, int d, const int64_t *m, const int64_t *n,
                                         const void *const *T, const void *const *const *L, void *const *S,
                                         kron_dtype dtype, kron_prec prec, void *ws, size_t ws_bytes,
                                         kron_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* KRON_H */
