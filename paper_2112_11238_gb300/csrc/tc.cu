// tc.cu -- split-precision contractions on the sm_103a tensor cores.
//
// One kernel template covers every contraction of the Tucker chain (Eq. (mmp)
// applied mode by mode, Definition "Tucker operator") and the adjoint's dL:
//
//     C[r, c] = sum_k A[r, k] * B[k, c]
//
// * A rows are fibres of the tensor operand, read straight from the column-
//   major tensor through a 2-level index map (no permute; the slab view of
//   the mu-unfolding is an index map, cf. the remark on permutations in
//   Section 2).  Converter warps load a 128 x BK tile, split every value into
//   TF32 or BF16 pieces and write each piece K-major with the 64-byte
//   swizzle into shared memory.
// * B (the small matrix op(L_mu)) is split and swizzled once per call into a
//   global "image" laid out exactly like its shared-memory tiles, and one
//   bulk copy (TMA unit) per pipeline stage brings a tile in.  For the
//   adjoint's dL both operands come from tensors and both are converted.
// * One thread issues tcgen05.mma for every (piece_a, piece_b) product of the
//   form, small products first, into an FP32 accumulator in tensor memory.
// * Four warps read the accumulator back with tcgen05.ld and store C through
//   its index map (FP32 or FP64).
//
// Pipelining: `stages` shared-memory stages guarded by full/empty mbarriers;
// every wait is bounded (ptx.cuh) so a fault never hangs the GPU.
#include <algorithm>
#include <mutex>

#include "tc_common.cuh"

namespace kron {

constexpr int kConvWarps = 16;      // converter warps
constexpr int kThreads = 64 + 32 * kConvWarps;

struct TcDev {
    const void *A;
    IdxMap rowA, kA;
    int64_t M;
    const void *B;
    IdxMap colB, kB;
    int64_t N;
    const uint8_t *bimg;
    void *C;
    IdxMap rowC, colC;
    int64_t czstride;  // element offset of C per blockIdx.z (split-K partials)
    int64_t K;
    int64_t KB;        // K-blocks in total
    int64_t kbps;      // K-blocks per blockIdx.z
    int BN;
    int stages;
    int nacc;          // accumulators in tensor memory (K-blocks round-robin)
    int a64, b64, c64, acc;
    int avec;          // A rows are contiguous along k and 16-byte aligned chunks
};

// Converts one R-row tile (rows given by precomputed offsets, -1 = padding)
// for the K-block starting at kbase into `dst` (piece tiles `piece_bytes`
// apart).  KC: the source is contiguous along k (consecutive threads take
// consecutive 16-byte chunks of a row); otherwise consecutive threads take
// consecutive rows.
template <int F, typename Tin, bool KC>
__device__ __forceinline__ void conv_tile(const Tin *__restrict__ src, const int64_t *rowoff, int R,
                                          const IdxMap &km, int64_t kbase, int64_t K, uint8_t *dst,
                                          uint32_t piece_bytes, int t) {
    constexpr int CH = 16 / FT<F>::ELEM;
    const int items = R * kChunks;
    for (int it = t; it < items; it += 32 * kConvWarps) {
        int row, ch;
        if constexpr (KC) {
            ch = it % kChunks;
            row = it / kChunks;
        } else {
            row = it % R;
            ch = it / R;
        }
        uint4 out[FT<F>::PIECES];
        load_split<F, Tin>(src, rowoff[row], km, kbase + ch * CH, K, out);
        const uint32_t off = swz(row, ch);
#pragma unroll
        for (int p = 0; p < FT<F>::PIECES; ++p)
            *reinterpret_cast<uint4 *>(dst + p * piece_bytes + off) = out[p];
    }
}

// Items (row, 16-byte chunk) of the 128-row A tile owned by converter thread t.
constexpr int kItemsA = kBM * kChunks / (32 * kConvWarps);

template <bool KC>
__device__ __forceinline__ void item_of(int it, int R, int &row, int &ch) {
    if constexpr (KC) {
        ch = it % kChunks;
        row = it / kChunks;
    } else {
        row = it % R;
        ch = it / R;
    }
}

template <int F, typename Tin, bool KC>
__device__ __forceinline__ void load_a(const Tin *__restrict__ src, const int64_t *rowoff, const IdxMap &km,
                                       int64_t kbase, int64_t K, bool vec, int t,
                                       Tin (&v)[kItemsA][16 / FT<F>::ELEM]) {
    constexpr int CH = 16 / FT<F>::ELEM;
#pragma unroll
    for (int i = 0; i < kItemsA; ++i) {
        int row, ch;
        item_of<KC>(t + i * 32 * kConvWarps, kBM, row, ch);
        load_chunk<F, Tin>(src, rowoff[row], km, kbase + ch * CH, K, vec, v[i]);
    }
}

template <int F, typename Tin, bool KC>
__device__ __forceinline__ void store_a(const Tin (&v)[kItemsA][16 / FT<F>::ELEM], uint8_t *dst, int t) {
#pragma unroll
    for (int i = 0; i < kItemsA; ++i) {
        int row, ch;
        item_of<KC>(t + i * 32 * kConvWarps, kBM, row, ch);
        uint4 out[FT<F>::PIECES];
        split_pack<F, Tin>(v[i], out);
        const uint32_t off = swz(row, ch);
#pragma unroll
        for (int q = 0; q < FT<F>::PIECES; ++q)
            *reinterpret_cast<uint4 *>(dst + q * (kBM * kRowBytes) + off) = out[q];
    }
}

// The converter warps' main loop for one source type: the loads of K-block
// kb+1 are issued right after K-block kb is handed to the MMA warp, so they
// are in flight while the warp waits for the next free stage.
template <int F, typename Tin, bool AKC, bool BIMG, bool BKC>
__device__ __forceinline__ void converter_loop(const TcDev &p, const Tin *__restrict__ A, const int64_t *rowA,
                                               const int64_t *rowB, uint8_t *sA, uint8_t *sB, uint64_t *full,
                                               uint64_t *empty, int64_t kb0, int64_t nkb, int S, uint32_t A_ST,
                                               uint32_t B_ST, uint32_t PIECE_B, int BN, int lane, int t) {
    constexpr int BK = kRowBytes / FT<F>::ELEM;
    Tin v[kItemsA][16 / FT<F>::ELEM];
    const bool vec = p.avec != 0;
    if (nkb > 0) load_a<F, Tin, AKC>(A, rowA, p.kA, kb0 * BK, p.K, vec, t, v);
    for (int64_t kb = 0; kb < nkb; ++kb) {
        const int s = (int)(kb % S);
        const uint32_t ph = (uint32_t)((kb / S) & 1);
        // lane 0 waits, the warp follows (keeps the warp converged)
        int ok = (lane == 0) ? (int)mbar_wait(smem_u32(&empty[s]), ph ^ 1u) : 1;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        const int64_t kbase = (kb0 + kb) * BK;
        store_a<F, Tin, AKC>(v, sA + (size_t)s * A_ST, t);
        if constexpr (!BIMG) {
            uint8_t *dB = sB + (size_t)s * B_ST;
            if (p.b64)
                conv_tile<F, double, BKC>(static_cast<const double *>(p.B), rowB, BN, p.kB, kbase, p.K, dB,
                                          PIECE_B, t);
            else
                conv_tile<F, float, BKC>(static_cast<const float *>(p.B), rowB, BN, p.kB, kbase, p.K, dB,
                                         PIECE_B, t);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&full[s]));
        if (kb + 1 < nkb) load_a<F, Tin, AKC>(A, rowA, p.kA, kbase + BK, p.K, vec, t, v);
    }
}

template <int F, bool AKC, bool BIMG, bool BKC>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(const TcDev p) {
    using T = FT<F>;
    constexpr int BK = kRowBytes / T::ELEM;
    constexpr uint32_t PIECE_A = kBM * kRowBytes;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_align1024(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int BN = p.BN, S = p.stages;
    const uint32_t A_ST = T::PIECES * PIECE_A;
    const uint32_t PIECE_B = (uint32_t)BN * kRowBytes;
    const uint32_t B_ST = T::PIECES * PIECE_B;
    uint8_t *sA = smem;
    uint8_t *sB = smem + (size_t)S * A_ST;
    int64_t *rowA = reinterpret_cast<int64_t *>(sB + (size_t)S * B_ST);
    int64_t *rowB = rowA + kBM;
    int64_t *rowC = rowB + 256;
    uint64_t *bars = reinterpret_cast<uint64_t *>(rowC + kBM);
    uint64_t *full = bars, *empty = bars + S, *accf = bars + 2 * S;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * S + 1);
    const uint32_t acc_cols = BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u));
    const int NACC = p.nacc;
    // per accumulator a: region 2a holds the hi*hi products, region 2a+1 the
    // smaller cross products (truncation in the FP32 accumulation then only
    // touches the big sum once per k-step)
    const uint32_t ncols = acc_cols * (uint32_t)NACC * 2u;

    const int64_t row0 = (int64_t)blockIdx.x * kBM;
    const int64_t n0 = (int64_t)blockIdx.y * BN;
    const int64_t kb0 = (int64_t)blockIdx.z * p.kbps;
    const int64_t nkb = min(p.KB, kb0 + p.kbps) - kb0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full[s]), kConvWarps + (BIMG ? 1 : 0));
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(accf), 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tslot), ncols);
        tmem_relinquish();
    }
    if (warp >= 2) {
        const int t = threadIdx.x - 64;
        for (int r = t; r < kBM; r += 32 * kConvWarps) {
            const int64_t rg = row0 + r;
            rowA[r] = rg < p.M ? imap(p.rowA, rg) : -1;
            rowC[r] = rg < p.M ? imap(p.rowC, rg) : -1;
        }
        if constexpr (!BIMG) {
            for (int r = t; r < BN; r += 32 * kConvWarps) {
                const int64_t cg = n0 + r;
                rowB[r] = cg < p.N ? imap(p.colB, cg) : -1;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if constexpr (BIMG) {
            if (lane == 0) {
                const uint8_t *img = p.bimg + (size_t)blockIdx.y * p.KB * B_ST;
                for (int64_t kb = 0; kb < nkb; ++kb) {
                    const int s = (int)(kb % S);
                    const uint32_t ph = (uint32_t)((kb / S) & 1);
                    if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u)) break;
                    mbar_arrive_expect_tx(smem_u32(&full[s]), B_ST);
                    bulk_g2s(smem_u32(sB + (size_t)s * B_ST), img + (size_t)(kb0 + kb) * B_ST, B_ST,
                             smem_u32(&full[s]));
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = make_idesc(T::FMT, kBM, (uint32_t)BN);
            bool ok = true;
            for (int64_t kb = 0; kb < nkb; ++kb) {
                const int s = (int)(kb % S);
                const uint32_t ph = (uint32_t)((kb / S) & 1);
                if (!mbar_wait(smem_u32(&full[s]), ph)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int64_t kval = min((int64_t)BK, p.K - (kb0 + kb) * BK);
                const int ksteps = (int)((kval + T::MMA_K - 1) / T::MMA_K);
                const uint32_t a_base = smem_u32(sA + (size_t)s * A_ST);
                const uint32_t b_base = smem_u32(sB + (size_t)s * B_ST);
                // K-block kb accumulates into accumulator kb % NACC, which
                // starts fresh on its first K-block.
                const uint32_t dhi = tmem + (uint32_t)(kb % NACC) * 2u * acc_cols;
                const uint32_t dlo = dhi + acc_cols;
                const bool fresh = kb < NACC;
                for (int ks = 0; ks < ksteps; ++ks) {
#pragma unroll
                    for (int pr = 0; pr < T::NPROD; ++pr) {
                        int pa, pb;
                        prod_pieces<F>(pr, pa, pb);
                        const uint64_t ad =
                            smem_desc_kmajor(a_base + pa * PIECE_A + ks * 32, kRowBytes);
                        const uint64_t bd =
                            smem_desc_kmajor(b_base + pb * PIECE_B + ks * 32, kRowBytes);
                        // hi*hi is the last product; the cross products come first
                        const bool is_hi = (pr == T::NPROD - 1);
                        const bool first = fresh && ks == 0 && (is_hi || pr == 0);
                        tc_mma<T::KIND>(is_hi ? dhi : dlo, ad, bd, idesc, first ? 0u : 1u);
                    }
                }
                tc_commit(smem_u32(&empty[s]));
            }
            if (ok) tc_commit(smem_u32(accf));
        }
        __syncwarp();
    } else {
        const int t = threadIdx.x - 64;
        if (p.a64)
            converter_loop<F, double, AKC, BIMG, BKC>(p, static_cast<const double *>(p.A), rowA, rowB, sA, sB, full,
                                                      empty, kb0, nkb, S, A_ST, B_ST, PIECE_B, BN, lane, t);
        else
            converter_loop<F, float, AKC, BIMG, BKC>(p, static_cast<const float *>(p.A), rowA, rowB, sA, sB, full,
                                                     empty, kb0, nkb, S, A_ST, B_ST, PIECE_B, BN, lane, t);
        // Epilogue: warps 2..5 cover the four 32-lane quarters of the accumulator.
        if (warp < 6) {
            int ok = (lane == 0) ? (int)mbar_wait(smem_u32(accf), 0) : 1;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            tc_fence_after();
            if (ok) {
                const int q = warp & 3;
                const int r = q * 32 + lane;
                const int64_t ro = rowC[r];
                const int64_t zoff = (int64_t)blockIdx.z * p.czstride;
                const int used = (int)min((int64_t)NACC, nkb);
                const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
                for (int c0 = 0; c0 < BN; c0 += 16) {
                    // fixed-order FP32 sum: per accumulator (cross + hi), then
                    // the accumulators in order
                    float sum[16];
                    for (int a = 0; a < used; ++a) {
                        uint32_t vh[16], vl[16];
                        tmem_ld16(lane_base + (uint32_t)(2 * a * acc_cols + c0), vh);
                        tmem_ld16(lane_base + (uint32_t)((2 * a + 1) * acc_cols + c0), vl);
                        tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const float v = __uint_as_float(vl[e]) + __uint_as_float(vh[e]);
                            sum[e] = (a == 0) ? v : sum[e] + v;
                        }
                    }
                    if (ro >= 0) {
                        const int cmax = (int)max((int64_t)0, min((int64_t)16, p.N - n0 - c0));
                        if (p.c64) store_row16<double>(static_cast<double *>(p.C) + zoff, ro, p.colC, n0 + c0, cmax, sum, p.acc != 0);
                        else store_row16<float>(static_cast<float *>(p.C) + zoff, ro, p.colC, n0 + c0, cmax, sum, p.acc != 0);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

// Builds the pre-split, pre-swizzled global image of B:
//   image[nt][kb][piece][BN rows x 64 bytes]   (row = output column c).
template <int F, typename Tin>
__global__ void bimage_kernel(const Tin *__restrict__ B, IdxMap colB, IdxMap kB, int64_t N, int64_t K,
                              int BN, int64_t KB, int64_t NT, uint8_t *img) {
    using T = FT<F>;
    constexpr int BK = kRowBytes / T::ELEM;
    constexpr int CH = 16 / T::ELEM;
    const int64_t total = NT * KB * BN * kChunks;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(idx % kChunks);
        int64_t rest = idx / kChunks;
        const int row = (int)(rest % BN);
        rest /= BN;
        const int64_t kb = rest % KB;
        const int64_t nt = rest / KB;
        const int64_t cg = nt * BN + row;
        const int64_t ro = cg < N ? imap(colB, cg) : -1;
        uint4 out[T::PIECES];
        load_split<F, Tin>(B, ro, kB, kb * BK + ch * CH, K, out);
        uint8_t *base = img + (size_t)((nt * KB + kb) * T::PIECES) * BN * kRowBytes;
        const uint32_t off = swz(row, ch);
#pragma unroll
        for (int q = 0; q < T::PIECES; ++q)
            *reinterpret_cast<uint4 *>(base + (size_t)q * BN * kRowBytes + off) = out[q];
    }
}

// Several images in one launch (up to KRON_MAX_D), the same bytes as
// bimage_kernel builds for each: the items of image j follow those of j - 1.
struct BimageSet {
    const void *B[KRON_MAX_D];
    IdxMap colB[KRON_MAX_D], kB[KRON_MAX_D];
    int64_t N[KRON_MAX_D], K[KRON_MAX_D], KB[KRON_MAX_D], begin[KRON_MAX_D + 1];
    uint8_t *img[KRON_MAX_D];
    int BN[KRON_MAX_D], b64[KRON_MAX_D];
    int count;
};

template <int F>
__global__ void bimage_set_kernel(const __grid_constant__ BimageSet S) {
    using T = FT<F>;
    constexpr int BK = kRowBytes / T::ELEM;
    constexpr int CH = 16 / T::ELEM;
    const int64_t total = S.begin[S.count];
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int j = 0;
        while (j + 1 < S.count && S.begin[j + 1] <= idx) ++j;
        const int BN = S.BN[j];
        const int64_t KB = S.KB[j];
        int64_t rest = idx - S.begin[j];
        const int ch = (int)(rest % kChunks);
        rest /= kChunks;
        const int row = (int)(rest % BN);
        rest /= BN;
        const int64_t kb = rest % KB;
        const int64_t nt = rest / KB;
        const int64_t cg = nt * BN + row;
        const int64_t ro = cg < S.N[j] ? imap(S.colB[j], cg) : -1;
        uint4 out[T::PIECES];
        if (S.b64[j]) load_split<F, double>(static_cast<const double *>(S.B[j]), ro, S.kB[j], kb * BK + ch * CH, S.K[j], out);
        else load_split<F, float>(static_cast<const float *>(S.B[j]), ro, S.kB[j], kb * BK + ch * CH, S.K[j], out);
        uint8_t *base = S.img[j] + (size_t)((nt * KB + kb) * T::PIECES) * BN * kRowBytes;
        const uint32_t off = swz(row, ch);
#pragma unroll
        for (int q = 0; q < T::PIECES; ++q)
            *reinterpret_cast<uint4 *>(base + (size_t)q * BN * kRowBytes + off) = out[q];
    }
}

// Fixed-order sum of split-K partials: C[r, c] (+)= sum_z P[z][r + M c].
// Sum of the split-K partials, in FP64 and in a fixed order (deterministic):
// a block takes 32 consecutive outputs; its thread (o, g) sums the splits
// z = g, g + 32, .. of output o in ascending z (loads of a warp: 32
// consecutive outputs of one split), then the 32 sums of an output are
// added in ascending g.
constexpr int kRedOut = 32, kRedGroups = 32;

__global__ void __launch_bounds__(kRedOut * kRedGroups) splitk_reduce_kernel(const float *__restrict__ P,
                                                                             int64_t splits, int64_t M, int64_t N,
                                                                             void *C, IdxMap rowC, IdxMap colC,
                                                                             int c64, int acc) {
    __shared__ double part[kRedGroups][kRedOut + 1];
    const int64_t total = M * N;
    const int o = threadIdx.x % kRedOut, g = threadIdx.x / kRedOut;
    for (int64_t base = (int64_t)blockIdx.x * kRedOut; base < total; base += (int64_t)gridDim.x * kRedOut) {
        const int64_t idx = base + o;
        double s = 0.0;
        if (idx < total)
            for (int64_t z = g; z < splits; z += kRedGroups) s += (double)P[z * total + idx];
        part[g][o] = s;
        __syncthreads();
        if (g == 0 && idx < total) {
            double t = 0.0;
            for (int h = 0; h < kRedGroups; ++h) t += part[h][o];
            const int64_t r = idx % M, c = idx / M;
            const int64_t off = imap(rowC, r) + imap(colC, c);
            if (c64) {
                double *d = static_cast<double *>(C) + off;
                *d = acc ? *d + t : t;
            } else {
                float *d = static_cast<float *>(C) + off;
                *d = acc ? (float)((double)*d + t) : (float)t;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host

cudaError_t tc_error_word(unsigned int *out, bool clear, cudaStream_t st) { return read_error_word(out, clear, st); }

static int pieces_of(int form) { return form == kFX32 ? 4 : ((form == kBF16x6 || form == kFX32H) ? 3 : 2); }
static int bk_of(int form) { return form == kTF32x3 ? kRowBytes / 4 : kRowBytes / 2; }
static int max_bn(int form) { return form == kBF16x6 ? 64 : (is_fx_form(form) ? 256 : 128); }

int tc_tile_n(int form, int64_t N) { return tc_tile_n_cap(form, N, 1 << 20); }

int tc_tile_n_cap(int form, int64_t N, int cap) {
    const int64_t mx = std::max<int64_t>(16, std::min<int64_t>(max_bn(form), cap));
    const int64_t nt = (N + mx - 1) / mx;
    int64_t bn = (N + nt - 1) / nt;
    bn = (bn + 15) / 16 * 16;
    return (int)std::max<int64_t>(bn, 16);
}

size_t tc_bimage_bytes(int form, int64_t N, int64_t K) { return tc_bimage_bytes_bn(form, N, K, tc_tile_n(form, N)); }

size_t tc_bimage_bytes_bn(int form, int64_t N, int64_t K, int bn) {
    const int64_t nt = (N + bn - 1) / bn;
    const int64_t kb = (K + bk_of(form) - 1) / bk_of(form);
    return (size_t)(nt * kb * pieces_of(form)) * bn * kRowBytes;
}

static size_t stage_bytes(int form, int bn) { return (size_t)pieces_of(form) * (kBM + bn) * kRowBytes; }
static size_t extra_bytes(int stages) { return 1024 + (kBM + 256 + kBM) * 8 + (2 * stages + 2) * 8; }
static constexpr size_t kSmemLimit = 227 * 1024;

static int pick_stages(int form, int bn, int64_t kb) {
    const size_t sb = stage_bytes(form, bn);
    int s = 1;
    while (s < 6 && (size_t)(s + 1) * sb + extra_bytes(s + 1) <= kSmemLimit) ++s;
    return (int)std::max<int64_t>(1, std::min<int64_t>(s, kb));
}

// Dynamic shared memory to request: at least `need`, and enough that the
// CTAs resident on one SM never ask for more than the 512 TMEM columns.
static int acc_cols_of(int bn) { return bn <= 32 ? 32 : (bn <= 64 ? 64 : (bn <= 128 ? 128 : 256)); }

// Accumulators per CTA: up to 4, within the 512 TMEM columns, never more
// than the K-blocks a CTA runs.
static int pick_nacc(int bn, int64_t kblocks) {
    // a power of two, so that the allocated columns are one
    const int64_t byc = 512 / (2 * acc_cols_of(bn));
    int64_t want = 1;
    while (want < kblocks && want < 4) want *= 2;
    return (int)std::min<int64_t>(want, byc);
}

static size_t smem_request(size_t need, int bn, int nacc) {
    const int ncols = acc_cols_of(bn) * nacc * 2;
    const size_t allowed = 512 / ncols;                  // CTAs whose columns fit
    const size_t sm_bytes = 228 * 1024;                  // shared memory of one SM
    const size_t floor_bytes = sm_bytes / (allowed + 1) + 1;
    return std::min(kSmemLimit, std::max(need, floor_bytes));
}

template <typename K>
static cudaError_t set_smem_attr(K kernel) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
}

static bool kcontig(const IdxMap &k) { return k.s0 == 1 && k.R0 != 1; }

template <int F, bool AKC, bool BIMG, bool BKC>
static cudaError_t launch_tc(const TcDev &d, dim3 grid, size_t smem, cudaStream_t st) {
    auto kern = tc_gemm_kernel<F, AKC, BIMG, BKC>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] { attr_err = set_smem_attr(kern); });
    if (attr_err != cudaSuccess) return attr_err;
    kern<<<grid, kThreads, smem, st>>>(d);
    return cudaGetLastError();
}

template <int F>
static cudaError_t dispatch_tc(const TcDev &d, bool akc, bool bimg, bool bkc, dim3 grid, size_t smem,
                               cudaStream_t st) {
    if (bimg) {
        return akc ? launch_tc<F, true, true, false>(d, grid, smem, st)
                   : launch_tc<F, false, true, false>(d, grid, smem, st);
    }
    if (akc && bkc) return launch_tc<F, true, false, true>(d, grid, smem, st);
    if (!akc && !bkc) return launch_tc<F, false, false, false>(d, grid, smem, st);
    if (akc) return launch_tc<F, true, false, false>(d, grid, smem, st);
    return launch_tc<F, false, false, true>(d, grid, smem, st);
}

static cudaError_t dispatch_form(int form, const TcDev &d, bool akc, bool bimg, bool bkc, dim3 grid,
                                 size_t smem, cudaStream_t st) {
    switch (form) {
        case kTF32x3: return dispatch_tc<kTF32x3>(d, akc, bimg, bkc, grid, smem, st);
        case kBF16x3: return dispatch_tc<kBF16x3>(d, akc, bimg, bkc, grid, smem, st);
        case kBF16x6: return dispatch_tc<kBF16x6>(d, akc, bimg, bkc, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t tc_build_bimage(int form, const Contraction &c, void *img, cudaStream_t st) {
    return tc_build_bimage_bn(form, c, img, tc_tile_n(form, c.N), st);
}

cudaError_t tc_build_bimage_bn(int form, const Contraction &c, void *img, int bn, cudaStream_t st) {
    const int64_t nt = (c.N + bn - 1) / bn;
    const int64_t kb = (c.K + bk_of(form) - 1) / bk_of(form);
    const int64_t total = nt * kb * bn * kChunks;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 152 * 16);
    auto *out = static_cast<uint8_t *>(img);
#define KRON_BIMG(FF)                                                                          \
    if (c.B_f64)                                                                               \
        bimage_kernel<FF, double><<<(unsigned)blocks, threads, 0, st>>>(                       \
            static_cast<const double *>(c.B), c.colB, c.kB, c.N, c.K, bn, kb, nt, out);        \
    else                                                                                       \
        bimage_kernel<FF, float><<<(unsigned)blocks, threads, 0, st>>>(                        \
            static_cast<const float *>(c.B), c.colB, c.kB, c.N, c.K, bn, kb, nt, out);
    switch (form) {
        case kTF32x3: KRON_BIMG(kTF32x3) break;
        case kBF16x3: KRON_BIMG(kBF16x3) break;
        case kBF16x6: KRON_BIMG(kBF16x6) break;
        default: return cudaErrorInvalidValue;
    }
#undef KRON_BIMG
    return cudaGetLastError();
}

cudaError_t tc_build_bimages(int form, int count, const Contraction *cs, void *const *imgs, const int *bns,
                             cudaStream_t st) {
    if (count < 1) return cudaSuccess;
    if (count > KRON_MAX_D) return cudaErrorInvalidValue;
    BimageSet S{};
    S.count = count;
    S.begin[0] = 0;
    for (int j = 0; j < count; ++j) {
        const Contraction &c = cs[j];
        const int bn = bns[j];
        S.B[j] = c.B;
        S.b64[j] = c.B_f64 ? 1 : 0;
        S.colB[j] = c.colB;
        S.kB[j] = c.kB;
        S.N[j] = c.N;
        S.K[j] = c.K;
        S.KB[j] = (c.K + bk_of(form) - 1) / bk_of(form);
        S.BN[j] = bn;
        S.img[j] = static_cast<uint8_t *>(imgs[j]);
        const int64_t nt = (c.N + bn - 1) / bn;
        S.begin[j + 1] = S.begin[j] + nt * S.KB[j] * bn * kChunks;
    }
    const int threads = 256;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((S.begin[count] + threads - 1) / threads, 152 * 16));
    switch (form) {
        case kTF32x3: bimage_set_kernel<kTF32x3><<<(unsigned)blocks, threads, 0, st>>>(S); break;
        case kBF16x3: bimage_set_kernel<kBF16x3><<<(unsigned)blocks, threads, 0, st>>>(S); break;
        case kBF16x6: bimage_set_kernel<kBF16x6><<<(unsigned)blocks, threads, 0, st>>>(S); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

static TcDev make_dev(int form, const Contraction &c, int bn) {
    TcDev d{};
    d.A = c.A;
    d.rowA = c.rowA;
    d.kA = c.kA;
    d.M = c.M;
    d.B = c.B;
    d.colB = c.colB;
    d.kB = c.kB;
    d.N = c.N;
    d.C = c.C;
    d.rowC = c.rowC;
    d.colC = c.colC;
    d.K = c.K;
    d.KB = (c.K + bk_of(form) - 1) / bk_of(form);
    d.kbps = d.KB;
    d.BN = bn;
    d.a64 = c.A_f64;
    d.b64 = c.B_f64;
    d.c64 = c.C_f64;
    d.acc = c.accumulate;
    {
        const int64_t v = c.A_f64 ? 2 : 4;  // elements per 16 bytes
        const bool unit_k = c.kA.R0 == 0 && c.kA.s0 == 1;
        const bool rows_ok = (c.rowA.s0 % v == 0) && (c.rowA.R0 == 0 || c.rowA.s1 % v == 0);
        const bool base_ok = (reinterpret_cast<uintptr_t>(c.A) % 16) == 0;
        d.avec = (unit_k && rows_ok && base_ok) ? 1 : 0;
    }
    d.czstride = 0;
    return d;
}

cudaError_t tc_contract_bimage(int form, const Contraction &c, const void *img, cudaStream_t st) {
    if (c.M == 0 || c.N == 0) return cudaSuccess;
    const int bn = tc_tile_n(form, c.N);
    TcDev d = make_dev(form, c, bn);
    d.bimg = static_cast<const uint8_t *>(img);
    d.stages = pick_stages(form, bn, d.KB);
    d.nacc = pick_nacc(bn, d.KB);
    const size_t smem = smem_request((size_t)d.stages * stage_bytes(form, bn) + extra_bytes(d.stages), bn, d.nacc);
    const dim3 grid((unsigned)((c.M + kBM - 1) / kBM), (unsigned)((c.N + bn - 1) / bn), 1);
    return dispatch_form(form, d, kcontig(c.kA), true, false, grid, smem, st);
}

static int64_t splitk_count(int64_t M, int64_t N, int64_t K, int form) {
    const int bn = tc_tile_n(form, N);
    const int64_t tiles = ((M + kBM - 1) / kBM) * ((N + bn - 1) / bn);
    const int64_t kb = (K + bk_of(form) - 1) / bk_of(form);
    int64_t splits = (2 * 152 + tiles - 1) / tiles;
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, kb));
    // every split must own at least one K-block
    const int64_t kbps = (kb + splits - 1) / splits;
    return (kb + kbps - 1) / kbps;
}

size_t tc_splitk_partial_bytes(int64_t M, int64_t N, int64_t K) {
    int64_t s = 1;
    for (int f = 0; f < 3; ++f) s = std::max(s, splitk_count(M, N, K, f));
    return (size_t)s * M * N * sizeof(float);
}

cudaError_t tc_contract_splitk(int form, const Contraction &c, float *partial, cudaStream_t st) {
    if (c.M == 0 || c.N == 0) return cudaSuccess;
    const int bn = tc_tile_n(form, c.N);
    TcDev d = make_dev(form, c, bn);
    const int64_t splits = splitk_count(c.M, c.N, c.K, form);
    d.kbps = (d.KB + splits - 1) / splits;
    d.C = partial;
    d.c64 = 0;
    d.acc = 0;
    d.rowC = IdxMap{0, 1, 0};
    d.colC = IdxMap{0, c.M, 0};
    d.czstride = c.M * c.N;
    d.stages = pick_stages(form, bn, d.kbps);
    d.nacc = pick_nacc(bn, d.kbps);
    const size_t smem = smem_request((size_t)d.stages * stage_bytes(form, bn) + extra_bytes(d.stages), bn, d.nacc);
    const dim3 grid((unsigned)((c.M + kBM - 1) / kBM), (unsigned)((c.N + bn - 1) / bn), (unsigned)splits);
    cudaError_t e = dispatch_form(form, d, kcontig(c.kA), false, kcontig(c.kB), grid, smem, st);
    if (e != cudaSuccess) return e;
    const int64_t total = c.M * c.N;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((total + kRedOut - 1) / kRedOut, 4096));
    splitk_reduce_kernel<<<(unsigned)blocks, kRedOut * kRedGroups, 0, st>>>(partial, splits, c.M, c.N, c.C, c.rowC,
                                                                            c.colC, c.C_f64, c.accumulate);
    return cudaGetLastError();
}

}  // namespace kron
