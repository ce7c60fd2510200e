// tcp.cu -- persistent, warp-specialised tensor-core kernel for mu-mode
// products (Eq. (mmp)), used by the Tucker chain, the stepper and the batched
// Tucker operators.
//
// One launch runs a table of "jobs"; each job is one contraction
//     C[r, c] = sum_k A[r, k] * op(L)[c, k]
// with A the tensor read through its index maps and converted/split on the
// fly, and op(L) read from its pre-split, pre-swizzled image.  A job may wait
// for another job of the same launch (the next mode of the same tensor), so a
// whole batch of Tucker operators runs in one launch.
//
// Roles (one CTA per SM, looping over tiles t = blockIdx.x + i * gridDim.x):
//   warp 0        bulk-copies the image tile of op(L) for every K-block
//   warp 1        issues tcgen05.mma (single thread) into tensor memory
//   warps 2..5    epilogue: tensor memory -> registers -> C, one row per thread
//   warps 6..13   converters: A tile (128 rows x one K-block) -> split pieces
//                 in 64-byte-swizzled K-major shared memory
// Stages are guarded by full/empty mbarriers, accumulators by acc_full /
// acc_empty mbarriers; with two accumulator buffers the epilogue of tile i
// overlaps the main loop of tile i+1.  With one (the fixed-point forms: two
// regions of 256 columns fill tensor memory) the MMA waits for the epilogue,
// so the converter warps, idle then, take two thirds of it, staging output
// boxes in the free A stages for TMA stores.  Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "tc_common.cuh"

namespace kron {

namespace {

constexpr int kConv = 8;                            // converter warps
constexpr int kEpi = 4;                             // epilogue warps
constexpr int kConv0 = 2 + kEpi;                      // first converter warp
constexpr int kPThreads = 32 * (kConv0 + kConv);     // 448 threads
constexpr int kItems = kBM * kChunks / (32 * kConv);  // (row, chunk) items per converter thread
constexpr int kMaxInline = 8;

struct TcJob {
    // raw A tiles by TMA (tma != 0): 2 = k-contiguous rows, box (BK, 128);
    // 3 = [slab][k][row] with tmaP rows per slab, box (128, BK, 1)
    CUtensorMap tmA;
    // fixed-point epilogue output by TMA stores of 32-row x 16-column boxes
    // staged in shared memory (tmc != 0): 2 = column-contiguous rows, box
    // (16, 32); 3 = [slab][column][row] with tmcP rows per slab, box (32, 16, 1)
    CUtensorMap tmC;
    int64_t tmaP, tmcP;
    int32_t tma, tmc;
    const void *A;
    IdxMap rowA, kA;
    int64_t M;
    const uint8_t *bimg;
    int64_t kb_img;    // K-blocks per N-tile in the image
    void *C;
    IdxMap rowC, colC;
    int64_t N, K;
    int32_t kb0, nkb;  // K-block range of the job
    int32_t BN;        // N-tile width (image layout)
    int32_t tiles_m, tiles_n, tile_begin;
    int32_t dep, dep_tiles;
    int32_t a64, c64, acc, avec, akc;
    int32_t publish;   // some later job waits for this one
    int32_t cp16;      // 4-byte source: 16-byte asynchronous copies are legal
    // fixed-point form: scale of A, scale of C (when C is fixed point),
    // row exponents of op(L) and the bound of its row sums
    const FxScale *fxA;
    FxScale *fxC;
    const int *fxF;
    const unsigned long long *fxG;
    int32_t cfix;      // C is 32-bit fixed point
};

// Raw (unsplit FP32) A tiles staged by cp.async ahead of the converters.
template <int F>
struct RawCfg {
    static constexpr int BK = kRowBytes / FT<F>::ELEM;
    static constexpr int BYTES = kBM * BK * 4;                 // one K-block of FP32 rows
    static constexpr int UNITS = BYTES / 16 / (32 * kConv);    // 16-byte units per converter thread
    static constexpr int STAGES = (F == kFX32) ? 2 : 4;
};

// Constants of the fixed-point form F: magnitude bits b of its integers
// (|X| < 2^b), the accumulator unit 2^(eA + f_c + UNIT) of a product of two
// fixed-point operands with scales eA and f_c, and the left shift VS of the
// level-0 accumulator in the 64-bit value path.
//   FX32:  four 8-bit digits, slices d_t 2^(-8t), x = 2^24 (sum of slices):
//          b = 31, UNIT = 48 - 62 = -14, level 0 an integer below 2^24.
//   FX32H: three digits (8, 11, 11 bits), slices d0 2^8, d1 2^-3, d2 2^-14,
//          x = 2^14 (sum of slices): b = 29, UNIT = 28 - 58 = -30, level 0 a
//          multiple of 2^16 (above 2^31 for long K: no 32-bit conversion).
template <int F>
struct FxForm {
    static constexpr int BITS = (F == kFX32H) ? 29 : 31;
    static constexpr int UNIT = (F == kFX32H) ? -30 : -14;
    static constexpr int VS = (F == kFX32H) ? 0 : 16;
};

// Left shift that brings the largest magnitude mA of a fixed-point operand to
// the top of the form's range (|X| < 2^b): the scale of every intermediate is
// chosen before its values exist, from a bound (the input's largest value
// times the largest row sum of |op(L)|) that is several times the actual
// largest output, so an intermediate can reach the next product with its top
// bits unused.  Shifted back up, its digit slices are full and the slice
// products left out are as small, relative to the data, as for the input
// tensor.  mA is an upper bound of the stored magnitudes, so the shifted
// values stay below 2^b.
template <int F>
__device__ __forceinline__ int fx_shift(unsigned mA) {
    if (mA == 0u) return 0;
    return max(0, FxForm<F>::BITS - (32 - __clz((int)mA)));
}

struct TcLaunch {
    TcJob inl[kMaxInline];  // small tables travel with the launch (tensor maps included)
    const TcJob *jobs;      // device table (when njobs > kMaxInline)
    int njobs, total_tiles;
    int *done;              // finished tiles per job, then one "a wait gave up" flag (zeroed before the launch)
    FxScale *reset_next;    // fixed point: scale word the next launch writes, cleared here
    int stages, nacc, nbuf, acc_cols, bn_max;
    int dep_hold;                      // test hook: extra tiles every dependency waits for
    unsigned long long dep_wait_ns;    // time limit of a dependency wait
    const int *tile_job;               // device table tile -> job (large job tables), or null
};

__device__ __forceinline__ const TcJob &job_at(const TcLaunch &L, int j) {
    return (L.njobs <= kMaxInline) ? L.inl[j] : L.jobs[j];
}

__device__ __forceinline__ int find_job(const TcLaunch &L, int t) {
    // large tables (the batched operators: thousands of jobs of a few tiles)
    // come with a tile -> job table: one load instead of a search
    if (L.tile_job != nullptr) return __ldg(L.tile_job + t);
    int lo = 0, hi = L.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (job_at(L, mid).tile_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void named_bar(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Item i of converter thread ct: (row, 16-byte chunk) of the 128-row tile.
__device__ __forceinline__ void item_rc(int i, int ct, bool kc, int &row, int &ch) {
    const int it = ct + i * 32 * kConv;
    if (kc) {
        ch = it % kChunks;
        row = it / kChunks;
    } else {
        row = it % kBM;
        ch = it / kBM;
    }
}

template <int F, typename Tin>
__device__ __forceinline__ void conv_load(const TcJob &J, const int64_t (&ro)[kItems], int64_t kbase, int ct,
                                          Tin (&v)[kItems][16 / FT<F>::ELEM]) {
    constexpr int CH = 16 / FT<F>::ELEM;
    const Tin *src = static_cast<const Tin *>(J.A);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int row, ch;
        item_rc(i, ct, J.akc != 0, row, ch);
        load_chunk<F, Tin, true>(src, ro[i], J.kA, kbase + ch * CH, J.K, J.avec != 0, v[i]);
    }
}

template <int F, typename Tin>
__device__ __forceinline__ void conv_store(const TcJob &J, const Tin (&v)[kItems][16 / FT<F>::ELEM], uint8_t *dst,
                                           int ct) {
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int row, ch;
        item_rc(i, ct, J.akc != 0, row, ch);
        uint4 out[FT<F>::PIECES];
        split_pack<F, Tin>(v[i], out);
        const uint32_t off = swz(row, ch);
#pragma unroll
        for (int q = 0; q < FT<F>::PIECES; ++q)
            *reinterpret_cast<uint4 *>(dst + q * (kBM * kRowBytes) + off) = out[q];
    }
}

// Converter warps: one tile's K-blocks; the loads of K-block kb+1 are issued
// right after K-block kb has been handed over.
template <int F, typename Tin>
__device__ __forceinline__ bool conv_tile_loop(const TcJob &J, int mt, uint8_t *sA, uint32_t A_ST, uint64_t *full,
                                               uint64_t *empty, int S, uint32_t &g, int lane, int ct) {
    constexpr int BK = kRowBytes / FT<F>::ELEM;
    int64_t ro[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int row, ch;
        item_rc(i, ct, J.akc != 0, row, ch);
        const int64_t rg = (int64_t)mt * kBM + row;
        ro[i] = rg < J.M ? imap(J.rowA, rg) : -1;
    }
    Tin v[kItems][16 / FT<F>::ELEM];
    conv_load<F, Tin>(J, ro, (int64_t)J.kb0 * BK, ct, v);
    for (int kb = 0; kb < J.nkb; ++kb, ++g) {
        const int s = (int)(g % (uint32_t)S);
        const uint32_t ph = (g / (uint32_t)S) & 1u;
        int ok = (lane == 0) ? (int)mbar_wait(smem_u32(&empty[s]), ph ^ 1u) : 1;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) return false;
        conv_store<F, Tin>(J, v, sA + (size_t)s * A_ST, ct);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&full[s]));
        if (kb + 1 < J.nkb) conv_load<F, Tin>(J, ro, (int64_t)(J.kb0 + kb + 1) * BK, ct, v);
    }
    return true;
}

// Unit u of converter thread ct (16 bytes of the raw FP32 tile): KC tiles are
// stored [row][k], the others [k][row].
template <int F>
__device__ __forceinline__ void raw_unit(int i, int ct, bool kc, int &row, int &k, uint32_t &dst_off) {
    using R = RawCfg<F>;
    const int u = ct + i * 32 * kConv;
    if (kc) {
        const int per_row = R::BK / 4;
        row = u / per_row;
        k = (u % per_row) * 4;
        dst_off = (uint32_t)(row * R::BK + k) * 4u;
    } else {
        k = u / (kBM / 4);
        row = (u % (kBM / 4)) * 4;
        dst_off = (uint32_t)(k * kBM + row) * 4u;
    }
}

// Issues the cp.async copies of one K-block of the raw FP32 A tile.
template <int F>
__device__ __forceinline__ void raw_issue(const TcJob &J, const int64_t (&base)[RawCfg<F>::UNITS],
                                          const int (&nrow)[RawCfg<F>::UNITS], int64_t row0, int64_t kbase,
                                          uint32_t raw_s, int ct) {
    using R = RawCfg<F>;
    const float *src = static_cast<const float *>(J.A);
    const bool kc = J.akc != 0;
#pragma unroll
    for (int i = 0; i < R::UNITS; ++i) {
        int row, k;
        uint32_t off;
        raw_unit<F>(i, ct, kc, row, k, off);
        const int64_t kg = kbase + k;
        const uint32_t dst = raw_s + off;
        if (kc) {
            // 4 consecutive k of one row
            const int nk = (int)max((int64_t)0, min((int64_t)4, J.K - kg));
            if (J.cp16) {
                const float *p = src + (base[i] >= 0 ? base[i] + kg : 0);
                cp_async16(dst, p, (base[i] >= 0) ? (uint32_t)(nk * 4) : 0u);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool ok = base[i] >= 0 && e < nk;
                    cp_async4(dst + 4 * e, src + (ok ? base[i] + imap(J.kA, kg + e) : 0), ok ? 4u : 0u);
                }
            }
        } else {
            // 4 consecutive rows at one k
            const bool kok = kg < J.K;
            const int nr = kok ? nrow[i] : 0;
            if (J.cp16) {
                const float *p = src + (nr > 0 ? base[i] + imap(J.kA, kg) : 0);
                cp_async16(dst, p, (uint32_t)(nr * 4));
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int64_t rg = row0 + row + e;
                    const bool ok = kok && rg < J.M;
                    const int64_t o = ok ? imap(J.rowA, rg) + imap(J.kA, kg) : 0;
                    cp_async4(dst + 4 * e, src + o, ok ? 4u : 0u);
                }
            }
        }
    }
}

// Float sources: raw tiles arrive through cp.async several K-blocks ahead;
// the converters split them from shared memory.
// fmul: 2^(left shift) of a fixed-point A (fx_shift of its scale word).
template <int F, bool TMA_OK, typename Join>
__device__ __forceinline__ bool conv_tile_loop_raw(const TcJob &J, const CUtensorMap *tm, uint64_t *rfull,
                                                   uint32_t &rc, int mt, uint8_t *sA, uint32_t A_ST, uint8_t *sRaw,
                                                   uint64_t *full, uint64_t *empty, int S, uint32_t &g, int lane,
                                                   int ct, int fmul, Join &&join) {
    using R = RawCfg<F>;
    constexpr int BK = R::BK;
    constexpr int CH = 16 / FT<F>::ELEM;
    const bool kc = J.akc != 0;
    const bool tma = TMA_OK && J.tma != 0;
    // per-unit source offsets (rows fixed over the tile)
    const int64_t row0 = (int64_t)mt * kBM;
    // TMA coordinates of the tile's rows (slab layout: row in slab, slab)
    const int trow = J.tma == 3 ? (int)(row0 % J.tmaP) : (int)row0;
    const int tslab = J.tma == 3 ? (int)(row0 / J.tmaP) : 0;
    int64_t base[R::UNITS];
    int nrow[R::UNITS];
#pragma unroll
    for (int i = 0; i < R::UNITS; ++i) {
        int row, k;
        uint32_t off;
        raw_unit<F>(i, ct, kc, row, k, off);
        const int64_t rg = (int64_t)mt * kBM + row;
        base[i] = rg < J.M ? imap(J.rowA, rg) : -1;
        nrow[i] = (int)max((int64_t)0, min((int64_t)4, J.M - rg));
    }
    named_bar(2, 32 * kConv);  // the raw ring is free (previous tile consumed)
    const uint32_t raw0 = smem_u32(sRaw);
    // TMA: one thread loads K-block kbi of the tile into ring slot (rc + kbi)
    auto tma_issue = [&](int kbi) {
        const uint32_t slot = (rc + (uint32_t)kbi) % R::STAGES;
        const uint32_t bar = smem_u32(&rfull[slot]);
        mbar_arrive_expect_tx(bar, R::BYTES);
        const int k0 = (J.kb0 + kbi) * BK;
        if (J.tma == 2) {
            tma_load_2d(raw0 + slot * R::BYTES, tm, k0, trow, bar);
        } else {
            tma_load_3d(raw0 + slot * R::BYTES, tm, trow, k0, tslab, bar);
        }
    };
    if (tma) {
        if (ct == 0)
            for (int j = 0; j < R::STAGES - 1 && j < J.nkb; ++j) tma_issue(j);
        // the MMA of this tile waits for the epilogue of the previous one:
        // take part in it first (the raw loads above run meanwhile)
        if (!join()) return false;
    } else {
#pragma unroll
        for (int j = 0; j < R::STAGES - 1; ++j) {
            if (j < J.nkb) raw_issue<F>(J, base, nrow, row0, (int64_t)(J.kb0 + j) * BK, raw0 + j * R::BYTES, ct);
            cp_async_commit();
        }
        if (!join()) {
            cp_async_wait<0>();
            return false;
        }
    }
    // conversion items of this thread
    int irow[kItems], ich[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) item_rc(i, ct, kc, irow[i], ich[i]);
    for (int kb = 0; kb < J.nkb; ++kb, ++g) {
        int rs;
        if (tma) {
            named_bar(2, 32 * kConv);  // every converter is done with K-block kb - 1
            const int kn = kb + R::STAGES - 1;
            if (ct == 0 && kn < J.nkb) tma_issue(kn);
            const uint32_t u = rc + (uint32_t)kb;
            rs = (int)(u % R::STAGES);
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&rfull[rs]), (u / R::STAGES) & 1u))) return false;
        } else {
            cp_async_wait<R::STAGES - 2>();
            named_bar(2, 32 * kConv);
            rs = kb % R::STAGES;
            const int kn = kb + R::STAGES - 1;
            if (kn < J.nkb)
                raw_issue<F>(J, base, nrow, row0, (int64_t)(J.kb0 + kn) * BK, raw0 + (kn % R::STAGES) * R::BYTES, ct);
            cp_async_commit();
        }
        const int s = (int)(g % (uint32_t)S);
        const uint32_t ph = (g / (uint32_t)S) & 1u;
        int ok = (lane == 0) ? (int)mbar_wait(smem_u32(&empty[s]), ph ^ 1u) : 1;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            cp_async_wait<0>();
            return false;
        }
        const float *raw = reinterpret_cast<const float *>(sRaw + rs * R::BYTES);
        uint8_t *dst = sA + (size_t)s * A_ST;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            float v[CH];
            if (kc) {
                const float *q = raw + irow[i] * BK + ich[i] * CH;
#pragma unroll
                for (int e = 0; e < CH; e += 4) *reinterpret_cast<float4 *>(&v[e]) = *reinterpret_cast<const float4 *>(q + e);
            } else {
#pragma unroll
                for (int e = 0; e < CH; ++e) v[e] = raw[(ich[i] * CH + e) * kBM + irow[i]];
            }
            uint4 out[FT<F>::PIECES];
            if constexpr (is_fx_f<F>()) {
                int32_t x[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] = __float_as_int(v[e]);
                fx_pack_f<F>(x, out, fmul);
            } else {
                split_pack<F, float>(v, out);
            }
            const uint32_t off = swz(irow[i], ich[i]);
#pragma unroll
            for (int q = 0; q < FT<F>::PIECES; ++q)
                *reinterpret_cast<uint4 *>(dst + q * (kBM * kRowBytes) + off) = out[q];
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&full[s]));
    }
    cp_async_wait<0>();
    if (tma) rc += (uint32_t)J.nkb;
    return true;
}

// x * 2^e as a double for |x| < 2^53, from integer operations only (the
// FP64 pipe is narrow); exponents outside the normal range take ldexp.
__device__ __forceinline__ double i64_scaled(long long x, int e) {
    if (x == 0) return 0.0;
    const unsigned long long a = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
    const int sh = __clzll((long long)a) - 11;  // leading one to bit 52
    const int E = 1075 + e - sh;
    if (sh < 0 || E <= 0 || E >= 2047) return ldexp((double)x, e);
    const unsigned long long bits = ((unsigned long long)(x < 0) << 63) | ((unsigned long long)E << 52) |
                                    ((a << sh) & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

// round(v) as a 64-bit integer (ties away from zero) for |v| < 2^62, from
// the bits of v.
__device__ __forceinline__ long long f32_round_i64(float v) {
    const uint32_t b = __float_as_uint(v);
    const int E = (int)((b >> 23) & 0xFFu);
    const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = E - 150;  // v = m * 2^sh
    unsigned long long r = 0;
    if (E == 0) r = 0;
    else if (sh >= 0) r = m << sh;
    else if (sh > -26) r = (m + (1ull << (-sh - 1))) >> (-sh);
    return (b >> 31) ? -(long long)r : (long long)r;
}

__device__ __forceinline__ int add_sat(int a, int b) {
    int r;
    asm("add.sat.s32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// Scales of one fixed-point job, the same for all of its tiles: A's scale
// eA and the output scale eC = eA_actual + g, where |A| < 2^eA_actual (from
// A's largest magnitude) and every row sum of |op(L)| is below 2^g, so that
// every output is below 2^b in magnitude up to rounding.
struct FxConsts {
    int j = -1;
    int eA = 0, eC = 0;
};

template <int F>
__device__ __forceinline__ void fx_consts(const TcJob &J, int j, FxConsts &k) {
    if (k.j == j) return;
    k.j = j;
    k.eA = J.fxA->e;
    const unsigned mA = J.fxA->maxabs;
    const int eAact = k.eA - FxForm<F>::BITS + (mA ? 32 - __clz((int)mA) : 0);
    const unsigned long long gb = *J.fxG;  // bits of the largest row sum (non-negative)
    const int g = gb ? (int)((gb >> 52) & 0x7FF) - 1022 : 0;
    k.eC = eAact + g;
    // the converters shift A left by fx_shift: its values carry the scale
    // 2^(eA - shift - b) from there on
    k.eA -= fx_shift<F>(mA);
}

// Fixed-point form epilogue for one tile row.  The two accumulator regions
// hold a0 (level 0, exact) and a1 (the other levels kept) in units of
// 2^(eA + f_c + UNIT).  Fixed-point output with scale eC:
//     X = round((a0 + a1) * 2^s),  s = eA + f_c + UNIT + b - eC,
// formed from the float pair (sum, err) = Fast2Sum(a0 * 2^s, a1 * 2^s) (both
// products are exact power-of-two scalings; Dekker's Fast2Sum is error-free
// when |a0| >= |a1|, the usual case, and within an ulp of the sum otherwise),
// then X = rint(sum) + rint(err) (|err| <= 2^7: rounded by the 1.5 * 2^23
// exponent trick), saturated for FX32 (FX32H stays below 2^29 + 2^8, no
// overflow).  The largest |X| of the tile is tracked on |sum| with a margin
// above the error term.  Two columns at a time in paired FP32 instructions.
// Value output (last mode): the sum 2^VS (a0 + a1) is formed in 64-bit
// integers (a0 exactly, a1 rounded) and scaled by 2^(eA + f_c + UNIT - VS).
// The 16-column chunks of the tile are shared by `nparts` warps of the same
// tensor-memory lane quarter; this one takes chunks part, part + nparts, ...
// stg: this warp's 4 KB of staging shared memory for TMA stores of C
// through tmC (null: plain stores); rw0 is the warp's first tile row.
// colw: one word per column of the tile in shared memory (the scale 2^s as
// a float for fixed-point output, the row exponent f_c otherwise); every
// warp fills the words of its own chunks (warps of other lane quarters
// with the same chunks write the same values), unless they already hold the
// words of the same job and column tile (fill_colw false).
template <int F>
__device__ __forceinline__ void fx_epilogue(const TcJob &J, const FxConsts &k, uint32_t lane_base, uint32_t ACOLS,
                                            int64_t ro, int64_t n0, int lane, int part, int nparts, uint8_t *stg,
                                            const CUtensorMap *tmC, int64_t rw0, uint32_t *colw, bool fill_colw) {
    const int eA = k.eA, eC = k.eC;
    const int lim = (int)min(J.N - n0, (int64_t)J.BN);
    const bool unit = (J.colC.R0 == 0 && J.colC.s0 == 1);
    const int64_t cs = J.colC.s0;
    const int step = 16 * nparts;
    using X = FxForm<F>;
    const int base = eA + X::UNIT + X::BITS - eC;
    // column words of this warp's chunks: lanes 0-15 one chunk, 16-31 the next
    for (int c = 16 * part + (lane >> 4) * step + (lane & 15); fill_colw && c - (lane & 15) < J.BN; c += 2 * step) {
        const int f = c < lim ? __ldg(J.fxF + n0 + c) : 0;
        // 2^s (s below -126 leaves only values that round to 0)
        colw[c] = J.cfix ? (uint32_t)((127 + min(100, max(-126, base + f))) << 23) : (uint32_t)f;
    }
    __syncwarp();
    // TMA coordinates of the warp's rows (slab layout: row in slab, slab)
    const int trow = (stg && J.tmc == 3) ? (int)(rw0 % J.tmcP) : (int)rw0;
    const int tslab = (stg && J.tmc == 3) ? (int)(rw0 / J.tmcP) : 0;
    unsigned mx = 0;
    float mxf = 0.f;
    int cnt = 0;       // boxes staged by this warp
    int64_t pcol = 0;  // column of the first box of the pending group
    // 16-column boxes in groups of nb (nb buffers of bbytes each): the first
    // box of a group waits until the previous group has been read, fill
    // writes this lane's row; a full group (or the last box) is fenced once
    // and handed to the TMA unit
    auto stage = [&](int nb, int bbytes, int64_t col, bool last, auto &&fill) {
        const int b = cnt % nb;
        if (b == 0 && cnt >= nb && lane == 0) bulk_wait_read<0>();
        __syncwarp();
        fill(stg + b * bbytes);
        if (b == 0) pcol = col;
        ++cnt;
        if (b == nb - 1 || last) {
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0 && rw0 < J.M) {  // boxes wholly past the last row are not stored
                for (int i = 0; i <= b; ++i) {
                    const uint32_t src = smem_u32(stg + i * bbytes);
                    // boxes of a group are `step` columns apart
                    const int cb = (int)(pcol + (int64_t)i * step);
                    if (J.tmc == 3) tma_store_3d(tmC, src, trow, cb, tslab);
                    else tma_store_2d(tmC, src, cb, trow);
                }
                bulk_commit();
            }
        }
    };
    for (int c0 = 16 * part; c0 < J.BN; c0 += step) {
        const bool last = c0 + step >= J.BN;
        uint32_t r0[16], r1[16], w[16];
        tmem_ld16(lane_base + (uint32_t)c0, r0);
        tmem_ld16(lane_base + ACOLS + (uint32_t)c0, r1);
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; e += 4) *reinterpret_cast<uint4 *>(&w[e]) = *reinterpret_cast<const uint4 *>(colw + c0 + e);
        if (J.cfix) {
            int32_t xv[16];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const uint64_t sc = pack2(w[e], w[e + 1]);
                const uint64_t h = mul_f32x2(pack2(r0[e], r0[e + 1]), sc);
                const uint64_t l = mul_f32x2(pack2(r1[e], r1[e + 1]), sc);
                const uint64_t sum = add_f32x2(h, l);
                const uint64_t err = sub_f32x2(l, sub_f32x2(sum, h));
                const uint64_t em = add_f32x2(err, 0x4B4000004B400000ull);  // + 1.5 * 2^23 each
                const float s0 = __uint_as_float((uint32_t)sum), s1 = __uint_as_float((uint32_t)(sum >> 32));
                const int e0 = (int)(uint32_t)em - 0x4B400000, e1 = (int)(uint32_t)(em >> 32) - 0x4B400000;
                if constexpr (F == kFX32H) {
                    xv[e] = __float2int_rn(s0) + e0;
                    xv[e + 1] = __float2int_rn(s1) + e1;
                } else {
                    xv[e] = add_sat(__float2int_rn(s0), e0);
                    xv[e + 1] = add_sat(__float2int_rn(s1), e1);
                }
                mxf = fmaxf(mxf, fmaxf(fabsf(s0), fabsf(s1)));
            }
            if (stg) {
                // groups of two 2 KB boxes; [column][row] or [row][column]
                stage(2, 2048, n0 + c0, last, [&](uint8_t *buf) {
                    if (J.tmc == 3) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) reinterpret_cast<int32_t *>(buf)[e * 32 + lane] = xv[e];
                    } else {
                        int4 *d = reinterpret_cast<int4 *>(buf + lane * 64);
#pragma unroll
                        for (int e = 0; e < 16; e += 4) d[e / 4] = make_int4(xv[e], xv[e + 1], xv[e + 2], xv[e + 3]);
                    }
                });
            } else if (ro >= 0) {
                int32_t *cp = static_cast<int32_t *>(J.C) + ro + (n0 + c0) * cs;
                if (unit && c0 + 16 <= lim && (reinterpret_cast<uintptr_t>(cp) & 15) == 0) {
#pragma unroll
                    for (int e = 0; e < 16; e += 4)
                        *reinterpret_cast<int4 *>(cp + e) = make_int4(xv[e], xv[e + 1], xv[e + 2], xv[e + 3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (c0 + e < lim) cp[e * cs] = xv[e];
                }
            }
        } else {
            double v[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int f = (int)w[e];
                const float s1 = __uint_as_float(r1[e]) * (float)(1 << X::VS);
                long long I0;
                if constexpr (X::VS > 0) I0 = (long long)__float2int_rz(__uint_as_float(r0[e])) << X::VS;
                else I0 = f32_round_i64(__uint_as_float(r0[e]));
                v[e] = i64_scaled(I0 + f32_round_i64(s1), eA + f + X::UNIT - X::VS);
            }
            // the accumulate flag is tested outside the stores: no loads of C otherwise
            if (stg) {
                // one 4 KB buffer of doubles (value output is FP64 when staged)
                stage(1, 4096, n0 + c0, last, [&](uint8_t *buf) {
                    if (J.tmc == 3) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) reinterpret_cast<double *>(buf)[e * 32 + lane] = v[e];
                    } else {
                        double2 *d = reinterpret_cast<double2 *>(buf + lane * 128);
#pragma unroll
                        for (int e = 0; e < 16; e += 2) d[e / 2] = make_double2(v[e], v[e + 1]);
                    }
                });
            } else if (ro < 0) {
            } else if (J.c64) {
                double *d = static_cast<double *>(J.C) + ro + (n0 + c0) * cs;
                if (J.acc) {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (c0 + e < lim) d[e * cs] += v[e];
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (c0 + e < lim) d[e * cs] = v[e];
                }
            } else {
                float *d = static_cast<float *>(J.C) + ro + (n0 + c0) * cs;
                if (J.acc) {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (c0 + e < lim) d[e * cs] = (float)((double)d[e * cs] + v[e]);
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (c0 + e < lim) d[e * cs] = (float)v[e];
                }
            }
        }
    }
    if (stg && lane == 0) {
        // the staging memory is handed back, and a tile read later in the
        // same launch must see the stores
        if (J.publish) bulk_wait<0>();
        else bulk_wait_read<0>();
    }
    __syncwarp();
    if (J.cfix) {
        // |X| <= |sum| + 2^7 + 1; capped at 2^31 (the rounding bound of
        // FX32, where the conversion saturates; FX32H stays below 2^29 + 2^8)
        mx = (unsigned)fminf(mxf + 256.0f, 2147483648.0f);
        if (mxf == 0.f) mx = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && mx) atomicMax(&J.fxC->maxabs, mx);
    }
}

// Epilogue share of one fixed-point tile (tile t, it-th tile of this CTA):
// waits for its accumulators, drains this warp's column share, releases the
// accumulators and publishes the tile.  `nbar` threads take part.
// stg: the warp's staging memory (used when the job stores C by TMA).
template <int F>
__device__ __forceinline__ bool fx_epi_tile(const TcLaunch &L, int t, int it, uint32_t tmem, uint32_t ACOLS, int NBUF,
                                            uint64_t *accf, uint64_t *acce, FxConsts &k, int q, int lane, bool lead,
                                            int part, int nparts, int nbar, uint8_t *stg, uint32_t *colt) {
    const int j = find_job(L, t);
    const TcJob J = job_at(L, j);
    const int lt = t - J.tile_begin;
    const int nt = lt % J.tiles_n, mt = lt / J.tiles_n;
    const int buf = it % NBUF;
    const uint32_t use = (uint32_t)(it / NBUF);
    int ok = (lane == 0) ? (int)mbar_wait(smem_u32(&accf[buf]), use & 1u) : 1;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return false;
    tc_fence_after();
    const int64_t rg = (int64_t)mt * kBM + q * 32 + lane;
    const int64_t ro = rg < J.M ? imap(J.rowC, rg) : -1;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * Regions<F>::N) * ACOLS;
    // one column tile per job and one table: the table still holds the
    // words of the previous tile when that was of the same job
    const bool fill = k.j != j || J.tiles_n > 1 || NBUF > 1;
    fx_consts<F>(J, j, k);
    if (J.cfix && lead && lane == 0) J.fxC->e = k.eC;
    const bool staged = stg != nullptr && J.tmc != 0;
    fx_epilogue<F>(J, k, lane_base, ACOLS, ro, (int64_t)nt * J.BN, lane, part, nparts, staged ? stg : nullptr,
                &job_at(L, j).tmC, (int64_t)mt * kBM + q * 32, colt + buf * 256, fill);
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&acce[buf]));
    if (J.publish) {
        named_bar(1, nbar);
        if (lead && lane == 0) {
            __threadfence();
            atomicAdd(&L.done[j], 1);
        }
    }
    return true;
}

// MODE (split forms; the fixed-point forms take 1): 2 = wide, some job reads
// an FP64 tensor (converted from registers), writes FP64 or accumulates into
// C; 1 = FP32 sources staged by TMA or cp.async, plain FP32 stores; 0 = as 1
// with cp.async staging only.  The smaller builds serve launches of many short
// jobs, which are bound by instruction fetch.
template <int F, int MODE>
__global__ void __launch_bounds__(kPThreads, 1) tcp_kernel(const __grid_constant__ TcLaunch L) {
    constexpr bool A64 = MODE == 2;
    using T = FT<F>;
    constexpr int BK = kRowBytes / T::ELEM;
    constexpr uint32_t PIECE_A = kBM * kRowBytes;
    constexpr uint32_t A_ST = T::PIECES * PIECE_A;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_align1024(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = L.stages, NACC = L.nacc, NBUF = L.nbuf;
    const uint32_t ACOLS = (uint32_t)L.acc_cols;
    const uint32_t B_ST = (uint32_t)T::PIECES * (uint32_t)L.bn_max * kRowBytes;
    uint8_t *sA = smem;
    uint8_t *sB = smem + (size_t)S * A_ST;
    uint8_t *sRaw = sB + (size_t)S * B_ST;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sRaw + (size_t)RawCfg<F>::STAGES * RawCfg<F>::BYTES);
    uint64_t *full = bars, *empty = bars + S, *accf = bars + 2 * S, *acce = bars + 2 * S + NBUF;
    uint64_t *rfull = bars + 2 * S + 2 * NBUF;  // raw A ring (TMA)
    uint32_t *tslot = reinterpret_cast<uint32_t *>(rfull + RawCfg<F>::STAGES);
    // fixed-point forms: one table of 256 column words per accumulator buffer
    uint32_t *colt = reinterpret_cast<uint32_t *>((reinterpret_cast<uintptr_t>(tslot + 1) + 15) & ~uintptr_t(15));
    constexpr int RG = Regions<F>::N;
    uint32_t ncols = ACOLS * (uint32_t)RG * (uint32_t)NACC * (uint32_t)NBUF;
    // programmatic dependent launch: the next launch may be scheduled now (it
    // gets an SM as soon as a CTA of this one exits) and runs its prologue
    // while this one finishes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    ncols = ncols <= 32 ? 32u : (ncols <= 64 ? 64u : (ncols <= 128 ? 128u : (ncols <= 256 ? 256u : 512u)));

    // one accumulator buffer (fixed point, 256-column tiles): the converter
    // warps, idle while the MMA waits for the epilogue, take two thirds of it
    const bool join = is_fx_f<F>() && NBUF == 1;
    const int n_epi = kEpi + (join ? kConv : 0);
    // in that mode every A stage is free during the epilogue (the converters
    // fill them only after it): 4 KB of staging per epilogue warp
    uint8_t *stg = (join && (uint32_t)S * A_ST >= 4096u * (kEpi + kConv) && warp >= 2)
                       ? sA + (size_t)(warp - 2) * 4096 : nullptr;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full[s]), kConv + 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(smem_u32(&accf[b]), 1);
            mbar_init(smem_u32(&acce[b]), (uint32_t)n_epi);
        }
        for (int r = 0; r < RawCfg<F>::STAGES; ++r) mbar_init(smem_u32(&rfull[r]), 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tslot), ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    // everything below may read what earlier launches wrote
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (L.reset_next && blockIdx.x == 0 && threadIdx.x == 0) {
        L.reset_next->maxabs = 0u;
        L.reset_next->e = 0;
    }

    if (warp == 0) {
        // ---------------------------------------------- op(L) image producer
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < L.total_tiles && ok; t += gridDim.x) {
                const TcJob J = job_at(L, find_job(L, t));
                const int lt = t - J.tile_begin;
                const int nt = lt % J.tiles_n;
                const uint32_t bytes = (uint32_t)T::PIECES * (uint32_t)J.BN * kRowBytes;
                const uint8_t *img = J.bimg + ((size_t)nt * J.kb_img + J.kb0) * bytes;
                for (int kb = 0; kb < J.nkb; ++kb, ++g) {
                    const int s = (int)(g % (uint32_t)S);
                    const uint32_t ph = (g / (uint32_t)S) & 1u;
                    if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(smem_u32(&full[s]), bytes);
                    bulk_g2s(smem_u32(sB + (size_t)s * B_ST), img + (size_t)kb * bytes, bytes, smem_u32(&full[s]));
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // -------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t g = 0;
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < L.total_tiles && ok; t += gridDim.x, ++it) {
                const TcJob J = job_at(L, find_job(L, t));
                const int buf = it % NBUF;
                const uint32_t use = (uint32_t)(it / NBUF);
                if (!mbar_wait(smem_u32(&acce[buf]), (use & 1u) ^ 1u)) break;
                tc_fence_after();
                const uint32_t idesc = make_idesc(T::FMT, kBM, (uint32_t)J.BN);
                const uint32_t PIECE_B = (uint32_t)J.BN * kRowBytes;
                const uint32_t dbase = tmem + (uint32_t)(buf * NACC * RG) * ACOLS;
                for (int kb = 0; kb < J.nkb; ++kb, ++g) {
                    const int s = (int)(g % (uint32_t)S);
                    const uint32_t ph = (g / (uint32_t)S) & 1u;
                    if (!mbar_wait(smem_u32(&full[s]), ph)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int64_t kval = min((int64_t)BK, J.K - (int64_t)(J.kb0 + kb) * BK);
                    const int ksteps = (int)((kval + T::MMA_K - 1) / T::MMA_K);
                    const uint32_t a_base = smem_u32(sA + (size_t)s * A_ST);
                    const uint32_t b_base = smem_u32(sB + (size_t)s * B_ST);
                    const uint32_t dset = dbase + (uint32_t)(kb % NACC) * (uint32_t)RG * ACOLS;
                    const bool fresh = kb < NACC;
                    for (int ks = 0; ks < ksteps; ++ks) {
#pragma unroll
                        for (int pr = 0; pr < T::NPROD; ++pr) {
                            int pa, pb;
                            prod_pieces<F>(pr, pa, pb);
                            const uint64_t ad = smem_desc_kmajor(a_base + pa * PIECE_A + ks * 32, kRowBytes);
                            const uint64_t bd = smem_desc_kmajor(b_base + pb * PIECE_B + ks * 32, kRowBytes);
                            const bool first = fresh && ks == 0 && first_in_region<F>(pr);
                            tc_mma<T::KIND>(dset + (uint32_t)region_of<F>(pr) * ACOLS, ad, bd, idesc, first ? 0u : 1u);
                        }
                    }
                    tc_commit(smem_u32(&empty[s]));
                }
                if (!ok) break;
                tc_commit(smem_u32(&accf[buf]));
            }
        }
        __syncwarp();
    } else if (warp < kConv0) {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;                // TMEM lane quarter this warp may access
        int it = 0;
        if constexpr (is_fx_f<F>()) {
            FxConsts k;
            for (int t = blockIdx.x; t < L.total_tiles; t += gridDim.x, ++it)
                if (!fx_epi_tile<F>(L, t, it, tmem, ACOLS, NBUF, accf, acce, k, q, lane, warp == 2, 0, join ? 3 : 1,
                                 32 * n_epi, stg, colt))
                    break;
        } else
        for (int t = blockIdx.x; t < L.total_tiles; t += gridDim.x, ++it) {
            const int j = find_job(L, t);
            const TcJob J = job_at(L, j);
            const int lt = t - J.tile_begin;
            const int nt = lt % J.tiles_n, mt = lt / J.tiles_n;
            const int buf = it % NBUF;
            const uint32_t use = (uint32_t)(it / NBUF);
            int ok = (lane == 0) ? (int)mbar_wait(smem_u32(&accf[buf]), use & 1u) : 1;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            const int64_t rg = (int64_t)mt * kBM + q * 32 + lane;
            const int64_t ro = rg < J.M ? imap(J.rowC, rg) : -1;
            const int64_t n0 = (int64_t)nt * J.BN;
            const int used = min(NACC, J.nkb);
            const uint32_t lane_base =
                tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * NACC * RG) * ACOLS;
            for (int c0 = 0; c0 < J.BN; c0 += 32) {
                // accumulator 0: hi + cross in FP32; further accumulators are
                // added in order
                uint32_t h[32], l[32];
                tmem_ld32(lane_base + (uint32_t)c0, h);
                tmem_ld32(lane_base + ACOLS + (uint32_t)c0, l);
                tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 32; ++e) h[e] = __float_as_uint(__uint_as_float(l[e]) + __uint_as_float(h[e]));
                for (int a = 1; a < used; ++a) {
                    uint32_t x[32];
                    tmem_ld32(lane_base + (uint32_t)(RG * a) * ACOLS + (uint32_t)c0, l);
                    tmem_ld32(lane_base + (uint32_t)(RG * a + 1) * ACOLS + (uint32_t)c0, x);
                    tmem_ld_wait();
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        h[e] = __float_as_uint(__uint_as_float(h[e]) + (__uint_as_float(x[e]) + __uint_as_float(l[e])));
                }
                if (ro >= 0) {
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        // columns of this tile only: the 32-column block may run past BN
                        const int64_t lim = min(J.N - n0, (int64_t)J.BN);
                        const int cmax = (int)max((int64_t)0, min((int64_t)16, lim - c0 - 16 * hh));
                        float s16[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) s16[e] = __uint_as_float(h[16 * hh + e]);
                        if (A64 && J.c64)
                            store_row16<double>(J.C, ro, J.colC, n0 + c0 + 16 * hh, cmax, s16, J.acc != 0);
                        else
                            store_row16<float>(J.C, ro, J.colC, n0 + c0 + 16 * hh, cmax, s16, A64 && J.acc != 0);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce[buf]));
            // publish the finished tile for jobs that wait on this one
            if (J.publish) {
                named_bar(1, 32 * kEpi);
                if (warp == 2 && lane == 0) {
                    __threadfence();
                    atomicAdd(&L.done[j], 1);
                }
            }
        }
    } else {
        // -------------------------------------------------------- converters
        const int ct = threadIdx.x - kConv0 * 32;
        uint32_t g = 0, rc = 0;
        // epilogue share of the previous tile, still due (join mode)
        int pend = -1, pend_it = 0;
        const int part = 1 + (warp - kConv0) / 4;
        FxConsts k;
        auto epi_prev = [&]() -> bool {
            if constexpr (!is_fx_f<F>()) {
                return true;
            } else {
                if (pend < 0) return true;
                const int t = pend;
                pend = -1;
                if (!fx_epi_tile<F>(L, t, pend_it, tmem, ACOLS, NBUF, accf, acce, k, warp & 3, lane, false, part, 3,
                                 32 * n_epi, stg, colt))
                    return false;
                // the A stages double as staging memory: wait until every
                // warp of the epilogue is done with it
                int ok = (lane == 0) ? (int)mbar_wait(smem_u32(&acce[pend_it % NBUF]), (uint32_t)(pend_it / NBUF) & 1u)
                                     : 1;
                return __shfl_sync(0xffffffffu, ok, 0) != 0;
            }
        };
        int it = 0;
        bool ok = true;
        // fixed point: the left shift of the current job's A (its scale word
        // was written by an earlier launch), read once per job
        int fmul = 1, fsh_job = -1;
        for (int t = blockIdx.x; t < L.total_tiles && ok; t += gridDim.x, ++it) {
            const int jt = find_job(L, t);
            const TcJob J = job_at(L, jt);
            if constexpr (is_fx_f<F>()) {
                if (jt != fsh_job) {
                    fmul = 1 << fx_shift<F>(J.fxA->maxabs);
                    fsh_job = jt;
                }
            }
            const CUtensorMap *tm = &job_at(L, jt).tmA;  // launch parameter space
            const int lt = t - J.tile_begin;
            const int mt = lt / J.tiles_n;
            if (J.dep >= 0) {
                // the tile waited for may be the previous tile of this CTA
                if (!epi_prev()) break;
                // wait until every tile of the job this one reads is stored
                // (bounded: at the limit the timeout is latched and the tile
                // goes ahead; once a dependency wait of this launch has given
                // up, the others give up after 1 ms)
                if (ct == 0) {
                    volatile int *dn = L.done + J.dep;
                    volatile int *gave_up = L.done + L.njobs;
                    const int need = J.dep_tiles + L.dep_hold;
                    const unsigned long long t0 = globaltimer_ns();
                    while (*dn < need) {
                        const unsigned long long dt = globaltimer_ns() - t0;
                        if (dt > L.dep_wait_ns) {
                            latch_error(kErrTimeout);
                            *gave_up = 1;
                            break;
                        }
                        if (dt > 1000000ull && *gave_up != 0) break;
                    }
                    __threadfence();
                }
                named_bar(2, 32 * kConv);
            }
            if constexpr (is_fx_f<F>()) {  // always 32-bit integers
                ok = conv_tile_loop_raw<F, true>(J, tm, rfull, rc, mt, sA, A_ST, sRaw, full, empty, S, g, lane, ct, fmul,
                                           epi_prev);
                if (join) {
                    pend = t;
                    pend_it = it;
                }
            } else {
                auto none = []() { return true; };
                if (A64 && J.a64)
                    ok = conv_tile_loop<F, double>(J, mt, sA, A_ST, full, empty, S, g, lane, ct);
                else
                    ok = conv_tile_loop_raw<F, MODE >= 1>(J, tm, rfull, rc, mt, sA, A_ST, sRaw, full, empty, S, g, lane, ct, 1,
                                               none);
            }
        }
        if (ok) epi_prev();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

}  // namespace

// ---------------------------------------------------------------- host side

cudaError_t tcp_error_word(unsigned int *out, bool clear, cudaStream_t st) { return read_error_word(out, clear, st); }

static std::atomic<int> g_dep_hold{0};
static std::atomic<unsigned long long> g_dep_wait_ns{0};

void tcp_debug_dependency_timeout(int hold, unsigned long long limit_ns) {
    g_dep_hold.store(hold ? 1 : 0);
    g_dep_wait_ns.store(limit_ns);
}

static int pieces_of_f(int form) { return form == kFX32 ? 4 : ((form == kBF16x6 || form == kFX32H) ? 3 : 2); }
static int bk_of_f(int form) { return form == kTF32x3 ? kRowBytes / 4 : kRowBytes / 2; }

size_t tcp_job_bytes() { return sizeof(TcJob); }

// Fills a job for contraction c (B side from `img`, built with tcp_tile_n).
static TcJob make_job(int form, const Contraction &c, const void *img, int bn = 0) {
    TcJob J{};
    J.A = c.A;
    J.rowA = c.rowA;
    J.kA = c.kA;
    J.M = c.M;
    J.bimg = static_cast<const uint8_t *>(img);
    J.C = c.C;
    J.rowC = c.rowC;
    J.colC = c.colC;
    J.N = c.N;
    J.K = c.K;
    const int bk = bk_of_f(form);
    J.kb_img = (c.K + bk - 1) / bk;
    J.kb0 = 0;
    J.nkb = (int32_t)J.kb_img;
    J.BN = bn > 0 ? bn : tc_tile_n(form, c.N);
    J.tiles_m = (int32_t)((c.M + kBM - 1) / kBM);
    J.tiles_n = (int32_t)((c.N + J.BN - 1) / J.BN);
    J.dep = -1;
    J.dep_tiles = 0;
    J.a64 = c.A_f64;
    J.c64 = c.C_f64;
    J.acc = c.accumulate;
    J.akc = (c.kA.s0 == 1 && c.kA.R0 != 1) ? 1 : 0;
    const int64_t v = c.A_f64 ? 2 : 4;
    const bool unit_k = c.kA.R0 == 0 && c.kA.s0 == 1;
    const bool rows_ok = (c.rowA.s0 % v == 0) && (c.rowA.R0 == 0 || c.rowA.s1 % v == 0);
    const bool base_ok = (reinterpret_cast<uintptr_t>(c.A) % 16) == 0;
    J.avec = (unit_k && rows_ok && base_ok) ? 1 : 0;
    // 16-byte cp.async of FP32 sources: k-contiguous rows need m % 4 == 0;
    // fibre-contiguous tiles need groups of 4 rows contiguous and aligned
    if (!c.A_f64 && base_ok) {
        if (J.akc)
            J.cp16 = (unit_k && c.rowA.s0 % 4 == 0 && (c.rowA.R0 == 0 || c.rowA.s1 % 4 == 0)) ? 1 : 0;
        else
            J.cp16 = (c.rowA.s0 == 1 && (c.rowA.R0 == 0 || (c.rowA.R0 % 4 == 0 && c.rowA.s1 % 4 == 0)) &&
                      c.kA.R0 == 0 && c.kA.s0 % 4 == 0) ? 1 : 0;
    }
    return J;
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on it).
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Raw A tiles by TMA where the layout allows it (4-byte source): either rows
// with contiguous k (one row stride), or slabs of tmaP contiguous rows (a
// multiple of the 128-row tile, so no tile straddles two slabs) with k at a
// fixed stride.  Strides must be multiples of 16 bytes.  Otherwise the
// converters copy the tiles themselves (cp.async).
static void setup_tma(int form, TcJob &J, const Contraction &c) {
    J.tma = 0;
    if (c.A_f64 || (reinterpret_cast<uintptr_t>(c.A) % 16) != 0 || c.M < 1 || c.K < 1) return;
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn) return;
    const cuuint32_t bk = (cuuint32_t)(form == kTF32x3 ? kRowBytes / 4 : kRowBytes / 2);
    const cuuint32_t estr[3] = {1, 1, 1};
    void *base = const_cast<void *>(c.A);
    if (J.akc) {
        if (!(c.kA.R0 == 0 && c.kA.s0 == 1 && c.rowA.R0 == 0 && c.rowA.s0 >= c.K && c.rowA.s0 % 4 == 0)) return;
        const cuuint64_t dims[2] = {(cuuint64_t)c.K, (cuuint64_t)c.M};
        const cuuint64_t strides[1] = {(cuuint64_t)c.rowA.s0 * 4};
        const cuuint32_t box[2] = {bk, (cuuint32_t)kBM};
        if (fn(&J.tmA, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
        J.tma = 2;
        return;
    }
    if (!(c.rowA.s0 == 1 && c.kA.R0 == 0 && c.kA.s0 % 4 == 0)) return;
    int64_t P = c.M, Q = 1, sq = c.kA.s0 * c.K;
    if (c.rowA.R0 != 0 && c.rowA.R0 < c.M) {
        P = c.rowA.R0;
        Q = (c.M + P - 1) / P;
        sq = c.rowA.s1;
        if (P % kBM != 0 || c.M % P != 0 || sq % 4 != 0) return;  // whole slabs only
    }
    if (c.kA.s0 < P) return;
    const cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)c.K, (cuuint64_t)Q};
    const cuuint64_t strides[2] = {(cuuint64_t)c.kA.s0 * 4, (cuuint64_t)sq * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kBM, bk, 1};
    if (fn(&J.tmA, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return;
    J.tmaP = P;
    J.tma = 3;
}

// TMA stores of the fixed-point epilogue output (not for accumulating jobs):
// rows contiguous within slabs of tmcP rows (a multiple of the 32 rows one
// warp stores, whole slabs), or columns contiguous with one row stride.
static void setup_tmc(TcJob &J, const Contraction &c) {
    J.tmc = 0;
    if (c.accumulate || (reinterpret_cast<uintptr_t>(c.C) % 16) != 0 || c.M < 1 || c.N < 1) return;
    if (!J.cfix && !c.C_f64) return;  // staged value output is FP64
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn) return;
    const int64_t es = J.cfix ? 4 : 8;
    const CUtensorMapDataType dt = J.cfix ? CU_TENSOR_MAP_DATA_TYPE_INT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const cuuint32_t estr[3] = {1, 1, 1};
    void *base = c.C;
    if (c.rowC.s0 == 1 && c.colC.R0 == 0) {
        const int64_t cs = c.colC.s0;
        int64_t P = c.M, Q = 1, sq = cs * c.N;
        if (c.rowC.R0 != 0 && c.rowC.R0 < c.M) {
            P = c.rowC.R0;
            Q = c.M / P;
            sq = c.rowC.s1;
            if (P % 32 != 0 || c.M % P != 0) return;
        }
        if (cs < P || (cs * es) % 16 != 0 || (sq * es) % 16 != 0) return;
        const cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)c.N, (cuuint64_t)Q};
        const cuuint64_t strides[2] = {(cuuint64_t)(cs * es), (cuuint64_t)(sq * es)};
        const cuuint32_t box[3] = {32, 16, 1};
        if (fn(&J.tmC, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
        J.tmcP = P;
        J.tmc = 3;
        return;
    }
    if (c.colC.R0 == 0 && c.colC.s0 == 1 && c.rowC.R0 == 0) {
        const int64_t rs = c.rowC.s0;
        if (rs < c.N || (rs * es) % 16 != 0) return;
        const cuuint64_t dims[2] = {(cuuint64_t)c.N, (cuuint64_t)c.M};
        const cuuint64_t strides[1] = {(cuuint64_t)(rs * es)};
        const cuuint32_t box[2] = {16, 32};
        if (fn(&J.tmC, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
        J.tmc = 2;
    }
}

static constexpr size_t kSmemMax = 227 * 1024;

// want_stages / want_nacc > 0: the caller's choice, clamped to what fits.
static void pick_config(int form, int bn_max, int nkb_max, int &stages, int &nacc, int &nbuf, int &acc_cols,
                        size_t &smem, int want_stages = 0, int want_nacc = 0) {
    acc_cols = bn_max <= 32 ? 32 : (bn_max <= 64 ? 64 : (bn_max <= 128 ? 128 : 256));
    // two accumulator buffers (epilogue overlapped) when tensor memory
    // allows, then more accumulator sets per tile (accuracy)
    const int rg = 2;
    const int budget = std::max(1, 512 / (rg * acc_cols));  // NACC * NBUF
    nbuf = std::min(2, budget);
    nacc = std::max(1, std::min(4, budget / nbuf));
    if (want_nacc > 0) nacc = std::min(nacc, want_nacc);
    // the fixed-point form keeps one exact accumulator set per tile
    if (nkb_max < 2 || is_fx_form(form)) nacc = 1;
    const size_t a_st = (size_t)pieces_of_f(form) * kBM * kRowBytes;
    const size_t b_st = (size_t)pieces_of_f(form) * bn_max * kRowBytes;
    // alignment slack, barriers and the tensor-memory slot; the fixed-point
    // forms add a 1 KB column table per accumulator buffer
    const size_t extra = 1024 + (size_t)(2 * 8 + 2 * 4 + 4 + 2) * 8 + (is_fx_form(form) ? (size_t)nbuf * 1024 : 0);
    size_t raw = 0;
    switch (form) {
        case kTF32x3: raw = (size_t)RawCfg<kTF32x3>::STAGES * RawCfg<kTF32x3>::BYTES; break;
        case kBF16x3: raw = (size_t)RawCfg<kBF16x3>::STAGES * RawCfg<kBF16x3>::BYTES; break;
        case kFX32: raw = (size_t)RawCfg<kFX32>::STAGES * RawCfg<kFX32>::BYTES; break;
        case kFX32H: raw = (size_t)RawCfg<kFX32H>::STAGES * RawCfg<kFX32H>::BYTES; break;
        default: raw = (size_t)RawCfg<kBF16x6>::STAGES * RawCfg<kBF16x6>::BYTES; break;
    }
    stages = 1;
    while (stages < 8 && (size_t)(stages + 1) * (a_st + b_st) + raw + extra <= kSmemMax) ++stages;
    if (want_stages > 0) stages = std::min(stages, want_stages);
    smem = (size_t)stages * (a_st + b_st) + raw + extra;
}

template <int F, int MODE>
static cudaError_t launch_f(const TcLaunch &L, int grid, size_t smem, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(tcp_kernel<F, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    });
    if (attr != cudaSuccess) return attr;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)kPThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tcp_kernel<F, MODE>, L);
}

static int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// Runs the jobs (tile_begin / dep fields filled by the caller).  `table` is a
// device copy of the jobs when there are more than kMaxInline of them;
// `done` holds one int per job, zeroed here.
static cudaError_t tcp_launch(int form, const TcJob *jobs, int njobs, int total_tiles, int bn_max, int nkb_max,
                              const void *table, int *done, cudaStream_t st, FxScale *reset_next = nullptr,
                              int want_stages = 0, int want_nacc = 0, const int *tile_job = nullptr) {
    if (total_tiles <= 0) return cudaSuccess;
    TcLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.njobs = njobs;
    L.total_tiles = total_tiles;
    L.done = done;
    L.reset_next = reset_next;
    L.tile_job = njobs > kMaxInline ? tile_job : nullptr;
    if (njobs <= kMaxInline)
        for (int j = 0; j < njobs; ++j) L.inl[j] = jobs[j];
    else
        L.jobs = static_cast<const TcJob *>(table);
    size_t smem;
    pick_config(form, bn_max, nkb_max, L.stages, L.nacc, L.nbuf, L.acc_cols, smem, want_stages, want_nacc);
    L.bn_max = bn_max;
    L.dep_hold = g_dep_hold.load();
    L.dep_wait_ns = g_dep_wait_ns.load();
    if (L.dep_wait_ns == 0) L.dep_wait_ns = kWaitLimitNs;
    if (done != nullptr) {
        cudaError_t e = cudaMemsetAsync(done, 0, sizeof(int) * ((size_t)njobs + 1), st);
        if (e != cudaSuccess) return e;
    }
    const int grid = std::min(total_tiles, num_sms());
    bool wide = false, tma = false;  // the build: FP64 sources, FP64 outputs or accumulation; TMA staging
    for (int j = 0; j < njobs; ++j) {
        wide = wide || jobs[j].a64 != 0 || jobs[j].c64 != 0 || jobs[j].acc != 0;
        tma = tma || jobs[j].tma != 0;
    }
    const int mode = wide ? 2 : (tma ? 1 : 0);
    switch (form) {
#define KRON_TCP_SPLIT(FORM)                                                       \
    case FORM:                                                                     \
        return mode == 2 ? launch_f<FORM, 2>(L, grid, smem, st)                   \
                         : (mode == 1 ? launch_f<FORM, 1>(L, grid, smem, st)      \
                                      : launch_f<FORM, 0>(L, grid, smem, st));
        KRON_TCP_SPLIT(kTF32x3)
        KRON_TCP_SPLIT(kBF16x3)
        KRON_TCP_SPLIT(kBF16x6)
#undef KRON_TCP_SPLIT
        case kFX32: return launch_f<kFX32, 1>(L, grid, smem, st);    // 32-bit integer sources only
        case kFX32H: return launch_f<kFX32H, 1>(L, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

// One fixed-point contraction of form `form`: A is fixed point (int32) with
// scale fxA, the image of op(L) comes with its row exponents and row-sum
// bound; C is fixed point with scale fxC (cfix) or a value tensor.
cudaError_t tcp_contract_fx(int form, const Contraction &c, const void *img, const FxScale *fxA, const int *fxF,
                            const unsigned long long *fxG, FxScale *fxC, cudaStream_t st, FxScale *reset_next) {
    if (c.M == 0 || c.N == 0) return cudaSuccess;
    TcJob J = make_job(form, c, img);
    J.fxA = fxA;
    J.fxF = fxF;
    J.fxG = fxG;
    J.fxC = fxC;
    J.cfix = fxC != nullptr;
    J.a64 = 0;
    J.tile_begin = 0;
    setup_tma(form, J, c);
    setup_tmc(J, c);
    const int tiles = J.tiles_m * J.tiles_n;
    return tcp_launch(form, &J, 1, tiles, J.BN, J.nkb, nullptr, nullptr, st, reset_next);
}

// Rows r0..M-1 of a row map are the same map shifted by imap(m, r0): one
// level, one slab holding all M rows, or r0 on a slab boundary.
static bool shifts_at(const IdxMap &m, int64_t r0, int64_t M) { return m.R0 == 0 || M <= m.R0 || r0 % m.R0 == 0; }

cudaError_t tcp_contract_fx_tail(int form, const Contraction &c, const void *img, const void *img_half,
                                 const FxScale *fxA, const int *fxF, const unsigned long long *fxG, FxScale *fxC,
                                 FxScale *reset_next, cudaStream_t st) {
    if (c.M == 0 || c.N == 0) return cudaSuccess;
    TcJob J = make_job(form, c, img);
    const int tiles = J.tiles_m * J.tiles_n;
    const int grid = num_sms();
    const int tail = tiles % grid;
    const int64_t R1 = (int64_t)(tiles - tail) * kBM;
    const bool split = img_half != nullptr && J.tiles_n == 1 && J.BN % 32 == 0 && tiles > grid && tail > 0 &&
                       2 * tail <= grid && !c.A_f64 && shifts_at(c.rowA, R1, c.M) && shifts_at(c.rowC, R1, c.M);
    if (!split) return tcp_contract_fx(form, c, img, fxA, fxF, fxG, fxC, st, reset_next);
    // job 0: the full rounds
    J.M = R1;
    J.tiles_m = tiles - tail;
    J.fxA = fxA;
    J.fxF = fxF;
    J.fxG = fxG;
    J.fxC = fxC;
    J.cfix = fxC != nullptr;
    J.a64 = 0;
    J.tile_begin = 0;
    setup_tma(form, J, c);
    setup_tmc(J, c);
    // job 1: the remaining rows in tiles of half the width
    Contraction cb = c;
    cb.M = c.M - R1;
    cb.A = static_cast<const int32_t *>(c.A) + imap(c.rowA, R1);
    const size_t esC = c.C_f64 ? 8 : 4;  // fixed-point output: int32 or a value tensor (FP32 / FP64)
    cb.C = static_cast<uint8_t *>(c.C) + (size_t)imap(c.rowC, R1) * esC;
    TcJob H = make_job(form, cb, img_half, J.BN / 2);
    H.fxA = fxA;
    H.fxF = fxF;
    H.fxG = fxG;
    H.fxC = fxC;
    H.cfix = fxC != nullptr;
    H.a64 = 0;
    H.tile_begin = J.tiles_m * J.tiles_n;
    setup_tma(form, H, cb);
    setup_tmc(H, cb);
    TcJob jobs[2] = {J, H};
    return tcp_launch(form, jobs, 2, H.tile_begin + H.tiles_m * H.tiles_n, J.BN, J.nkb, nullptr, nullptr, st,
                      reset_next);
}

// One contraction with the B side from an image built by tc_build_bimage.
cudaError_t tcp_contract(int form, const Contraction &c, const void *img, cudaStream_t st) {
    if (c.M == 0 || c.N == 0) return cudaSuccess;
    TcJob J = make_job(form, c, img);
    J.tile_begin = 0;
    if (!c.A_f64) setup_tma(form, J, c);
    const int tiles = J.tiles_m * J.tiles_n;
    return tcp_launch(form, &J, 1, tiles, J.BN, J.nkb, nullptr, nullptr, st);
}

// ---------------------------------------------------------- job tables

void tcp_jobs_begin(TcpJobs &jobs, int form) {
    jobs.form = form;
    jobs.host.clear();
    jobs.tile_job.clear();
    jobs.total_tiles = 0;
    jobs.bn_max = 16;
    jobs.nkb_max = 1;
}

int tcp_jobs_add(TcpJobs &jobs, const Contraction &c, const void *img, int dep, int bn) {
    TcJob J = make_job(jobs.form, c, img, bn);
    J.tile_begin = jobs.total_tiles;
    J.dep = dep;
    if (dep >= 0) {
        TcJob *D = reinterpret_cast<TcJob *>(jobs.host.data()) + dep;
        J.dep_tiles = D->tiles_m * D->tiles_n;
        D->publish = 1;
    }
    jobs.total_tiles += J.tiles_m * J.tiles_n;
    jobs.tile_job.insert(jobs.tile_job.end(), (size_t)J.tiles_m * J.tiles_n, (int)(jobs.host.size() / sizeof(TcJob)));
    jobs.bn_max = std::max(jobs.bn_max, (int)J.BN);
    jobs.nkb_max = std::max(jobs.nkb_max, (int)J.nkb);
    const size_t off = jobs.host.size();
    jobs.host.resize(off + sizeof(TcJob));
    std::memcpy(jobs.host.data() + off, &J, sizeof(TcJob));
    return (int)(off / sizeof(TcJob));
}

size_t tcp_jobs_table_bytes(const TcpJobs &jobs) { return jobs.host.size(); }

cudaError_t tcp_jobs_run(const TcpJobs &jobs, const void *table, int *done, cudaStream_t st, const int *tile_job) {
    const int njobs = (int)(jobs.host.size() / sizeof(TcJob));
    return tcp_launch(jobs.form, reinterpret_cast<const TcJob *>(jobs.host.data()), njobs, jobs.total_tiles,
                      jobs.bn_max, jobs.nkb_max, table, done, st, nullptr, jobs.stages, jobs.nacc, tile_job);
}

}  // namespace kron
