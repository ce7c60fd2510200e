// tcg.cu -- a group of up to three consecutive small mu-mode products fused
// in one launch, the intermediates kept on chip (Definition "Tucker
// operator", Eq. (tuckerop): the d products in sequence; the remark in
// Section 2 that consecutive products need not go through memory in
// between, there merging the permutations).
//
// The group applies modes a, a+1, ..., a+g-1 (g <= 3, every m, n <= 32) of a
// column-major tensor whose modes before a have already been applied.  With
// P = prod of the sizes before a and Q = prod of the sizes after the group,
// the tensor is X[p, j_0, .., j_{g-1}, q]; a work unit is PB consecutive p
// (PB a power of two; 1 when P = 1, so that a unit is one contiguous slab)
// and one q.  Per unit, one CTA:
//   1. loads X[p0 .. p0+PB-1, :, :, :, q] into an FP32 staging array in
//      shared memory, one row per fibre of the first mode and the contracted
//      index k along the row (odd pitch: conflict-free for any lane order);
//   2. for each mode t of the group: splits the staged values into the
//      form's pieces (3xTF32 / BF16x3 / BF16x6) in the K-major 64-byte-
//      swizzled layout of the tcgen05 descriptors (up to four 128-row tiles);
//      tile by tile, one thread issues the MMAs of the tile against the
//      mode's op(L) image (kept in shared memory for the whole launch) into
//      tensor memory (hi * hi apart from the smaller products, as in the other
//      kernels; two B pieces per MMA where they sit side by side in the image)
//      while the next tile is converted; four groups of four warps,
//      one tile each, read the accumulators back and write the outputs into
//      the staging array as the rows of the next mode, or, after the last
//      mode, to global memory;
// so the group reads X and writes its output once.  Rows are ordered p
// fastest, then the other local indices in increasing order, so the global
// loads and stores run along p (or along the slab when P = 1).
// Every wait is bounded; a CTA's decision to stop is taken by one thread and
// shared through shared memory, so no thread is left at a barrier.
#include <algorithm>
#include <mutex>

#include "tc_common.cuh"

namespace kron {

namespace {

constexpr int kGThreads = 512;   // sixteen warps: four groups of one warp per tensor-memory lane quarter
constexpr int kPitch = 33;       // staging row pitch in floats (odd)
constexpr int kGMaxTiles = 4;    // rows per mode <= 512
constexpr uint32_t kTile = kBM * kRowBytes;  // one piece of one K-block of a 128-row tile

struct GLaunch {
    const float *src;
    void *dst;
    int dst64;
    int g;
    int cur[3][3];      // cur[t][dim]: sizes of the local dims when mode t is applied
    int K[3], N[3], BN[3], KB[3], rows[3], tiles[3];
    const uint8_t *img[3];   // images of op(L_t) in global memory
    uint32_t simg[3];        // their offsets in shared memory
    uint32_t img_bytes[3];
    int64_t P, Q;
    int PB, lpb;
    int64_t pblocks, units;
    int64_t Gin, Gout;       // elements of one (p, q) slab before / after the group
    uint32_t magic0;         // ceil(2^32 / cur[0][0]); unused when cur[0][0] = 1 (2^32 has no 32-bit form)
    uint32_t op_off, stage_off, bar_off;
    uint32_t stage2_off;     // FP32 variant: the second staging array
    const void *Lsrc[3];     // FP32 variant: L_t in global memory, ld, op = L^T, FP64 storage
    int64_t ldL[3];
    int ltrans, l64;
    uint32_t etab_off[3];    // per mode: table of the epilogue's per-row offsets (shared memory)
    int64_t estep[3];        // per mode: the offset's step per output column
    int kbmax;
    int bulk0;               // P = 1 and the slab copies as one bulk copy (16-byte multiple and aligned):
                             // mode 0's rows are then staged with pitch m_0 (the slab as it is)
};

__device__ __forceinline__ void named_bar(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// The dims other than t, in increasing order (g <= 3): their indices.
__device__ __forceinline__ void others(int g, int t, int &da, int &db) {
    da = db = -1;
    int c = 0;
    for (int d = 0; d < g; ++d) {
        if (d == t) continue;
        if (c == 0) da = d;
        else db = d;
        ++c;
    }
}

// Copies unit u of the group's input into the staging array with 4-byte
// asynchronous copies (element e = pb + PB (j_0 + cur0 (j_1 + cur1 j_2))
// goes to row pb + PB (j_1 + cur1 j_2), column j_0); threads t0, t0 + nt, ..
// take part.  Padding p (past P) is not copied: its rows only feed outputs
// that are never stored.
__device__ __forceinline__ void load_unit(const GLaunch &L, int64_t u, float *stage, int t0, int nt, uint64_t *bar_in) {
    if (L.bulk0) {
        // one slab, contiguous in memory and in the staging array (pitch m_0):
        // one bulk copy by the TMA unit, completing on bar_in
        if (t0 == 0) {
            const uint32_t bytes = (uint32_t)(L.Gin * 4);
            fence_proxy_async_smem();  // the stage's previous readers came first
            mbar_arrive_expect_tx(smem_u32(bar_in), bytes);
            bulk_g2s(smem_u32(stage), L.src + L.Gin * u, bytes, smem_u32(bar_in));
        }
        return;
    }
    const int64_t pblk = u % L.pblocks, q = u / L.pblocks;
    const int64_t p0 = pblk * L.PB;
    const int PB = L.PB;
    const int64_t pvalid = min((int64_t)PB, L.P - p0);
    const uint32_t E = (uint32_t)((int64_t)PB * L.Gin);
    const float *src = L.src + p0 + L.P * L.Gin * q;
    const uint32_t c0 = (uint32_t)L.cur[0][0];
    const uint32_t s0 = smem_u32(stage);
    for (uint32_t e = t0; e < E; e += nt) {
        const int pb = (int)(e & (uint32_t)(PB - 1));
        const uint32_t rest = e >> L.lpb;
        if (pb >= pvalid) continue;
        const uint32_t o = c0 == 1u ? rest : __umulhi(rest, L.magic0);  // rest / cur0
        const uint32_t srow = (uint32_t)pb + (uint32_t)PB * o;
        cp_async4(s0 + (srow * kPitch + (rest - o * c0)) * 4u, src + pb + L.P * (int64_t)rest, 4u);
    }
    cp_async_commit();
}

// Where the epilogue of mode t puts the outputs of row `row`: for a mode
// before the last, the word offset in the staging array of the next mode's
// row for output column 0 (the column adds estep[t] per step); for the last
// mode, the element offset in C apart from p0 and q (p0 + off + P Gout q).
// Rows are decoded as pb (fastest), then the dims other than t in increasing
// order.  The same for every unit: built once per CTA.
__device__ __forceinline__ int64_t epi_offset(const GLaunch &L, int t, int row) {
    const int PB = L.PB;
    const int pb = row & (PB - 1);
    int o = row >> L.lpb;
    int da, db;
    others(L.g, t, da, db);
    int j[3] = {0, 0, 0};
    if (da >= 0) {
        const int sa = L.cur[t][da];
        j[da] = o % sa;
        o /= sa;
    }
    if (db >= 0) j[db] = o;
    if (t < L.g - 1) {
        // next mode t + 1: rows over the dims other than t + 1 (sizes
        // cur[t + 1]), k = j[t + 1]; linear in j[t]
        int na, nb;
        others(L.g, t + 1, na, nb);
        const int sa = L.cur[t + 1][na >= 0 ? na : 0];
        const int ja = (na == t) ? 0 : (na >= 0 ? j[na] : 0);
        const int jb = (nb == t) ? 0 : (nb >= 0 ? j[nb] : 0);
        return (int64_t)(pb + PB * (ja + sa * jb)) * kPitch + j[t + 1];
    }
    // C: p + P (j_0 + n_0 (j_1 + n_1 j_2) + Gout q), j[t] = column
    int64_t idx = 0, mult = 1;
    for (int d = 0; d < L.g; ++d) {
        if (d != t) idx += mult * j[d];
        mult *= (d == t) ? L.N[t] : L.cur[t][d];
    }
    return pb + L.P * idx;
}

// Stores the N outputs of one row, column c at dst + c * step, in chunks of
// 16, 8 and 8 columns (chunks past N are skipped as a whole).
template <typename To>
__device__ __forceinline__ void store_outputs(To *dst, int64_t step, int N, const uint32_t (&r0)[32],
                                              const uint32_t (&r1)[32]) {
#pragma unroll
    for (int c = 0; c < 16; ++c)
        if (c < N) dst[c * step] = (To)(__uint_as_float(r1[c]) + __uint_as_float(r0[c]));
    if (N > 16) {
#pragma unroll
        for (int c = 16; c < 24; ++c)
            if (c < N) dst[c * step] = (To)(__uint_as_float(r1[c]) + __uint_as_float(r0[c]));
    }
    if (N > 24) {
#pragma unroll
        for (int c = 24; c < 32; ++c)
            if (c < N) dst[c * step] = (To)(__uint_as_float(r1[c]) + __uint_as_float(r0[c]));
    }
}

template <int F>
__global__ void __launch_bounds__(kGThreads, 1) tcg_kernel(const __grid_constant__ GLaunch L) {
    using T = FT<F>;
    constexpr int CH = 16 / T::ELEM;     // values per 16-byte chunk
    constexpr int BK = kRowBytes / T::ELEM;
    constexpr int kConvT = kGThreads - 32;  // converter threads (all warps but the last)
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_align1024(smem_raw);
    uint8_t *op = smem + L.op_off;
    float *stage = reinterpret_cast<float *>(smem + L.stage_off);
    uint64_t *bar_mma = reinterpret_cast<uint64_t *>(smem + L.bar_off);  // per tile: its MMAs completed
    uint64_t *bar_conv = bar_mma + kGMaxTiles;                            // per tile: its operand is written
    uint64_t *bar_in = bar_conv + kGMaxTiles;                             // the unit's input (bulk copy)
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_in + 1);
    int *flag = reinterpret_cast<int *>(tslot + 1);
    int *gflag = flag + 1;  // per tile: its waits ended in time
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == kGThreads / 32 - 1;

    if (tid == 0) {
        for (int i = 0; i < kGMaxTiles; ++i) {
            mbar_init(smem_u32(&bar_mma[i]), 1);
            mbar_init(smem_u32(&bar_conv[i]), kConvT / 32);
            gflag[i] = 1;
        }
        mbar_init(smem_u32(bar_in), 1);
        fence_mbar_init();
        *flag = 1;
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tslot), 512);
        tmem_relinquish();
    }
    // the images of op(L_t): small, loaded once (16-byte words)
    for (int t = 0; t < L.g; ++t) {
        const uint4 *s = reinterpret_cast<const uint4 *>(L.img[t]);
        uint4 *d = reinterpret_cast<uint4 *>(smem + L.simg[t]);
        for (uint32_t i = tid; i < L.img_bytes[t] / 16; i += kGThreads) d[i] = __ldg(s + i);
    }
    // the epilogue's per-row offsets of every mode
    for (int t = 0; t < L.g; ++t) {
        if (t < L.g - 1) {
            int *tab = reinterpret_cast<int *>(smem + L.etab_off[t]);
            for (int row = tid; row < L.rows[t]; row += kGThreads) tab[row] = (int)epi_offset(L, t, row);
        } else {
            long long *tab = reinterpret_cast<long long *>(smem + L.etab_off[t]);
            for (int row = tid; row < L.rows[t]; row += kGThreads) tab[row] = epi_offset(L, t, row);
        }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phases = 0;  // bit i: parity of tile i's two barriers
    uint32_t in_phase = 0;
    if (blockIdx.x < L.units) load_unit(L, blockIdx.x, stage, tid, kGThreads, bar_in);

    for (int64_t u = blockIdx.x; u < L.units; u += gridDim.x) {
        const int64_t pblk = u % L.pblocks, q = u / L.pblocks;
        const int64_t p0 = pblk * L.PB;
        const int PB = L.PB;
        const int64_t pvalid = min((int64_t)PB, L.P - p0);
        // ---- 1. the unit's input (copies issued during the previous unit)
        if (L.bulk0) {
            if (tid == 0 && !mbar_wait(smem_u32(bar_in), in_phase)) *flag = 0;
            in_phase ^= 1u;
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (*flag == 0) break;
        for (int t = 0; t < L.g; ++t) {
            const int K = L.K[t], N = L.N[t], rows = L.rows[t], tiles = L.tiles[t];
            const int kb_n = L.KB[t];
            const bool last = (t == L.g - 1);
            // ---- 2a. converters, tile by tile: staged rows -> pieces in the
            // K-major swizzled layout; each warp signals the tile's barrier.
            // Chunks past the last K-step of the MMAs are never read.
            if (!mma_warp) {
                // mode 0 of a bulk-copied slab is staged with pitch m_0
                const int pitch = (t == 0 && L.bulk0) ? L.K[0] : kPitch;
                const bool vec_rows = t == 0 && L.bulk0;
                const int kread = (K + T::MMA_K - 1) / T::MMA_K * T::MMA_K;
                const int nch = (kread + CH - 1) / CH;  // chunks read by the MMAs
                for (int tile = 0; tile < tiles; ++tile) {
                    // rows past the last fibre are not converted: the MMA turns
                    // whatever they hold into output rows that are never stored
                    // (every output row depends on its own operand row only)
                    const int rt = min(kBM, rows - tile * kBM);
                    const int items = kBM * nch;
                    for (int it = tid; it < items; it += kConvT) {
                        const int r = it % kBM, ch = it / kBM;
                        if (r >= rt) continue;
                        const int row = tile * kBM + r;
                        const int k0 = ch * CH;
                        const float *src = stage + row * pitch + k0;
                        float v[CH];
                        if (k0 + CH <= K && vec_rows) {
                            // pitch m_0, a multiple of four: 16-byte rows of
                            // eight lanes fall in distinct banks
#pragma unroll
                            for (int e = 0; e < CH; e += 4) *reinterpret_cast<float4 *>(&v[e]) = *reinterpret_cast<const float4 *>(src + e);
                        } else if (k0 + CH <= K) {
#pragma unroll
                            for (int e = 0; e < CH; ++e) v[e] = src[e];
                        } else {
#pragma unroll
                            for (int e = 0; e < CH; ++e) v[e] = k0 + e < K ? src[e] : 0.f;
                        }
                        uint4 out[T::PIECES];
                        split_pack<F, float>(v, out);
                        uint8_t *base = op + ((size_t)(tile * L.kbmax + (ch >> 2)) * T::PIECES) * kTile;
                        const uint32_t off = swz(r, ch & 3);
#pragma unroll
                        for (int p = 0; p < T::PIECES; ++p) *reinterpret_cast<uint4 *>(base + p * kTile + off) = out[p];
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&bar_conv[tile]));
                }
                // every converter has read the stage: the epilogue may write
                // the next mode's rows there, or, after the last mode, the
                // next unit's input may go there while this unit finishes
                named_bar(5, kConvT);
                if (last && u + gridDim.x < L.units) load_unit(L, u + gridDim.x, stage, tid, kConvT, bar_in);
            } else if (lane == 0) {
                // ---- 2b. the MMAs of each tile as soon as it is converted
                // op(L)'s pieces lie one after the other in its image (32 rows
                // each), so one MMA of N = 64 multiplies an A piece by two B
                // pieces at once; tensor memory per tile: Z = hi * hi, X = the
                // products of piece-index sum 1, Y (BF16x6) sum 2, 32 columns each
                const uint32_t idesc1 = make_idesc(T::FMT, kBM, (uint32_t)kTcgBN);
                const uint32_t idesc2 = make_idesc(T::FMT, kBM, (uint32_t)(2 * kTcgBN));
                const uint32_t img = smem_u32(smem + L.simg[t]);
                constexpr uint32_t PIECE_B = (uint32_t)kTcgBN * kRowBytes;
                const uint64_t adesc0 = smem_desc_kmajor(smem_u32(op), kRowBytes);
                const uint64_t bdesc0 = smem_desc_kmajor(img, kRowBytes);
                for (int tile = 0; tile < tiles; ++tile) {
                    if (!mbar_wait(smem_u32(&bar_conv[tile]), (phases >> tile) & 1u)) {
                        gflag[tile] = 0;
                        continue;  // its MMA barrier never completes: the tile's group times out too
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(tile * 128);
                    for (int kb = 0; kb < kb_n; ++kb) {
                        const int kval = min(BK, K - kb * BK);
                        const int ksteps = (kval + T::MMA_K - 1) / T::MMA_K;
                        // descriptor address fields advance by bytes / 16
                        const uint32_t a_off = (uint32_t)((tile * L.kbmax + kb) * T::PIECES) * kTile;
                        const uint32_t b_off = (uint32_t)(kb * T::PIECES) * PIECE_B;
                        for (int ks = 0; ks < ksteps; ++ks) {
                            const uint32_t acc = (kb == 0 && ks == 0) ? 0u : 1u;
                            auto a = [&](int p) { return adesc0 + ((a_off + p * kTile + ks * 32) >> 4); };
                            auto b = [&](int p) { return bdesc0 + ((b_off + p * PIECE_B + ks * 32) >> 4); };
                            if constexpr (T::PIECES == 2) {
                                tc_mma<T::KIND>(d, a(0), b(0), idesc2, acc);        // Z = a0 b0, X = a0 b1
                                tc_mma<T::KIND>(d + 32u, a(1), b(0), idesc1, 1u);   // X += a1 b0
                            } else {
                                tc_mma<T::KIND>(d, a(0), b(0), idesc1, acc);        // Z = a0 b0
                                tc_mma<T::KIND>(d + 32u, a(0), b(1), idesc2, acc);  // X = a0 b1, Y = a0 b2
                                tc_mma<T::KIND>(d + 32u, a(1), b(0), idesc2, 1u);   // X += a1 b0, Y += a1 b1
                                tc_mma<T::KIND>(d + 64u, a(2), b(0), idesc1, 1u);   // Y += a2 b0
                            }
                        }
                    }
                    tc_commit(smem_u32(&bar_mma[tile]));
                }
            }
            __syncwarp();  // the issuing lane rejoins its warp
            // ---- 2c. epilogue: each group of four warps (one per lane
            // quarter) takes one tile; its first thread waits for the tile's
            // MMAs, the group follows
            const int wg = warp >> 2;
            if (wg < tiles) {
                if ((tid & 127) == 0 && !mbar_wait(smem_u32(&bar_mma[wg]), (phases >> wg) & 1u)) gflag[wg] = 0;
                __syncwarp();
                named_bar(1 + wg, 128);
            }
            phases ^= (1u << tiles) - 1u;
            const bool good = wg < tiles && gflag[wg] != 0;
            const int qd = warp & 3;
            if (good) {
                const int tile = wg;
                tc_fence_after();
                // r1 = X (+ Y), the smaller products, then r0 = Z = hi * hi
                uint32_t r0[32], r1[32];
                const uint32_t ta = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(tile * 128);
                tmem_ld32(ta + 32u, r1);
                if constexpr (T::PIECES == 3) {
                    tmem_ld32(ta + 64u, r0);
                    tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < 32; ++c) r1[c] = __float_as_uint(__uint_as_float(r0[c]) + __uint_as_float(r1[c]));
                }
                tmem_ld32(ta, r0);
                tmem_ld_wait();
                const int row = tile * kBM + qd * 32 + lane;
                if (row < rows && (row & (PB - 1)) < pvalid) {
                    if (!last) {
                        const int off = reinterpret_cast<const int *>(smem + L.etab_off[t])[row];
                        store_outputs<float>(stage + off, L.estep[t], N, r0, r1);
                    } else {
                        const int64_t base = p0 + reinterpret_cast<const long long *>(smem + L.etab_off[t])[row] +
                                             L.P * L.Gout * q;
                        if (L.dst64) store_outputs<double>(static_cast<double *>(L.dst) + base, L.estep[t], N, r0, r1);
                        else store_outputs<float>(static_cast<float *>(L.dst) + base, L.estep[t], N, r0, r1);
                    }
                }
            }
            tc_fence_before();
            __syncthreads();
            // a tile whose wait ran out stops the CTA (decided the same way by
            // every thread: the flags were written before the barrier)
            for (int i = 0; i < tiles; ++i)
                if (gflag[i] == 0) *flag = 0;
            __syncthreads();
            if (*flag == 0) break;
        }
        if (*flag == 0) break;
    }
    cp_async_wait<0>();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// The FP32 CUDA-core variant of the fused group (same units, staging, rows
// and offsets): mode t reads the staged rows of one array and writes the next
// mode's rows into the other.  A weight that every lane of a warp needs costs
// a full register write-back per lane when it is loaded, so each thread
// takes a block of kFR rows x 4 output columns: per k it loads kFR row
// values and one 16-byte word of op(L_t)^T ([k][c], 32 columns) for
// 4 kFR fused multiply-adds.  Every output is one chain over k = 0 .. K-1
// in ascending order from zero.  The rows of a thread are rg, rg + RG, ..
// (RG = ceil(rows / kFR)), so that lanes with consecutive rg read rows of
// distinct banks and store consecutive outputs; the loops over k are
// unrolled to 32 (K <= 32), so that every shared-memory address is a
// register plus a constant.
constexpr int kFR = 4;
constexpr int kFWP4 = 8;  // op(L_t)^T rows: 32 floats (eight 16-byte words)

__global__ void __launch_bounds__(kGThreads, 1) tcf_kernel(const __grid_constant__ GLaunch L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_align1024(smem_raw);
    float *const stg0 = reinterpret_cast<float *>(smem + L.stage_off);
    float *const stg1 = reinterpret_cast<float *>(smem + L.stage2_off);
    auto stg = [&](int i) { return (i & 1) ? stg1 : stg0; };
    uint64_t *bar_in = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    int *flag = reinterpret_cast<int *>(bar_in + 1);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(smem_u32(bar_in), 1);
        fence_mbar_init();
        *flag = 1;
    }
    // op(L_t)^T in FP32: [k][c] with 32 columns, zero past N
    for (int t = 0; t < L.g; ++t) {
        float *d = reinterpret_cast<float *>(smem + L.simg[t]);
        const int K = L.K[t], N = L.N[t], wp = 4 * kFWP4;
        for (int i = tid; i < K * wp; i += kGThreads) {
            const int k = i / wp, c = i % wp;
            float v = 0.f;
            if (c < N) {
                const int64_t o = L.ltrans ? (int64_t)k + L.ldL[t] * c : (int64_t)c + L.ldL[t] * k;
                v = L.l64 ? (float)static_cast<const double *>(L.Lsrc[t])[o] : static_cast<const float *>(L.Lsrc[t])[o];
            }
            d[i] = v;
        }
    }
    for (int t = 0; t < L.g; ++t) {
        if (t < L.g - 1) {
            int *tab = reinterpret_cast<int *>(smem + L.etab_off[t]);
            for (int row = tid; row < L.rows[t]; row += kGThreads) tab[row] = (int)epi_offset(L, t, row);
        } else {
            long long *tab = reinterpret_cast<long long *>(smem + L.etab_off[t]);
            for (int row = tid; row < L.rows[t]; row += kGThreads) tab[row] = epi_offset(L, t, row);
        }
    }
    __syncthreads();
    uint32_t in_phase = 0;
    int b = 0;  // the staging array holding the unit's input
    if (blockIdx.x < L.units) load_unit(L, blockIdx.x, stg0, tid, kGThreads, bar_in);

    for (int64_t u = blockIdx.x; u < L.units; u += gridDim.x) {
        const int64_t pblk = u % L.pblocks, q = u / L.pblocks;
        const int64_t p0 = pblk * L.PB;
        const int PB = L.PB;
        const int64_t pvalid = min((int64_t)PB, L.P - p0);
        if (L.bulk0) {
            if (tid == 0 && !mbar_wait(smem_u32(bar_in), in_phase)) *flag = 0;
            in_phase ^= 1u;
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (*flag == 0) break;
        for (int t = 0; t < L.g; ++t) {
            const int K = L.K[t], N = L.N[t], rows = L.rows[t];
            const bool last = (t == L.g - 1);
            const float *in = stg(b + t);
            // mode 0 of a bulk-copied slab is staged with pitch m_0 (a multiple of four)
            const bool vec = t == 0 && L.bulk0;
            const int pitch = vec ? L.K[0] : kPitch;
            // the array the last mode does not read takes the next unit's input
            if (last && u + gridDim.x < L.units) load_unit(L, u + gridDim.x, stg(b + t + 1), tid, kGThreads, bar_in);
            const int RG = (rows + kFR - 1) / kFR;
            const int CG = (N + 3) / 4;
            const float4 *W4 = reinterpret_cast<const float4 *>(smem + L.simg[t]);
            for (int task = tid; task < RG * CG; task += kGThreads) {
                const int cg = task / RG, rg = task - cg * RG;
                // rows past the last are read as row rg (in bounds) and never stored
                int ro[kFR];  // the rows' word offsets in the staging array
#pragma unroll
                for (int j = 0; j < kFR; ++j) {
                    const int row = rg + j * RG;
                    ro[j] = (row < rows ? row : rg) * pitch;
                }
                float acc[kFR][4];
#pragma unroll
                for (int j = 0; j < kFR; ++j)
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
                const float4 *wc = W4 + cg;  // op(L_t)^T row k at wc[k * kFWP4]
                if (vec) {
#pragma unroll
                    for (int k = 0; k < 32; k += 4) {
                        if (k >= K) break;
                        float4 w[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) w[e] = wc[(k + e) * kFWP4];
#pragma unroll
                        for (int h = 0; h < kFR; h += 4) {
                            float4 xv[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) xv[j] = *reinterpret_cast<const float4 *>(in + ro[h + j] + k);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    const float x = e == 0 ? xv[j].x : e == 1 ? xv[j].y : e == 2 ? xv[j].z : xv[j].w;
                                    acc[h + j][0] = fmaf(x, w[e].x, acc[h + j][0]);
                                    acc[h + j][1] = fmaf(x, w[e].y, acc[h + j][1]);
                                    acc[h + j][2] = fmaf(x, w[e].z, acc[h + j][2]);
                                    acc[h + j][3] = fmaf(x, w[e].w, acc[h + j][3]);
                                }
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        if (k >= K) break;
                        const float4 w = wc[k * kFWP4];
#pragma unroll
                        for (int j = 0; j < kFR; ++j) {
                            const float x = in[ro[j] + k];
                            acc[j][0] = fmaf(x, w.x, acc[j][0]);
                            acc[j][1] = fmaf(x, w.y, acc[j][1]);
                            acc[j][2] = fmaf(x, w.z, acc[j][2]);
                            acc[j][3] = fmaf(x, w.w, acc[j][3]);
                        }
                    }
                }
                const int c0 = 4 * cg;
                const int64_t step = L.estep[t];
#pragma unroll
                for (int j = 0; j < kFR; ++j) {
                    const int row = rg + j * RG;
                    if (row >= rows || (row & (PB - 1)) >= pvalid) continue;
                    if (!last) {
                        float *dst = stg(b + t + 1) + reinterpret_cast<const int *>(smem + L.etab_off[t])[row] + c0 * step;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (c0 + i < N) dst[i * step] = acc[j][i];
                    } else {
                        const int64_t base = p0 + reinterpret_cast<const long long *>(smem + L.etab_off[t])[row] +
                                             L.P * L.Gout * q + c0 * step;
                        if (L.dst64) {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if (c0 + i < N) static_cast<double *>(L.dst)[base + i * step] = (double)acc[j][i];
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if (c0 + i < N) static_cast<float *>(L.dst)[base + i * step] = acc[j][i];
                        }
                    }
                }
            }
            __syncthreads();
        }
        b = (b + L.g) & 1;
    }
    cp_async_wait<0>();
    __syncthreads();
}

constexpr size_t kGSmemMax = 227 * 1024;

}  // namespace

static int g_pieces(int form) { return form == kBF16x6 ? 3 : 2; }
static int g_bk(int form) { return form == kTF32x3 ? kRowBytes / 4 : kRowBytes / 2; }

// Fills the launch for a group with p-blocks of at most pb_cap; false if it
// does not fit (sizes, shared memory).
// form kFusedFP32: the CUDA-core variant (no operand tiles, no images: op(L)
// in FP32 in shared memory; two staging arrays, mode t reading one and
// writing the other).
constexpr int kFusedFP32 = -2;

static bool tcg_plan_pb(int form, const GroupSpec &gs, int pb_cap, GLaunch &L, size_t &smem) {
    const bool fp32 = form == kFusedFP32;
    if (!fp32 && form != kTF32x3 && form != kBF16x3 && form != kBF16x6) return false;
    if (gs.g < 1 || gs.g > 3 || gs.P < 1 || gs.Q < 1) return false;
    L = GLaunch{};
    L.g = gs.g;
    int sz[3] = {1, 1, 1};
    for (int t = 0; t < gs.g; ++t) {
        if (gs.m[t] < 1 || gs.m[t] > 32 || gs.n[t] < 1 || gs.n[t] > 32) return false;
        sz[t] = (int)gs.m[t];
    }
    const int bk = fp32 ? 32 : g_bk(form);
    int64_t rows_max = 1;
    for (int t = 0; t < gs.g; ++t) {
        for (int d = 0; d < 3; ++d) L.cur[t][d] = d < gs.g ? sz[d] : 1;
        int64_t r = 1;
        for (int d = 0; d < gs.g; ++d)
            if (d != t) r *= sz[d];
        L.rows[t] = (int)r;  // times PB below
        rows_max = std::max(rows_max, r);
        L.K[t] = (int)gs.m[t];
        L.N[t] = (int)gs.n[t];
        L.BN[t] = kTcgBN;  // the image's N-tile (tc_build_bimage_bn with kTcgBN)
        L.KB[t] = (int)((gs.m[t] + bk - 1) / bk);
        sz[t] = (int)gs.n[t];
    }
    // p-block: one slab when P = 1; else the largest power of two with at
    // most 512 rows per mode (four tiles), at least 8 (32-byte runs) when P
    // allows
    // (at least 4 when P > 1: the loads take four consecutive p at a time)
    int PB = 1;
    if (gs.P > 1) {
        PB = 4;
        while (PB < pb_cap && (int64_t)PB * 2 * rows_max <= kGMaxTiles * kBM && PB * 2 <= gs.P) PB *= 2;
        if (PB < 8 && gs.P >= 8) return false;
    }
    if ((int64_t)PB * rows_max > kGMaxTiles * kBM) return false;
    L.PB = PB;
    L.lpb = 0;
    while ((1 << L.lpb) < PB) ++L.lpb;
    int kbmax = 1, tiles_max = 1;
    for (int t = 0; t < gs.g; ++t) {
        L.rows[t] *= PB;
        L.tiles[t] = (L.rows[t] + kBM - 1) / kBM;
        tiles_max = std::max(tiles_max, L.tiles[t]);
        kbmax = std::max(kbmax, L.KB[t]);
    }
    L.kbmax = kbmax;
    L.P = gs.P;
    L.Q = gs.Q;
    L.pblocks = (gs.P + PB - 1) / PB;
    L.units = L.pblocks * gs.Q;
    L.Gin = 1;
    L.Gout = 1;
    for (int t = 0; t < gs.g; ++t) {
        L.Gin *= gs.m[t];
        L.Gout *= gs.n[t];
    }
    L.magic0 = gs.m[0] == 1 ? 0u : (uint32_t)(((1ull << 32) + (uint64_t)gs.m[0] - 1) / (uint64_t)gs.m[0]);
    // shared memory: operand tiles, staging, images, barrier + slots
    size_t off = 0;
    L.op_off = 0;
    if (!fp32) off += (size_t)tiles_max * kbmax * g_pieces(form) * kTile;
    int64_t stage_rows = 0;
    for (int t = 0; t < gs.g; ++t) stage_rows = std::max<int64_t>(stage_rows, L.rows[t]);
    const size_t stage_bytes = ((size_t)stage_rows * kPitch * 4 + 1023) / 1024 * 1024;
    L.stage_off = (uint32_t)off;
    off += stage_bytes;
    if (fp32) {
        L.stage2_off = (uint32_t)off;
        off += stage_bytes;
        for (int t = 0; t < gs.g; ++t) {
            L.Lsrc[t] = gs.L[t];
            L.ldL[t] = gs.ldL[t];
            L.simg[t] = (uint32_t)off;  // op(L_t)^T in FP32, [k][c] with 32 columns
            L.img_bytes[t] = (uint32_t)(L.K[t] * 32 * 4);
            off += (L.img_bytes[t] + 127) / 128 * 128;
        }
        L.ltrans = gs.trans ? 1 : 0;
        L.l64 = gs.l64 ? 1 : 0;
    } else {
        for (int t = 0; t < gs.g; ++t) {
            L.img[t] = static_cast<const uint8_t *>(gs.img[t]);
            L.simg[t] = (uint32_t)off;
            L.img_bytes[t] = (uint32_t)(L.KB[t] * g_pieces(form) * L.BN[t] * kRowBytes);
            off += (L.img_bytes[t] + 1023) / 1024 * 1024;
        }
    }
    // the epilogue's per-row tables (int offsets before the last mode, 64-bit after)
    for (int t = 0; t < gs.g; ++t) {
        L.etab_off[t] = (uint32_t)off;
        off += ((size_t)L.rows[t] * (t < gs.g - 1 ? 4 : 8) + 127) / 128 * 128;
    }
    // and their steps per output column: before the last mode, PB times the
    // stride of dim t among the next mode's row dims (in increasing order),
    // in staging words; after it, P times the product of the sizes before t
    for (int t = 0; t < gs.g; ++t) {
        if (t < gs.g - 1) {
            int64_t stride = 1, rc = 0;
            for (int d = 0; d < gs.g; ++d) {
                if (d == t + 1) continue;
                if (d == t) rc = stride;
                stride *= L.cur[t + 1][d];
            }
            L.estep[t] = (int64_t)PB * rc * kPitch;
        } else {
            int64_t cs = 1;
            for (int d = 0; d < t; ++d) cs *= L.cur[t][d];
            L.estep[t] = gs.P * cs;
        }
    }
    L.bar_off = (uint32_t)off;
    off += 128;  // two barriers per tile, tensor-memory slot, flags
    smem = off + 1024;  // alignment slack
    return smem <= kGSmemMax;
}

// One CTA per SM (sixteen warps): the largest p-block that fits, so that a
// unit has as many tiles (work between two waits) as possible.
static bool tcg_plan(int form, const GroupSpec &gs, GLaunch &L, size_t &smem) {
    for (int cap = 512; cap >= 8; cap /= 2) {
        if (tcg_plan_pb(form, gs, cap, L, smem)) return true;
        if (gs.P == 1) break;  // one slab per unit: nothing to shrink
    }
    return false;
}

bool tcf_fits(const GroupSpec &gs) {
    GLaunch L;
    size_t smem = 0;
    return tcg_plan(kFusedFP32, gs, L, smem);
}

static cudaError_t tcf_launch(const GLaunch &L, size_t smem, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(tcf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmemMax);
    });
    if (attr != cudaSuccess) return attr;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>(L.units, (int64_t)std::max(1, sms));
    tcf_kernel<<<(unsigned)grid, kGThreads, smem, st>>>(L);
    return cudaGetLastError();
}

cudaError_t tcf_run(const GroupSpec &gs, const float *src, void *dst, bool dst64, cudaStream_t st) {
    GLaunch L;
    size_t smem = 0;
    if (!tcg_plan(kFusedFP32, gs, L, smem)) return cudaErrorInvalidValue;
    if (L.units == 0) return cudaSuccess;
    L.src = src;
    L.dst = dst;
    L.dst64 = dst64 ? 1 : 0;
    const bool base16 = (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    L.bulk0 = (base16 && L.P == 1 && L.Gin % 4 == 0 && L.K[0] % 4 == 0) ? 1 : 0;
    return tcf_launch(L, smem, st);
}

bool tcg_fits(int form, const GroupSpec &gs) {
    GLaunch L;
    size_t smem = 0;
    return tcg_plan(form, gs, L, smem);
}

template <int F>
static cudaError_t tcg_launch_f(const GLaunch &L, size_t smem, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(tcg_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmemMax);
    });
    if (attr != cudaSuccess) return attr;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one resident CTA per SM: each takes all 512 columns of tensor memory
    (void)per_sm;
    per_sm = 1;
    const int64_t grid = std::min<int64_t>(L.units, (int64_t)std::max(1, sms) * per_sm);
    tcg_kernel<F><<<(unsigned)grid, kGThreads, smem, st>>>(L);
    return cudaGetLastError();
}

cudaError_t tcg_run(int form, const GroupSpec &gs, const float *src, void *dst, bool dst64, cudaStream_t st) {
    GLaunch L;
    size_t smem = 0;
    if (!tcg_plan(form, gs, L, smem)) return cudaErrorInvalidValue;
    if (L.units == 0) return cudaSuccess;
    L.src = src;
    L.dst = dst;
    L.dst64 = dst64 ? 1 : 0;
    // four consecutive elements of a group start 16-byte aligned: P = 1 with
    // slabs of a multiple of four, or p-blocks (PB >= 4) with P a multiple of four
    const bool base16 = (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    L.bulk0 = (base16 && L.P == 1 && L.Gin % 4 == 0 && L.K[0] % 4 == 0) ? 1 : 0;
    switch (form) {
        case kTF32x3: return tcg_launch_f<kTF32x3>(L, smem, st);
        case kBF16x3: return tcg_launch_f<kBF16x3>(L, smem, st);
        case kBF16x6: return tcg_launch_f<kBF16x6>(L, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace kron
