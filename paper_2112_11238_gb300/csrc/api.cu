// api.cu -- the extern "C" boundary of libkron (declared in include/kron.h):
// argument validation, plans, workspace layout, and the host drivers of the
// mu-mode product, the Tucker chain, its adjoint and the exponential stepper.
// Every step of the computation runs in the kernels of tc.cu / simt.cu /
// expm.cu / batched.cu; this file only decides what to launch.
#include <algorithm>
#include <mutex>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace kron;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

kron_status cuda_status(cudaError_t e) { return e == cudaSuccess ? KRON_OK : KRON_ERR_CUDA; }

bool valid_dtype(kron_dtype t) { return t == KRON_F64 || t == KRON_F32; }
bool valid_prec(kron_prec p) { return p >= KRON_PREC_FP64 && p <= KRON_PREC_FX32H; }
size_t esize(kron_dtype t) { return t == KRON_F64 ? 8 : 4; }

// Element size of the intermediates of a precision.
size_t inter_size(kron_prec p) { return p == KRON_PREC_FP64 ? 8 : 4; }

int64_t prod(const int64_t *v, int lo, int hi) {
    int64_t p = 1;
    for (int k = lo; k < hi; ++k) p *= v[k];
    return p;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Geometry of one mu-mode product inside a chain: the input has sizes cur[],
// mode mu (0-based) of size m is mapped to n.
struct ModeGeom {
    int64_t P, Q, m, n;
};

ModeGeom mode_geom(int d, const int64_t *cur, int mu, int64_t n) {
    return ModeGeom{prod(cur, 0, mu), prod(cur, mu + 1, d), cur[mu], n};
}

// Contraction of a mu-mode product for the tensor-core path: rows are the
// fibres (p, q) of the tensor, columns the n outputs of a fibre, k the mode.
Contraction tc_mode_contraction(const ModeGeom &g, const void *src, bool src64, const void *L,
                                bool L64, int64_t ldL, bool transL, void *dst, bool dst64) {
    Contraction c;
    c.M = g.P * g.Q;
    c.N = g.n;
    c.K = g.m;
    c.A = src;
    c.A_f64 = src64;
    if (g.P == 1) {
        c.rowA = IdxMap{0, g.m, 0};
        c.rowC = IdxMap{0, g.n, 0};
    } else {
        c.rowA = IdxMap{g.P, 1, g.P * g.m};
        c.rowC = IdxMap{g.P, 1, g.P * g.n};
    }
    c.kA = IdxMap{0, g.P, 0};
    c.B = L;
    c.B_f64 = L64;
    if (!transL) {
        c.colB = IdxMap{0, 1, 0};
        c.kB = IdxMap{0, ldL, 0};
    } else {
        c.colB = IdxMap{0, ldL, 0};
        c.kB = IdxMap{0, 1, 0};
    }
    c.C = dst;
    c.C_f64 = dst64;
    c.colC = IdxMap{0, g.P, 0};
    return c;
}

// Contraction of a mu-mode product for the CUDA-core path.  For mu with
// P == 1 the roles are swapped (rows = outputs of a fibre, columns = fibres)
// so that both loads and stores stay contiguous.
Contraction simt_mode_contraction(const ModeGeom &g, const void *src, bool src64, const void *L,
                                  bool L64, int64_t ldL, bool transL, void *dst, bool dst64) {
    if (g.P != 1) return tc_mode_contraction(g, src, src64, L, L64, ldL, transL, dst, dst64);
    Contraction c;
    c.M = g.n;
    c.N = g.Q;
    c.K = g.m;
    c.A = L;
    c.A_f64 = L64;
    if (!transL) {
        c.rowA = IdxMap{0, 1, 0};
        c.kA = IdxMap{0, ldL, 0};
    } else {
        c.rowA = IdxMap{0, ldL, 0};
        c.kA = IdxMap{0, 1, 0};
    }
    c.B = src;
    c.B_f64 = src64;
    c.colB = IdxMap{0, g.m, 0};
    c.kB = IdxMap{0, 1, 0};
    c.C = dst;
    c.C_f64 = dst64;
    c.rowC = IdxMap{0, 1, 0};
    c.colC = IdxMap{0, g.n, 0};
    return c;
}

kron_status check_shape(int d, const int64_t *m, const int64_t *n) {
    if (d < 1 || d > KRON_MAX_D || !m || !n) return KRON_ERR_INVALID_ARG;
    long double in = 1, out = 1;
    for (int k = 0; k < d; ++k) {
        if (m[k] < 1 || n[k] < 1) return KRON_ERR_INVALID_ARG;
        in *= (long double)m[k];
        out *= (long double)n[k];
    }
    // every intermediate is bounded by prod(max(m, n))
    long double mx = 1;
    for (int k = 0; k < d; ++k) mx *= (long double)std::max(m[k], n[k]);
    if (mx > (long double)(1ll << 40)) return KRON_ERR_UNSUPPORTED;
    (void)in;
    (void)out;
    return KRON_OK;
}

}  // namespace

struct kron_plan_s {
    int d;
    int64_t m[KRON_MAX_D], n[KRON_MAX_D];
    kron_dtype dtype;
    kron_prec prec;
    unsigned flags;
    int order[KRON_MAX_D];
    // workspace layout of kron_tucker
    size_t img_off[KRON_MAX_D], img_bytes[KRON_MAX_D];
    size_t buf_off[2], buf_bytes;
    // fixed-point form: row exponents and row-sum bounds of every image, the
    // fixed-point copy of T, three scale words and a scratch word
    size_t fxf_off[KRON_MAX_D], fxg_off[KRON_MAX_D], fxin_off, fxsc_off;
    size_t ws_bytes;
};

namespace {

// Applies the chain of the plan in its order.  src (dtype of the plan) ->
// dst (dtype); intermediates in ws buffers.  Images of the split L live in
// ws at the plan's offsets.
kron_status run_chain_fx(const kron_plan_s *pl, const void *T, const void *const *L, const int64_t *ldL,
                         void *S, uint8_t *ws, cudaStream_t st, bool trans, bool acc_last) {
    const int d = pl->d;
    const bool io64 = pl->dtype == KRON_F64;
    FxScale *sc = reinterpret_cast<FxScale *>(ws + pl->fxsc_off);  // [0] input, [1], [2] buffers
    auto *scratch = reinterpret_cast<unsigned long long *>(sc + 3);
    auto *xin = reinterpret_cast<int32_t *>(ws + pl->fxin_off);
    const int form = form_of(pl->prec);
    if (fx_from_float(form, T, io64, prod(pl->m, 0, d), xin, &sc[0], scratch, st) != cudaSuccess)
        return KRON_ERR_CUDA;
    int64_t cur[KRON_MAX_D];
    for (int k = 0; k < d; ++k) cur[k] = pl->m[k];
    const void *src = xin;
    const FxScale *ssrc = &sc[0];
    for (int s = 0; s < d; ++s) {
        const int mu = pl->order[s];
        const ModeGeom g = mode_geom(d, cur, mu, pl->n[mu]);
        const bool last = (s == d - 1);
        void *dst = last ? S : (void *)(ws + pl->buf_off[s & 1]);
        FxScale *sdst = last ? nullptr : &sc[1 + (s & 1)];
        Contraction c = tc_mode_contraction(g, src, false, L[mu], io64, ldL[mu], trans, dst, last ? io64 : false);
        c.accumulate = last && acc_last;
        void *img = ws + pl->img_off[mu];
        int *f = reinterpret_cast<int *>(ws + pl->fxf_off[mu]);
        auto *gb = reinterpret_cast<unsigned long long *>(ws + pl->fxg_off[mu]);
        cudaError_t e = fx_build_bimage(form, c, img, f, gb, st);
        if (e == cudaSuccess && sdst) e = fx_reset(sdst, st);
        if (e == cudaSuccess) e = tcp_contract_fx(form, c, img, ssrc, f, gb, sdst, st);
        if (e != cudaSuccess) return KRON_ERR_CUDA;
        cur[mu] = pl->n[mu];
        src = dst;
        ssrc = sdst;
    }
    return KRON_OK;
}

// Size of the fused group of small modes that starts at chain step s (the
// modes order[s], order[s] + 1, .. applied one after the other), 0 if none:
// split forms and FP32, up to three modes (FP32: at least two, from a whole
// slab), the largest group whose sizes fit the fused kernel.  cur: the sizes before step s.  A group may not end with the
// chain's last step when that step accumulates into S.
int chain_group(const kron_plan_s *pl, int s, const int64_t *cur, bool acc_last, GroupSpec &gs) {
    const bool fp32 = pl->prec == KRON_PREC_FP32;
    if ((!is_split(pl->prec) && !fp32) || (pl->flags & KRON_PLAN_UNFUSED)) return 0;
    const int d = pl->d, mu = pl->order[s];
    // FP32: a single mode runs faster on the per-mode kernel
    for (int gg = std::min(3, d - s); gg >= (fp32 ? 2 : 1); --gg) {
        bool ok = !(acc_last && s + gg == d);
        for (int t = 0; t < gg && ok; ++t) ok = pl->order[s + t] == mu + t;
        if (!ok) continue;
        GroupSpec c;
        c.g = gg;
        c.P = prod(cur, 0, mu);
        c.Q = prod(cur, mu + gg, d);
        for (int t = 0; t < gg; ++t) {
            c.m[t] = cur[mu + t];
            c.n[t] = pl->n[mu + t];
        }
        // FP32: only whole slabs (P = 1; the strided groups stream slower
        // than the per-mode kernel)
        if (fp32 ? (c.P == 1 && tcf_fits(c)) : tcg_fits(form_of(pl->prec), c)) {
            gs = c;
            return gg;
        }
    }
    return 0;
}

// acc_last: the last product adds into S instead of overwriting it.
kron_status run_chain(const kron_plan_s *pl, const void *T, const void *const *L, const int64_t *ldL,
                      void *S, uint8_t *ws, cudaStream_t st, bool trans, bool acc_last = false) {
    if (is_fx(pl->prec)) return run_chain_fx(pl, T, L, ldL, S, ws, st, trans, acc_last);
    const int d = pl->d;
    const bool io64 = pl->dtype == KRON_F64;
    const bool split = is_split(pl->prec);
    const int form = form_of(pl->prec);
    const bool i64 = pl->prec == KRON_PREC_FP64;
    int64_t cur[KRON_MAX_D];
    for (int k = 0; k < d; ++k) cur[k] = pl->m[k];
    if (split) {
        // the images of every op(L_mu) the chain uses, in one launch: the
        // chain's steps are walked once ahead (fused group: 32-column tiles)
        Contraction ic[KRON_MAX_D];
        void *iimg[KRON_MAX_D];
        int ibn[KRON_MAX_D];
        int cnt = 0;
        int64_t pc[KRON_MAX_D];
        for (int k = 0; k < d; ++k) pc[k] = pl->m[k];
        bool p64 = io64;
        for (int s = 0; s < d;) {
            GroupSpec gs;
            const int gsz = !p64 ? chain_group(pl, s, pc, acc_last, gs) : 0;
            const int steps = gsz > 0 ? gsz : 1;
            for (int t = 0; t < steps; ++t) {
                const int nu = pl->order[s + t];
                ic[cnt] = tc_mode_contraction(mode_geom(d, pc, nu, pl->n[nu]), nullptr, false, L[nu], io64, ldL[nu],
                                              trans, nullptr, false);
                iimg[cnt] = ws + pl->img_off[nu];
                ibn[cnt] = gsz > 0 ? kTcgBN : tc_tile_n(form, pl->n[nu]);
                ++cnt;
                pc[nu] = pl->n[nu];
            }
            s += steps;
            p64 = (s == d) ? io64 : false;
        }
        if (tc_build_bimages(form, cnt, ic, iimg, ibn, st) != cudaSuccess) return KRON_ERR_CUDA;
    }
    const void *src = T;
    bool src64 = io64;
    int writes = 0;  // intermediates written so far (ping-pong buffers)
    for (int s = 0; s < d; ++s) {
        const int mu = pl->order[s];
        const ModeGeom g = mode_geom(d, cur, mu, pl->n[mu]);
        // split forms: consecutive small modes mu, mu + 1, .. applied in a row
        // run as one fused group with the intermediates on chip
        // (FP32: the same groups on the CUDA cores)
        GroupSpec gs;
        const bool fp32 = pl->prec == KRON_PREC_FP32;
        const int gsz = ((split || fp32) && !src64) ? chain_group(pl, s, cur, acc_last, gs) : 0;
        if (gsz > 0 && fp32) {
            for (int t = 0; t < gsz; ++t) {
                gs.L[t] = L[mu + t];
                gs.ldL[t] = ldL[mu + t];
            }
            gs.trans = trans;
            gs.l64 = io64;
            const bool last = (s + gsz == d);
            void *dst = last ? S : (void *)(ws + pl->buf_off[writes & 1]);
            const bool dst64 = last ? io64 : false;
            if (tcf_run(gs, static_cast<const float *>(src), dst, dst64, st) != cudaSuccess) return KRON_ERR_CUDA;
            for (int t = 0; t < gsz; ++t) cur[mu + t] = pl->n[mu + t];
            src = dst;
            src64 = dst64;
            ++writes;
            s += gsz - 1;
            continue;
        }
        for (int t = 0; t < gsz; ++t) gs.img[t] = ws + pl->img_off[mu + t];
        if (gsz > 0) {
            const bool last = (s + gsz == d);
            void *dst = last ? S : (void *)(ws + pl->buf_off[writes & 1]);
            const bool dst64 = last ? io64 : false;
            if (tcg_run(form, gs, static_cast<const float *>(src), dst, dst64, st) != cudaSuccess) return KRON_ERR_CUDA;
            for (int t = 0; t < gsz; ++t) cur[mu + t] = pl->n[mu + t];
            src = dst;
            src64 = dst64;
            ++writes;
            s += gsz - 1;
            continue;
        }
        const bool last = (s == d - 1);
        void *dst = last ? S : (void *)(ws + pl->buf_off[writes & 1]);
        const bool dst64 = last ? io64 : (split ? false : i64);
        cudaError_t e;
        if (split) {
            Contraction c = tc_mode_contraction(g, src, src64, L[mu], io64, ldL[mu], trans, dst, dst64);
            c.accumulate = last && acc_last;
            e = tcp_contract(form, c, ws + pl->img_off[mu], st);  // image built above
        } else if (simt_small_fits(i64, g.m, g.n)) {
            // small factor: one thread per fibre, op(L) in shared memory
            Contraction c = tc_mode_contraction(g, src, src64, L[mu], io64, ldL[mu], trans, dst, dst64);
            c.accumulate = last && acc_last;
            e = simt_contract_small(i64, c, st);
        } else {
            Contraction c =
                simt_mode_contraction(g, src, src64, L[mu], io64, ldL[mu], trans, dst, dst64);
            c.accumulate = last && acc_last;
            e = simt_contract(i64, c, st);
        }
        if (e != cudaSuccess) return KRON_ERR_CUDA;
        cur[mu] = pl->n[mu];
        src = dst;
        src64 = dst64;
        ++writes;
    }
    return KRON_OK;
}

void plan_layout(kron_plan_s *pl) {
    const int d = pl->d;
    size_t off = 0;
    const int form = form_of(pl->prec);
    for (int k = 0; k < d; ++k) {
        pl->img_off[k] = off;
        pl->img_bytes[k] = form >= 0 ? tc_bimage_bytes(form, pl->n[k], pl->m[k]) : 0;
        // small modes of the split forms may run in a fused group, whose image
        // has N-tiles of kTcgBN columns
        if (is_split(pl->prec) && pl->n[k] <= kTcgBN && pl->m[k] <= kTcgBN)
            pl->img_bytes[k] = std::max(pl->img_bytes[k], tc_bimage_bytes_bn(form, pl->n[k], pl->m[k], kTcgBN));
        off += align_up(pl->img_bytes[k]);
    }
    // largest intermediate (outputs of steps 0..d-2)
    int64_t cur[KRON_MAX_D];
    for (int k = 0; k < d; ++k) cur[k] = pl->m[k];
    int64_t mx = 0;
    for (int s = 0; s < d - 1; ++s) {
        cur[pl->order[s]] = pl->n[pl->order[s]];
        mx = std::max(mx, prod(cur, 0, d));
    }
    pl->buf_bytes = align_up((size_t)mx * inter_size(pl->prec));
    pl->buf_off[0] = off;
    pl->buf_off[1] = off + pl->buf_bytes;
    off += 2 * pl->buf_bytes;
    if (is_fx(pl->prec)) {
        for (int k = 0; k < d; ++k) {
            pl->fxf_off[k] = off;
            off += align_up((size_t)pl->n[k] * sizeof(int));
            pl->fxg_off[k] = off;
            off += kAlign;
        }
        pl->fxin_off = off;
        off += align_up((size_t)prod(pl->m, 0, d) * sizeof(int32_t));
        pl->fxsc_off = off;
        off += kAlign;
    }
    pl->ws_bytes = std::max<size_t>(off, kAlign);
}

void choose_order(kron_plan_s *pl) {
    const int d = pl->d;
    int perm[KRON_MAX_D];
    for (int k = 0; k < d; ++k) perm[k] = pl->order[k] = k;
    if (pl->flags & KRON_PLAN_NATURAL_ORDER) return;
    long double best = -1;
    do {
        int64_t cur[KRON_MAX_D];
        for (int k = 0; k < d; ++k) cur[k] = pl->m[k];
        long double fl = 0;
        for (int s = 0; s < d; ++s) {
            const int mu = perm[s];
            fl += 2.0L * pl->n[mu] * (long double)prod(cur, 0, d);
            cur[mu] = pl->n[mu];
        }
        if (best < 0 || fl < best * (1 - 1e-12L)) {
            best = fl;
            for (int k = 0; k < d; ++k) pl->order[k] = perm[k];
        }
    } while (std::next_permutation(perm, perm + d));
}

}  // namespace

extern "C" {

const char *kron_status_string(kron_status s) {
    switch (s) {
        case KRON_OK: return "KRON_OK";
        case KRON_ERR_INVALID_ARG: return "KRON_ERR_INVALID_ARG";
        case KRON_ERR_UNSUPPORTED: return "KRON_ERR_UNSUPPORTED";
        case KRON_ERR_ALIGNMENT: return "KRON_ERR_ALIGNMENT";
        case KRON_ERR_WORKSPACE: return "KRON_ERR_WORKSPACE";
        case KRON_ERR_CUDA: return "KRON_ERR_CUDA";
        case KRON_ERR_TIMEOUT: return "KRON_ERR_TIMEOUT";
        case KRON_ERR_NUMERIC: return "KRON_ERR_NUMERIC";
    }
    return "KRON_ERR_UNKNOWN";
}

int kron_version(void) { return 100; }

kron_status kron_get_device_error(kron_stream_t stream, int *code, int clear) {
    if (!code) return KRON_ERR_INVALID_ARG;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    unsigned a = 0, b = 0, c = 0;
    if (tc_error_word(&a, clear != 0, cs) != cudaSuccess) return KRON_ERR_CUDA;
    if (tcp_error_word(&b, clear != 0, cs) != cudaSuccess) return KRON_ERR_CUDA;
    if (expm_error_word(&c, clear != 0, cs) != cudaSuccess) return KRON_ERR_CUDA;
    const unsigned w = a | b | c;
    *code = (int)w;
    if (w & 1u) return KRON_ERR_TIMEOUT;
    if (w & 2u) return KRON_ERR_NUMERIC;
    return KRON_OK;
}

kron_status kron_debug_dependency_timeout(int hold, double limit_ms) {
    if (!(limit_ms >= 0.0) || limit_ms > 10000.0) return KRON_ERR_INVALID_ARG;
    tcp_debug_dependency_timeout(hold != 0, (unsigned long long)(limit_ms * 1e6));
    return KRON_OK;
}

// ------------------------------------------------------------ mu-mode product

kron_status kron_mump_workspace_size(int d, const int64_t *m, int mu, int64_t n, kron_dtype dtype,
                                     kron_prec prec, size_t *bytes) {
    if (!bytes || !valid_dtype(dtype) || !valid_prec(prec)) return KRON_ERR_INVALID_ARG;
    if (d < 1 || d > KRON_MAX_D || !m || mu < 0 || mu >= d || n < 1) return KRON_ERR_INVALID_ARG;
    for (int k = 0; k < d; ++k)
        if (m[k] < 1) return KRON_ERR_INVALID_ARG;
    const int form = form_of(prec);
    *bytes = align_up(form >= 0 ? tc_bimage_bytes(form, n, m[mu]) : 0);
    if (is_fx(prec))  // + row exponents, row-sum bound, fixed-point T, scales
        *bytes += align_up((size_t)n * sizeof(int)) + kAlign + align_up((size_t)prod(m, 0, d) * 4) + kAlign;
    if (*bytes == 0) *bytes = kAlign;
    return KRON_OK;
}

kron_status kron_mump(int d, const int64_t *m, int mu, int64_t n, const void *T, const void *L,
                      int64_t ldL, int transL, void *S, kron_dtype dtype, kron_prec prec, void *ws,
                      size_t ws_bytes, kron_stream_t stream) {
    size_t need = 0;
    kron_status st = kron_mump_workspace_size(d, m, mu, n, dtype, prec, &need);
    if (st != KRON_OK) return st;
    if (!T || !L || !S) return KRON_ERR_INVALID_ARG;
    if (transL ? ldL < m[mu] : ldL < n) return KRON_ERR_INVALID_ARG;
    const size_t es = esize(dtype);
    if (!aligned(T, es) || !aligned(L, es) || !aligned(S, es)) return KRON_ERR_ALIGNMENT;
    if (is_split(prec) || is_fx(prec)) {
        if (!ws) return KRON_ERR_INVALID_ARG;
        if (!aligned(ws, kAlign)) return KRON_ERR_ALIGNMENT;
        if (ws_bytes < need) return KRON_ERR_WORKSPACE;
    }
    const ModeGeom g = mode_geom(d, m, mu, n);
    const bool io64 = dtype == KRON_F64;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (is_fx(prec)) {
        auto *w = static_cast<uint8_t *>(ws);
        const int form = form_of(prec);
        size_t off = align_up(tc_bimage_bytes(form, n, m[mu]));
        int *f = reinterpret_cast<int *>(w + off);
        off += align_up((size_t)n * sizeof(int));
        auto *gb = reinterpret_cast<unsigned long long *>(w + off);
        off += kAlign;
        auto *X = reinterpret_cast<int32_t *>(w + off);
        off += align_up((size_t)prod(m, 0, d) * 4);
        auto *sc = reinterpret_cast<FxScale *>(w + off);
        auto *scratch = reinterpret_cast<unsigned long long *>(sc + 1);
        Contraction c = tc_mode_contraction(g, X, false, L, io64, ldL, transL != 0, S, io64);
        e = fx_from_float(form, T, io64, prod(m, 0, d), X, sc, scratch, cs);
        if (e == cudaSuccess) e = fx_build_bimage(form, c, w, f, gb, cs);
        if (e == cudaSuccess) e = tcp_contract_fx(form, c, w, sc, f, gb, nullptr, cs);
    } else if (is_split(prec)) {
        const int form = form_of(prec);
        Contraction c = tc_mode_contraction(g, T, io64, L, io64, ldL, transL != 0, S, io64);
        e = tc_build_bimage(form, c, ws, cs);
        if (e == cudaSuccess) e = tcp_contract(form, c, ws, cs);
    } else {
        Contraction c = simt_mode_contraction(g, T, io64, L, io64, ldL, transL != 0, S, io64);
        e = simt_contract(prec == KRON_PREC_FP64, c, cs);
    }
    return cuda_status(e);
}

// ------------------------------------------------------------------- plans

kron_status kron_plan_create(kron_plan *plan, int d, const int64_t *m, const int64_t *n, kron_dtype dtype,
                             kron_prec prec, unsigned flags) {
    if (!plan) return KRON_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!valid_dtype(dtype) || !valid_prec(prec)) return KRON_ERR_INVALID_ARG;
    if (flags & ~(KRON_PLAN_TRANS_L | KRON_PLAN_NATURAL_ORDER | KRON_PLAN_UNFUSED)) return KRON_ERR_INVALID_ARG;
    kron_status st = check_shape(d, m, n);
    if (st != KRON_OK) return st;
    auto *pl = new (std::nothrow) kron_plan_s();
    if (!pl) return KRON_ERR_INVALID_ARG;
    pl->d = d;
    for (int k = 0; k < d; ++k) {
        pl->m[k] = m[k];
        pl->n[k] = n[k];
    }
    pl->dtype = dtype;
    pl->prec = prec;
    pl->flags = flags;
    choose_order(pl);
    plan_layout(pl);
    *plan = pl;
    return KRON_OK;
}

kron_status kron_plan_destroy(kron_plan plan) {
    delete plan;
    return KRON_OK;
}

kron_status kron_plan_workspace_size(kron_plan plan, size_t *bytes) {
    if (!plan || !bytes) return KRON_ERR_INVALID_ARG;
    *bytes = plan->ws_bytes;
    return KRON_OK;
}

kron_status kron_plan_launches(kron_plan plan, int *sizes, int *count) {
    if (!plan || !sizes || !count) return KRON_ERR_INVALID_ARG;
    const int d = plan->d;
    int64_t cur[KRON_MAX_D];
    for (int k = 0; k < d; ++k) cur[k] = plan->m[k];
    bool src64 = plan->dtype == KRON_F64;
    int c = 0;
    for (int s = 0; s < d;) {
        GroupSpec gs;
        int g = src64 ? 0 : chain_group(plan, s, cur, false, gs);
        if (g == 0) g = 1;
        for (int t = 0; t < g; ++t) cur[plan->order[s + t]] = plan->n[plan->order[s + t]];
        sizes[c++] = g;
        s += g;
        src64 = false;  // the intermediates are FP32 (split forms) or of the plan's precision
        if (plan->prec == KRON_PREC_FP64) src64 = true;
    }
    *count = c;
    return KRON_OK;
}

kron_status kron_plan_order(kron_plan plan, int *order) {
    if (!plan || !order) return KRON_ERR_INVALID_ARG;
    for (int k = 0; k < plan->d; ++k) order[k] = plan->order[k];
    return KRON_OK;
}

double kron_plan_flops(kron_plan plan) {
    if (!plan) return 0.0;
    int64_t cur[KRON_MAX_D];
    for (int k = 0; k < plan->d; ++k) cur[k] = plan->m[k];
    double fl = 0;
    for (int s = 0; s < plan->d; ++s) {
        const int mu = plan->order[s];
        fl += 2.0 * (double)plan->n[mu] * (double)prod(cur, 0, plan->d);
        cur[mu] = plan->n[mu];
    }
    return fl;
}

static kron_status check_L(const kron_plan_s *pl, const void *const *L, const int64_t *ldL, bool trans) {
    if (!L || !ldL) return KRON_ERR_INVALID_ARG;
    const size_t es = esize(pl->dtype);
    for (int k = 0; k < pl->d; ++k) {
        if (!L[k]) return KRON_ERR_INVALID_ARG;
        if (!aligned(L[k], es)) return KRON_ERR_ALIGNMENT;
        if (trans ? ldL[k] < pl->m[k] : ldL[k] < pl->n[k]) return KRON_ERR_INVALID_ARG;
    }
    return KRON_OK;
}

static kron_status check_ws(const void *ws, size_t ws_bytes, size_t need) {
    if (need > 0 && !ws) return KRON_ERR_INVALID_ARG;
    if (ws && !aligned(ws, kAlign)) return KRON_ERR_ALIGNMENT;
    if (ws_bytes < need) return KRON_ERR_WORKSPACE;
    return KRON_OK;
}

kron_status kron_tucker(kron_plan plan, const void *T, const void *const *L, const int64_t *ldL, void *S,
                        void *ws, size_t ws_bytes, kron_stream_t stream) {
    if (!plan || !T || !S) return KRON_ERR_INVALID_ARG;
    const bool trans = (plan->flags & KRON_PLAN_TRANS_L) != 0;
    kron_status st = check_L(plan, L, ldL, trans);
    if (st != KRON_OK) return st;
    const size_t es = esize(plan->dtype);
    if (!aligned(T, es) || !aligned(S, es)) return KRON_ERR_ALIGNMENT;
    st = check_ws(ws, ws_bytes, plan->ws_bytes);
    if (st != KRON_OK) return st;
    return run_chain(plan, T, L, ldL, S, static_cast<uint8_t *>(ws),
                     reinterpret_cast<cudaStream_t>(stream), trans);
}

// ------------------------------------------------------ complex Tucker
//
// Workspace: [M_mu x d: real 2n x 2m matrices][images x d][X0][X1]
namespace {

struct CtLayout {
    size_t M[KRON_MAX_D], img[KRON_MAX_D], buf[2], total;
};

CtLayout ct_layout(const kron_plan_s *pl) {
    CtLayout s{};
    const int d = pl->d;
    const int form = form_of(pl->prec);
    const size_t es = esize(pl->dtype);
    size_t off = 0;
    for (int k = 0; k < d; ++k) {
        s.M[k] = off;
        off += align_up((size_t)(4 * pl->n[k] * pl->m[k]) * es);
    }
    for (int k = 0; k < d; ++k) {
        s.img[k] = off;
        off += align_up(form >= 0 ? tc_bimage_bytes(form, 2 * pl->n[k], 2 * pl->m[k]) : 0);
    }
    int64_t cur[KRON_MAX_D];
    for (int k = 0; k < d; ++k) cur[k] = pl->m[k];
    int64_t mx = 0;
    for (int st = 0; st < d - 1; ++st) {
        cur[pl->order[st]] = pl->n[pl->order[st]];
        mx = std::max(mx, prod(cur, 0, d));
    }
    const size_t bb = align_up((size_t)(2 * mx) * inter_size(pl->prec));
    s.buf[0] = off;
    s.buf[1] = off + bb;
    off += 2 * bb;
    s.total = std::max<size_t>(off, kAlign);
    return s;
}

// A complex mu-mode product as one real contraction over the (real,
// imaginary) view of the tensors: rows are the fibres (p, q) (real offset
// 2p + 2Pmq), the contracted index c + 2k runs over the part c and the mode
// index k (real offset c + 2Pk), the output column c' + 2j likewise; the B
// operand is the real 2n x 2m matrix made by complex_expand.  For P == 1
// the (part, index) pairs are contiguous and the maps have one level.
Contraction c_mode_contraction(const ModeGeom &g, const void *src, bool src64, const void *M, bool M64, void *dst,
                               bool dst64) {
    Contraction c;
    c.M = g.P * g.Q;
    c.N = 2 * g.n;
    c.K = 2 * g.m;
    c.A = src;
    c.A_f64 = src64;
    if (g.P == 1) {
        c.rowA = IdxMap{0, 2 * g.m, 0};
        c.rowC = IdxMap{0, 2 * g.n, 0};
        c.kA = IdxMap{0, 1, 0};
        c.colC = IdxMap{0, 1, 0};
    } else {
        c.rowA = IdxMap{g.P, 2, 2 * g.P * g.m};
        c.rowC = IdxMap{g.P, 2, 2 * g.P * g.n};
        c.kA = IdxMap{2, 1, 2 * g.P};
        c.colC = IdxMap{2, 1, 2 * g.P};
    }
    c.B = M;
    c.B_f64 = M64;
    c.colB = IdxMap{0, 1, 0};
    c.kB = IdxMap{0, 2 * g.n, 0};
    c.C = dst;
    c.C_f64 = dst64;
    return c;
}

kron_status run_chain_c(const kron_plan_s *pl, const void *T, void *S, uint8_t *ws, const CtLayout &lay,
                        cudaStream_t st) {
    const int d = pl->d;
    const bool io64 = pl->dtype == KRON_F64;
    const bool split = is_split(pl->prec);
    const int form = form_of(pl->prec);
    const bool i64 = pl->prec == KRON_PREC_FP64;
    int64_t cur[KRON_MAX_D];
    for (int k = 0; k < d; ++k) cur[k] = pl->m[k];
    const void *src = T;
    bool src64 = io64;
    for (int s = 0; s < d; ++s) {
        const int mu = pl->order[s];
        const ModeGeom g = mode_geom(d, cur, mu, pl->n[mu]);
        const bool last = (s == d - 1);
        void *dst = last ? S : (void *)(ws + lay.buf[s & 1]);
        const bool dst64 = last ? io64 : (split ? false : i64);
        Contraction c = c_mode_contraction(g, src, src64, ws + lay.M[mu], io64, dst, dst64);
        cudaError_t e;
        if (split) {
            void *img = ws + lay.img[mu];
            e = tc_build_bimage(form, c, img, st);
            if (e == cudaSuccess) e = tcp_contract(form, c, img, st);
        } else {
            e = simt_contract(i64, c, st);
        }
        if (e != cudaSuccess) return KRON_ERR_CUDA;
        cur[mu] = pl->n[mu];
        src = dst;
        src64 = dst64;
    }
    return KRON_OK;
}

}  // namespace

kron_status kron_ctucker_workspace_size(kron_plan plan, size_t *bytes) {
    if (!plan || !bytes) return KRON_ERR_INVALID_ARG;
    if (is_fx(plan->prec)) return KRON_ERR_UNSUPPORTED;
    *bytes = ct_layout(plan).total;
    return KRON_OK;
}

kron_status kron_ctucker(kron_plan plan, const void *T, const void *const *L, const int64_t *ldL, int conj, void *S,
                         void *ws, size_t ws_bytes, kron_stream_t stream) {
    if (!plan || !T || !S || !L || !ldL || (conj != 0 && conj != 1)) return KRON_ERR_INVALID_ARG;
    if (is_fx(plan->prec)) return KRON_ERR_UNSUPPORTED;
    const bool trans = (plan->flags & KRON_PLAN_TRANS_L) != 0;
    const size_t es2 = 2 * esize(plan->dtype);  // one complex element
    if (!aligned(T, es2) || !aligned(S, es2)) return KRON_ERR_ALIGNMENT;
    for (int k = 0; k < plan->d; ++k) {
        if (!L[k]) return KRON_ERR_INVALID_ARG;
        if (!aligned(L[k], es2)) return KRON_ERR_ALIGNMENT;
        if (trans ? ldL[k] < plan->m[k] : ldL[k] < plan->n[k]) return KRON_ERR_INVALID_ARG;
    }
    const CtLayout lay = ct_layout(plan);
    kron_status st = check_ws(ws, ws_bytes, lay.total);
    if (st != KRON_OK) return st;
    auto *w = static_cast<uint8_t *>(ws);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const bool io64 = plan->dtype == KRON_F64;
    for (int k = 0; k < plan->d; ++k)
        if (complex_expand(L[k], io64, ldL[k], plan->n[k], plan->m[k], trans, conj != 0, w + lay.M[k], cs) !=
            cudaSuccess)
            return KRON_ERR_CUDA;
    return run_chain_c(plan, T, S, w, lay, cs);
}

// ----------------------------------------------------------------- adjoint
//
// Workspace: [img fwd x d][img trans x d][X0][X1][G0][G1][partial]
namespace {
struct AdjLayout {
    size_t img_f[KRON_MAX_D], img_t[KRON_MAX_D];
    size_t x[2], g[2], partial, total;
    size_t xbytes, gbytes;
};

AdjLayout adjoint_layout(const kron_plan_s *pl) {
    AdjLayout a{};
    const int d = pl->d;
    const int form = form_of(pl->prec);
    const size_t isz = inter_size(pl->prec);
    size_t off = 0;
    for (int k = 0; k < d; ++k) {
        a.img_f[k] = off;
        off += align_up(form >= 0 ? tc_bimage_bytes(form, pl->n[k], pl->m[k]) : 0);
        a.img_t[k] = off;
        off += align_up(form >= 0 ? tc_bimage_bytes(form, pl->m[k], pl->n[k]) : 0);
    }
    // X_mu (mu >= 1): sizes n_1..n_{mu-1}, m_mu..m_d ; G_mu: n_1..n_{mu-1}, m_mu.. and n_mu..
    int64_t mx = 1;
    int64_t cur[KRON_MAX_D];
    for (int k = 0; k < d; ++k) cur[k] = pl->m[k];
    for (int s = 0; s <= d; ++s) {
        mx = std::max(mx, prod(cur, 0, d));
        if (s < d) cur[s] = pl->n[s];
    }
    a.xbytes = a.gbytes = align_up((size_t)mx * isz);
    a.x[0] = off; off += a.xbytes;
    a.x[1] = off; off += a.xbytes;
    a.g[0] = off; off += a.gbytes;
    a.g[1] = off; off += a.gbytes;
    size_t pb = 0;
    for (int mu = 0; mu < d; ++mu) {
        // dL_mu contraction: M = n_mu, N = m_mu, K = prod of the others
        int64_t K = 1;
        for (int k = 0; k < mu; ++k) K *= pl->n[k];
        for (int k = mu + 1; k < d; ++k) K *= pl->m[k];
        const size_t b = form >= 0 ? tc_splitk_partial_bytes(pl->n[mu], pl->m[mu], K)
                                   : simt_splitk_partial_bytes(pl->prec == KRON_PREC_FP64, pl->n[mu],
                                                               pl->m[mu], K);
        pb = std::max(pb, b);
    }
    a.partial = off;
    off += align_up(pb);
    a.total = std::max<size_t>(off, kAlign);
    return a;
}

// One mode product inside the adjoint (either path).
cudaError_t adj_mode(const kron_plan_s *pl, const ModeGeom &g, const void *src, bool src64, const void *L,
                     int64_t ldL, bool trans, void *dst, bool dst64, uint8_t *img, cudaStream_t st) {
    const bool io64 = pl->dtype == KRON_F64;
    if (is_split(pl->prec)) {
        const int form = form_of(pl->prec);
        Contraction c = tc_mode_contraction(g, src, src64, L, io64, ldL, trans, dst, dst64);
        cudaError_t e = tc_build_bimage(form, c, img, st);
        if (e != cudaSuccess) return e;
        return tcp_contract(form, c, img, st);
    }
    Contraction c = simt_mode_contraction(g, src, src64, L, io64, ldL, trans, dst, dst64);
    return simt_contract(pl->prec == KRON_PREC_FP64, c, st);
}
}  // namespace

kron_status kron_adjoint_workspace_size(kron_plan plan, size_t *bytes) {
    if (!plan || !bytes) return KRON_ERR_INVALID_ARG;
    *bytes = adjoint_layout(plan).total;
    return KRON_OK;
}

kron_status kron_tucker_adjoint(kron_plan plan, const void *T, const void *const *L, const int64_t *ldL,
                                const void *dS, void *dT, void *const *dL, void *ws, size_t ws_bytes,
                                kron_stream_t stream) {
    if (!plan || !dS) return KRON_ERR_INVALID_ARG;
    if (plan->flags & KRON_PLAN_TRANS_L) return KRON_ERR_UNSUPPORTED;
    if (is_fx(plan->prec)) return KRON_ERR_UNSUPPORTED;
    kron_status st = check_L(plan, L, ldL, false);
    if (st != KRON_OK) return st;
    const int d = plan->d;
    bool want_dL = false;
    if (dL)
        for (int k = 0; k < d; ++k) want_dL |= dL[k] != nullptr;
    if (want_dL && !T) return KRON_ERR_INVALID_ARG;
    const size_t es = esize(plan->dtype);
    if (!aligned(dS, es) || (dT && !aligned(dT, es)) || (T && !aligned(T, es))) return KRON_ERR_ALIGNMENT;
    if (dL)
        for (int k = 0; k < d; ++k)
            if (dL[k] && !aligned(dL[k], es)) return KRON_ERR_ALIGNMENT;
    const AdjLayout lay = adjoint_layout(plan);
    st = check_ws(ws, ws_bytes, lay.total);
    if (st != KRON_OK) return st;
    auto *w = static_cast<uint8_t *>(ws);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const bool io64 = plan->dtype == KRON_F64;
    const bool i64 = plan->prec == KRON_PREC_FP64;
    const bool split = is_split(plan->prec);
    const int form = form_of(plan->prec);

    // G holds the cotangent of X_{mu+1}; sizes gcur.
    int64_t gcur[KRON_MAX_D];
    for (int k = 0; k < d; ++k) gcur[k] = plan->n[k];
    const void *G = dS;
    bool G64 = io64;
    int gsel = 0;
    for (int mu = d - 1; mu >= 0; --mu) {
        if (dL && dL[mu]) {
            // X_mu = T x_1 L_1 ... x_{mu-1} L_{mu-1}, recomputed from T
            int64_t xcur[KRON_MAX_D];
            for (int k = 0; k < d; ++k) xcur[k] = plan->m[k];
            const void *X = T;
            bool X64 = io64;
            for (int nu = 0; nu < mu; ++nu) {
                const ModeGeom g = mode_geom(d, xcur, nu, plan->n[nu]);
                void *dst = w + lay.x[nu & 1];
                if (adj_mode(plan, g, X, X64, L[nu], ldL[nu], false, dst, i64, w + lay.img_f[nu], cs) !=
                    cudaSuccess)
                    return KRON_ERR_CUDA;
                xcur[nu] = plan->n[nu];
                X = dst;
                X64 = i64;
            }
            // dL_mu(i, j) = sum_{p,q} G(p, i, q) X(p, j, q): M = n_mu, N = m_mu
            const int64_t P = prod(xcur, 0, mu), Q = prod(xcur, mu + 1, d);
            const int64_t nm = plan->n[mu], mm = plan->m[mu];
            Contraction c;
            c.M = nm;
            c.N = mm;
            c.K = P * Q;
            c.A = G;
            c.A_f64 = G64;
            c.rowA = IdxMap{0, P, 0};
            c.kA = (P == 1) ? IdxMap{0, nm, 0} : IdxMap{P, 1, P * nm};
            c.B = X;
            c.B_f64 = X64;
            c.colB = IdxMap{0, P, 0};
            c.kB = (P == 1) ? IdxMap{0, mm, 0} : IdxMap{P, 1, P * mm};
            c.C = dL[mu];
            c.C_f64 = io64;
            c.rowC = IdxMap{0, 1, 0};
            c.colC = IdxMap{0, nm, 0};
            cudaError_t e = split ? tc_contract_splitk(form, c, reinterpret_cast<float *>(w + lay.partial), cs)
                                  : simt_contract_splitk(i64, c, w + lay.partial, cs);
            if (e != cudaSuccess) return KRON_ERR_CUDA;
        }
        if (mu == 0 && !dT) break;
        // G_mu = G_{mu+1} x_mu L_mu^T
        const ModeGeom g = mode_geom(d, gcur, mu, plan->m[mu]);
        const bool lastg = (mu == 0);
        void *dst = lastg ? dT : (void *)(w + lay.g[gsel]);
        const bool dst64 = lastg ? io64 : i64;
        if (adj_mode(plan, g, G, G64, L[mu], ldL[mu], true, dst, dst64, w + lay.img_t[mu], cs) != cudaSuccess)
            return KRON_ERR_CUDA;
        gcur[mu] = plan->m[mu];
        G = dst;
        G64 = dst64;
        gsel ^= 1;
    }
    return KRON_OK;
}

// ------------------------------------------------------- matrix exponential

kron_status kron_expm_workspace_size(int64_t n, size_t *bytes) {
    if (!bytes || n < 1 || n > 1024) return KRON_ERR_INVALID_ARG;
    *bytes = align_up(expm_workspace_bytes(n));
    return KRON_OK;
}

kron_status kron_expm(int64_t n, const double *A, int64_t ldA, double tau, double *E, void *ws,
                      size_t ws_bytes, kron_stream_t stream) {
    size_t need = 0;
    kron_status st = kron_expm_workspace_size(n, &need);
    if (st != KRON_OK) return st;
    if (!A || !E || ldA < n) return KRON_ERR_INVALID_ARG;
    if (!aligned(A, 8) || !aligned(E, 8)) return KRON_ERR_ALIGNMENT;
    st = check_ws(ws, ws_bytes, need);
    if (st != KRON_OK) return st;
    return cuda_status(expm_pade13(n, A, ldA, tau, E, ws, reinterpret_cast<cudaStream_t>(stream)));
}

// ------------------------------------------------------- Kronecker-sum action
//
// S = sum_mu V x_mu op(L_mu) (Eq. (actkron)): d mode products that all read
// V; the first writes S, the others accumulate.  Workspace: [image][fixed
// point: row exponents, row-sum bound, fixed-point V, scale words].
namespace {
struct KsvLayout {
    size_t img, fxf, fxg, fxv, fxsc, total;
};

KsvLayout kronsumv_layout(const kron_plan_s *pl) {
    KsvLayout l{};
    const int form = form_of(pl->prec);
    size_t img = 0;
    int64_t nmax = 1;
    for (int k = 0; k < pl->d; ++k) {
        if (form >= 0) img = std::max(img, tc_bimage_bytes(form, pl->n[k], pl->n[k]));
        nmax = std::max(nmax, pl->n[k]);
    }
    size_t off = 0;
    l.img = off;
    off += align_up(img);
    if (is_fx(pl->prec)) {
        l.fxf = off;
        off += align_up((size_t)nmax * sizeof(int));
        l.fxg = off;
        off += kAlign;
        l.fxv = off;
        off += align_up((size_t)prod(pl->n, 0, pl->d) * 4);
        l.fxsc = off;
        off += kAlign;
    }
    l.total = std::max(off, kAlign);
    return l;
}

bool square_plan(const kron_plan_s *pl) {
    for (int k = 0; k < pl->d; ++k)
        if (pl->m[k] != pl->n[k]) return false;
    return true;
}
}  // namespace

kron_status kron_kronsumv_workspace_size(kron_plan plan, size_t *bytes) {
    if (!plan || !bytes) return KRON_ERR_INVALID_ARG;
    if (!square_plan(plan)) return KRON_ERR_INVALID_ARG;
    *bytes = kronsumv_layout(plan).total;
    return KRON_OK;
}

kron_status kron_kronsumv(kron_plan plan, const void *V, const void *const *L, const int64_t *ldL, void *S,
                          void *ws, size_t ws_bytes, kron_stream_t stream) {
    if (!plan || !V || !S || V == S) return KRON_ERR_INVALID_ARG;
    if (!square_plan(plan)) return KRON_ERR_INVALID_ARG;
    const bool trans = (plan->flags & KRON_PLAN_TRANS_L) != 0;
    kron_status st = check_L(plan, L, ldL, trans);
    if (st != KRON_OK) return st;
    const size_t es = esize(plan->dtype);
    if (!aligned(V, es) || !aligned(S, es)) return KRON_ERR_ALIGNMENT;
    const KsvLayout lay = kronsumv_layout(plan);
    st = check_ws(ws, ws_bytes, lay.total);
    if (st != KRON_OK) return st;
    auto *w = static_cast<uint8_t *>(ws);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const int d = plan->d;
    const bool io64 = plan->dtype == KRON_F64;
    const int form = form_of(plan->prec);
    cudaError_t e = cudaSuccess;
    int32_t *X = nullptr;
    FxScale *sc = nullptr;
    if (is_fx(plan->prec)) {
        X = reinterpret_cast<int32_t *>(w + lay.fxv);
        sc = reinterpret_cast<FxScale *>(w + lay.fxsc);
        e = fx_from_float(form, V, io64, prod(plan->n, 0, d), X, sc, reinterpret_cast<unsigned long long *>(sc + 1),
                          cs);
    }
    for (int mu = 0; mu < d && e == cudaSuccess; ++mu) {
        const ModeGeom g = mode_geom(d, plan->n, mu, plan->n[mu]);
        if (is_fx(plan->prec)) {
            Contraction c = tc_mode_contraction(g, X, false, L[mu], io64, ldL[mu], trans, S, io64);
            c.accumulate = mu > 0;
            int *f = reinterpret_cast<int *>(w + lay.fxf);
            auto *gb = reinterpret_cast<unsigned long long *>(w + lay.fxg);
            e = fx_build_bimage(form, c, w + lay.img, f, gb, cs);
            if (e == cudaSuccess) e = tcp_contract_fx(form, c, w + lay.img, sc, f, gb, nullptr, cs);
        } else if (is_split(plan->prec)) {
            Contraction c = tc_mode_contraction(g, V, io64, L[mu], io64, ldL[mu], trans, S, io64);
            c.accumulate = mu > 0;
            e = tc_build_bimage(form, c, w + lay.img, cs);
            if (e == cudaSuccess) e = tcp_contract(form, c, w + lay.img, cs);
        } else {
            Contraction c = simt_mode_contraction(g, V, io64, L[mu], io64, ldL[mu], trans, S, io64);
            c.accumulate = mu > 0;
            e = simt_contract(plan->prec == KRON_PREC_FP64, c, cs);
        }
    }
    return cuda_status(e);
}

// ------------------------------------------------------------ inverse Tucker
//
// S = V x_1 op(P_1)^{-1} ... x_d op(P_d)^{-1} (Eq. (preconnd)).  Workspace:
// [inversion x d][inverses in FP32 (FP32 plans)][chain of the plan]
// [refinement: S and P_mu in FP64 (FP32 plans), forward result Y (FP64),
//  residual R (plan dtype), chain of an FP64 plan].
namespace {
struct ItLayout {
    size_t inv[KRON_MAX_D], pin32[KRON_MAX_D], chain, s64, p64[KRON_MAX_D], y64, r, chain64, total;
    kron_plan_s pl64;  // the same shapes in FP64 (residual of the refinement)
};

ItLayout itucker_layout(const kron_plan_s *pl, int refine) {
    ItLayout l{};
    const int d = pl->d;
    const bool f32 = pl->dtype == KRON_F32;
    const int64_t N = prod(pl->n, 0, d);
    size_t off = 0;
    for (int k = 0; k < d; ++k) {
        l.inv[k] = off;
        off += align_up(inv_workspace_bytes(pl->n[k]));
    }
    for (int k = 0; k < d; ++k) {
        l.pin32[k] = off;
        if (f32) off += align_up((size_t)pl->n[k] * pl->n[k] * 4);
    }
    l.chain = off;
    off += align_up(pl->ws_bytes);
    if (refine > 0) {
        l.pl64 = *pl;
        l.pl64.dtype = KRON_F64;
        l.pl64.prec = KRON_PREC_FP64;
        plan_layout(&l.pl64);
        l.s64 = off;
        if (f32) off += align_up((size_t)N * 8);
        for (int k = 0; k < d; ++k) {
            l.p64[k] = off;
            if (f32) off += align_up((size_t)pl->n[k] * pl->n[k] * 8);
        }
        l.y64 = off;
        off += align_up((size_t)N * 8);
        l.r = off;
        off += align_up((size_t)N * esize(pl->dtype));
        l.chain64 = off;
        off += align_up(l.pl64.ws_bytes);
    }
    l.total = std::max(off, kAlign);
    return l;
}

// dst[i + ldd j] = src[i + lds j] for an r x c block, FP64/FP32 either side.
__global__ void cast2d_kernel(const void *src, bool s64, int64_t lds, void *dst, bool d64, int64_t ldd, int64_t r,
                              int64_t c) {
    const int64_t total = r * c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % r, j = e / r;
        const double v = s64 ? static_cast<const double *>(src)[i + lds * j]
                             : (double)static_cast<const float *>(src)[i + lds * j];
        if (d64) static_cast<double *>(dst)[i + ldd * j] = v;
        else static_cast<float *>(dst)[i + ldd * j] = (float)v;
    }
}

cudaError_t cast2d(const void *src, bool s64, int64_t lds, void *dst, bool d64, int64_t ldd, int64_t r, int64_t c,
                   cudaStream_t st) {
    const int64_t total = r * c;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
    cast2d_kernel<<<blocks, 256, 0, st>>>(src, s64, lds, dst, d64, ldd, r, c);
    return cudaGetLastError();
}

// R = V - Y (Y FP64), R and V in the plan dtype.
__global__ void residual_kernel(const void *V, const double *Y, void *R, bool io64, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (io64) static_cast<double *>(R)[i] = static_cast<const double *>(V)[i] - Y[i];
        else static_cast<float *>(R)[i] = (float)((double)static_cast<const float *>(V)[i] - Y[i]);
    }
}
}  // namespace

// FP64 inverses of the P_mu (one launch) into the layout; Li / ldi receive
// the matrices the chain uses (FP64, or FP32 copies for FP32 plans).
cudaError_t itucker_prepare(const kron_plan_s *plan, const void *const *P, const int64_t *ldP, uint8_t *w,
                            const ItLayout &lay, const void **Li, int64_t *ldi, cudaStream_t cs) {
    const int d = plan->d;
    const bool io64 = plan->dtype == KRON_F64;
    void *iws[KRON_MAX_D] = {};
    for (int k = 0; k < d; ++k) iws[k] = w + lay.inv[k];
    cudaError_t e = inv_gj_batch(d, plan->n, P, ldP, io64, iws, cs);
    for (int k = 0; k < d && e == cudaSuccess; ++k) {
        const double *inv = inv_result(plan->n[k], iws[k]);
        ldi[k] = plan->n[k];
        if (io64) {
            Li[k] = inv;
        } else {
            e = cast2d(inv, true, plan->n[k], w + lay.pin32[k], false, plan->n[k], plan->n[k], plan->n[k], cs);
            Li[k] = w + lay.pin32[k];
        }
    }
    return e;
}

kron_status kron_itucker_workspace_size(kron_plan plan, int refine, size_t *bytes) {
    if (!plan || !bytes || refine < 0 || refine > 8) return KRON_ERR_INVALID_ARG;
    if (!square_plan(plan)) return KRON_ERR_INVALID_ARG;
    for (int k = 0; k < plan->d; ++k)
        if (plan->n[k] > 1024) return KRON_ERR_UNSUPPORTED;
    *bytes = itucker_layout(plan, refine).total;
    return KRON_OK;
}

kron_status kron_itucker(kron_plan plan, const void *V, const void *const *P, const int64_t *ldP, int refine,
                         void *S, void *ws, size_t ws_bytes, kron_stream_t stream) {
    size_t need = 0;
    kron_status st = kron_itucker_workspace_size(plan, refine, &need);
    if (st != KRON_OK) return st;
    if (!V || !S || V == S) return KRON_ERR_INVALID_ARG;
    const bool trans = (plan->flags & KRON_PLAN_TRANS_L) != 0;
    st = check_L(plan, P, ldP, trans);
    if (st != KRON_OK) return st;
    const size_t es = esize(plan->dtype);
    if (!aligned(V, es) || !aligned(S, es)) return KRON_ERR_ALIGNMENT;
    st = check_ws(ws, ws_bytes, need);
    if (st != KRON_OK) return st;
    const ItLayout lay = itucker_layout(plan, refine);
    auto *w = static_cast<uint8_t *>(ws);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const int d = plan->d;
    const bool io64 = plan->dtype == KRON_F64;
    const int64_t N = prod(plan->n, 0, d);
    // FP64 inverses, one launch
    const void *Li[KRON_MAX_D];
    int64_t ldi[KRON_MAX_D];
    cudaError_t e = itucker_prepare(plan, P, ldP, w, lay, Li, ldi, cs);
    if (e != cudaSuccess) return KRON_ERR_CUDA;
    st = run_chain(plan, V, Li, ldi, S, w + lay.chain, cs, trans);
    if (st != KRON_OK) return st;
    // refinement: R = V - S x_mu op(P_mu) in FP64, S += R x_mu op(P_mu)^{-1}
    const void *P64[KRON_MAX_D];
    int64_t ld64[KRON_MAX_D];
    for (int k = 0; k < d; ++k) {
        P64[k] = P[k];
        ld64[k] = ldP[k];
    }
    if (refine > 0 && !io64) {
        for (int k = 0; k < d && e == cudaSuccess; ++k) {
            const int64_t r = trans ? plan->m[k] : plan->n[k];  // rows of the stored P
            e = cast2d(P[k], false, ldP[k], w + lay.p64[k], true, r, r, r, cs);
            P64[k] = w + lay.p64[k];
            ld64[k] = r;
        }
        if (e != cudaSuccess) return KRON_ERR_CUDA;
    }
    for (int it = 0; it < refine; ++it) {
        const void *S64 = S;
        if (!io64) {
            if (cast2d(S, false, N, w + lay.s64, true, N, N, 1, cs) != cudaSuccess) return KRON_ERR_CUDA;
            S64 = w + lay.s64;
        }
        auto *Y = reinterpret_cast<double *>(w + lay.y64);
        st = run_chain(&lay.pl64, S64, P64, ld64, Y, w + lay.chain64, cs, trans);
        if (st != KRON_OK) return st;
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 152 * 8));
        residual_kernel<<<blocks, 256, 0, cs>>>(V, Y, w + lay.r, io64, N);
        if (cudaGetLastError() != cudaSuccess) return KRON_ERR_CUDA;
        st = run_chain(plan, w + lay.r, Li, ldi, S, w + lay.chain, cs, trans, true);
        if (st != KRON_OK) return st;
    }
    return KRON_OK;
}

// --------------------------------------------- PCG for Kronecker-sum systems
//
// Workspace: [r][z][p][q] (N values of the plan dtype), [scalars][dot
// partials], [kron_kronsumv workspace], [kron_itucker workspace].
namespace {
struct PcgLayout {
    size_t r, z, p, q, sc, part, ksv, itk, total;
};

PcgLayout pcg_layout(const kron_plan_s *pl, bool pre) {
    PcgLayout l{};
    const size_t vb = align_up((size_t)prod(pl->n, 0, pl->d) * esize(pl->dtype));
    size_t off = 0;
    l.r = off;
    off += vb;
    l.z = off;
    off += vb;
    l.p = off;
    off += vb;
    l.q = off;
    off += vb;
    l.sc = off;
    off += kAlign;
    l.part = off;
    off += align_up(pcg_partial_doubles() * sizeof(double));
    l.ksv = off;
    off += align_up(kronsumv_layout(pl).total);
    l.itk = off;
    if (pre) off += align_up(itucker_layout(pl, 0).total);
    l.total = off;
    return l;
}
}  // namespace

kron_status kron_kronsum_pcg_workspace_size(kron_plan plan, int precondition, size_t *bytes) {
    if (!plan || !bytes) return KRON_ERR_INVALID_ARG;
    if (!square_plan(plan)) return KRON_ERR_INVALID_ARG;
    if (precondition)
        for (int k = 0; k < plan->d; ++k)
            if (plan->n[k] > 1024) return KRON_ERR_UNSUPPORTED;
    *bytes = pcg_layout(plan, precondition != 0).total;
    return KRON_OK;
}

kron_status kron_kronsum_pcg(kron_plan plan, const void *const *M, const int64_t *ldM, const void *const *P,
                             const int64_t *ldP, const void *B, void *X, double tol, int maxit, int *iters,
                             double *relres, void *ws, size_t ws_bytes, kron_stream_t stream) {
    const bool pre = P != nullptr;
    size_t need = 0;
    kron_status st = kron_kronsum_pcg_workspace_size(plan, pre ? 1 : 0, &need);
    if (st != KRON_OK) return st;
    if (!B || !X || B == X || !(tol >= 0.0) || maxit < 0) return KRON_ERR_INVALID_ARG;
    const bool trans = (plan->flags & KRON_PLAN_TRANS_L) != 0;
    st = check_L(plan, M, ldM, trans);
    if (st == KRON_OK && pre) st = check_L(plan, P, ldP, trans);
    if (st != KRON_OK) return st;
    const size_t es = esize(plan->dtype);
    if (!aligned(B, es) || !aligned(X, es)) return KRON_ERR_ALIGNMENT;
    st = check_ws(ws, ws_bytes, need);
    if (st != KRON_OK) return st;
    const PcgLayout lay = pcg_layout(plan, pre);
    auto *w = static_cast<uint8_t *>(ws);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const bool f64 = plan->dtype == KRON_F64;
    const int64_t N = prod(plan->n, 0, plan->d);
    void *r = w + lay.r, *z = w + lay.z, *p = w + lay.p, *q = w + lay.q;
    double *sc = reinterpret_cast<double *>(w + lay.sc);  // [0] b.b [1] r.z [2] p.q [3] r.r [4] new r.z
    double *part = reinterpret_cast<double *>(w + lay.part);
    const size_t ksv_bytes = kronsumv_layout(plan).total;
    auto matvec = [&](const void *v, void *out) {
        return kron_kronsumv(plan, v, M, ldM, out, w + lay.ksv, ksv_bytes, stream);
    };
    // the preconditioner's inverses once per solve
    const ItLayout itl = itucker_layout(plan, 0);
    const void *Li[KRON_MAX_D];
    int64_t ldi[KRON_MAX_D];
    if (pre && itucker_prepare(plan, P, ldP, w + lay.itk, itl, Li, ldi, cs) != cudaSuccess) return KRON_ERR_CUDA;
    auto precond = [&](const void *v, void *out) -> kron_status {
        if (pre) return run_chain(plan, v, Li, ldi, out, w + lay.itk + itl.chain, cs, trans);
        return cuda_status(cudaMemcpyAsync(out, v, (size_t)N * es, cudaMemcpyDeviceToDevice, cs));
    };
    auto host = [&](const double *dev, double *out) {
        cudaError_t e = cudaMemcpyAsync(out, dev, sizeof(double), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        return e;
    };
    int done = 0;
    double bb = 0.0, rr = 0.0;
    // r = b - M x ; z = P^{-1} r ; p = z
    st = matvec(X, q);
    if (st != KRON_OK) return st;
    cudaError_t e = pcg_axpby(f64, N, 1.0, nullptr, nullptr, B, 0.0, nullptr, nullptr, r, cs);
    if (e == cudaSuccess) e = pcg_axpby(f64, N, -1.0, nullptr, nullptr, q, 1.0, nullptr, nullptr, r, cs);
    if (e == cudaSuccess) e = pcg_dot(B, B, f64, N, part, &sc[0], cs);
    if (e == cudaSuccess) e = pcg_dot(r, r, f64, N, part, &sc[3], cs);
    if (e == cudaSuccess) e = host(&sc[0], &bb);
    if (e == cudaSuccess) e = host(&sc[3], &rr);
    if (e != cudaSuccess) return KRON_ERR_CUDA;
    if (bb == 0.0) {  // b = 0: x = 0
        e = cudaMemsetAsync(X, 0, (size_t)N * es, cs);
        if (iters) *iters = 0;
        if (relres) *relres = 0.0;
        return cuda_status(e);
    }
    const double bn = std::sqrt(bb);
    if (std::sqrt(rr) > tol * bn && maxit > 0) {
        st = precond(r, z);
        if (st != KRON_OK) return st;
        e = pcg_axpby(f64, N, 1.0, nullptr, nullptr, z, 0.0, nullptr, nullptr, p, cs);
        if (e == cudaSuccess) e = pcg_dot(r, z, f64, N, part, &sc[1], cs);
        if (e != cudaSuccess) return KRON_ERR_CUDA;
        while (done < maxit) {
            st = matvec(p, q);
            if (st != KRON_OK) return st;
            e = pcg_dot(p, q, f64, N, part, &sc[2], cs);
            // x += (rz / pq) p ; r -= (rz / pq) q
            if (e == cudaSuccess) e = pcg_axpby(f64, N, 1.0, &sc[1], &sc[2], p, 1.0, nullptr, nullptr, X, cs);
            if (e == cudaSuccess) e = pcg_axpby(f64, N, -1.0, &sc[1], &sc[2], q, 1.0, nullptr, nullptr, r, cs);
            if (e == cudaSuccess) e = pcg_dot(r, r, f64, N, part, &sc[3], cs);
            if (e == cudaSuccess) e = host(&sc[3], &rr);
            if (e != cudaSuccess) return KRON_ERR_CUDA;
            ++done;
            if (std::sqrt(rr) <= tol * bn || !std::isfinite(rr)) break;
            st = precond(r, z);
            if (st != KRON_OK) return st;
            // p = z + (rz_new / rz) p
            e = pcg_dot(r, z, f64, N, part, &sc[4], cs);
            if (e == cudaSuccess) e = pcg_axpby(f64, N, 1.0, nullptr, nullptr, z, 1.0, &sc[4], &sc[1], p, cs);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&sc[1], &sc[4], sizeof(double), cudaMemcpyDeviceToDevice, cs);
            if (e != cudaSuccess) return KRON_ERR_CUDA;
        }
    }
    if (iters) *iters = done;
    if (relres) *relres = std::sqrt(rr) / bn;
    return KRON_OK;
}

// ------------------------------------------------ exponential-of-Kronecker-sum stepper
//
// Workspace: [expm ws][E_0..E_{d-1} (FP64)][images x d][state0][state1]
namespace {
struct StepLayout {
    size_t expm, expm_each, E[KRON_MAX_D], img[KRON_MAX_D], st[2], stbytes, total;
    size_t fxf[KRON_MAX_D], fxg[KRON_MAX_D], fxsc;  // fixed-point form
    size_t imgh[KRON_MAX_D];                        // fixed point: half-width images (tail tiles)
};

StepLayout step_layout(const kron_plan_s *pl) {
    StepLayout s{};
    size_t off = 0;
    int64_t nmax = 1;
    for (int k = 0; k < pl->d; ++k) nmax = std::max(nmax, pl->n[k]);
    s.expm = off;  // one expm workspace per mode: the exponentials run in one launch
    s.expm_each = align_up(expm_workspace_bytes(nmax));
    off += (size_t)pl->d * s.expm_each;
    for (int k = 0; k < pl->d; ++k) {
        s.E[k] = off;
        off += align_up((size_t)pl->n[k] * pl->n[k] * 8);
    }
    const int form = form_of(pl->prec);
    for (int k = 0; k < pl->d; ++k) {
        s.img[k] = off;
        off += align_up(form >= 0 ? tc_bimage_bytes(form, pl->n[k], pl->n[k]) : 0);
    }
    s.stbytes = align_up((size_t)prod(pl->n, 0, pl->d) * std::max(inter_size(pl->prec), esize(pl->dtype)));
    s.st[0] = off;
    off += s.stbytes;
    s.st[1] = off;
    off += s.stbytes;
    if (is_fx(pl->prec)) {
        for (int k = 0; k < pl->d; ++k) {
            s.fxf[k] = off;
            off += align_up((size_t)pl->n[k] * sizeof(int));
            s.fxg[k] = off;
            off += kAlign;
            s.imgh[k] = off;
            const int bn = tc_tile_n(form, pl->n[k]);
            if (bn % 32 == 0) off += align_up(tc_bimage_bytes_bn(form, pl->n[k], pl->n[k], bn / 2));
        }
        s.fxsc = off;
        off += kAlign;
    }
    s.total = off;
    return s;
}

// Fixed-point stepper: U (float) -> fixed point once, then every mode
// product fixed point -> fixed point (state ping-pong), the last one back to
// the storage type.
// state_ready: when not null, an event the stream waits for before U is first
// read (the exponentials' images do not need U and go ahead of it).
kron_status run_steps_fx(const kron_plan_s *pl, const double *const *E, const int64_t *ldE, int nsteps, void *U,
                         uint8_t *w, const StepLayout &lay, cudaStream_t cs, cudaEvent_t state_ready) {
    const int d = pl->d;
    const bool io64 = pl->dtype == KRON_F64;
    const int total = nsteps * d;
    if (total == 0) return KRON_OK;
    // three rotating scale words: product k reads sc[k % 3] and writes
    // sc[(k + 1) % 3], and clears sc[(k + 2) % 3] for product k + 1 once the
    // launches before it are complete (no memset between the launches)
    FxScale *sc = reinterpret_cast<FxScale *>(w + lay.fxsc);
    auto *scratch = reinterpret_cast<unsigned long long *>(sc + 3);
    const int form = form_of(pl->prec);
    for (int k = 0; k < d; ++k) {
        const ModeGeom g{1, 1, pl->n[k], pl->n[k]};
        Contraction c = tc_mode_contraction(g, nullptr, false, E[k], true, ldE[k], false, nullptr, false);
        if (fx_build_bimage(form, c, w + lay.img[k], reinterpret_cast<int *>(w + lay.fxf[k]),
                            reinterpret_cast<unsigned long long *>(w + lay.fxg[k]), cs) != cudaSuccess)
            return KRON_ERR_CUDA;
        // half-width image for the tail tiles (same row exponents and bound)
        const int bn = tc_tile_n(form, pl->n[k]);
        if (bn % 32 == 0 &&
            fx_build_bimage_bn(form, c, w + lay.imgh[k], reinterpret_cast<int *>(w + lay.fxf[k]),
                               reinterpret_cast<unsigned long long *>(w + lay.fxg[k]), bn / 2, cs) != cudaSuccess)
            return KRON_ERR_CUDA;
    }
    const int64_t N = prod(pl->n, 0, d);
    if (state_ready && cudaStreamWaitEvent(cs, state_ready, 0) != cudaSuccess) return KRON_ERR_CUDA;
    if (fx_from_float(form, U, io64, N, reinterpret_cast<int32_t *>(w + lay.st[0]), &sc[0], scratch, cs) !=
        cudaSuccess)
        return KRON_ERR_CUDA;
    if (fx_reset(&sc[1], cs) != cudaSuccess) return KRON_ERR_CUDA;
    int cur = 0, idx = 0;
    for (int s = 0; s < nsteps; ++s) {
        for (int j = 0; j < d; ++j, ++idx) {
            const int mu = pl->order[j];
            const ModeGeom g = mode_geom(d, pl->n, mu, pl->n[mu]);
            const bool last = (idx == total - 1);
            void *dst = last ? U : (void *)(w + lay.st[cur ^ 1]);
            FxScale *sdst = last ? nullptr : &sc[(idx + 1) % 3];
            FxScale *snext = (idx + 2 < total) ? &sc[(idx + 2) % 3] : nullptr;
            Contraction c = tc_mode_contraction(g, w + lay.st[cur], false, E[mu], true, ldE[mu], false, dst,
                                                last ? io64 : false);
            const bool half = tc_tile_n(form, pl->n[mu]) % 32 == 0;
            const cudaError_t e =
                tcp_contract_fx_tail(form, c, w + lay.img[mu], half ? w + lay.imgh[mu] : nullptr, &sc[idx % 3],
                                     reinterpret_cast<const int *>(w + lay.fxf[mu]),
                                     reinterpret_cast<const unsigned long long *>(w + lay.fxg[mu]), sdst, snext, cs);
            if (e != cudaSuccess) return KRON_ERR_CUDA;
            cur ^= 1;
        }
    }
    return KRON_OK;
}

kron_status check_step_plan(const kron_plan_s *pl) {
    if (pl->flags & KRON_PLAN_TRANS_L) return KRON_ERR_UNSUPPORTED;
    for (int k = 0; k < pl->d; ++k)
        if (pl->m[k] != pl->n[k]) return KRON_ERR_INVALID_ARG;
    return KRON_OK;
}

kron_status run_steps(const kron_plan_s *pl, const double *const *E, const int64_t *ldE, int nsteps, void *U,
                      uint8_t *w, const StepLayout &lay, cudaStream_t cs, cudaEvent_t state_ready = nullptr) {
    if (is_fx(pl->prec)) return run_steps_fx(pl, E, ldE, nsteps, U, w, lay, cs, state_ready);
    const int d = pl->d;
    const bool io64 = pl->dtype == KRON_F64;
    const bool split = is_split(pl->prec);
    const int form = form_of(pl->prec);
    const bool i64 = pl->prec == KRON_PREC_FP64;
    const int total = nsteps * d;
    if (total == 0) return KRON_OK;
    // Images of the split E_mu, built once for all steps.
    if (split) {
        for (int k = 0; k < d; ++k) {
            const ModeGeom g{1, 1, pl->n[k], pl->n[k]};
            Contraction c = tc_mode_contraction(g, nullptr, false, E[k], true, ldE[k], false, nullptr, false);
            if (tc_build_bimage(form, c, w + lay.img[k], cs) != cudaSuccess) return KRON_ERR_CUDA;
        }
    }
    if (state_ready && cudaStreamWaitEvent(cs, state_ready, 0) != cudaSuccess) return KRON_ERR_CUDA;
    const void *src = U;
    bool src64 = io64;
    int sel = 0;
    int idx = 0;
    for (int s = 0; s < nsteps; ++s) {
        for (int j = 0; j < d; ++j, ++idx) {
            const int mu = pl->order[j];
            const ModeGeom g = mode_geom(d, pl->n, mu, pl->n[mu]);
            const bool last = (idx == total - 1);
            // a single contraction would read and write U: go through a buffer
            const bool via_buf = last && total == 1;
            void *dst = (last && !via_buf) ? U : (void *)(w + lay.st[sel]);
            const bool dst64 = last ? io64 : i64;
            cudaError_t e;
            if (split) {
                Contraction c = tc_mode_contraction(g, src, src64, E[mu], true, ldE[mu], false, dst, dst64);
                e = tcp_contract(form, c, w + lay.img[mu], cs);
            } else {
                Contraction c = simt_mode_contraction(g, src, src64, E[mu], true, ldE[mu], false, dst, dst64);
                e = simt_contract(i64, c, cs);
            }
            if (e != cudaSuccess) return KRON_ERR_CUDA;
            if (via_buf) {
                const size_t bytes = (size_t)prod(pl->n, 0, d) * esize(pl->dtype);
                if (cudaMemcpyAsync(U, dst, bytes, cudaMemcpyDeviceToDevice, cs) != cudaSuccess)
                    return KRON_ERR_CUDA;
            }
            src = dst;
            src64 = dst64;
            sel ^= 1;
        }
    }
    return KRON_OK;
}
}  // namespace

kron_status kron_expkronsum_workspace_size(kron_plan plan, size_t *bytes) {
    if (!plan || !bytes) return KRON_ERR_INVALID_ARG;
    kron_status st = check_step_plan(plan);
    if (st != KRON_OK) return st;
    *bytes = step_layout(plan).total;
    return KRON_OK;
}

kron_status kron_expkronsum_apply(kron_plan plan, const double *const *E, const int64_t *ldE, int nsteps,
                                  void *U, void *ws, size_t ws_bytes, kron_stream_t stream) {
    if (!plan || !E || !ldE || !U || nsteps < 0) return KRON_ERR_INVALID_ARG;
    kron_status st = check_step_plan(plan);
    if (st != KRON_OK) return st;
    for (int k = 0; k < plan->d; ++k) {
        if (!E[k] || ldE[k] < plan->n[k]) return KRON_ERR_INVALID_ARG;
        if (!aligned(E[k], 8)) return KRON_ERR_ALIGNMENT;
    }
    if (!aligned(U, esize(plan->dtype))) return KRON_ERR_ALIGNMENT;
    const StepLayout lay = step_layout(plan);
    st = check_ws(ws, ws_bytes, lay.total);
    if (st != KRON_OK) return st;
    return run_steps(plan, E, ldE, nsteps, U, static_cast<uint8_t *>(ws), lay,
                     reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {

// Copies of the host-state stepper: one stream per device, created on first
// use, on which the state's host-to-device copy runs beside the exponentials.
cudaStream_t copy_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
        streams[dev] = nullptr;
    return streams[dev];
}

// kron_expkronsum_step with an optional event waited for before the state
// is first read.
kron_status expkronsum_step(kron_plan plan, const double *const *A, const int64_t *ldA, double tau, int nsteps,
                            void *U, void *ws, size_t ws_bytes, cudaStream_t cs, cudaEvent_t state_ready) {
    if (!plan || !A || !ldA || !U || nsteps < 0) return KRON_ERR_INVALID_ARG;
    kron_status st = check_step_plan(plan);
    if (st != KRON_OK) return st;
    for (int k = 0; k < plan->d; ++k) {
        if (!A[k] || ldA[k] < plan->n[k]) return KRON_ERR_INVALID_ARG;
        if (!aligned(A[k], 8)) return KRON_ERR_ALIGNMENT;
        if (plan->n[k] > 1024) return KRON_ERR_UNSUPPORTED;
    }
    if (!aligned(U, esize(plan->dtype))) return KRON_ERR_ALIGNMENT;
    const StepLayout lay = step_layout(plan);
    st = check_ws(ws, ws_bytes, lay.total);
    if (st != KRON_OK) return st;
    auto *w = static_cast<uint8_t *>(ws);
    const double *Ep[KRON_MAX_D];
    int64_t ldE[KRON_MAX_D];
    // the distinct A_mu, all exponentials in one launch
    int cnt = 0;
    int64_t bn[KRON_MAX_D], bld[KRON_MAX_D];
    const double *bA[KRON_MAX_D];
    double *bE[KRON_MAX_D];
    void *bws[KRON_MAX_D];
    for (int k = 0; k < plan->d; ++k) {
        int same = -1;
        for (int j = 0; j < k; ++j)
            if (A[j] == A[k] && ldA[j] == ldA[k] && plan->n[j] == plan->n[k]) same = j;
        ldE[k] = plan->n[k];
        if (same >= 0) {
            Ep[k] = Ep[same];
            continue;
        }
        double *Ek = reinterpret_cast<double *>(w + lay.E[k]);
        bn[cnt] = plan->n[k];
        bA[cnt] = A[k];
        bld[cnt] = ldA[k];
        bE[cnt] = Ek;
        bws[cnt] = w + lay.expm + (size_t)cnt * lay.expm_each;
        ++cnt;
        Ep[k] = Ek;
    }
    if (expm_pade13_batch(cnt, bn, bA, bld, tau, bE, bws, cs) != cudaSuccess) return KRON_ERR_CUDA;
    return run_steps(plan, Ep, ldE, nsteps, U, w, lay, cs, state_ready);
}

}  // namespace

extern "C" {

kron_status kron_expkronsum_step(kron_plan plan, const double *const *A, const int64_t *ldA, double tau,
                                 int nsteps, void *U, void *ws, size_t ws_bytes, kron_stream_t stream) {
    return expkronsum_step(plan, A, ldA, tau, nsteps, U, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream),
                           nullptr);
}

kron_status kron_expkronsum_step_host(kron_plan plan, const double *const *A, const int64_t *ldA, double tau,
                                      int nsteps, const void *U_in, void *U_out, void *U_dev, void *ws,
                                      size_t ws_bytes, kron_stream_t stream) {
    if (!plan || !A || !ldA || !U_in || !U_out || !U_dev || nsteps < 0) return KRON_ERR_INVALID_ARG;
    kron_status st = check_step_plan(plan);
    if (st != KRON_OK) return st;
    if (!aligned(U_dev, esize(plan->dtype))) return KRON_ERR_ALIGNMENT;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t cp = copy_stream();
    if (!cp) return KRON_ERR_CUDA;
    const size_t bytes = (size_t)prod(plan->n, 0, plan->d) * esize(plan->dtype);
    // fork: the copy into U_dev waits for the stream's earlier work (which
    // may still use U_dev); join: the steps wait for the copy
    cudaEvent_t fork = nullptr, join = nullptr;
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return KRON_ERR_CUDA;
    if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
        cudaEventDestroy(fork);
        return KRON_ERR_CUDA;
    }
    st = KRON_OK;
    if (cudaEventRecord(fork, cs) != cudaSuccess || cudaStreamWaitEvent(cp, fork, 0) != cudaSuccess ||
        cudaMemcpyAsync(U_dev, U_in, bytes, cudaMemcpyHostToDevice, cp) != cudaSuccess ||
        cudaEventRecord(join, cp) != cudaSuccess)
        st = KRON_ERR_CUDA;
    if (st == KRON_OK) st = expkronsum_step(plan, A, ldA, tau, nsteps, U_dev, ws, ws_bytes, cs, join);
    // a step that failed before waiting for the copy must still join it
    if (st != KRON_OK) cudaStreamWaitEvent(cs, join, 0);
    if (st == KRON_OK && cudaMemcpyAsync(U_out, U_dev, bytes, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
        st = KRON_ERR_CUDA;
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
    return st;
}

}  // extern "C"
