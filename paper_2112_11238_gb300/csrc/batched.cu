// batched.cu -- many independent Tucker operators of uneven sizes in one
// persistent launch (Section 3.2, Eq. (tensinterp); the batched evaluation
// of tensor-product interpolants, cf. Section 4.3).
//
// A plan fixes the shapes.  Every problem b becomes d jobs of the persistent
// tensor-core kernel (tcp.cu), one per mode in the problem's cost-minimising
// order; the job of mode step s waits for step s-1 of the same problem.  Jobs
// are ordered in waves (step s of problem group g runs in wave g + s) so that
// the intermediates of a group are consumed while they are still in L2.
//
// bind() writes the device job table (pointers of that binding) into the
// workspace; run() is two launches -- one that splits and swizzles every L_mu
// into its image, and the persistent kernel -- plus a memset of the job
// counters, so a bound run can be captured in a CUDA graph.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "tc_common.cuh"

namespace kron {

namespace {

constexpr size_t kAl = 256;
inline size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }

// One L_mu to split into an image.
struct ImgJob {
    const void *L;
    int64_t ld, N, K;
    uint8_t *img;
    int32_t BN;
    int32_t l64;
    int64_t items;   // (nt, kb, row, chunk) items of this image
    int64_t begin;   // prefix sum of items
};

template <int F>
__global__ void batched_bimage_kernel(const ImgJob *__restrict__ jobs, int njobs, int64_t total) {
    using T = FT<F>;
    constexpr int BK = kRowBytes / T::ELEM;
    constexpr int CH = 16 / T::ELEM;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].begin <= idx) lo = mid;
            else hi = mid - 1;
        }
        const ImgJob &J = jobs[lo];
        int64_t r = idx - J.begin;
        const int ch = (int)(r % kChunks);
        r /= kChunks;
        const int row = (int)(r % J.BN);
        r /= J.BN;
        const int64_t KB = (J.K + BK - 1) / BK;
        const int64_t kb = r % KB;
        const int64_t nt = r / KB;
        const int64_t c = nt * J.BN + row;
        const int64_t ro = c < J.N ? c : -1;  // L is n x m with ld: element (c, k) at c + ld * k
        const IdxMap km{0, J.ld, 0};
        uint4 out[T::PIECES];
        if (J.l64) load_split<F, double>(static_cast<const double *>(J.L), ro, km, kb * BK + ch * CH, J.K, out);
        else load_split<F, float>(static_cast<const float *>(J.L), ro, km, kb * BK + ch * CH, J.K, out);
        uint8_t *base = J.img + (size_t)((nt * KB + kb) * T::PIECES) * J.BN * kRowBytes;
        const uint32_t off = swz(row, ch);
#pragma unroll
        for (int q = 0; q < T::PIECES; ++q) *reinterpret_cast<uint4 *>(base + (size_t)q * J.BN * kRowBytes + off) = out[q];
    }
}

}  // namespace
}  // namespace kron

using namespace kron;

struct kron_batched_plan_s {
    int batch = 0, d = 0;
    kron_dtype dtype = KRON_F32;
    kron_prec prec = KRON_PREC_3XTF32;
    int form = 0;
    std::vector<int64_t> m, n;          // batch * d
    std::vector<int> order;             // batch * d
    // job sequence: (problem, step) in launch order
    std::vector<std::pair<int, int>> seq;
    // workspace layout
    std::vector<size_t> img_off;        // batch * d (per mode)
    std::vector<size_t> buf_off;        // batch * (d - 1) intermediates
    size_t imgjob_off = 0, imgjob_bytes = 0;
    size_t table_off = 0, table_bytes = 0;
    size_t tilejob_off = 0, tilejob_bytes = 0;
    int64_t tiles_max = 0;
    size_t done_off = 0, done_bytes = 0;
    size_t ws_bytes = 0;
    double flops = 0;
    int64_t img_items = 0;
    // bound state
    TcpJobs jobs;
    std::vector<ImgJob> imgjobs;
    uint8_t *pinned = nullptr;          // staging for the uploads
    size_t pinned_bytes = 0;
    bool bound = false;
    void *bound_ws = nullptr;
    // the bound operands (kept for re-binding under another configuration)
    std::vector<const void *> bT, bL;
    std::vector<void *> bS;
    // launch configuration (0: the built-in rule): N-tile width cap,
    // pipeline stages, accumulator sets per tile
    int tune_bn = 0, tune_stages = 0, tune_nacc = 0;
};

namespace {

int64_t prodv(const int64_t *v, int d) {
    int64_t p = 1;
    for (int k = 0; k < d; ++k) p *= v[k];
    return p;
}

void problem_order(int d, const int64_t *m, const int64_t *n, int *order) {
    int perm[KRON_MAX_D];
    for (int k = 0; k < d; ++k) perm[k] = order[k] = k;
    long double best = -1;
    do {
        int64_t cur[KRON_MAX_D];
        for (int k = 0; k < d; ++k) cur[k] = m[k];
        long double fl = 0;
        for (int s = 0; s < d; ++s) {
            fl += 2.0L * n[perm[s]] * (long double)prodv(cur, d);
            cur[perm[s]] = n[perm[s]];
        }
        if (best < 0 || fl < best * (1 - 1e-12L)) {
            best = fl;
            for (int k = 0; k < d; ++k) order[k] = perm[k];
        }
    } while (std::next_permutation(perm, perm + d));
}

int kb_of(int form) { return form == kTF32x3 ? kRowBytes / 4 : kRowBytes / 2; }

// N-tile width caps the tuner tries (the built-in rule is the largest).
constexpr int kTileCaps[] = {32, 64, 128};

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// Builds the plan; with_pinned: also the pinned staging buffer of bind (the
// one-shot call uploads from pageable host memory instead).
kron_status batched_plan_init(kron_batched_plan *plan, int batch, int d, const int64_t *m, const int64_t *n,
                              kron_dtype dtype, kron_prec prec, unsigned flags, bool with_pinned) {
    if (!plan) return KRON_ERR_INVALID_ARG;
    *plan = nullptr;
    if (batch < 1 || batch > 65536 || d < 1 || d > KRON_MAX_D || !m || !n || flags != 0) return KRON_ERR_INVALID_ARG;
    if (dtype != KRON_F64 && dtype != KRON_F32) return KRON_ERR_INVALID_ARG;
    if (prec < KRON_PREC_FP64 || prec > KRON_PREC_BF16X6) return KRON_ERR_INVALID_ARG;
    if (!is_split(prec)) return KRON_ERR_UNSUPPORTED;
    for (int64_t i = 0; i < (int64_t)batch * d; ++i)
        if (m[i] < 1 || n[i] < 1 || m[i] > (1 << 20) || n[i] > (1 << 20)) return KRON_ERR_INVALID_ARG;
    auto *pl = new (std::nothrow) kron_batched_plan_s();
    if (!pl) return KRON_ERR_INVALID_ARG;
    pl->batch = batch;
    pl->d = d;
    pl->dtype = dtype;
    pl->prec = prec;
    pl->form = form_of(prec);
    pl->m.assign(m, m + (size_t)batch * d);
    pl->n.assign(n, n + (size_t)batch * d);
    pl->order.resize((size_t)batch * d);
    const size_t isz = 4;  // FP32 intermediates
    size_t off = 0;
    pl->img_off.resize((size_t)batch * d);
    pl->buf_off.assign((size_t)batch * std::max(d - 1, 1), 0);
    std::vector<size_t> inter_bytes(batch, 0);
    for (int b = 0; b < batch; ++b) {
        const int64_t *mb = &pl->m[(size_t)b * d];
        const int64_t *nb = &pl->n[(size_t)b * d];
        problem_order(d, mb, nb, &pl->order[(size_t)b * d]);
        int64_t cur[KRON_MAX_D];
        for (int k = 0; k < d; ++k) cur[k] = mb[k];
        for (int s = 0; s < d; ++s) {
            const int mu = pl->order[(size_t)b * d + s];
            // tiles of this mode at the narrowest tile width (16)
            pl->tiles_max += ((prodv(cur, d) / cur[mu] + 127) / 128) * ((nb[mu] + 15) / 16);
            pl->flops += 2.0 * (double)nb[mu] * (double)prodv(cur, d);
            cur[mu] = nb[mu];
            if (s < d - 1) {
                pl->buf_off[(size_t)b * (d - 1) + s] = off;
                const size_t by = al((size_t)prodv(cur, d) * isz);
                off += by;
                inter_bytes[b] += by;
            }
        }
        for (int k = 0; k < d; ++k) {
            // room for the image at every N-tile width the tuner may pick
            pl->img_off[(size_t)b * d + k] = off;
            size_t ib = 0;
            for (int cap : kTileCaps)
                ib = std::max(ib, tc_bimage_bytes_bn(pl->form, nb[k], mb[k], tc_tile_n_cap(pl->form, nb[k], cap)));
            off += al(ib);
        }
    }
    // waves: groups of problems whose intermediates take about 32 MB
    std::vector<int> group(batch, 0);
    int ng = 0;
    size_t acc = 0;
    for (int b = 0; b < batch; ++b) {
        if (acc > 0 && acc + inter_bytes[b] > (32u << 20)) {
            ++ng;
            acc = 0;
        }
        group[b] = ng;
        acc += inter_bytes[b];
    }
    ++ng;
    for (int w = 0; w < ng + d - 1; ++w)
        for (int s = 0; s < d; ++s) {
            const int g = w - s;
            if (g < 0 || g >= ng) continue;
            for (int b = 0; b < batch; ++b)
                if (group[b] == g) pl->seq.emplace_back(b, s);
        }
    const size_t njobs = pl->seq.size();
    pl->imgjob_off = off;
    pl->imgjob_bytes = al(sizeof(ImgJob) * (size_t)batch * d);
    off += pl->imgjob_bytes;
    pl->table_off = off;
    pl->table_bytes = al(tcp_job_bytes() * njobs);
    off += pl->table_bytes;
    // the job of every tile, right after the job table (one upload for both)
    pl->tilejob_off = off;
    pl->tilejob_bytes = al(sizeof(int) * (size_t)pl->tiles_max);
    off += pl->tilejob_bytes;
    pl->done_off = off;
    pl->done_bytes = al(sizeof(int) * (njobs + 1));  // + the launch's "a wait gave up" flag
    off += pl->done_bytes;
    pl->ws_bytes = off;
    pl->pinned_bytes = pl->imgjob_bytes + pl->table_bytes + pl->tilejob_bytes;
    if (with_pinned && cudaMallocHost(reinterpret_cast<void **>(&pl->pinned), pl->pinned_bytes) != cudaSuccess) {
        delete pl;
        return KRON_ERR_CUDA;
    }
    *plan = pl;
    return KRON_OK;
}

kron_status batched_build(kron_batched_plan plan, void *ws, kron_stream_t stream);

}  // namespace

extern "C" {

kron_status kron_batched_plan_create(kron_batched_plan *plan, int batch, int d, const int64_t *m, const int64_t *n,
                                     kron_dtype dtype, kron_prec prec, unsigned flags) {
    return batched_plan_init(plan, batch, d, m, n, dtype, prec, flags, true);
}

kron_status kron_batched_plan_destroy(kron_batched_plan plan) {
    if (!plan) return KRON_OK;
    if (plan->pinned) {
        // the staging buffer may still feed an upload in flight
        cudaDeviceSynchronize();
        cudaFreeHost(plan->pinned);
    }
    delete plan;
    return KRON_OK;
}

kron_status kron_batched_workspace_size(kron_batched_plan plan, size_t *bytes) {
    if (!plan || !bytes) return KRON_ERR_INVALID_ARG;
    *bytes = plan->ws_bytes;
    return KRON_OK;
}

double kron_batched_flops(kron_batched_plan plan) { return plan ? plan->flops : 0.0; }

kron_status kron_batched_bind(kron_batched_plan plan, const void *const *T, const void *const *L, void *const *S,
                              void *ws, size_t ws_bytes, kron_stream_t stream) {
    if (!plan || !T || !L || !S || !ws) return KRON_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % kAl) return KRON_ERR_ALIGNMENT;
    if (ws_bytes < plan->ws_bytes) return KRON_ERR_WORKSPACE;
    const int d = plan->d, batch = plan->batch;
    const size_t es = plan->dtype == KRON_F64 ? 8 : 4;
    for (int b = 0; b < batch; ++b) {
        if (!T[b] || !S[b]) return KRON_ERR_INVALID_ARG;
        if (reinterpret_cast<uintptr_t>(T[b]) % es || reinterpret_cast<uintptr_t>(S[b]) % es) return KRON_ERR_ALIGNMENT;
        for (int k = 0; k < d; ++k) {
            const void *l = L[(size_t)b * d + k];
            if (!l) return KRON_ERR_INVALID_ARG;
            if (reinterpret_cast<uintptr_t>(l) % es) return KRON_ERR_ALIGNMENT;
        }
    }
    plan->bT.assign(T, T + batch);
    plan->bL.assign(L, L + (size_t)batch * d);
    plan->bS.assign(S, S + batch);
    return batched_build(plan, ws, stream);
}

}  // extern "C"

namespace {

// Job tables of the bound operands under the plan's launch configuration,
// uploaded into the workspace on `stream`.
kron_status batched_build(kron_batched_plan plan, void *ws, kron_stream_t stream) {
    const int d = plan->d, batch = plan->batch;
    const void *const *L = plan->bL.data();
    const void *const *T = plan->bT.data();
    void *const *S = plan->bS.data();
    const int cap = plan->tune_bn > 0 ? plan->tune_bn : (1 << 20);
    auto *w = static_cast<uint8_t *>(ws);
    const bool io64 = plan->dtype == KRON_F64;
    // image jobs
    plan->imgjobs.assign((size_t)batch * d, ImgJob{});
    int64_t begin = 0;
    for (int b = 0; b < batch; ++b)
        for (int k = 0; k < d; ++k) {
            ImgJob &J = plan->imgjobs[(size_t)b * d + k];
            J.L = L[(size_t)b * d + k];
            J.N = plan->n[(size_t)b * d + k];
            J.K = plan->m[(size_t)b * d + k];
            J.ld = J.N;
            J.img = w + plan->img_off[(size_t)b * d + k];
            J.BN = tc_tile_n_cap(plan->form, J.N, cap);
            J.l64 = io64;
            const int64_t nt = (J.N + J.BN - 1) / J.BN;
            const int64_t kb = (J.K + kb_of(plan->form) - 1) / kb_of(plan->form);
            J.items = nt * kb * J.BN * kChunks;
            J.begin = begin;
            begin += J.items;
        }
    plan->img_items = begin;
    // tensor-core jobs in launch order; job index of (b, s) for dependencies
    tcp_jobs_begin(plan->jobs, plan->form);
    plan->jobs.stages = plan->tune_stages;
    plan->jobs.nacc = plan->tune_nacc;
    std::vector<int> jid((size_t)batch * d, -1);
    for (const auto &bs : plan->seq) {
        const int b = bs.first, s = bs.second;
        const int64_t *mb = &plan->m[(size_t)b * d];
        const int64_t *nb = &plan->n[(size_t)b * d];
        const int *ord = &plan->order[(size_t)b * d];
        int64_t cur[KRON_MAX_D];
        for (int k = 0; k < d; ++k) cur[k] = mb[k];
        for (int j = 0; j < s; ++j) cur[ord[j]] = nb[ord[j]];
        const int mu = ord[s];
        int64_t P = 1, Q = 1;
        for (int k = 0; k < mu; ++k) P *= cur[k];
        for (int k = mu + 1; k < d; ++k) Q *= cur[k];
        const int64_t mm = cur[mu], nn = nb[mu];
        const void *src = (s == 0) ? T[b] : (const void *)(w + plan->buf_off[(size_t)b * (d - 1) + s - 1]);
        const bool src64 = (s == 0) ? io64 : false;
        void *dst = (s == d - 1) ? S[b] : (void *)(w + plan->buf_off[(size_t)b * (d - 1) + s]);
        const bool dst64 = (s == d - 1) ? io64 : false;
        Contraction c;
        c.M = P * Q;
        c.N = nn;
        c.K = mm;
        c.A = src;
        c.A_f64 = src64;
        if (P == 1) {
            c.rowA = IdxMap{0, mm, 0};
            c.rowC = IdxMap{0, nn, 0};
        } else {
            c.rowA = IdxMap{P, 1, P * mm};
            c.rowC = IdxMap{P, 1, P * nn};
        }
        c.kA = IdxMap{0, P, 0};
        c.C = dst;
        c.C_f64 = dst64;
        c.colC = IdxMap{0, P, 0};
        const int dep = (s == 0) ? -1 : jid[(size_t)b * d + s - 1];
        jid[(size_t)b * d + s] = tcp_jobs_add(plan->jobs, c, w + plan->img_off[(size_t)b * d + mu], dep,
                                              tc_tile_n_cap(plan->form, nn, cap));
    }
    if ((int64_t)plan->jobs.tile_job.size() > plan->tiles_max) return KRON_ERR_INVALID_ARG;  // not reached
    // upload both tables: one copy from the pinned staging buffer, or (no
    // staging buffer) from pageable memory, which the copy has consumed when
    // cudaMemcpyAsync returns
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (plan->pinned) {
        if (cudaStreamSynchronize(cs) != cudaSuccess) return KRON_ERR_CUDA;  // staging buffer reuse
        std::memcpy(plan->pinned, plan->imgjobs.data(), sizeof(ImgJob) * plan->imgjobs.size());
        std::memcpy(plan->pinned + plan->imgjob_bytes, plan->jobs.host.data(), plan->jobs.host.size());
        std::memcpy(plan->pinned + plan->imgjob_bytes + plan->table_bytes, plan->jobs.tile_job.data(),
                    sizeof(int) * plan->jobs.tile_job.size());
        if (cudaMemcpyAsync(w + plan->imgjob_off, plan->pinned, plan->pinned_bytes, cudaMemcpyHostToDevice, cs) !=
            cudaSuccess)
            return KRON_ERR_CUDA;
    } else {
        std::vector<uint8_t> stage(plan->imgjob_bytes + plan->table_bytes + plan->tilejob_bytes, 0);
        std::memcpy(stage.data(), plan->imgjobs.data(), sizeof(ImgJob) * plan->imgjobs.size());
        std::memcpy(stage.data() + plan->imgjob_bytes, plan->jobs.host.data(), plan->jobs.host.size());
        std::memcpy(stage.data() + plan->imgjob_bytes + plan->table_bytes, plan->jobs.tile_job.data(),
                    sizeof(int) * plan->jobs.tile_job.size());
        if (cudaMemcpyAsync(w + plan->imgjob_off, stage.data(), stage.size(), cudaMemcpyHostToDevice, cs) !=
            cudaSuccess)
            return KRON_ERR_CUDA;
    }
    plan->bound = true;
    plan->bound_ws = ws;
    return KRON_OK;
}

}  // namespace

extern "C" {

kron_status kron_batched_run(kron_batched_plan plan, void *ws, size_t ws_bytes, kron_stream_t stream) {
    if (!plan || !ws) return KRON_ERR_INVALID_ARG;
    if (!plan->bound || ws != plan->bound_ws) return KRON_ERR_INVALID_ARG;
    if (ws_bytes < plan->ws_bytes) return KRON_ERR_WORKSPACE;
    auto *w = static_cast<uint8_t *>(ws);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const int64_t total = plan->img_items;
    const int threads = 256;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + threads - 1) / threads, 152 * 32));
    const auto *ij = reinterpret_cast<const ImgJob *>(w + plan->imgjob_off);
    const int nij = (int)plan->imgjobs.size();
    switch (plan->form) {
        case kTF32x3: batched_bimage_kernel<kTF32x3><<<blocks, threads, 0, cs>>>(ij, nij, total); break;
        case kBF16x3: batched_bimage_kernel<kBF16x3><<<blocks, threads, 0, cs>>>(ij, nij, total); break;
        case kBF16x6: batched_bimage_kernel<kBF16x6><<<blocks, threads, 0, cs>>>(ij, nij, total); break;
        default: return KRON_ERR_UNSUPPORTED;
    }
    if (cudaGetLastError() != cudaSuccess) return KRON_ERR_CUDA;
    if (tcp_jobs_run(plan->jobs, w + plan->table_off, reinterpret_cast<int *>(w + plan->done_off), cs,
                     reinterpret_cast<const int *>(w + plan->tilejob_off)) != cudaSuccess)
        return KRON_ERR_CUDA;
    return KRON_OK;
}

// One-shot form: plan, bind and run in one call (host-side plan only; the
// tables go to the workspace from pageable host memory, so nothing is
// allocated on the device or pinned).
kron_status kron_tucker_batched_workspace_size(int batch, int d, const int64_t *m, const int64_t *n,
                                               kron_dtype dtype, kron_prec prec, size_t *bytes) {
    if (!bytes) return KRON_ERR_INVALID_ARG;
    kron_batched_plan pl = nullptr;
    kron_status st = batched_plan_init(&pl, batch, d, m, n, dtype, prec, 0, false);
    if (st != KRON_OK) return st;
    *bytes = pl->ws_bytes;
    delete pl;
    return KRON_OK;
}

kron_status kron_tucker_batched(int batch, int d, const int64_t *m, const int64_t *n, const void *const *T,
                                const void *const *const *L, void *const *S, kron_dtype dtype, kron_prec prec,
                                void *ws, size_t ws_bytes, kron_stream_t stream) {
    if (!T || !L || !S) return KRON_ERR_INVALID_ARG;
    kron_batched_plan pl = nullptr;
    kron_status st = batched_plan_init(&pl, batch, d, m, n, dtype, prec, 0, false);
    if (st != KRON_OK) return st;
    std::vector<const void *> flat((size_t)batch * d, nullptr);
    for (int b = 0; b < batch && st == KRON_OK; ++b) {
        if (!L[b]) st = KRON_ERR_INVALID_ARG;
        else
            for (int k = 0; k < d; ++k) flat[(size_t)b * d + k] = L[b][k];
    }
    if (st == KRON_OK) st = kron_batched_bind(pl, T, flat.data(), S, ws, ws_bytes, stream);
    if (st == KRON_OK) st = kron_batched_run(pl, ws, ws_bytes, stream);
    delete pl;  // no staging buffer: nothing on the device refers to the plan
    return st;
}

// ------------------------------------------------------------- autotuning
//
// kron_batched_autotune times candidate launch configurations of a bound
// plan -- the N-tile width cap (image layout and MMA width), the pipeline
// stages and the accumulator sets per tile of the persistent kernel -- on
// the bound operands, keeps the fastest, and records it in the file named by
// KRON_AUTOTUNE_CACHE (one JSON object per line), keyed by the GPU's name and
// the plan's shapes, dtype and precision; a later plan with the same key
// takes the recorded choice without timing.

}  // extern "C"

namespace {

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
    const auto *b = static_cast<const uint8_t *>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

std::string tune_key(const kron_batched_plan_s *pl) {
    int dev = 0;
    cudaDeviceProp prop{};
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::string gpu(prop.name);
    for (char &c : gpu)
        if (c == '"' || c == '\\' || c == '|') c = '_';
    uint64_t h = fnv1a(pl->m.data(), pl->m.size() * sizeof(int64_t));
    h = fnv1a(pl->n.data(), pl->n.size() * sizeof(int64_t), h);
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s|d=%d|batch=%d|shapes=%016llx|dtype=%d|prec=%d", gpu.c_str(), pl->d, pl->batch,
                  (unsigned long long)h, (int)pl->dtype, (int)pl->prec);
    return std::string(buf);
}

std::mutex g_cache_mu;

// The last record of `key` in the cache file.
bool cache_lookup(const char *path, const std::string &key, int &bn, int &stages, int &nacc) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    const std::string tag = "\"key\": \"" + key + "\"";
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        if (!std::strstr(line, tag.c_str())) continue;
        int a = 0, b = 0, c = 0;
        const char *p = std::strstr(line, "\"bn\":");
        const char *q = std::strstr(line, "\"stages\":");
        const char *r = std::strstr(line, "\"nacc\":");
        if (p && q && r && std::sscanf(p, "\"bn\": %d", &a) == 1 && std::sscanf(q, "\"stages\": %d", &b) == 1 &&
            std::sscanf(r, "\"nacc\": %d", &c) == 1) {
            bn = a;
            stages = b;
            nacc = c;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, int bn, int stages, int nacc, float ms) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"key\": \"%s\", \"bn\": %d, \"stages\": %d, \"nacc\": %d, \"ms\": %.6f}\n", key.c_str(), bn,
                 stages, nacc, (double)ms);
    std::fclose(f);
}

}  // namespace

extern "C" {

kron_status kron_batched_autotune(kron_batched_plan plan, void *ws, size_t ws_bytes, kron_stream_t stream,
                                  int *from_cache) {
    if (!plan || !ws) return KRON_ERR_INVALID_ARG;
    if (!plan->bound || ws != plan->bound_ws) return KRON_ERR_INVALID_ARG;
    if (ws_bytes < plan->ws_bytes) return KRON_ERR_WORKSPACE;
    if (from_cache) *from_cache = 0;
    const char *path = std::getenv("KRON_AUTOTUNE_CACHE");
    const std::string key = tune_key(plan);
    int bn = 0, stages = 0, nacc = 0;
    if (path && *path && cache_lookup(path, key, bn, stages, nacc)) {
        plan->tune_bn = bn;
        plan->tune_stages = stages;
        plan->tune_nacc = nacc;
        if (from_cache) *from_cache = 1;
        return batched_build(plan, ws, stream);
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return KRON_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return KRON_ERR_CUDA;
    }
    // candidates: every tile-width cap the form allows, stages 2 or as many
    // as fit, one accumulator set, two, or as many as fit
    const int caps_max = plan->form == kBF16x6 ? 64 : 128;
    float best = -1.f;
    int bb = 0, bs = 0, ba = 0;
    kron_status st = KRON_OK;
    for (int cap : kTileCaps) {
        if (cap > caps_max || st != KRON_OK) continue;
        for (int sg : {2, 0})
            for (int na : {1, 2, 0}) {
                if (st != KRON_OK) break;
                plan->tune_bn = cap;
                plan->tune_stages = sg;
                plan->tune_nacc = na;
                st = batched_build(plan, ws, stream);
                if (st == KRON_OK) st = kron_batched_run(plan, ws, ws_bytes, stream);  // warm-up
                if (st == KRON_OK && cudaEventRecord(e0, cs) != cudaSuccess) st = KRON_ERR_CUDA;
                for (int r = 0; r < 3 && st == KRON_OK; ++r) st = kron_batched_run(plan, ws, ws_bytes, stream);
                if (st == KRON_OK && cudaEventRecord(e1, cs) != cudaSuccess) st = KRON_ERR_CUDA;
                float ms = 0.f;
                if (st == KRON_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    st = KRON_ERR_CUDA;
                if (st == KRON_OK && (best < 0.f || ms < best)) {
                    best = ms;
                    bb = cap;
                    bs = sg;
                    ba = na;
                }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != KRON_OK) return st;
    plan->tune_bn = bb;
    plan->tune_stages = bs;
    plan->tune_nacc = ba;
    if (path && *path) cache_store(path, key, bb, bs, ba, best / 3.f);
    return batched_build(plan, ws, stream);
}

kron_status kron_batched_tuning(kron_batched_plan plan, int *bn_cap, int *stages, int *nacc) {
    if (!plan || !bn_cap || !stages || !nacc) return KRON_ERR_INVALID_ARG;
    *bn_cap = plan->tune_bn;
    *stages = plan->tune_stages;
    *nacc = plan->tune_nacc;
    return KRON_OK;
}

}  // extern "C"
