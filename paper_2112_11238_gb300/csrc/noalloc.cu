// noalloc.cu -- a mu-mode product that needs no workspace from the caller.
//
// kron_mump needs device scratch for the split, swizzled image of op(L), and
// takes it from the caller's workspace.  Some callers cannot hand out device
// memory: a host application whose memory pool owns all of the device memory
// and gives none to libraries, or a latency-critical loop that must not call
// cudaMalloc because an allocation can synchronise the device.  For them
// kron_mump_noalloc keeps that scratch in a fixed array compiled into this
// library (every GPU that loads the library holds it until the process exits)
// and allocates nothing.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;  // 1 MiB

// The scratch shared by every call on a device (file scope, device memory).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// per device: the context the address was looked up in, and the address
void *g_scratch_ctx[kMaxDevices] = {};
void *g_scratch_ptr[kMaxDevices] = {};

// cuCtxGetCurrent from the driver (no link-time dependency on it).
using CtxGetCurrentFn = int (*)(void **);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    });
    return fn;
}

// Device address of the scratch array on the current device.  Host code
// cannot use the array's name as a device address (it names a host-side
// stand-in), so the address is looked up with cudaGetSymbolAddress, with the
// device current, once per device and context: a device reset destroys the
// primary context and, with it, the module holding the array, and the next
// context may place it elsewhere, so a changed context means a new lookup.
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    // (before the first runtime call that needs it, no context is current:
    // then the address is looked up afresh, which also creates the context)
    void *ctx = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    const bool have_ctx = get != nullptr && get(&ctx) == 0 && ctx != nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!have_ctx || !g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = have_ctx ? ctx : nullptr;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

using namespace kron;

extern "C" {

kron_status kron_mump_noalloc(int d, const int64_t *m, int mu, int64_t n, const void *T, const void *L,
                              int64_t ldL, int transL, void *S, kron_dtype dtype, kron_prec prec,
                              kron_stream_t stream) {
    if (d < 1 || d > KRON_MAX_D || !m || mu < 0 || mu >= d || n < 1 || !T || !L || !S) return KRON_ERR_INVALID_ARG;
    if (dtype != KRON_F64 && dtype != KRON_F32) return KRON_ERR_INVALID_ARG;
    for (int k = 0; k < d; ++k)
        if (m[k] < 1) return KRON_ERR_INVALID_ARG;
    if (!is_split(prec)) return KRON_ERR_UNSUPPORTED;  // only the split forms keep their scratch this small
    if (transL ? ldL < m[mu] : ldL < n) return KRON_ERR_INVALID_ARG;
    const size_t es = dtype == KRON_F64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(T) % es || reinterpret_cast<uintptr_t>(L) % es ||
        reinterpret_cast<uintptr_t>(S) % es)
        return KRON_ERR_ALIGNMENT;
    const int form = form_of(prec);
    if (tc_bimage_bytes(form, n, m[mu]) > kNoAllocScratchBytes) return KRON_ERR_WORKSPACE;
    void *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return KRON_ERR_CUDA;
    // T viewed as (P, m_mu, Q): rows are the fibres, columns the n outputs
    int64_t P = 1, Q = 1;
    for (int k = 0; k < mu; ++k) P *= m[k];
    for (int k = mu + 1; k < d; ++k) Q *= m[k];
    const int64_t mm = m[mu];
    const bool io64 = dtype == KRON_F64;
    Contraction c;
    c.M = P * Q;
    c.N = n;
    c.K = mm;
    c.A = T;
    c.A_f64 = io64;
    c.rowA = (P == 1) ? IdxMap{0, mm, 0} : IdxMap{P, 1, P * mm};
    c.rowC = (P == 1) ? IdxMap{0, n, 0} : IdxMap{P, 1, P * n};
    c.kA = IdxMap{0, P, 0};
    c.B = L;
    c.B_f64 = io64;
    c.colB = transL ? IdxMap{0, ldL, 0} : IdxMap{0, 1, 0};
    c.kB = transL ? IdxMap{0, 1, 0} : IdxMap{0, ldL, 0};
    c.C = S;
    c.C_f64 = io64;
    c.colC = IdxMap{0, P, 0};
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    // the whole image is rewritten by every call, so nothing needs clearing
    cudaError_t e = tc_build_bimage(form, c, scratch, cs);
    if (e == cudaSuccess) e = tcp_contract(form, c, scratch, cs);
    return e == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

}  // extern "C"
