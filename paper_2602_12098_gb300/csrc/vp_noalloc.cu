// vp_precode_noalloc: one slot (factorise + select paths + precode) that
// allocates nothing. It is meant for callers that cannot let a library call
// cudaMalloc: real-time slot loops (cudaMalloc may synchronise the device and
// take unbounded time inside a slot's deadline), processes whose device memory
// is reserved up front by another allocator, and hosts that hand this library
// device buffers only. The per-channel state that a plan would
// keep in cudaMalloc'd memory lives instead in the file-scope array
// g_noalloc_state below, sized for a fixed maximum; the kernels are the
// plan path's own kernels, run on that storage.
#include <mutex>

#include "vp_internal.cuh"

namespace {

// 8 MiB of per-channel state. Every GPU that loads this library holds it
// until the process exits.
constexpr size_t kNoAllocBytes = size_t(8) << 20;
__device__ __align__(256) unsigned char g_noalloc_state[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};   // device address of g_noalloc_state, per device

// The host-side name g_noalloc_state is only a stand-in for the device array:
// the address a kernel may use comes from cudaGetSymbolAddress, once per
// device, with that device current.
vp_status scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_state) != cudaSuccess || !p) {
            cudaGetLastError();
            return VP_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return VP_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

namespace vp {

// Lays the state of C channels out from `base` (256-byte aligned pieces);
// returns the bytes used. base = null only measures.
size_t carve_state(unsigned char* base, int C, int K, int Mp, int n, DeviceState* d)
{
    const size_t nch = (size_t)vp::n_chunks(n);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base ? base + off : nullptr;
        off = align256(off + bytes);
        return p;
    };
    d->utp = reinterpret_cast<float4*>(take(sizeof(float4) * C * K * K));
    d->utc = reinterpret_cast<float2*>(take(sizeof(float2) * C * K * K));
    d->w = reinterpret_cast<float*>(take(sizeof(float) * C * K));
    d->ul = take((size_t)C * K);
    d->pt = reinterpret_cast<float2*>(take(sizeof(float2) * C * K * Mp));
    d->ptlo = reinterpret_cast<float2*>(take(sizeof(float2) * C * K * Mp));
    d->paths = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * C * n));
    d->maxq = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * C * nch));
    d->ecode = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * C * n));
    d->emeta = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * C * n));
    d->pcode = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * C * vp::kMaxPrefix));
    d->phdr = reinterpret_cast<int4*>(take(sizeof(int4) * C));
    d->st = take((size_t)C);
    d->nflag = reinterpret_cast<int*>(take(sizeof(int)));
    d->flags = reinterpret_cast<int*>(take(sizeof(int) * C));
    return off;
}

// One slot on the plan's state: factorise C channels, select paths, copy the
// status bytes, and precode S vectors per channel. Returns the first failing
// launch's error.
cudaError_t enqueue_slot(const vp_plan* p, const float2* H, int C, const uint8_t* sym, int S, float2* x, int8_t* l,
                         float* gamma, uint8_t* status, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->d.nflag, 0, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = launch_factor32(p, H, C, nullptr, nullptr, nullptr, s)) != cudaSuccess) return e;
    if ((e = launch_factor64(p, H, C, nullptr, nullptr, nullptr, s)) != cudaSuccess) return e;
    if ((e = launch_pathsel(p, C, s)) != cudaSuccess) return e;
    if (status && (e = cudaMemcpyAsync(status, p->d.st, (size_t)C, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    if (S > 0 && (e = launch_search(p, sym, S, nullptr, C * S, x, l, gamma, s)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace vp

extern "C" {

size_t vp_noalloc_capacity_bytes(void) { return kNoAllocBytes; }

int vp_noalloc_max_channels(const vp_plan* plan)
{
    if (!plan) return 0;
    const int mp = vp::p_rows(plan);
    vp::DeviceState probe;
    // the state grows with C, so the largest fitting C is found by bisection
    int lo = 0, hi = 1;
    while (vp::carve_state(nullptr, hi, plan->K, mp, plan->n_paths, &probe) <= kNoAllocBytes) {
        lo = hi;
        if (hi > (1 << 28)) return lo;
        hi *= 2;
    }
    while (hi - lo > 1) {
        const int mid = lo + (hi - lo) / 2;
        if (vp::carve_state(nullptr, mid, plan->K, mp, plan->n_paths, &probe) <= kNoAllocBytes) lo = mid;
        else hi = mid;
    }
    return lo;
}

vp_status vp_precode_noalloc(const vp_plan* plan, const void* H, int C, const uint8_t* sym_idx, int S, void* x,
                             int8_t* l, float* gamma, uint8_t* status, void* stream)
{
    if (!plan || !H || !sym_idx || !x || !l || !gamma || C < 1 || S < 0) return VP_ERR_INVALID_ARG;
    if ((long long)C * S > 0x7fffffffLL) return VP_ERR_INVALID_ARG;
    if (plan->K > plan->M && !(plan->lambda > 0.f)) return VP_ERR_INVALID_ARG;
    const int mp = vp::p_rows(plan);
    vp::DeviceState probe;
    if (vp::carve_state(nullptr, C, plan->K, mp, plan->n_paths, &probe) > kNoAllocBytes) return VP_ERR_CAPACITY;
    void* base = nullptr;
    vp_status st = scratch_address(&base);
    if (st != VP_OK) return st;

    vp_plan p = *plan;                    // parameters only; the state points into the array
    vp::carve_state(static_cast<unsigned char*>(base), C, p.K, mp, p.n_paths, &p.d);
    p.cap = C;
    p.C = C;
    if (vp::enqueue_slot(&p, static_cast<const float2*>(H), C, sym_idx, S, static_cast<float2*>(x), l, gamma, status,
                         static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return VP_ERR_CUDA;
    return VP_OK;
}

}  // extern "C"
