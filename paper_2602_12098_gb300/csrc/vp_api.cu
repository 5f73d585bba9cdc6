// C-ABI of libvp: plan lifecycle, argument checks and kernel sequencing.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "vp_internal.cuh"

namespace {

bool valid_qam(int q) { return q == 4 || q == 16 || q == 64 || q == 256; }

long long pow9(int K)
{
    long long r = 1;
    for (int i = 0; i < K; ++i) r *= 9;
    return r;
}

void free_state(vp::DeviceState& d)
{
    cudaFree(d.utp);
    cudaFree(d.utc);
    cudaFree(d.w);
    cudaFree(d.ul);
    cudaFree(d.pt);
    cudaFree(d.ptlo);
    cudaFree(d.paths);
    cudaFree(d.maxq);
    cudaFree(d.ecode);
    cudaFree(d.emeta);
    cudaFree(d.pcode);
    cudaFree(d.phdr);
    cudaFree(d.st);
    cudaFree(d.nflag);
    cudaFree(d.flags);
    d = vp::DeviceState();
}

template <class T>
bool dalloc(T** p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16) == cudaSuccess;
}

vp_status ensure_capacity(vp_plan* p, int C)
{
    const int mp = vp::p_rows(p);
    if (C <= p->cap && mp == p->cap_mp) return VP_OK;
    cudaDeviceSynchronize();                 // no enqueued work may still read the old state
    free_state(p->d);
    p->cap = 0;
    p->cap_mp = 0;
    const size_t K = p->K, M = (size_t)mp, n = p->n_paths, nch = vp::n_chunks(p->n_paths);
    vp::DeviceState d;
    bool ok = dalloc(&d.utp, (size_t)C * K * K) && dalloc(&d.utc, (size_t)C * K * K) &&
              dalloc(&d.w, (size_t)C * K) && dalloc(&d.ul, (size_t)C * K) && dalloc(&d.pt, (size_t)C * K * M) && dalloc(&d.ptlo, (size_t)C * K * M) &&
              dalloc(&d.paths, (size_t)C * n) && dalloc(&d.maxq, (size_t)C * nch) && dalloc(&d.ecode, (size_t)C * n) &&
              dalloc(&d.emeta, (size_t)C * n) && dalloc(&d.pcode, (size_t)C * vp::kMaxPrefix) &&
              dalloc(&d.phdr, (size_t)C) && dalloc(&d.st, (size_t)C) &&
              dalloc(&d.nflag, 1) && dalloc(&d.flags, (size_t)C);
    if (!ok) {
        free_state(d);
        cudaGetLastError();
        return VP_ERR_OOM;
    }
    p->d = d;
    p->cap = C;
    p->cap_mp = mp;
    return VP_OK;
}

template <class T>
vp_status ensure_buf(T** p, size_t* have, size_t need)
{
    if (need <= *have) return VP_OK;
    cudaDeviceSynchronize();
    cudaFree(*p);
    *p = nullptr;
    *have = 0;
    if (cudaMalloc(reinterpret_cast<void**>(p), need) != cudaSuccess) {
        cudaGetLastError();
        return VP_ERR_OOM;
    }
    *have = need;
    return VP_OK;
}

// Device address of page-locked host memory that the GPU can read and write
// in place (over NVLink-C2C on Grace systems), or null (pageable memory, or
// the mapping is not available).
void* mapped(const void* hp)
{
    if (!hp) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, hp) != cudaSuccess || at.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return nullptr;
    }
    void* dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, const_cast<void*>(hp), 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return dp;
}

}  // namespace

namespace vp {

cudaError_t allow_dynamic_smem(const void* kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> raised;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = raised[std::make_pair(kernel, dev)];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

}  // namespace vp

extern "C" {

const char* vp_status_string(vp_status s)
{
    switch (s) {
    case VP_OK: return "ok";
    case VP_ERR_INVALID_ARG: return "invalid argument";
    case VP_ERR_CUDA: return "CUDA error";
    case VP_ERR_OOM: return "out of device memory";
    case VP_ERR_TIMEOUT: return "device wait timed out";
    case VP_ERR_NOT_FACTORIZED: return "no factorised channels";
    case VP_ERR_CAPACITY: return "exceeds the fixed storage (vp_precode_noalloc array or server pool)";
    }
    return "unknown status";
}

vp_status vp_plan_create(int K, int M, int qam, int n_paths, float tau, vp_plan** out)
{
    if (!out) return VP_ERR_INVALID_ARG;
    *out = nullptr;
    if (K < 1 || K > VP_MAX_K || M < 1 || M > VP_MAX_M || !valid_qam(qam)) return VP_ERR_INVALID_ARG;
    if (n_paths < 1 || n_paths > VP_MAX_PATHS || (long long)n_paths > pow9(K)) return VP_ERR_INVALID_ARG;
    if (!(tau >= 0.f) || !std::isfinite(tau)) return VP_ERR_INVALID_ARG;
    vp_plan* p = new (std::nothrow) vp_plan();
    if (!p) return VP_ERR_OOM;
    p->K = K;
    p->M = M;
    p->qam = qam;
    p->n_paths = n_paths;
    p->tau = (tau == 0.f) ? 2.0f * std::sqrt((float)qam) : tau;
    *out = p;
    return VP_OK;
}

vp_status vp_plan_set_fp64_threshold(vp_plan* p, float kappa_hat)
{
    if (!p || std::isnan(kappa_hat) || kappa_hat < 0.f) return VP_ERR_INVALID_ARG;
    p->kappa_thr = kappa_hat;
    return VP_OK;
}

vp_status vp_plan_set_lambda(vp_plan* p, float lambda)
{
    if (!p || !(lambda >= 0.f) || !std::isfinite(lambda)) return VP_ERR_INVALID_ARG;
    p->lambda = lambda;
    p->C = 0;   // the resident state no longer matches: factorise again
    return VP_OK;
}

vp_status vp_plan_set_demap(vp_plan* p, int demap)
{
    if (!p || (demap != VP_DEMAP_EXACT && demap != VP_DEMAP_LUT)) return VP_ERR_INVALID_ARG;
    if (demap == VP_DEMAP_LUT && p->frac_bits > 0) return VP_ERR_INVALID_ARG;
    p->demap = demap;
    return VP_OK;
}

vp_status vp_plan_set_fixed_point(vp_plan* p, int frac_bits)
{
    if (!p || frac_bits < 0 || frac_bits > 15) return VP_ERR_INVALID_ARG;
    if (frac_bits > 0 && p->demap != VP_DEMAP_EXACT) return VP_ERR_INVALID_ARG;
    p->frac_bits = frac_bits;
    return VP_OK;
}

vp_status vp_plan_set_tensor_product(vp_plan* p, int enable)
{
    if (!p || (enable != 0 && enable != 1)) return VP_ERR_INVALID_ARG;
    p->tensor_product = enable;
    return VP_OK;
}

vp_status vp_plan_destroy(vp_plan* p)
{
    if (!p) return VP_OK;
    cudaDeviceSynchronize();
    free_state(p->d);
    cudaFree(p->h_H);
    cudaFree(p->h_sym);
    cudaFree(p->h_x);
    cudaFree(p->h_l);
    cudaFree(p->h_g);
    delete p;
    return VP_OK;
}

vp_status vp_factorize(vp_plan* p, const void* H, int C, void* U, void* P, uint8_t* user_of_level,
                       uint8_t* status, void* stream)
{
    if (!p || !H || C < 1) return VP_ERR_INVALID_ARG;
    if (p->K > p->M && !(p->lambda > 0.f)) return VP_ERR_INVALID_ARG;   // H H^H singular without lambda
    vp_status st = ensure_capacity(p, C);
    if (st != VP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float2* h = static_cast<const float2*>(H);
    p->last_launches = 0;
    if (cudaMemsetAsync(p->d.nflag, 0, sizeof(int), s) != cudaSuccess) return VP_ERR_CUDA;
    if (vp::launch_factor32(p, h, C, static_cast<float2*>(U), static_cast<float2*>(P), user_of_level, s) != cudaSuccess)
        return VP_ERR_CUDA;
    if (vp::launch_factor64(p, h, C, static_cast<float2*>(U), static_cast<float2*>(P), user_of_level, s) != cudaSuccess)
        return VP_ERR_CUDA;
    if (vp::launch_pathsel(p, C, s) != cudaSuccess) return VP_ERR_CUDA;
    p->last_launches = 3;
    if (status && cudaMemcpyAsync(status, p->d.st, (size_t)C, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return VP_ERR_CUDA;
    p->C = C;
    return VP_OK;
}

vp_status vp_precode(vp_plan* p, const uint8_t* sym_idx, int S, const int32_t* vec_offsets, int n_vec, void* x,
                     int8_t* l, float* gamma, void* stream)
{
    if (!p || !sym_idx || !x || !l || !gamma || n_vec < 0) return VP_ERR_INVALID_ARG;
    if (p->C < 1) return VP_ERR_NOT_FACTORIZED;
    if (!vec_offsets) {
        if (S < 0 || (long long)S * p->C != (long long)n_vec) return VP_ERR_INVALID_ARG;
    }
    p->last_launches = 0;
    if (n_vec == 0) return VP_OK;
    if (vp::launch_search(p, sym_idx, S, vec_offsets, n_vec, static_cast<float2*>(x), l, gamma,
                          static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return VP_ERR_CUDA;
    p->last_launches = 1;
    return VP_OK;
}

vp_status vp_get_paths(vp_plan* p, uint64_t* codes, void* stream)
{
    if (!p || !codes) return VP_ERR_INVALID_ARG;
    if (p->C < 1) return VP_ERR_NOT_FACTORIZED;
    if (cudaMemcpyAsync(codes, p->d.paths, sizeof(uint64_t) * (size_t)p->C * p->n_paths, cudaMemcpyDeviceToDevice,
                        static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return VP_ERR_CUDA;
    return VP_OK;
}

vp_status vp_run_slot_host(vp_plan* p, const void* H_host, int C, const uint8_t* sym_host, int S, void* x_host,
                           int8_t* l_host, float* gamma_host, void* stream)
{
    if (!p || !H_host || !sym_host || !x_host || C < 1 || S < 0) return VP_ERR_INVALID_ARG;
    const size_t V = (size_t)C * S;
    const size_t hb = sizeof(float2) * (size_t)C * p->K * p->M;
    const size_t sb = V * p->K, xb = sizeof(float2) * V * p->M, lb = V * p->K * 2, gb = sizeof(float) * V;
    vp_status st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = ensure_buf(&p->h_H, &p->h_H_bytes, hb)) != VP_OK) return st;
    if ((st = ensure_buf(&p->h_sym, &p->h_sym_bytes, sb + 1)) != VP_OK) return st;
    if ((st = ensure_buf(&p->h_x, &p->h_x_bytes, xb + 1)) != VP_OK) return st;
    if ((st = ensure_buf(&p->h_l, &p->h_l_bytes, lb + 1)) != VP_OK) return st;
    if ((st = ensure_buf(&p->h_g, &p->h_g_bytes, gb + 1)) != VP_OK) return st;
    if (cudaMemcpyAsync(p->h_H, H_host, hb, cudaMemcpyHostToDevice, s) != cudaSuccess) return VP_ERR_CUDA;
    if (sb && cudaMemcpyAsync(p->h_sym, sym_host, sb, cudaMemcpyHostToDevice, s) != cudaSuccess) return VP_ERR_CUDA;
    if ((st = vp_factorize(p, p->h_H, C, nullptr, nullptr, nullptr, nullptr, stream)) != VP_OK) return st;
    const int nf = p->last_launches;
    // page-locked, mapped output buffers are written by the search kernel in
    // place (over NVLink-C2C on Grace systems), saving the copies back
    void* xd = mapped(x_host);
    void* ld = mapped(l_host);
    void* gd = mapped(gamma_host);
    if ((st = vp_precode(p, p->h_sym, S, nullptr, (int)V, xd ? xd : p->h_x, ld ? static_cast<int8_t*>(ld) : p->h_l,
                         gd ? static_cast<float*>(gd) : p->h_g, stream)) != VP_OK)
        return st;
    p->last_launches += nf;
    if (!xd && xb && cudaMemcpyAsync(x_host, p->h_x, xb, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return VP_ERR_CUDA;
    if (l_host && !ld && lb && cudaMemcpyAsync(l_host, p->h_l, lb, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return VP_ERR_CUDA;
    if (gamma_host && !gd && gb && cudaMemcpyAsync(gamma_host, p->h_g, gb, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return VP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VP_ERR_CUDA;
    return VP_OK;
}

int vp_last_launch_count(const vp_plan* p) { return p ? p->last_launches : 0; }

}  // extern "C"
