// Internal declarations of libvp (GPU side only; never included by the oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vp.h"

namespace vp {

constexpr int kMaxK = VP_MAX_K;
constexpr int kMaxM = VP_MAX_M;
constexpr int kMaxPaths = VP_MAX_PATHS;
// The search evaluates the top T <= kSplitMax levels once per distinct path
// prefix (at most kMaxPrefix of them, one lane each).
constexpr int kMaxPrefix = 32;
constexpr int kSplitMax = 3;

// Resident per-channel state of a plan (device pointers, capacity `cap` channels).
struct DeviceState {
    float4* utp = nullptr;     // [cap][K][K] unit-upper U~ = U_lk / U_ll, as (re, im, im, re)
    float2* utc = nullptr;     // [cap][K][K] U~ transposed (utc[m][l] = U~[l][m]), for the per-vector prologue
    float* w = nullptr;        // [cap][K]    w_l = U_ll^2 = 1 / R_ll^2
    uint8_t* ul = nullptr;     // [cap][K]    user at level l
    float2* pt = nullptr;      // [cap][K][Mp] P^T in user order: pt[c][k][m] = P[m][k] (leading part)
    float2* ptlo = nullptr;    // [cap][K][Mp] trailing part: P = pt + ptlo (zero where P is FP32-accurate)
                               // Mp = M, or M + K with lambda > 0 (rows M.. map u to the
                               // regularisation part of w = Qbar^H Rt u, Alg. 2)
    uint64_t* paths = nullptr; // [cap][n]    path codes, rank order
    uint64_t* maxq = nullptr;  // [cap][nchunk] per 32-path chunk of the evaluation order, per level: max digit
    uint64_t* ecode = nullptr; // [cap][n]    path codes in evaluation order
    uint32_t* emeta = nullptr; // [cap][n]    MoP rank | shared-prefix index << 16, evaluation order
    uint64_t* pcode = nullptr; // [cap][kMaxPrefix] a code of each shared prefix
    int4* phdr = nullptr;      // [cap]       shared levels T, prefix count, per-level max digit of the prefixes
    uint8_t* st = nullptr;     // [cap]       VP_CH_* bits
    int* nflag = nullptr;      // [1]         number of channels sent to the FP64 path
    int* flags = nullptr;      // [cap]       their indices
};

// One problem of an uneven batch (one channel and its S data vectors), as
// the kernels read it from the device table of vp_precode_batch. The state
// pointers point into the batch workspace.
struct BatchProblem {
    const float2* H;      // [K][M]
    const uint8_t* sym;   // [S][K]
    float2* x;            // [S][M]
    int8_t* l;            // [S][K][2]
    float* gamma;         // [S]
    uint8_t* status;      // [1] or null
    float4* utp;
    float2* utc;
    float* w;
    uint8_t* ul;
    float2* pt;
    float2* ptlo;
    uint64_t* paths;
    uint64_t* maxq;
    uint64_t* ecode;
    uint32_t* emeta;
    uint64_t* pcode;
    int4* phdr;
    uint8_t* st;
    int K, M, n, m_qam, S;
    float tau, kappa_thr;
    int pad_;
};

// Resident state of one channel (pointers offset to that channel).
struct ChanState {
    float4* utp;
    float2* utc;
    float* w;
    uint8_t* ul;
    float2* pt;
    float2* ptlo;
    uint64_t* paths;
    uint64_t* maxq;
    uint64_t* ecode;
    uint32_t* emeta;
    uint64_t* pcode;
    int4* phdr;
    uint8_t* st;
};

__host__ __device__ inline int n_chunks(int n_paths) { return (n_paths + 31) / 32; }

// K tile of the search kernel (levels unrolled); the shared top levels are
// used when K fills its tile (K = 8, 12, 16).
__host__ __device__ inline int search_tile(int K) { return K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : K <= 12 ? 12 : 16; }

// The K 4-bit digits of a path code in reverse level order (an involution).
__device__ __forceinline__ uint64_t nibble_reverse(uint64_t c, int K)
{
    c = __brevll(c);                                                                 // bits reversed
    c = ((c >> 1) & 0x5555555555555555ull) | ((c & 0x5555555555555555ull) << 1);
    c = ((c >> 2) & 0x3333333333333333ull) | ((c & 0x3333333333333333ull) << 2);    // nibbles restored
    return K == 16 ? c : c >> (64 - 4 * K);
}

__host__ __device__ inline ChanState chan_state(const DeviceState& d, size_t c, int K, int Mp, int n)
{
    ChanState s;
    s.utp = d.utp + c * K * K;
    s.utc = d.utc + c * K * K;
    s.w = d.w + c * K;
    s.ul = d.ul + c * K;
    s.pt = d.pt + c * K * Mp;
    s.ptlo = d.ptlo + c * K * Mp;
    s.paths = d.paths + c * n;
    s.maxq = d.maxq + c * n_chunks(n);
    s.ecode = d.ecode + c * n;
    s.emeta = d.emeta + c * n;
    s.pcode = d.pcode + c * kMaxPrefix;
    s.phdr = d.phdr + c;
    s.st = d.st + c;
    return s;
}

__host__ __device__ inline ChanState chan_state(const BatchProblem& p)
{
    ChanState s;
    s.utp = p.utp;
    s.utc = p.utc;
    s.w = p.w;
    s.ul = p.ul;
    s.pt = p.pt;
    s.ptlo = p.ptlo;
    s.paths = p.paths;
    s.maxq = p.maxq;
    s.ecode = p.ecode;
    s.emeta = p.emeta;
    s.pcode = p.pcode;
    s.phdr = p.phdr;
    s.st = p.st;
    return s;
}

}  // namespace vp

struct vp_plan {
    int K = 0, M = 0, qam = 0, n_paths = 0;
    float tau = 0.f;
    float kappa_thr = 1e4f;
    float lambda = 0.f;   // Tikhonov parameter (Hbar = [H lambda*I])
    int demap = VP_DEMAP_EXACT;
    int frac_bits = 0;                  // fixed-point search with 16-bit words (0 = floating point)
    int tensor_product = 0;             // w = P u on the tensor cores (vp_plan_set_tensor_product)
    int cap = 0;   // channel capacity of `d`
    int cap_mp = 0;  // rows of P that `d` was allocated for
    int C = 0;     // channels of the last vp_factorize
    vp::DeviceState d;
    // staging buffers of vp_run_slot_host
    void* h_H = nullptr; size_t h_H_bytes = 0;
    uint8_t* h_sym = nullptr; size_t h_sym_bytes = 0;
    void* h_x = nullptr; size_t h_x_bytes = 0;
    int8_t* h_l = nullptr; size_t h_l_bytes = 0;
    float* h_g = nullptr; size_t h_g_bytes = 0;
    int last_launches = 0;
};

namespace vp {

// Rows of the precoding map w = Qbar^H Rt u kept per channel: the M antennas,
// plus the K regularisation rows when lambda > 0.
inline int p_rows(const vp_plan* p) { return p->M + (p->lambda > 0.f ? p->K : 0); }

// Limits of one problem shape (those of vp_plan_create with lambda = 0).
inline bool shape_ok(int K, int M, int qam, int n_paths, float tau)
{
    if (K < 1 || K > VP_MAX_K || M < K || M > VP_MAX_M) return false;
    if (!(qam == 4 || qam == 16 || qam == 64 || qam == 256)) return false;
    long long p9 = 1;
    for (int i = 0; i < K && p9 <= VP_MAX_PATHS; ++i) p9 *= 9;
    if (n_paths < 1 || n_paths > VP_MAX_PATHS || (long long)n_paths > p9) return false;
    return tau >= 0.f && tau < 3.0e38f;
}

inline int qam_side(int qam)
{
    int m = 1;
    while (m * m < qam) ++m;
    return m;
}

// Per-channel state of C channels laid out from `base` in 256-byte aligned
// pieces; returns the bytes used (base = null only measures).
size_t carve_state(unsigned char* base, int C, int K, int Mp, int n, DeviceState* d);

// One slot on p's state (vp_factorize + vp_precode without the optional
// outputs): memset, factor32, factor64, pathsel, status copy, search.
cudaError_t enqueue_slot(const vp_plan* p, const float2* H, int C, const uint8_t* sym, int S, float2* x, int8_t* l,
                         float* gamma, uint8_t* status, cudaStream_t s);

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device (once per kernel, device and size; thread-safe). A no-op under the
// default 48 KB.
cudaError_t allow_dynamic_smem(const void* kernel, size_t bytes);

// Programmatic dependent launch: a kernel launched by launch_dependent may
// be scheduled while the kernel before it on the stream is still running
// (once every block of that kernel has called pdl_trigger or exited), so its
// launch and block start-up overlap the predecessor's last blocks. Every
// kernel calls pdl_wait before it reads anything that earlier work on the
// stream produced (it returns once the predecessor grid has completed and
// its writes are visible; without the launch attribute it returns at once),
// and pdl_trigger when its block's work is done: after the wait, so that
// completion is transitive along a chain of such launches, and late, since
// dependent blocks waiting beside the kernel's own work slowed it down.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                    Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Kernel launchers (each returns cudaSuccess or the launch error).
cudaError_t launch_factor32(const vp_plan* p, const float2* H, int C, float2* U_out, float2* P_out,
                            uint8_t* ul_out, cudaStream_t s);
cudaError_t launch_factor64(const vp_plan* p, const float2* H, int C, float2* U_out, float2* P_out,
                            uint8_t* ul_out, cudaStream_t s);
cudaError_t launch_pathsel(const vp_plan* p, int C, cudaStream_t s);
cudaError_t launch_search(const vp_plan* p, const uint8_t* sym, int S, const int32_t* vec_off,
                          int n_vec, float2* x, int8_t* l, float* gamma, cudaStream_t s);

// Batch launchers: `ids[0..count)` are indices into the device table `probs`.
// factor32: every listed problem has this K and M. FP64 candidates are
// appended (as table indices) to flags / nflag.
cudaError_t launch_factor32_batch(const BatchProblem* probs, const int* ids, int count, int K, int M,
                                  int* nflag, int* flags, cudaStream_t s);
// factor64: the problems listed in flags[0..*nflag); at most max_flagged of them.
cudaError_t launch_factor64_batch(const BatchProblem* probs, const int* nflag, const int* flags, int max_flagged,
                                  cudaStream_t s);
// pathsel: every listed problem has n_paths <= n_max.
// tpc: threads per channel (32, 64, 128 or 256; 0 = chosen by the list length)
cudaError_t launch_pathsel_batch(const BatchProblem* probs, const int* ids, int count, int n_max, cudaStream_t s,
                                 int tpc = 0);
// search: every listed problem has K <= KT (KT in {2, 4, 8, 12, 16}) and the
// given maxima of K*M, n_paths and S.
// nw: warps per block (1..7; 0 = chosen from s_max)
cudaError_t launch_search_batch(const BatchProblem* probs, const int* ids, int count, int KT, int km_max,
                                int n_max, int s_max, cudaStream_t s, int nw = 0);
// The whole search stage of a batch in one persistent launch: ids[0..count)
// in the order taken (heaviest first), problems of every K tile; `counter` is
// a device int that must be 0 at launch. Knobs (0 = built in): nw warps per
// block (1..7), blocks_per_sm resident (1..4: problems in flight per SM),
// stage16 = 1 stage the 16-level tile's path codes in shared memory, 2 read
// them in place.
cudaError_t launch_search_persist(const BatchProblem* probs, const int* ids, int count, int km_max, int n_max,
                                  int s_max, int* counter, cudaStream_t s, int nw = 0, int blocks_per_sm = 0,
                                  int stage16 = 0);

// ---------------------------------------------------------------------------
// Small device helpers shared by the kernels of this library.

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul_conj_a(float2 a, float2 b)   // conj(a) * b
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c)  // a*b + c
{
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// Error-free transformations (Dekker / Knuth): a*b = p + e and a+b = s + e exactly.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e)
{
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += a * b, with a*b formed exactly and the running sum compensated.
__device__ __forceinline__ void dot2_acc(float a, float b, float& hi, float& lo)
{
    float p, e, s, f;
    two_prod(a, b, p, e);
    two_sum(hi, p, s, f);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, f));
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 zfma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

// QAM index -> odd-integer point (exact in float): m = sqrt(qam).
__device__ __forceinline__ float2 qam_point(int idx, int m)
{
    return make_float2((float)(2 * (idx % m) - (m - 1)), (float)(2 * (idx / m) - (m - 1)));
}

}  // namespace vp
