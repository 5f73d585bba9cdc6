// Most-promising-path selection (Section III-A-2): the n position vectors p
// with the smallest Metric of Promise M(p) = sum_l w_l (p_l - 1) (Eq. mop),
// by breadth-first K-Best over the levels.
//
// One block per channel. The weights are scaled by a power of two into
// integers, q_l = w_l * 2^(55-e) with max_l w_l < 2^e (exact for every FP32
// weight within 2^32 of the largest), so every partial metric is an exact
// uint64 sum, ties in the real metric stay ties, and (metric, code) is a
// strict total order. With it K-Best keeps exactly the n smallest vectors,
// whatever the level order.
//
// Levels are visited in increasing weight (K-Best is exact in any level
// order under this total order), which lets fewer children enter the later
// levels. Level step: the children of the survivors S are S + k (q_l, 1 << 4l),
// k = 0..8, all shifted copies of the sorted list S. Their n smallest follow
// from three doubling merges and one more (S+{0,1} -> S+{0..3} -> S+{0..7},
// then with S+8), each cut to n entries: the n smallest of a union only need
// the n smallest of each part. A merge is skipped when the shifted copy
// starts after the current n-th entry. Each merge is a merge-path pass of
// one warp (8 outputs per lane at n = 256), synchronised with __syncwarp.
#include "vp_internal.cuh"

namespace vp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct PathArgs {
    int C, K, n, nch;
    int ns;                     // skewed list length of the launch's largest n
    int gstride;                // shared memory of one channel group, in 8-byte words
    DeviceState d;
    const BatchProblem* probs;  // batch mode: channel i of the launch is problem ids[i]
    const int* ids;
};

// Shared-memory lists use a skewed index (one pad word per 8 entries): the
// lanes of a merge own contiguous output ranges, and without the pad their
// 64-bit accesses would fall on two banks only.
__device__ __forceinline__ int sk(int i) { return i + (i >> 3); }

__device__ __forceinline__ bool key_less(uint64_t am, uint64_t ac, uint64_t bm, uint64_t bc)
{
    return am < bm || (am == bm && ac < bc);
}

// First `nout` outputs of the merge of sorted A[0..na) with the sorted list
// B[0..nb) shifted by (dm, dc), into O; thread t of the channel's `tpc`
// threads writes outputs [t*per, (t+1)*per). The metric decides; the code is
// compared only when two metrics are equal.
__device__ void merge_shift(const uint64_t* Am, const uint64_t* Ac, int na,
                            const uint64_t* Bm, const uint64_t* Bc, int nb, uint64_t dm, uint64_t dc,
                            uint64_t* Om, uint64_t* Oc, int nout, int t, int tpc)
{
    const int per = (nout + tpc - 1) / tpc;
    const int d0 = min(t * per, nout);
    const int d1 = min(d0 + per, nout);
    if (d0 >= d1) return;
    int lo = max(0, d0 - nb), hi = min(d0, na);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int bj = d0 - mid - 1;
        const uint64_t am = Am[sk(mid)], bmv = Bm[sk(bj)] + dm;
        const bool lt = am < bmv || (am == bmv && Ac[sk(mid)] < Bc[sk(bj)] + dc);
        if (lt) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = d0 - lo;
    uint64_t am = i < na ? Am[sk(i)] : ~0ull;
    uint64_t bmv = j < nb ? Bm[sk(j)] + dm : ~0ull;
    for (int d = d0; d < d1; ++d) {
        bool takeA;
        if (j >= nb) takeA = true;
        else if (i >= na) takeA = false;
        else takeA = am < bmv || (am == bmv && Ac[sk(i)] < Bc[sk(j)] + dc);
        if (takeA) {
            Om[sk(d)] = am;
            Oc[sk(d)] = Ac[sk(i)];
            ++i;
            am = i < na ? Am[sk(i)] : ~0ull;
        } else {
            Om[sk(d)] = bmv;
            Oc[sk(d)] = Bc[sk(j)] + dc;
            ++j;
            bmv = j < nb ? Bm[sk(j)] + dm : ~0ull;
        }
    }
}

// Evaluation order of a channel's paths for the search, computed once per
// channel (every vector of the channel uses it):
//  1. shared top levels: presence bitmaps of the top-1/2/3-level prefixes
//     give the largest T <= kSplitMax whose distinct prefixes fit one pass of
//     kMaxPrefix lanes (when K fills its search tile and there are 2+
//     chunks); a path's prefix index is its prefix's rank in the bitmap;
//  2. evaluation order: the paths sorted by their digits from level 1 up (the
//     light levels, where the candidates differ most), so that a 32-path
//     chunk shares small digits and needs the cheap DEMAP branches (results
//     do not depend on the order: ties are broken by MoP rank);
//  3. per chunk and level the largest digit, and over the prefixes.
// The group's list buffers are reused (the paths were already written to
// `out`, which is read back after the barrier).
__host__ __device__ inline int pow2_ceil(int n)
{
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}
__host__ __device__ inline size_t eval_order_bytes(int n) { return 12 * (size_t)pow2_ceil(n) + 8 + 1664; }

// (key, val) pairs ordered by key, then val (padding entries are equal pairs)
__device__ __forceinline__ bool kv_less(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb)
{
    return ka < kb || (ka == kb && va < vb);
}

// Ascending bitonic sort of key[0..np2) / val[0..np2) (np2 = E * tpc) held in
// registers, E consecutive entries per thread (entry i = t E + e): partners
// within a thread are compared in registers, within a warp through
// shuffles, and across the group's warps through shared memory (key / val
// are the staging area). The same network as the shared-memory sort.
template <int E>
__device__ void bitonic_regs(uint64_t* key, uint32_t* val, int np2, int t, int tpc)
{
    auto gsync = [&]() {
        if (tpc == 32) __syncwarp(kFull);
        else __syncthreads();
    };
    uint64_t k[E];
    uint32_t v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        k[e] = key[t * E + e];
        v[e] = val[t * E + e];
    }
    gsync();
    for (int kk = 2; kk <= np2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j < E) {                                      // partner in the same thread
#pragma unroll
                for (int jj = E >> 1; jj >= 1; jj >>= 1) {    // compile-time distance: registers stay registers
                    if (jj != j) continue;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int f = e ^ jj;
                        if (f > e) {
                            const int i = t * E + e;
                            const bool up = (i & kk) == 0;
                            if (kv_less(k[f], v[f], k[e], v[e]) == up) {
                                const uint64_t tk = k[e]; k[e] = k[f]; k[f] = tk;
                                const uint32_t tv = v[e]; v[e] = v[f]; v[f] = tv;
                            }
                        }
                    }
                }
            } else {
                const int tm = j / E;                         // partner thread t ^ tm
                if (tm < 32) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int i = t * E + e;
                        const uint64_t ok = __shfl_xor_sync(kFull, k[e], tm);
                        const uint32_t ov = __shfl_xor_sync(kFull, v[e], tm);
                        const bool up = (i & kk) == 0, low = (i & j) == 0;
                        const bool other_less = kv_less(ok, ov, k[e], v[e]);
                        if (other_less == (up == low)) { k[e] = ok; v[e] = ov; }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        key[t * E + e] = k[e];
                        val[t * E + e] = v[e];
                    }
                    gsync();
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int i = t * E + e;
                        const uint64_t ok = key[(t ^ tm) * E + e];
                        const uint32_t ov = val[(t ^ tm) * E + e];
                        const bool up = (i & kk) == 0, low = (i & j) == 0;
                        const bool other_less = kv_less(ok, ov, k[e], v[e]);
                        if (other_less == (up == low)) { k[e] = ok; v[e] = ov; }
                    }
                    gsync();
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        key[t * E + e] = k[e];
        val[t * E + e] = v[e];
    }
    gsync();
}

__device__ void eval_order(const ChanState& cs, const uint64_t* out, uint64_t* base, int n, int K, int nch, int t,
                           int tpc)
{
    constexpr int kBits = 16 * 16 * 16;                          // top three digits
    auto gsync = [&]() {
        if (tpc == 32) __syncwarp(kFull);
        else __syncthreads();
    };
    const int lane = t & 31, wig = t >> 5, nwarp = tpc >> 5;
    const int np2 = pow2_ceil(n);
    uint64_t* key = base;                                                  // [np2] sort keys
    uint32_t* val = reinterpret_cast<uint32_t*>(base + np2);               // [np2] rank | prefix << 16
    uint64_t* pcs = base + np2 + (np2 + 1) / 2;                            // [kMaxPrefix] prefix codes
    uint32_t* bm3 = reinterpret_cast<uint32_t*>(pcs + kMaxPrefix);         // [128] prefixes of 3 levels
    int* wpre = reinterpret_cast<int*>(bm3 + kBits / 32);                  // [128] set bits before a word
    uint32_t* bm2 = reinterpret_cast<uint32_t*>(wpre + kBits / 32);        // [8]
    uint32_t* bm1 = bm2 + 8;                                               // [1]
    gsync();
    for (int i = t; i < kBits / 32; i += tpc) bm3[i] = 0u;
    for (int i = t; i < 8; i += tpc) bm2[i] = 0u;
    if (t == 0) bm1[0] = 0u;
    gsync();
    const bool split = K == search_tile(K) && K >= 8 && nch >= 2;
    if (split) {
        for (int i = t; i < n; i += tpc) {
            const unsigned p3 = (unsigned)(out[i] >> (4 * (K - 3))) & 0xfffu;
            atomicOr(&bm3[p3 >> 5], 1u << (p3 & 31));
            atomicOr(&bm2[(p3 >> 4) >> 5], 1u << ((p3 >> 4) & 31));
            atomicOr(&bm1[0], 1u << (p3 >> 8));
        }
    }
    gsync();
    int T = 0;
    if (split) {
        // every warp counts the set bits (lane l: words 4l..4l+3 of the 3-level map)
        const int c4 = __popc(bm3[4 * lane]) + __popc(bm3[4 * lane + 1]) + __popc(bm3[4 * lane + 2]) +
                       __popc(bm3[4 * lane + 3]);
        int incl = c4;                                           // inclusive scan over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const int n3 = __shfl_sync(kFull, incl, 31);
        int c2 = lane < 8 ? __popc(bm2[lane]) : 0, i2 = c2;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const int v = __shfl_up_sync(kFull, i2, o);
            if (lane >= o) i2 += v;
        }
        const int n2 = __shfl_sync(kFull, i2, 7);
        const int n1 = __popc(bm1[0]);
        T = n3 <= kMaxPrefix ? 3 : (n2 <= kMaxPrefix ? 2 : (n1 <= kMaxPrefix ? 1 : 0));
        if (wig == 0) {                                          // words' exclusive prefix counts
            if (T == 3) {
                int r = incl - c4;
                for (int q = 0; q < 4; ++q) {
                    wpre[4 * lane + q] = r;
                    r += __popc(bm3[4 * lane + q]);
                }
            } else if (T == 2 && lane < 8) {
                wpre[lane] = i2 - c2;
            }
        }
    }
    gsync();
    const int npf = T == 3 ? wpre[kBits / 32 - 1] + __popc(bm3[kBits / 32 - 1])
                  : T == 2 ? wpre[7] + __popc(bm2[7])
                  : T == 1 ? __popc(bm1[0]) : 1;
    for (int i = t; i < np2; i += tpc) {
        if (i >= n) {
            key[i] = ~0ull;
            val[i] = 0u;
            continue;
        }
        const uint64_t c = out[i];
        int p = 0;
        if (T > 0) {
            const unsigned pv = (unsigned)(c >> (4 * (K - T))) & ((1u << (4 * T)) - 1u);
            if (T == 3) p = wpre[pv >> 5] + __popc(bm3[pv >> 5] & ((1u << (pv & 31)) - 1u));
            else if (T == 2) p = wpre[pv >> 5] + __popc(bm2[pv >> 5] & ((1u << (pv & 31)) - 1u));
            else p = __popc(bm1[0] & ((1u << pv) - 1u));
            pcs[p] = c;                                          // any code with this prefix
        }
        key[i] = nibble_reverse(c, K);
        val[i] = (uint32_t)i | ((uint32_t)p << 16);
    }
    if (T == 0 && t == 0) pcs[0] = 0ull;
    gsync();
    const int E = np2 / tpc;
    if (nch > 1 && np2 >= tpc && E <= 8) {                       // ascending sort in registers
        if (E == 1) bitonic_regs<1>(key, val, np2, t, tpc);
        else if (E == 2) bitonic_regs<2>(key, val, np2, t, tpc);
        else if (E == 4) bitonic_regs<4>(key, val, np2, t, tpc);
        else bitonic_regs<8>(key, val, np2, t, tpc);
    } else
    for (int k = 2; k <= (nch > 1 ? np2 : 1); k <<= 1) {         // ascending bitonic sort, keys distinct
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = t; i < (np2 >> 1); i += tpc) {
                const int ix = ((i & ~(j - 1)) << 1) | (i & (j - 1));
                const int iy = ix + j;
                const bool up = (ix & k) == 0;
                const uint64_t c0 = key[ix], c1 = key[iy];
                if ((c0 > c1) == up && c0 != c1) {
                    key[ix] = c1;
                    key[iy] = c0;
                    const uint32_t v = val[ix];
                    val[ix] = val[iy];
                    val[iy] = v;
                }
            }
            gsync();
        }
    }
    for (int i = t; i < n; i += tpc) {
        const uint64_t c = nibble_reverse(key[i], K);
        key[i] = c;
        cs.ecode[i] = c;
        cs.emeta[i] = val[i];
    }
    for (int i = t; i < kMaxPrefix; i += tpc) cs.pcode[i] = i < npf ? pcs[i] : 0ull;
    gsync();
    for (int ch = wig; ch < nch; ch += nwarp) {
        const int i = ch * 32 + lane;
        const uint64_t code = i < n ? key[i] : 0ull;
        uint64_t mq = 0;
        for (int l = 0; l < K; ++l)
            mq |= (uint64_t)__reduce_max_sync(kFull, (unsigned)((code >> (4 * l)) & 15u)) << (4 * l);
        if (lane == 0) cs.maxq[ch] = mq;
    }
    if (wig == 0) {
        const uint64_t code = lane < npf ? pcs[lane] : 0ull;
        uint64_t mq = 0;
        for (int l = K - T; l < K; ++l)
            mq |= (uint64_t)__reduce_max_sync(kFull, (unsigned)((code >> (4 * l)) & 15u)) << (4 * l);
        if (lane == 0) cs.phdr[0] = make_int4(T, npf, (int)(uint32_t)mq, (int)(uint32_t)(mq >> 32));
    }
}

// A channel is worked on by `tpc` threads: one warp (a block then holds `cpb`
// channels) or a whole block of 2-4 warps (cpb = 1), which shortens the
// dependent merge chains of a channel. Shared memory: 48 n bytes per channel.
__global__ void pathsel_kernel(PathArgs a, int cpb)
{
    extern __shared__ uint64_t shm[];
    __shared__ uint64_t qws[8][kMaxK];
    __shared__ int ords[8][kMaxK];
    pdl_wait();                                                  // weights and status of the factor kernels
    const int tpc = blockDim.x / cpb;                            // threads per channel
    const int grp = threadIdx.x / tpc, t = threadIdx.x % tpc;
    const int lane = threadIdx.x & 31, wig = t >> 5;             // lane, warp within the channel's group
    const int ci = blockIdx.x * cpb + grp;
    if (ci >= a.C) return;
    int n = a.n, K = a.K, nch = a.nch;
    ChanState cs;
    if (a.probs) {
        const BatchProblem& p = a.probs[a.ids[ci]];
        n = p.n;
        K = p.K;
        nch = n_chunks(n);
        cs = chan_state(p);
    } else {
        cs = chan_state(a.d, (size_t)ci, K, 0, n);
    }
    const int ns = sk(n);                                        // skewed length of one list
    uint64_t* base = shm + (size_t)grp * a.gstride;
    // buffer b (0..2): metrics at base + 2 b ns, codes at base + (2 b + 1) ns
    // (pointer arithmetic: an indexed pointer array would live in local memory)
#define BM(b) (base + 2 * (b) * ns)
#define BC(b) (base + (2 * (b) + 1) * ns)
    uint64_t* qw = qws[grp];
    int* ord = ords[grp];
    uint64_t* out = cs.paths;
    uint64_t* mqo = cs.maxq;

    if (cs.st[0] & (VP_CH_NONFINITE | VP_CH_SINGULAR)) {
        for (int i = t; i < n; i += tpc) out[i] = 0;
        for (int i = t; i < nch; i += tpc) mqo[i] = 0;
        if (t == 0) cs.phdr[0] = make_int4(0, 1, 0, 0);
        return;
    }
    if (wig == 0) {
        const float wl = lane < K ? cs.w[lane] : 0.f;
        float wmax = wl;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(kFull, wmax, o));
        int e;
        frexpf(wmax, &e);                      // wmax < 2^e, so 8 K w 2^(55-e) < 2^62
        if (lane < K) qw[lane] = __double2ull_rn(ldexp((double)wl, 55 - e));
        // levels in increasing weight (ties: lower level): fewer children enter the later levels
        if (lane < K) {
            int rank = 0;
            for (int k = 0; k < K; ++k) {
                const float wk = cs.w[k];
                rank += (wk < wl) || (wk == wl && k < lane);
            }
            ord[rank] = lane;
        }
        if (lane == 0) { BM(0)[0] = 0; BC(0)[0] = 0; }
    }
    if (tpc == 32) __syncwarp(kFull); else __syncthreads();

    int iS = 0, s = 1;
    for (int li = 0; li < K; ++li) {
        const int l = ord[li];
        const uint64_t q = qw[l];
        const uint64_t d1 = 1ull << (4 * l);
        int ix = iS, nx = s;
        for (int step = 0; step < 4; ++step) {
            // steps 0..2: X + 2^step * delta; step 3: S + 8 * delta
            const uint64_t mul = step < 3 ? (1ull << step) : 8ull;
            const int ib = step < 3 ? ix : iS;
            const int nb = step < 3 ? nx : s;
            const uint64_t dm = mul * q, dc = mul * d1;
            const bool skip = nx >= n && key_less(BM(ix)[sk(n - 1)], BC(ix)[sk(n - 1)], BM(ib)[0] + dm, BC(ib)[0] + dc);
            if (skip) continue;
            const int io = (ix == iS) ? (iS + 1) % 3 : 3 - ix - iS;
            const int nout = min(nx + nb, n);
            merge_shift(BM(ix), BC(ix), nx, BM(ib), BC(ib), nb, dm, dc, BM(io), BC(io), nout, t, tpc);
            if (tpc == 32) __syncwarp(kFull); else __syncthreads();
            ix = io;
            nx = nout;
        }
        iS = ix;
        s = nx;
    }

    const uint64_t* Sc = BC(iS);
#undef BM
#undef BC
    for (int i = t; i < n; i += tpc) out[i] = (i < s) ? Sc[sk(i)] : 0;
    eval_order(cs, out, base, n, K, nch, t, tpc);
    pdl_trigger();
}

cudaError_t run_pathsel(PathArgs a, int n_max, cudaStream_t s, int tpc_set = 0)
{
    const int ns = n_max + (n_max >> 3);
    a.ns = ns;
    size_t per = (size_t)6 * ns * sizeof(uint64_t);
    if (per < eval_order_bytes(n_max)) per = (eval_order_bytes(n_max) + 15) & ~size_t(15);
    // long lists: a block of warps per channel (2 warps up to 256 paths, 4 for
    // 512-1024, measured best on GB300); short ones: a warp per channel
    a.gstride = (int)(per / sizeof(uint64_t));
    int tpc = n_max >= 512 ? 128 : (n_max >= 128 ? 64 : 32);
    if (tpc_set == 32 || tpc_set == 64 || tpc_set == 128 || tpc_set == 256) tpc = tpc_set;
    int cpb = 1;
    if (tpc == 32) {
        cpb = (int)((48 * 1024) / per);
        cpb = cpb < 1 ? 1 : (cpb > 8 ? 8 : cpb);
    }
    const size_t shbytes = per * cpb;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(pathsel_kernel), shbytes);
    if (e != cudaSuccess) return e;
    return launch_dependent(pathsel_kernel, dim3((a.C + cpb - 1) / cpb), dim3(tpc * cpb), shbytes, s, a, cpb);
}

}  // namespace

cudaError_t launch_pathsel(const vp_plan* p, int C, cudaStream_t s)
{
    PathArgs a;
    a.C = C;
    a.K = p->K;
    a.n = p->n_paths;
    a.nch = n_chunks(p->n_paths);
    a.d = p->d;
    a.probs = nullptr;
    a.ids = nullptr;
    return run_pathsel(a, p->n_paths, s);
}

cudaError_t launch_pathsel_batch(const BatchProblem* probs, const int* ids, int count, int n_max, cudaStream_t s,
                                 int tpc)
{
    PathArgs a = PathArgs();
    a.C = count;
    a.probs = probs;
    a.ids = ids;
    return run_pathsel(a, n_max, s, tpc);
}

}  // namespace vp
