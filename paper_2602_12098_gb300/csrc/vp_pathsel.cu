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
// Level step: the children of the survivors S are S + k (q_l, 1 << 4l),
// k = 0..8, all shifted copies of the sorted list S. Their n smallest follow
// from three doubling merges and one more (S+{0,1} -> S+{0..3} -> S+{0..7},
// then with S+8), each cut to n entries: the n smallest of a union only need
// the n smallest of each part. A merge is skipped when the shifted copy
// starts after the current n-th entry. Each merge is a merge-path pass.
#include "vp_internal.cuh"

namespace vp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct PathArgs {
    int C, K, n, nch;
    DeviceState d;
};

__device__ __forceinline__ bool key_less(uint64_t am, uint64_t ac, uint64_t bm, uint64_t bc)
{
    return am < bm || (am == bm && ac < bc);
}

// First `nout` outputs of the merge of sorted A[0..na) with the sorted list
// B[0..nb) shifted by (dm, dc), into O. Threads split the output range.
__device__ void merge_shift(const uint64_t* Am, const uint64_t* Ac, int na,
                            const uint64_t* Bm, const uint64_t* Bc, int nb, uint64_t dm, uint64_t dc,
                            uint64_t* Om, uint64_t* Oc, int nout, int tid, int T)
{
    const int per = (nout + T - 1) / T;
    const int d0 = min(tid * per, nout);
    const int d1 = min(d0 + per, nout);
    if (d0 >= d1) return;
    int lo = max(0, d0 - nb), hi = min(d0, na);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int bj = d0 - mid - 1;
        if (key_less(Am[mid], Ac[mid], Bm[bj] + dm, Bc[bj] + dc)) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = d0 - lo;
    for (int d = d0; d < d1; ++d) {
        const bool takeA = (j >= nb) || (i < na && key_less(Am[i], Ac[i], Bm[j] + dm, Bc[j] + dc));
        if (takeA) { Om[d] = Am[i]; Oc[d] = Ac[i]; ++i; }
        else { Om[d] = Bm[j] + dm; Oc[d] = Bc[j] + dc; ++j; }
    }
}

__global__ void pathsel_kernel(PathArgs a)
{
    extern __shared__ uint64_t shm[];
    __shared__ uint64_t qw[kMaxK];
    const int n = a.n, K = a.K, T = blockDim.x, tid = threadIdx.x;
    uint64_t* bm[3] = {shm, shm + 2 * n, shm + 4 * n};       // metrics of the three buffers
    uint64_t* bc[3] = {shm + n, shm + 3 * n, shm + 5 * n};   // codes
    const int c = blockIdx.x;
    uint64_t* out = a.d.paths + (size_t)c * n;
    uint64_t* mqo = a.d.maxq + (size_t)c * a.nch;

    if (a.d.st[c] & (VP_CH_NONFINITE | VP_CH_SINGULAR)) {
        for (int i = tid; i < n; i += T) out[i] = 0;
        for (int i = tid; i < a.nch; i += T) mqo[i] = 0;
        return;
    }
    if (tid == 0) {
        float wmax = 0.f;
        for (int l = 0; l < K; ++l) wmax = fmaxf(wmax, a.d.w[(size_t)c * K + l]);
        int e;
        frexpf(wmax, &e);                      // wmax < 2^e, so 8 K w 2^(55-e) < 2^62
        for (int l = 0; l < K; ++l)
            qw[l] = __double2ull_rn(ldexp((double)a.d.w[(size_t)c * K + l], 55 - e));
        bm[0][0] = 0;
        bc[0][0] = 0;
    }
    __syncthreads();

    int iS = 0, s = 1;
    for (int l = 0; l < K; ++l) {
        const uint64_t q = qw[l];
        const uint64_t d1 = 1ull << (4 * l);
        int ix = iS, nx = s;
        for (int step = 0; step < 4; ++step) {
            // steps 0..2: X + 2^step * delta; step 3: S + 8 * delta
            const uint64_t mul = step < 3 ? (1ull << step) : 8ull;
            const int ib = step < 3 ? ix : iS;
            const int nb = step < 3 ? nx : s;
            const uint64_t dm = mul * q, dc = mul * d1;
            const bool skip = nx >= n && key_less(bm[ix][n - 1], bc[ix][n - 1], bm[ib][0] + dm, bc[ib][0] + dc);
            if (skip) continue;
            const int io = (ix == iS) ? (iS + 1) % 3 : 3 - ix - iS;
            const int nout = min(nx + nb, n);
            merge_shift(bm[ix], bc[ix], nx, bm[ib], bc[ib], nb, dm, dc, bm[io], bc[io], nout, tid, T);
            __syncthreads();
            ix = io;
            nx = nout;
        }
        iS = ix;
        s = nx;
    }

    const uint64_t* Sc = bc[iS];
    for (int i = tid; i < n; i += T) out[i] = (i < s) ? Sc[i] : 0;
    const int warp = tid >> 5, lane = tid & 31;
    for (int ch = warp; ch < a.nch; ch += T >> 5) {
        const int i = ch * 32 + lane;
        const uint64_t code = (i < s) ? Sc[i] : 0;
        uint64_t mq = 0;
        for (int l = 0; l < K; ++l) {
            const unsigned dgt = (unsigned)((code >> (4 * l)) & 15u);
            mq |= (uint64_t)__reduce_max_sync(kFull, dgt) << (4 * l);
        }
        if (lane == 0) mqo[ch] = mq;
    }
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
    const size_t shbytes = (size_t)6 * p->n_paths * sizeof(uint64_t);
    static size_t attr_set = 0;
    if (shbytes > 40 * 1024 && shbytes > attr_set) {
        cudaError_t e = cudaFuncSetAttribute(pathsel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)shbytes);
        if (e != cudaSuccess) return e;
        attr_set = shbytes;
    }
    int T = 32;
    if (p->n_paths > 64) T = 128;
    if (p->n_paths > 256) T = 256;
    pathsel_kernel<<<C, T, shbytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vp
