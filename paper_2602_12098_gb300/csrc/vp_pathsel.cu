// Most-promising-path selection (Section III-A-2): the n position vectors p
// with the smallest Metric of Promise M(p) = sum_l w_l (p_l - 1) (Eq. mop),
// by breadth-first K-Best over the levels.
//
// One block per channel. The weights are turned into integers
// q_l = round(w_l / max_l w_l * 2^40), so every partial metric is an exact
// uint64 sum and the order (metric, code) is a strict total order. With it,
// K-Best keeps exactly the n smallest vectors, whatever the level order.
//
// Level step: the survivors S (sorted) spawn children S + k*q_l, k = 1..8.
// Only children below the current n-th survivor can enter. Their ranks among
// themselves come from binary searches in the 8 shifted copies of S (each
// copy is sorted), and one merge-path pass merges them into S.
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

// First `nout` outputs of the merge of sorted A[0..na) and B[0..nb) into O.
__device__ void merge_path(const uint64_t* Am, const uint64_t* Ac, int na,
                           const uint64_t* Bm, const uint64_t* Bc, int nb,
                           uint64_t* Om, uint64_t* Oc, int nout, int tid, int T)
{
    const int per = (nout + T - 1) / T;
    const int d0 = min(tid * per, nout);
    const int d1 = min(d0 + per, nout);
    if (d0 >= d1) return;
    int lo = max(0, d0 - nb), hi = min(d0, na);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key_less(Am[mid], Ac[mid], Bm[d0 - mid - 1], Bc[d0 - mid - 1])) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = d0 - lo;
    for (int d = d0; d < d1; ++d) {
        const bool takeA = (j >= nb) || (i < na && key_less(Am[i], Ac[i], Bm[j], Bc[j]));
        if (takeA) { Om[d] = Am[i]; Oc[d] = Ac[i]; ++i; }
        else { Om[d] = Bm[j]; Oc[d] = Bc[j]; ++j; }
    }
}

__global__ void pathsel_kernel(PathArgs a)
{
    extern __shared__ uint64_t shm[];
    __shared__ uint64_t qw[kMaxK];
    __shared__ int cnt[9];
    __shared__ int pre[10];
    const int n = a.n, K = a.K, T = blockDim.x, tid = threadIdx.x;
    uint64_t* Sm = shm;
    uint64_t* Sc = Sm + n;
    uint64_t* Em = Sc + n;
    uint64_t* Ec = Em + n;
    uint64_t* Nm = Ec + n;
    uint64_t* Nc = Nm + n;
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
        for (int l = 0; l < K; ++l)
            qw[l] = __double2ull_rn((double)a.d.w[(size_t)c * K + l] / (double)wmax * 1099511627776.0);
        Sm[0] = 0;
        Sc[0] = 0;
    }
    __syncthreads();

    int s = 1;
    for (int l = 0; l < K; ++l) {
        const uint64_t q = qw[l];
        const int sh4 = 4 * l;
        if (tid >= 1 && tid <= 8) {
            const int k = tid;
            int ck;
            if (s < n) {
                ck = s;                                  // every child is a candidate
            } else {
                const uint64_t lim = Sm[n - 1];
                const uint64_t kq = (uint64_t)k * q;
                if (kq >= lim) {
                    ck = 0;
                } else {                                 // #{i : Sm[i] + kq < lim}
                    const uint64_t th = lim - kq;
                    int lo = 0, hi = n;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (Sm[mid] < th) lo = mid + 1; else hi = mid;
                    }
                    ck = lo;
                }
            }
            cnt[k] = ck;
        }
        __syncthreads();
        if (tid == 0) {
            pre[1] = 0;
            for (int k = 1; k <= 8; ++k) pre[k + 1] = pre[k] + cnt[k];
        }
        __syncthreads();
        const int E = pre[9];
        if (E == 0) continue;                            // no child enters: digit 0 everywhere

        for (int e = tid; e < E; e += T) {
            int k = 1;
            while (e >= pre[k + 1]) ++k;
            const int i = e - pre[k];
            const uint64_t em = Sm[i] + (uint64_t)k * q;
            const uint64_t ec = Sc[i];
            int rank = i;
            for (int k2 = 1; k2 <= 8; ++k2) {
                const int len = cnt[k2];
                if (k2 == k || len == 0) continue;
                const uint64_t sq = (uint64_t)k2 * q;
                int lo = 0, hi = len;
                while (lo < hi) {                        // count children (j, k2) before (i, k)
                    const int mid = (lo + hi) >> 1;
                    const uint64_t mm = Sm[mid] + sq;
                    const bool lt = mm < em || (mm == em && (k2 < k || (k2 == k && Sc[mid] < ec)));
                    if (lt) lo = mid + 1; else hi = mid;
                }
                rank += lo;
            }
            if (rank < n) {
                Em[rank] = em;
                Ec[rank] = ec | ((uint64_t)k << sh4);
            }
        }
        __syncthreads();
        const int ne = E < n ? E : n;
        const int outn = (s + ne) < n ? (s + ne) : n;
        merge_path(Sm, Sc, s, Em, Ec, ne, Nm, Nc, outn, tid, T);
        __syncthreads();
        uint64_t* t0 = Sm; Sm = Nm; Nm = t0;
        uint64_t* t1 = Sc; Sc = Nc; Nc = t1;
        s = outn;
    }

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
