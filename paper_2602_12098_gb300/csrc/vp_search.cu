// Parallel post-processing of Alg. 2: for each data vector, every candidate
// path descends the tree from level K (Section II-B PED recursion) and the
// best candidate gives l, gamma and the precoded vector x.
//
// Mapping: one block per channel (its factor, paths and P staged in shared
// memory), one warp per data vector, one lane per candidate path (32 paths
// per pass). Per lane the residuals r_m (m below the current level) live in
// registers in units of tau (r' = r / tau is the effective point s_hat_l of
// Eq. (17)); choosing t_l at level l updates them column-wise,
//   r'_m -= U~_ml t_l,  m < l,
// with two packed FP32 FMAs per complex term, and t_l is the p_l-th nearest point of
// {-1,0,1}+j{-1,0,1} to r'_l (DEMAP), ties to the smaller (Re t, Im t).
// The PED grows by w_l tau^2 |r'_l - t_l|^2.
// The zero perturbation is candidate 0; the warp's (PED, index) minimum wins
// (ties: lower index). x = P (s + tau l) / sqrt(gamma) with gamma = ||P u||^2,
// the product P u formed with exact products and compensated sums.
#include "vp_internal.cuh"

namespace vp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct SearchArgs {
    const uint8_t* sym;
    const int32_t* off;
    int S, n_vec, C;
    float2* x;
    int8_t* l;
    float* gamma;
    int K, M, n, nch, m_qam;
    float tau, inv_tau;
    DeviceState d;
    // batch mode (probs != null): block i works on problem ids[i] of the table;
    // KM, NP give the shared-memory layout (the launch's largest K*M and n)
    const BatchProblem* probs;
    const int* ids;
    int KM, NP;
};

// DEMAP selection: the q-th (0-based) nearest point t of {-1,0,1}+j{-1,0,1}
// to the effective point c = (x, y), ties to the smaller alphabet index
// 3(tr+1) + (ti+1), i.e. to the lexicographically smaller (tr, ti).
//
// Ties. Measuring from c - (eps_x, eps_y) with eps_x >> eps_y > 0 tiny orders
// equal-distance points exactly by (tr, ti), so every comparison below is a
// plain '<' on the shifted point. Exact ties only occur for dyadic centres
// (|x|, |y| < 1/2, e.g. s/tau at the first level), where 2^-23 and 2^-25 are
// representable shifts far below the spacing of distinct distances.
//
// Per axis (region r = [x > -1/2] + [x > 0] + [x > 1/2]) the points in
// increasing distance are n_0, n_1, n_2 (kNTab), and their squared distances
// exceed that of n_0 by 0, D1 = |1 - 2|x||, D2 = max(1 + 2|x|, 4|x|). The 9
// points form a 3x3 table of sums Dx_i + Dy_j (cell (i, j) = (n_i(x), n_j(y))).
// Against the origin cell the 8 others are
//   A=(1,0): D1x  B=(0,1): D1y  C=(2,0): D2x  D=(0,2): D2y  E=(1,1): D1x+D1y
//   F=(1,2): D1x+D2y  G=(2,1): D2x+D1y  H=(2,2): largest,
// and every pair not ordered by the table's structure is one of
//   f0 A<B, f1 C<B, f2 A<D, f3 C<D, f4 E<C, f5 E<D, f6 F<C, f7 G<D, f8 F<G,
// so the rank of each cell is a short sum of these bits.
constexpr float kEpsX = 0x1p-23f;
constexpr float kEpsY = 0x1p-25f;
// (n_i(r) + 1) in 2 bits at bit 2(3r + i): r0 (-1,0,1), r1 (0,-1,1), r2 (0,1,-1), r3 (1,0,-1)
constexpr uint32_t kNTab = 0x189864u;

__device__ __forceinline__ int region4(float x) { return (x > -0.5f) + (x > 0.f) + (x > 0.5f); }
__device__ __forceinline__ int npt(int r, int i) { return (int)((kNTab >> (2 * (3 * r + i))) & 3u) - 1; }
__device__ __forceinline__ float gap1(float x) { return fabsf(fmaf(-2.f, fabsf(x), 1.f)); }
__device__ __forceinline__ float gap2(float x) { return fmaxf(fmaf(2.f, fabsf(x), 1.f), 4.f * fabsf(x)); }

// cell (ci, cj) of 0-based rank q >= 1 from the nine comparisons
__device__ __forceinline__ void rank_cell(float D1x, float D2x, float D1y, float D2y, int q, int& ci, int& cj)
{
    const float vE = D1x + D1y, vF = D1x + D2y, vG = D2x + D1y;
    const int f0 = D1x < D1y, f1 = D2x < D1y, f2 = D1x < D2y, f3 = D2x < D2y, f4 = vE < D2x;
    const int f5 = vE < D2y, f6 = vF < D2x, f7 = vG < D2y, f8 = vF < vG;
    const int k = q - 1;
    const int rA = 2 - f0 - f2, rB = f0 + f1, rC = 3 - f1 - f3 + f4 + f6, rD = 1 + f2 + f3 + f5 + f7;
    const int rE = 4 - f4 - f5, rF = 6 - f6 - f8, rG = 5 - f7 + f8;
    ci = 2; cj = 2;                                                   // H
    if (rG == k) { ci = 2; cj = 1; }
    if (rF == k) { ci = 1; cj = 2; }
    if (rE == k) { ci = 1; cj = 1; }
    if (rD == k) { ci = 0; cj = 2; }
    if (rC == k) { ci = 2; cj = 0; }
    if (rB == k) { ci = 0; cj = 1; }
    if (rA == k) { ci = 1; cj = 0; }
}

// t for rank q at effective point (cx, cy); `mq` = the warp's largest q at this
// level (uniform) picks the cheapest branch that is exact for every lane.
__device__ __forceinline__ void select_point(float cx, float cy, int q, int mq, int& tr, int& ti)
{
    const float px = cx - kEpsX, py = cy - kEpsY;
    if (mq == 0) {
        tr = (px > 0.5f) - (px <= -0.5f);
        ti = (py > 0.5f) - (py <= -0.5f);
        return;
    }
    if (mq == 1) {                                                    // rank 0 or 1: round, or step to A or B
        const bool f0 = gap1(px) < gap1(py);
        const int ci = (q == 1 && f0) ? 1 : 0, cj = (q == 1 && !f0) ? 1 : 0;
        tr = npt(region4(px), ci);
        ti = npt(region4(py), cj);
        return;
    }
    const float D1x = gap1(px), D2x = gap2(px), D1y = gap1(py), D2y = gap2(py);
    int ci, cj;
    if (mq == 2) {
        const bool f0 = D1x < D1y;                                    // rank 1: A or B
        const bool g = f0 ? (D1y < D2x) : (D1x < D2y);                // rank 2: the other, or C / D
        const int c2i = f0 ? (g ? 0 : 2) : (g ? 1 : 0);
        const int c2j = f0 ? (g ? 1 : 0) : (g ? 0 : 2);
        ci = q == 0 ? 0 : (q == 1 ? (f0 ? 1 : 0) : c2i);
        cj = q == 0 ? 0 : (q == 1 ? (f0 ? 0 : 1) : c2j);
    } else {
        rank_cell(D1x, D2x, D1y, D2y, q, ci, cj);
        if (q == 0) { ci = 0; cj = 0; }
    }
    tr = npt(region4(px), ci);
    ti = npt(region4(py), cj);
}

template <int KT, bool BATCH>
__global__ void __launch_bounds__(224, 4) search_kernel(SearchArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int NW = blockDim.x >> 5;
    const int c = blockIdx.x;
    int K, M, n, nch, m_qam;
    float tau, inv_tau;
    int v0, v1;
    ChanState cs;
    const uint8_t* sym;
    float2* xo;
    int8_t* lo;
    float* go;
    if (BATCH) {
        const BatchProblem& p = a.probs[a.ids[c]];
        K = p.K; M = p.M; n = p.n; nch = n_chunks(p.n); m_qam = p.m_qam;
        tau = p.tau; inv_tau = 1.0f / p.tau;
        v0 = 0; v1 = p.S;
        cs = chan_state(p);
        sym = p.sym; xo = p.x; lo = p.l; go = p.gamma;
        if (threadIdx.x == 0 && p.status) p.status[0] = p.st[0];
    } else {
        K = a.K; M = a.M; n = a.n; nch = a.nch; m_qam = a.m_qam;
        tau = a.tau; inv_tau = a.inv_tau;
        if (a.off) {
            v0 = min(max(a.off[c], 0), a.n_vec);
            v1 = min(max(a.off[c + 1], v0), a.n_vec);
        } else {
            v0 = c * a.S;
            v1 = v0 + a.S;
        }
        cs = chan_state(a.d, (size_t)c, K, M, n);
        sym = a.sym; xo = a.x; lo = a.l; go = a.gamma;
    }
    const int KM = BATCH ? a.KM : K * M, NP = BATCH ? a.NP : n;
    float4* utp = reinterpret_cast<float4*>(smraw);                 // [KT][KT]
    float2* utc = reinterpret_cast<float2*>(utp + KT * KT);        // [KT][KT]
    float2* pt = utc + KT * KT;                                    // [K][M] leading part of P^T
    float2* ptl = pt + KM;                                         // [K][M] trailing part
    float2* bvec = ptl + KM;                                       // [NW][KT]
    uint64_t* paths = reinterpret_cast<uint64_t*>(bvec + NW * KT); // [n]
    uint64_t* maxq = paths + NP;                                   // [nch]
    float* wv = reinterpret_cast<float*>(maxq + n_chunks(NP));     // [KT]
    int* ulv = reinterpret_cast<int*>(wv + KT);                    // [KT]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (cs.st[0] & (VP_CH_NONFINITE | VP_CH_SINGULAR)) {
        for (int v = v0 + warp; v < v1; v += NW) {
            if (lane < M) xo[(size_t)v * M + lane] = make_float2(0.f, 0.f);
            if (lane < K) {
                lo[((size_t)v * K + lane) * 2] = 0;
                lo[((size_t)v * K + lane) * 2 + 1] = 0;
            }
            if (lane == 0) go[v] = 0.f;
        }
        return;
    }

    for (int i = threadIdx.x; i < KT * KT; i += blockDim.x) {
        const int r = i / KT, q = i % KT;
        const bool in = r < K && q < K;
        utp[i] = in ? cs.utp[r * K + q] : make_float4(0.f, 0.f, 0.f, 0.f);
        utc[i] = in ? cs.utc[r * K + q] : make_float2(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < K * M; i += blockDim.x) {
        pt[i] = cs.pt[i];
        ptl[i] = cs.ptlo[i];
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) paths[i] = cs.paths[i];
    for (int i = threadIdx.x; i < nch; i += blockDim.x) maxq[i] = cs.maxq[i];
    for (int i = threadIdx.x; i < KT; i += blockDim.x) {
        wv[i] = i < K ? cs.w[i] * tau * tau : 0.f;   // w_l tau^2
        ulv[i] = i < K ? (int)cs.ul[i] : 0;
    }
    __syncthreads();

    float2* bw = bvec + warp * KT;
    for (int v = v0 + warp; v < v1; v += NW) {
        // symbols in level order (lane k <-> level k) and b_k = s_k + sum_{m>k} U~_km s_m
        float2 s = make_float2(0.f, 0.f);
        if (lane < K) s = qam_point((int)sym[(size_t)v * K + ulv[lane]], m_qam);
        float2 b = s;
        for (int m = 1; m < K; ++m) {
            const float2 sm = make_float2(__shfl_sync(kFull, s.x, m), __shfl_sync(kFull, s.y, m));
            if (lane < m) b = cfma(utc[m * KT + lane], sm, b);
        }
        // residuals are kept in units of tau: r' = r / tau is the effective point of Eq. (17)
        b = make_float2(b.x * inv_tau, b.y * inv_tau);
        if (lane < KT) bw[lane] = (lane < K) ? b : make_float2(0.f, 0.f);
        float g0 = (lane < K) ? wv[lane] * cabs2(b) : 0.f;     // zero candidate: ||U s||^2
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) g0 += __shfl_xor_sync(kFull, g0, o);
        __syncwarp(kFull);

        float bp = INFINITY;
        int bi = 0x7fffffff;
        uint32_t blc0 = 0, blc1 = 0;
        for (int ch = 0; ch < nch; ++ch) {
            const int jp = ch * 32 + lane;
            const bool vld = jp < n;
            const uint64_t code = vld ? paths[jp] : 0ull;
            const uint32_t cw0 = (uint32_t)code, cw1 = (uint32_t)(code >> 32);
            const uint64_t mq = maxq[ch];
            const uint32_t mq0 = (uint32_t)mq, mq1 = (uint32_t)(mq >> 32);
            float2 r[KT];
#pragma unroll
            for (int m = 0; m < KT; ++m) r[m] = bw[m];
            float ped = 0.f;
            uint32_t lc0 = 0, lc1 = 0;
#pragma unroll
            for (int lv = KT - 1; lv >= 0; --lv) {
                if (lv < K) {
                    const int sh = 4 * (lv & 7);
                    const int q = (int)(((lv < 8) ? cw0 : cw1) >> sh) & 15;
                    const int mql = (int)(((lv < 8) ? mq0 : mq1) >> sh) & 15;
                    const float cx = r[lv].x, cy = r[lv].y;
                    int tr, ti;
                    select_point(cx, cy, q, mql, tr, ti);
                    const float ftr = (float)tr, fti = (float)ti;
                    const float dx = cx - ftr, dy = cy - fti;
                    ped = fmaf(wv[lv], fmaf(dx, dx, dy * dy), ped);
                    const uint32_t dig = (uint32_t)((tr + 1) | ((ti + 1) << 2)) << sh;
                    if (lv < 8) lc0 |= dig; else lc1 |= dig;
                    if (lv > 0) {
                        const float2 c1 = make_float2(-ftr, -ftr);
                        const float2 c2 = make_float2(fti, -fti);
#pragma unroll
                        for (int m = 0; m < lv; ++m) {
                            const float4 u = utp[m * KT + lv];
                            r[m] = __ffma2_rn(make_float2(u.x, u.y), c1, r[m]);
                            r[m] = __ffma2_rn(make_float2(u.z, u.w), c2, r[m]);
                        }
                    }
                }
            }
            if (vld && ped < bp) { bp = ped; bi = jp + 1; blc0 = lc0; blc1 = lc1; }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const float obp = __shfl_xor_sync(kFull, bp, o);
            const int obi = __shfl_xor_sync(kFull, bi, o);
            if (obp < bp || (obp == bp && obi < bi)) { bp = obp; bi = obi; }
        }
        const bool zero_wins = !(bp < g0);
        const int src = zero_wins ? 0 : ((bi - 1) & 31);
        uint32_t w0 = __shfl_sync(kFull, blc0, src), w1 = __shfl_sync(kFull, blc1, src);
        if (zero_wins) { w0 = 0x55555555u; w1 = 0x55555555u; }

        // l (user order) and u = s + tau l = s - tau t in level order
        float2 u = make_float2(0.f, 0.f);
        if (lane < K) {
            const int nib = (int)(((lane < 8 ? w0 : w1) >> (4 * (lane & 7))) & 15u);
            const int tr = (nib & 3) - 1, ti = (nib >> 2) - 1;
            u = make_float2(s.x - (float)tr * tau, s.y - (float)ti * tau);
            const int usr = ulv[lane];
            lo[((size_t)v * K + usr) * 2] = (int8_t)(-tr);
            lo[((size_t)v * K + usr) * 2 + 1] = (int8_t)(-ti);
        }
        // y = P u with P = pt + ptl: exact products and compensated sums (u holds
        // small integers, so P u keeps ~48 bits before the final rounding)
        float yr = 0.f, yre = 0.f, yi = 0.f, yie = 0.f;
        for (int lv = 0; lv < K; ++lv) {
            const float ur = __shfl_sync(kFull, u.x, lv), ui = __shfl_sync(kFull, u.y, lv);
            if (lane < M) {
                const int idx = ulv[lv] * M + lane;
                const float2 ph = pt[idx], pl = ptl[idx];
                dot2_acc(ph.x, ur, yr, yre);
                dot2_acc(-ph.y, ui, yr, yre);
                dot2_acc(ph.x, ui, yi, yie);
                dot2_acc(ph.y, ur, yi, yie);
                yre = fmaf(pl.x, ur, fmaf(-pl.y, ui, yre));
                yie = fmaf(pl.x, ui, fmaf(pl.y, ur, yie));
            }
        }
        const float2 y = make_float2(__fadd_rn(yr, yre), __fadd_rn(yi, yie));
        float g = (lane < M) ? cabs2(y) : 0.f;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) g += __shfl_xor_sync(kFull, g, o);
        const float rs = __frsqrt_rn(g);
        if (lane < M) xo[(size_t)v * M + lane] = make_float2(y.x * rs, y.y * rs);
        if (lane == 0) go[v] = g;
        __syncwarp(kFull);
    }
}

template <int KT>
cudaError_t launch_kt(const SearchArgs& a, int C, int threads, cudaStream_t s)
{
    const int NW = threads / 32;
    const int KM = a.probs ? a.KM : a.K * a.M, NP = a.probs ? a.NP : a.n;
    const size_t sh = sizeof(float4) * KT * KT + sizeof(float2) * KT * KT + 2 * sizeof(float2) * KM +
                      sizeof(float2) * NW * KT + sizeof(uint64_t) * (NP + n_chunks(NP)) + sizeof(float) * KT +
                      sizeof(int) * KT;
    if (a.probs) {
        static size_t attr = 0;
        if (sh > 40 * 1024 && sh > attr) {
            cudaError_t e = cudaFuncSetAttribute(search_kernel<KT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
            if (e != cudaSuccess) return e;
            attr = sh;
        }
        search_kernel<KT, true><<<C, threads, sh, s>>>(a);
    } else {
        static size_t attr = 0;
        if (sh > 40 * 1024 && sh > attr) {
            cudaError_t e = cudaFuncSetAttribute(search_kernel<KT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
            if (e != cudaSuccess) return e;
            attr = sh;
        }
        search_kernel<KT, false><<<C, threads, sh, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_search(const vp_plan* p, const uint8_t* sym, int S, const int32_t* vec_off, int n_vec,
                          float2* x, int8_t* l, float* gamma, cudaStream_t s)
{
    SearchArgs a;
    a.sym = sym;
    a.off = vec_off;
    a.S = S;
    a.n_vec = n_vec;
    a.C = p->C;
    a.x = x;
    a.l = l;
    a.gamma = gamma;
    a.K = p->K;
    a.M = p->M;
    a.n = p->n_paths;
    a.nch = n_chunks(p->n_paths);
    int m = 1;
    while (m * m < p->qam) ++m;
    a.m_qam = m;
    a.tau = p->tau;
    a.inv_tau = 1.0f / p->tau;
    a.d = p->d;
    a.probs = nullptr;
    a.ids = nullptr;
    a.KM = 0;
    a.NP = 0;
    // warps per block (<= 7, the register budget of 4 blocks per SM): a
    // divisor-friendly count of the vectors per channel
    const int per = vec_off ? (n_vec + p->C - 1) / p->C : S;
    int nw = 7;
    if (per <= 7) nw = per < 1 ? 1 : per;
    else if (per % 7 != 0 && per % 6 == 0) nw = 6;
    const int threads = nw * 32;
    const int K = p->K;
    if (K <= 2) return launch_kt<2>(a, p->C, threads, s);
    if (K <= 4) return launch_kt<4>(a, p->C, threads, s);
    if (K <= 8) return launch_kt<8>(a, p->C, threads, s);
    if (K <= 12) return launch_kt<12>(a, p->C, threads, s);
    return launch_kt<16>(a, p->C, threads, s);
}

cudaError_t launch_search_batch(const BatchProblem* probs, const int* ids, int count, int KT, int km_max,
                                int n_max, int s_max, cudaStream_t s)
{
    SearchArgs a = SearchArgs();
    a.probs = probs;
    a.ids = ids;
    a.C = count;
    a.KM = km_max;
    a.NP = n_max;
    int nw = 7;
    if (s_max <= 7) nw = s_max < 1 ? 1 : s_max;
    else if (s_max % 7 != 0 && s_max % 6 == 0) nw = 6;
    const int threads = nw * 32;
    switch (KT) {
    case 2: return launch_kt<2>(a, count, threads, s);
    case 4: return launch_kt<4>(a, count, threads, s);
    case 8: return launch_kt<8>(a, count, threads, s);
    case 12: return launch_kt<12>(a, count, threads, s);
    case 16: return launch_kt<16>(a, count, threads, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace vp
