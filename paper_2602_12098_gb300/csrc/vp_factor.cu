// Channel factorisation: (H H^H)^-1 = U^H U with U = R^-1 upper triangular,
// in the min-norm-first sorted order of Alg. 1 (Section III-A-1) with the
// index reversal of Section IV-B (first-picked user at the last level).
//
// factor32_kernel: FP32 column-pivoted Householder QR of A = H^H (equivalent
//   to the sorted RQ of H: H_perm = R Q). The pivot at each step is the
//   remaining user with the smallest residual norm, which is Alg. 1's rule.
//   Orthogonal reflections keep the error near FP32 rounding (the Gram
//   matrix route squares the condition number). One half-warp per channel,
//   lane j holds column j of A in registers.
// factor64_kernel: channels whose estimated cond(H H^H) (power iteration on R
//   and U) passes the plan threshold are redone with FP64: the Gram matrix
//   (compensated FP32 sums, exact for FP32 input), pivoted reverse Cholesky
//   with the same min-pivot rule, U = R^-1 and one Newton step
//   U <- U (2I - R U) (the residual I - R U in FP64, the small correction
//   U (I - R U) in FP32), then P = H^H U^H U as a hi/lo FP32 pair.
//
// Outputs per channel (level order unless noted): U~ = U_lk / U_ll (unit
// upper), w_l = U_ll^2, the user of each level, and P^T in user order.
#include "vp_internal.cuh"

namespace vp {
namespace {

constexpr int kLanes = 16;        // lanes per channel
constexpr int kChPerBlock32 = 4;  // FP32 kernel: 64 threads
constexpr unsigned kFull = 0xffffffffu;

struct FactorArgs {
    const float2* H;
    int C, K, M, n;
    int Mp;          // rows of P kept (M, or M + K with lambda > 0)
    float lambda;    // Tikhonov parameter (plan layout only; the batch table has lambda = 0)
    float kappa_thr;
    DeviceState d;
    float2* U_out;
    float2* P_out;
    uint8_t* ul_out;
    // batch mode (probs != null): channel i of the launch is problem ids[i] of
    // the table; its state lives in the workspace, no U / P / ul outputs
    const BatchProblem* probs;
    const int* ids;
    const int* nflag_in;   // FP64 list (batch: in the workspace; plain: d.nflag / d.flags)
    int* nflag;
    int* flags;
};

// Inputs and outputs of one channel.
struct FChan {
    const float2* H;   // [K][M]
    ChanState s;
    float2* U_out;     // [K][K] or null
    float2* P_out;     // [M][K] or null
    uint8_t* ul_out;   // [K] or null
};

__device__ __forceinline__ FChan fchan(const FactorArgs& a, int c, int K, int M)
{
    FChan f;
    if (a.probs) {
        const BatchProblem& p = a.probs[c];
        f.H = p.H;
        f.s = chan_state(p);
        f.U_out = nullptr;
        f.P_out = nullptr;
        f.ul_out = nullptr;
    } else {
        f.H = a.H + (size_t)c * K * M;
        f.s = chan_state(a.d, (size_t)c, K, a.Mp, a.n);
        f.U_out = a.U_out ? a.U_out + (size_t)c * K * K : nullptr;
        f.P_out = a.P_out ? a.P_out + (size_t)c * M * K : nullptr;
        f.ul_out = a.ul_out ? a.ul_out + (size_t)c * K : nullptr;
    }
    return f;
}

constexpr int kRow32 = kMaxK + 1;   // padded row length of the triangular factors in shared memory

template <int MT>
struct Smem32 {
    float2 refl[kMaxK][MT];    // Householder vector of step t (zero above row t)
    float2 ru[kMaxK][kMaxK];   // ru[t][j]: entry of row t of R' in the column of user j
    float2 rl[kMaxK][kRow32];  // R, level order (rows padded: lane j reading row j hits distinct banks)
    float2 uu[kMaxK][kRow32];  // U = R^-1, level order (padded likewise)
    float2 phi[kMaxK];         // phase of R'_tt
    float beta[kMaxK];
    float rdiag[kMaxK];        // |R'_tt|
    int piv[kMaxK];            // user pivoted at step t
};

__device__ __forceinline__ void write_channel_outputs_zero(const FChan& f, int K, int M, int Mp, int j)
{
    if (j < K) {
        for (int k = 0; k < K; ++k) {
            f.s.utp[j * K + k] = make_float4(0.f, 0.f, 0.f, 0.f);
            f.s.utc[j * K + k] = make_float2(0.f, 0.f);
            if (f.U_out) f.U_out[j * K + k] = make_float2(0.f, 0.f);
        }
        for (int m = 0; m < Mp; ++m) {
            f.s.pt[j * Mp + m] = make_float2(0.f, 0.f);
            f.s.ptlo[j * Mp + m] = make_float2(0.f, 0.f);
            if (f.P_out && m < M) f.P_out[m * K + j] = make_float2(0.f, 0.f);
        }
        f.s.w[j] = 0.f;
        f.s.ul[j] = (uint8_t)j;
        if (f.ul_out) f.ul_out[j] = (uint8_t)j;
    }
}

// sigma_max(A)^2 and sigma_max(B)^2 of two upper-triangular K x K matrices
// held in shared memory, by power iteration on A^H A and B^H B (lower bounds
// that converge from below). The two iterations are independent and run
// interleaved, each with its own operations in its own order. Every lane of
// the warp calls it; lane j < K holds component j of the iterates; K <= KT.
// The iterates are exchanged through the channel's scratch rows `xv`
// (rows 0-3: v_A, v_B, w_A, w_B), read back as shared-memory broadcasts.
template <int KT>
__device__ void power_sigma2_pair(const float2 (*A)[kRow32], const float2 (*B)[kRow32], float2 (*xv)[kMaxK], int K,
                                  int j, float& la, float& lb)
{
    const bool act = j < K;
    float2 va = make_float2(act ? 1.f + 0.0625f * (float)j : 0.f, 0.f), vb = va;
    la = 0.f;
    lb = 0.f;
    for (int it = 0; it < 6; ++it) {
        if (act) {
            xv[0][j] = va;
            xv[1][j] = vb;
        }
        __syncwarp(kFull);
        float2 wa = make_float2(0.f, 0.f), wb = wa;              // w = A v
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            if (k < K && act && k >= j) {
                wa = cfma(A[j][k], xv[0][k], wa);
                wb = cfma(B[j][k], xv[1][k], wb);
            }
        }
        if (act) {
            xv[2][j] = wa;
            xv[3][j] = wb;
        }
        __syncwarp(kFull);
        float2 za = make_float2(0.f, 0.f), zb = za;              // z = A^H w
#pragma unroll
        for (int i = 0; i < KT; ++i) {
            if (i < K && act && i <= j) {
                za = cfma(make_float2(A[i][j].x, -A[i][j].y), xv[2][i], za);
                zb = cfma(make_float2(B[i][j].x, -B[i][j].y), xv[3][i], zb);
            }
        }
        float nwa = cabs2(wa), nva = cabs2(va), nza = cabs2(za);
        float nwb = cabs2(wb), nvb = cabs2(vb), nzb = cabs2(zb);
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) {
            nwa += __shfl_xor_sync(kFull, nwa, off, kLanes);
            nva += __shfl_xor_sync(kFull, nva, off, kLanes);
            nza += __shfl_xor_sync(kFull, nza, off, kLanes);
            nwb += __shfl_xor_sync(kFull, nwb, off, kLanes);
            nvb += __shfl_xor_sync(kFull, nvb, off, kLanes);
            nzb += __shfl_xor_sync(kFull, nzb, off, kLanes);
        }
        la = nwa / nva;                                          // Rayleigh quotients
        lb = nwb / nvb;
        const float sa = rsqrtf(nza), sb = rsqrtf(nzb);
        va = make_float2(za.x * sa, za.y * sa);
        vb = make_float2(zb.x * sb, zb.y * sb);
    }
}

// MT: rows of A (M, or M + K with lambda > 0) rounded up; KT >= K: the
// unrolled step loops stop at KT, so small K runs a small kernel body.
template <int MT, int KT>
__global__ void __launch_bounds__(kLanes * kChPerBlock32) factor32_kernel(FactorArgs a)
{
    __shared__ Smem32<MT> smem[kChPerBlock32];
    pdl_wait();
    const int slot = threadIdx.x / kLanes;
    const int j = threadIdx.x % kLanes;
    const int hw = (threadIdx.x >> 4) & 1;                 // half of the warp
    const unsigned hmask = 0xFFFFu << (16 * hw);
    const int ci = blockIdx.x * kChPerBlock32 + slot;
    const bool valid = ci < a.C;
    const int K = a.K, M = a.M, Mp = a.Mp;
    const int c = valid ? (a.ids ? a.ids[ci] : ci) : 0;   // channel (plain) or table index (batch)
    const FChan f = fchan(a, c, K, M);
    const bool act = j < K;
    Smem32<MT>& sm = smem[slot];

    // column j of A = H^H (row j of H, read as 16-byte pairs of entries when
    // the rows are 16-byte aligned)
    float2 av[MT];
    bool finite = true;
    const bool v4 = ((M & 1) == 0) && ((reinterpret_cast<uintptr_t>(f.H) & 15u) == 0u);
#pragma unroll
    for (int m = 0; m < MT; m += 2) {
        float2 h0 = make_float2(0.f, 0.f), h1 = h0;
        if (valid && act && m < M) {
            if (v4) {
                const float4 q = *reinterpret_cast<const float4*>(f.H + j * M + m);
                h0 = make_float2(q.x, q.y);
                h1 = make_float2(q.z, q.w);
            } else {
                h0 = f.H[j * M + m];
                if (m + 1 < M) h1 = f.H[j * M + m + 1];
            }
        }
        finite = finite && isfinite(h0.x) && isfinite(h0.y) && isfinite(h1.x) && isfinite(h1.y);
        av[m] = make_float2(h0.x, -h0.y);
        if (m + 1 < MT) av[m + 1] = make_float2(h1.x, -h1.y);
        if (act && m == M + j && a.lambda > 0.f) av[m] = make_float2(a.lambda, 0.f);   // Hbar = [H lambda*I]
        if (act && m + 1 == M + j && a.lambda > 0.f && m + 1 < MT) av[m + 1] = make_float2(a.lambda, 0.f);
    }
    const bool nonfinite = (__ballot_sync(kFull, !finite) & hmask) != 0u;
    if (nonfinite) {
#pragma unroll
        for (int m = 0; m < MT; ++m) av[m] = make_float2(0.f, 0.f);
    }

    bool placed = !act;
    bool degenerate = false;
#pragma unroll
    for (int t = 0; t < KT; ++t) {
        if (t < K) {
            float nu = 0.f;
#pragma unroll
            for (int m = t; m < MT; ++m) nu = fmaf(av[m].x, av[m].x, fmaf(av[m].y, av[m].y, nu));
            float key = placed ? INFINITY : nu;
            int kj = j;
#pragma unroll
            for (int off = 8; off >= 1; off >>= 1) {
                const float ok = __shfl_xor_sync(kFull, key, off, kLanes);
                const int oj = __shfl_xor_sync(kFull, kj, off, kLanes);
                if (ok < key || (ok == key && oj < kj)) { key = ok; kj = oj; }
            }
            const int p = kj;

            float2 vv[MT];
#pragma unroll
            for (int m = 0; m < MT; ++m) vv[m] = make_float2(0.f, 0.f);
            float beta = 0.f;
            if (j == p) {
                const float2 x0 = av[t];
                const float amag = sqrtf(nu);
                const float x0abs = sqrtf(cabs2(x0));
                const float2 ph = (x0abs > 0.f) ? make_float2(x0.x / x0abs, x0.y / x0abs)
                                                : make_float2(1.f, 0.f);
                const float2 alpha = make_float2(-ph.x * amag, -ph.y * amag);
                const float vn2 = 2.f * fmaf(amag, x0abs, nu);
                beta = (vn2 > 0.f) ? 2.f / vn2 : 0.f;
#pragma unroll
                for (int m = t; m < MT; ++m)
                    vv[m] = (m == t) ? make_float2(x0.x - alpha.x, x0.y - alpha.y) : av[m];
                degenerate = degenerate || !(nu > 0.f);
                av[t] = alpha;
#pragma unroll
                for (int m = t + 1; m < MT; ++m) av[m] = make_float2(0.f, 0.f);
                placed = true;
                sm.piv[t] = j;
                sm.rdiag[t] = amag;
                sm.phi[t] = make_float2(-ph.x, -ph.y);
                sm.beta[t] = beta;
#pragma unroll
                for (int m = 0; m < MT; ++m) sm.refl[t][m] = vv[m];
            }
            // the reflector reaches the other lanes as shared-memory broadcasts
            __syncwarp(kFull);
#pragma unroll
            for (int m = t; m < MT; ++m) vv[m] = sm.refl[t][m];
            beta = sm.beta[t];
            if (!placed) {
                float2 s = make_float2(0.f, 0.f);
#pragma unroll
                for (int m = t; m < MT; ++m) s = make_float2(s.x + (vv[m].x * av[m].x + vv[m].y * av[m].y),
                                                             s.y + (vv[m].x * av[m].y - vv[m].y * av[m].x));
                s.x *= beta;
                s.y *= beta;
#pragma unroll
                for (int m = t; m < MT; ++m) {
                    av[m].x -= vv[m].x * s.x - vv[m].y * s.y;
                    av[m].y -= vv[m].x * s.y + vv[m].y * s.x;
                }
            }
            if (act) sm.ru[t][j] = av[t];
        }
    }
    __syncwarp(kFull);

    // R in level order: level i <-> step K-1-i
    if (act) {
        const int i = j;
        const int ui = sm.piv[K - 1 - i];
        for (int k = 0; k < K; ++k) {
            float2 v = make_float2(0.f, 0.f);
            if (k > i) {
                const int tk = K - 1 - k;
                const float2 r = sm.ru[tk][ui];
                v = cmul(sm.phi[tk], make_float2(r.x, -r.y));
            } else if (k == i) {
                v = make_float2(sm.rdiag[K - 1 - i], 0.f);
            }
            sm.rl[i][k] = v;
        }
    }
    __syncwarp(kFull);

    // U = R^-1, lane k computes column k by back substitution
    if (act) {
        const int k = j;
        sm.uu[k][k] = make_float2(1.f / sm.rl[k][k].x, 0.f);
        for (int i = k - 1; i >= 0; --i) {
            float2 s = make_float2(0.f, 0.f);
            for (int m = i + 1; m <= k; ++m) s = cfma(sm.rl[i][m], sm.uu[m][k], s);
            const float rii = sm.rl[i][i].x;
            sm.uu[i][k] = make_float2(-s.x / rii, -s.y / rii);
        }
        for (int i = k + 1; i < K; ++i) sm.uu[i][k] = make_float2(0.f, 0.f);
    }
    __syncwarp(kFull);

    // cond(H H^H) = (sigma_max(R) sigma_max(U))^2, estimated by power iteration;
    // channels above the plan threshold (or degenerate) go to the FP64 path
    float sr, su;
    power_sigma2_pair<KT>(sm.rl, sm.uu, sm.ru, K, j, sr, su);    // ru is free after R's level order
    const float kappa = sr * su;
    const bool degen = (__ballot_sync(kFull, degenerate) & hmask) != 0u;
    const float thr = (a.probs && valid) ? a.probs[c].kappa_thr : a.kappa_thr;
    const bool to64 = !nonfinite && (degen || !(kappa <= thr));
    if (!valid) return;

    if (nonfinite) {
        write_channel_outputs_zero(f, K, M, Mp, j);
        if (j == 0) f.s.st[0] = (uint8_t)VP_CH_NONFINITE;
        return;
    }
    if (to64) {
        if (j == 0) {
            const int idx = atomicAdd(a.nflag, 1);
            a.flags[idx] = c;
            f.s.st[0] = (uint8_t)VP_CH_FP64;
        }
        return;
    }

    if (act) {
        const float uii = sm.uu[j][j].x;
        f.s.w[j] = uii * uii;
        const uint8_t ui = (uint8_t)sm.piv[K - 1 - j];
        f.s.ul[j] = ui;
        if (f.ul_out) f.ul_out[j] = ui;
        // lane k writes column k of each row i (row-major stores coalesced across the lanes)
        const int k = j;
        for (int i = 0; i < K; ++i) {
            const float rii = sm.rl[i][i].x;
            const float2 u = sm.uu[i][k];
            const float2 ut = (k > i) ? make_float2(u.x * rii, u.y * rii)
                                      : (k == i ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f));
            f.s.utp[i * K + k] = make_float4(ut.x, ut.y, ut.y, ut.x);
            f.s.utc[k * K + i] = ut;
            if (f.U_out) f.U_out[i * K + k] = u;
        }
    }

    // P_level = Q^H U = H_0 ... H_{K-1} [D J U; 0]; lane k builds column k
    if (act) {
        const int k = j;
        float2 z[MT];
#pragma unroll
        for (int t = 0; t < MT; ++t)
            z[t] = (t < K) ? cmul(sm.phi[t], sm.uu[K - 1 - t][k]) : make_float2(0.f, 0.f);
#pragma unroll
        for (int t = KT - 1; t >= 0; --t) {
            if (t < K) {
                float2 s = make_float2(0.f, 0.f);
#pragma unroll
                for (int m = t; m < MT; ++m) s = cfma(make_float2(sm.refl[t][m].x, -sm.refl[t][m].y), z[m], s);
                const float b = sm.beta[t];
                s.x *= b;
                s.y *= b;
#pragma unroll
                for (int m = t; m < MT; ++m) {
                    const float2 v = sm.refl[t][m];
                    z[m].x -= v.x * s.x - v.y * s.y;
                    z[m].y -= v.x * s.y + v.y * s.x;
                }
            }
        }
        const int u = sm.piv[K - 1 - k];
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            if (m < Mp) {
                f.s.pt[u * Mp + m] = z[m];
                f.s.ptlo[u * Mp + m] = make_float2(0.f, 0.f);
                if (f.P_out && m < M) f.P_out[m * K + u] = z[m];
            }
        }
    }
    if (j == 0) f.s.st[0] = 0;
    pdl_trigger();
}

// ---------------------------------------------------------------------------
// FP64 path for the flagged channels: a block of NT threads per channel,
// strided over the entries of each (triangular) matrix operation. GB300 issues FP64 FMAs
// at 1/64 of the FP32 rate, so FP64 is kept to the pivoted Cholesky of the
// Gram matrix, U = R^-1 and one Newton step, with the lanes of every FP64
// instruction packed; the Gram matrix, A = U2^H U2 and P = H^H A are
// accumulated in compensated FP32 (exact products, ~48-bit sums).

// Threads on one flagged channel (one channel per block, 27 KB of shared
// memory): two warps split every entry loop; the small reductions (largest
// diagonal, pivot) run on each warp over the same shared values. Measured on
// GB300 (outputs identical for 1, 2 and 4 warps): 2 warps cut vp_factorize
// by 8 us on the Kronecker 16x16 slot (625 flagged channels) and by 14 us on
// an i.i.d. 16x16 slot (252); 4 warps gained nothing more.
constexpr int kNT64 = 64;

struct Smem64 {
    float2 h[kMaxK][kMaxM];      // H rows (user order)
    double2 s[kMaxK][kMaxK];     // Gram / Schur complement (both triangles, user index); later E
    double2 lc[kMaxK][kMaxK];    // lc[t][u]: column of R at level t, by user; later substitution sums
    double2 r[kMaxK][kMaxK];     // R, level order
    double2 u[kMaxK][kMaxK];     // U = R^-1, then U2 after the Newton step
    float2 uh[kMaxK][kMaxK];     // U2 as FP32 hi + lo
    float2 ul[kMaxK][kMaxK];
    float2 ahi[kMaxK][kMaxK];    // A = U2^H U2 as FP32 hi + lo
    float2 alo[kMaxK][kMaxK];
    double2 pc[kMaxK];           // pivot column of the current step (by remaining position)
    double rd[kMaxK];
    double rinv[kMaxK];
    int uol[kMaxK];
    int rem[kMaxK];              // remaining users
};

// e-th entry (e < n(n+1)/2) of a lower triangle: a >= b
__device__ __forceinline__ void tri_index(int e, int& a, int& b)
{
    int r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    while (r * (r + 1) / 2 > e) --r;
    a = r;
    b = e - r * (r + 1) / 2;
}

// (hi, lo) += x * y for a complex FP32 pair y = yh + yl (x exact FP32)
__device__ __forceinline__ void cdot2(float2 x, float2 yh, float2 yl, float& re, float& ree, float& im, float& ime)
{
    dot2_acc(x.x, yh.x, re, ree);
    dot2_acc(-x.y, yh.y, re, ree);
    dot2_acc(x.x, yh.y, im, ime);
    dot2_acc(x.y, yh.x, im, ime);
    ree = fmaf(x.x, yl.x, fmaf(-x.y, yl.y, ree));
    ime = fmaf(x.x, yl.y, fmaf(x.y, yl.x, ime));
}

// One flagged channel per block (grid-stride over the flag list); every
// thread runs the same control flow, so the block barriers are uniform.
template <int NT>
__global__ void __launch_bounds__(NT) factor64_kernel(FactorArgs a)
{
    __shared__ Smem64 sm;
    const int tid = threadIdx.x, lane = threadIdx.x & 31;
    pdl_wait();                                    // the flag list of the FP32 factor
    const int nflag = *a.nflag_in;
    auto gsync = [&]() { if (NT == 32) __syncwarp(); else __syncthreads(); };

    for (int slot = blockIdx.x; slot < nflag; slot += gridDim.x) {
        const int c = a.flags[slot];
        const int K = a.probs ? a.probs[c].K : a.K;
        const int M = a.probs ? a.probs[c].M : a.M;
        const int Mp = a.probs ? M : a.Mp;
        const float lam = a.probs ? 0.f : a.lambda;
        const FChan f = fchan(a, c, K, M);
        for (int i = tid; i < K * M; i += NT) sm.h[i / M][i % M] = f.H[i];
        if (tid < K) sm.rem[tid] = tid;
        gsync();
        // Gram matrix (compensated FP32, exact for FP32 input), both triangles in FP64
        for (int e = tid; e < K * (K + 1) / 2; e += NT) {
            int r, q;
            tri_index(e, r, q);
            float re = 0.f, ree = 0.f, im = 0.f, ime = 0.f;
            for (int m = 0; m < M; ++m) {
                const float2 x = sm.h[r][m], y = sm.h[q][m];
                dot2_acc(x.x, y.x, re, ree);
                dot2_acc(x.y, y.y, re, ree);
                dot2_acc(x.y, y.x, im, ime);
                dot2_acc(-x.x, y.y, im, ime);
            }
            double2 g = make_double2((double)re + (double)ree, (double)im + (double)ime);
            if (r == q) g.x += (double)lam * (double)lam;          // H H^H + lambda^2 I
            sm.s[r][q] = g;
            sm.s[q][r] = zconj(g);
        }
        gsync();
        double dmax = lane < K ? sm.s[lane][lane].x : 0.0;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(kFull, dmax, o));

        // pivoted reverse Cholesky (level t from K-1 down: smallest Schur diagonal, ties to the lowest user)
        bool singular = false;
        for (int t = K - 1; t >= 0; --t) {
            const int m = t + 1;                                       // remaining users before the pivot
            // smallest diagonal: the doubles compared as ordered integers (sign-folded bit
            // patterns), which keeps the comparisons off the FP64 pipe
            long long ik = 0x7ff0000000000000ll;                        // +infinity
            int ku = 0x7fffffff, kp = lane;
            if (lane < m) {
                ku = sm.rem[lane];
                const long long b = __double_as_longlong(sm.s[ku][ku].x);
                ik = b ^ ((b >> 63) & 0x7fffffffffffffffll);
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const long long ok = __shfl_xor_sync(kFull, ik, o);
                const int ou = __shfl_xor_sync(kFull, ku, o), op = __shfl_xor_sync(kFull, kp, o);
                if (ok < ik || (ok == ik && ou < ku)) { ik = ok; ku = ou; kp = op; }
            }
            const double key = __longlong_as_double(ik ^ ((ik >> 63) & 0x7fffffffffffffffll));
            // a NaN diagonal orders above +infinity here, so with every remaining
            // diagonal NaN the winner is an inactive lane (ku not a user): singular
            if (ku < 0 || ku >= K || kp >= m || !(key > 1e-12 * dmax)) { singular = true; break; }   // uniform
            const int p = ku;
            // remove p from the remaining list (move the last one into its position)
            const int last = sm.rem[m - 1];
            gsync();
            if (tid == 0) {
                // 1 / sqrt(key): FP32 estimate, two Newton steps in FP64 (y <- y (3 - k y^2) / 2,
                // each doubling the correct bits), then sqrt(key) = key / sqrt(key); one thread
                // only, since the FP64 pipe is the contended unit of this kernel
                double irt = (double)rsqrtf((float)key);
                if (!(irt > 0.0 && irt < INFINITY)) irt = 1.0 / sqrt(key);   // key outside the FP32 range
                irt = irt * (1.5 - 0.5 * key * irt * irt);
                irt = irt * (1.5 - 0.5 * key * irt * irt);
                sm.rem[kp] = last;
                sm.rd[t] = key * irt;
                sm.rinv[t] = irt;
                sm.uol[t] = p;
            }
            gsync();
            if (tid < m - 1) {
                const double irt = sm.rinv[t];
                const double2 v = sm.s[sm.rem[tid]][p];
                const double2 l = make_double2(v.x * irt, v.y * irt);
                sm.pc[tid] = l;
                sm.lc[t][sm.rem[tid]] = l;
            }
            gsync();
            for (int e = tid; e < (m - 1) * m / 2; e += NT) {        // Schur update, packed lower triangle
                int ia, ib;
                tri_index(e, ia, ib);
                const int ua = sm.rem[ia], ub = sm.rem[ib];
                const double2 pr = zmul(sm.pc[ia], zconj(sm.pc[ib]));
                const double2 v = make_double2(sm.s[ua][ub].x - pr.x, sm.s[ua][ub].y - pr.y);
                sm.s[ua][ub] = v;
                sm.s[ub][ua] = zconj(v);
            }
            gsync();
        }

        if (!singular) {
            for (int e = tid; e < K * K; e += NT) {                    // R in level order
                const int r = e / K, q = e % K;
                sm.r[r][q] = (q > r) ? sm.lc[q][sm.uol[r]] : (q == r ? make_double2(sm.rd[r], 0.0) : make_double2(0.0, 0.0));
            }
            gsync();
            for (int e = tid; e < K * K; e += NT) sm.lc[e / K][e % K] = make_double2(0.0, 0.0);
            gsync();
            // U = R^-1 by rows from the bottom: U_m. = (e_m - sum_{j>m} R_mj U_j.) / R_mm
            for (int m = K - 1; m >= 0; --m) {
                if (tid < K) {
                    const int k = tid;
                    const double2 acc = sm.lc[m][k];
                    const double ri = sm.rinv[m];
                    sm.u[m][k] = (k < m) ? make_double2(0.0, 0.0)
                                         : make_double2(((k == m ? 1.0 : 0.0) - acc.x) * ri, -acc.y * ri);
                }
                gsync();
                const int w = K - m;                                    // entries (i < m, k >= m)
                for (int e = tid; e < m * w; e += NT) {
                    const int i = e / w, k = m + e % w;
                    sm.lc[i][k] = zfma(sm.r[i][m], sm.u[m][k], sm.lc[i][k]);
                }
                gsync();
            }
            // one Newton step U2 = U (2I - R U) = U + U E with E = I - R U (both upper
            // triangular): E in FP64, accumulated by rank-1 steps (E_ik -= R_im U_mk,
            // i <= m <= k); E is of the order of the FP64 rounding of U, so the
            // correction U E is formed in FP32 (its rounding is far below U2's own), in
            // the scratch arrays of the hi / lo parts: U in uh, E in ul, U E in ahi
            for (int e = tid; e < K * K; e += NT) {
                const int r = e / K, q = e % K;
                sm.s[r][q] = make_double2(r == q ? 1.0 : 0.0, 0.0);
            }
            gsync();
            for (int m = 0; m < K; ++m) {
                const int w = K - m;
                for (int e = tid; e < (m + 1) * w; e += NT) {
                    const int i = e / w, k = m + e % w;
                    const double2 pr = zmul(sm.r[i][m], sm.u[m][k]);
                    sm.s[i][k].x -= pr.x;
                    sm.s[i][k].y -= pr.y;
                }
                gsync();
            }
            for (int e = tid; e < K * (K + 1) / 2; e += NT) {
                int k, i;
                tri_index(e, k, i);                                     // i <= k
                sm.ul[i][k] = make_float2((float)sm.s[i][k].x, (float)sm.s[i][k].y);
                sm.uh[i][k] = make_float2((float)sm.u[i][k].x, (float)sm.u[i][k].y);
            }
            gsync();
            for (int e = tid; e < K * (K + 1) / 2; e += NT) {
                int k, i;
                tri_index(e, k, i);
                float2 c = make_float2(0.f, 0.f);
                for (int m = i; m <= k; ++m) c = cfma(sm.uh[i][m], sm.ul[m][k], c);
                sm.ahi[i][k] = c;
            }
            gsync();
            for (int e = tid; e < K * K; e += NT) {                    // U2 (upper), in lc
                const int r = e / K, q = e % K;
                const double2 v = sm.u[r][q];
                sm.lc[r][q] = (q >= r) ? make_double2(v.x + (double)sm.ahi[r][q].x, v.y + (double)sm.ahi[r][q].y)
                                       : make_double2(0.0, 0.0);
            }
            gsync();
            // U2 (in lc) as FP32 hi + lo; outputs: row r of U~, w_r, user of level r
            if (tid < K) sm.rd[tid] = 1.0 / sm.lc[tid][tid].x;     // 1 / U2_rr
            gsync();
            for (int e = tid; e < K * K; e += NT) {
                const int r = e / K, q = e % K;
                const double2 v = sm.lc[r][q];
                const float hx = (float)v.x, hy = (float)v.y;
                sm.uh[r][q] = make_float2(hx, hy);
                sm.ul[r][q] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
                const double urr = sm.lc[r][r].x, iurr = sm.rd[r];
                const float2 ut = (q > r) ? make_float2((float)(v.x * iurr), (float)(v.y * iurr))
                                          : (q == r ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f));
                f.s.utp[r * K + q] = make_float4(ut.x, ut.y, ut.y, ut.x);
                f.s.utc[q * K + r] = ut;
                if (f.U_out) f.U_out[r * K + q] = make_float2(hx, hy);
                if (q == 0) {
                    f.s.w[r] = (float)(urr * urr);
                    f.s.ul[r] = (uint8_t)sm.uol[r];
                    if (f.ul_out) f.ul_out[r] = (uint8_t)sm.uol[r];
                }
            }
            gsync();
            // A = U2^H U2 (Hermitian) in compensated FP32: A_ik = sum_{m <= min(i,k)} conj(U2_mi) U2_mk
            for (int e = tid; e < K * (K + 1) / 2; e += NT) {
                int i, k;
                tri_index(e, i, k);                                     // i >= k
                float re = 0.f, ree = 0.f, im = 0.f, ime = 0.f;
                for (int m = 0; m <= k; ++m) {
                    const float2 xh = sm.uh[m][i], xl = sm.ul[m][i];
                    const float2 cx = make_float2(xh.x, -xh.y);
                    cdot2(cx, sm.uh[m][k], sm.ul[m][k], re, ree, im, ime);
                    ree = fmaf(xl.x, sm.uh[m][k].x, fmaf(xl.y, sm.uh[m][k].y, ree));    // conj(xl) * yh
                    ime = fmaf(xl.x, sm.uh[m][k].y, fmaf(-xl.y, sm.uh[m][k].x, ime));
                }
                const float2 hi = make_float2(__fadd_rn(re, ree), __fadd_rn(im, ime));
                const float2 lo = make_float2(__fsub_rn(ree, __fsub_rn(hi.x, re)), __fsub_rn(ime, __fsub_rn(hi.y, im)));
                sm.ahi[i][k] = hi;
                sm.alo[i][k] = lo;
                sm.ahi[k][i] = make_float2(hi.x, -hi.y);
                sm.alo[k][i] = make_float2(lo.x, -lo.y);
            }
            gsync();
            // P_level[m][k] = sum_j conj(H_perm[j][m]) A[j][k], compensated FP32
            for (int e = tid; e < M * K; e += NT) {
                const int m = e / K, k = e % K;
                float re = 0.f, ree = 0.f, im = 0.f, ime = 0.f;
                for (int j = 0; j < K; ++j) {
                    const float2 hv = sm.h[sm.uol[j]][m];
                    cdot2(make_float2(hv.x, -hv.y), sm.ahi[j][k], sm.alo[j][k], re, ree, im, ime);
                }
                const float2 hi = make_float2(__fadd_rn(re, ree), __fadd_rn(im, ime));
                const float2 lo = make_float2(__fsub_rn(ree, __fsub_rn(hi.x, re)), __fsub_rn(ime, __fsub_rn(hi.y, im)));
                const int uk = sm.uol[k];
                f.s.pt[uk * Mp + m] = hi;
                f.s.ptlo[uk * Mp + m] = lo;
                if (f.P_out) f.P_out[m * K + uk] = hi;
            }
            // regularisation rows (lambda > 0): row M + u of P is lambda A[level of u][.]
            for (int e = tid; e < (Mp - M) * K; e += NT) {
                const int u = e / K, k = e % K;
                int lu = 0;
                for (int i = 0; i < K; ++i) lu = (sm.uol[i] == u) ? i : lu;
                const float2 ah = sm.ahi[lu][k], al = sm.alo[lu][k];
                float hx, ex, hy, ey;
                two_prod(lam, ah.x, hx, ex);
                two_prod(lam, ah.y, hy, ey);
                const int uk = sm.uol[k];
                f.s.pt[uk * Mp + M + u] = make_float2(hx, hy);
                f.s.ptlo[uk * Mp + M + u] = make_float2(fmaf(lam, al.x, ex), fmaf(lam, al.y, ey));
            }
            if (tid == 0) f.s.st[0] = (uint8_t)VP_CH_FP64;
        } else {
            if (tid < 16) write_channel_outputs_zero(f, K, M, Mp, tid);
            if (tid == 0) f.s.st[0] = (uint8_t)(VP_CH_FP64 | VP_CH_SINGULAR);
        }
        gsync();
    }
    pdl_trigger();
}

FactorArgs make_args(const vp_plan* p, const float2* H, int C, float2* U_out, float2* P_out, uint8_t* ul_out)
{
    FactorArgs a;
    a.H = H;
    a.C = C;
    a.K = p->K;
    a.M = p->M;
    a.n = p->n_paths;
    a.Mp = p_rows(p);
    a.lambda = p->lambda;
    a.kappa_thr = p->kappa_thr;
    a.d = p->d;
    a.U_out = U_out;
    a.P_out = P_out;
    a.ul_out = ul_out;
    a.probs = nullptr;
    a.ids = nullptr;
    a.nflag_in = p->d.nflag;
    a.nflag = p->d.nflag;
    a.flags = p->d.flags;
    return a;
}

cudaError_t run_factor32(const FactorArgs& a, cudaStream_t s)
{
    const int blocks = (a.C + kChPerBlock32 - 1) / kChPerBlock32;
    const int threads = kLanes * kChPerBlock32;
    const int rows = a.lambda > 0.f ? a.M + a.K : a.M;   // rows of A = Hbar^H
    const int kt = a.K <= 4 ? 4 : (a.K <= 8 ? 8 : 16);
    if (rows <= 4) factor32_kernel<4, 4><<<blocks, threads, 0, s>>>(a);
    else if (rows <= 8 && kt == 4) factor32_kernel<8, 4><<<blocks, threads, 0, s>>>(a);
    else if (rows <= 8) factor32_kernel<8, 8><<<blocks, threads, 0, s>>>(a);
    else if (rows <= 16 && kt == 4) factor32_kernel<16, 4><<<blocks, threads, 0, s>>>(a);
    else if (rows <= 16 && kt == 8) factor32_kernel<16, 8><<<blocks, threads, 0, s>>>(a);
    else if (rows <= 16) factor32_kernel<16, 16><<<blocks, threads, 0, s>>>(a);
    else if (kt == 4) factor32_kernel<32, 4><<<blocks, threads, 0, s>>>(a);
    else if (kt == 8) factor32_kernel<32, 8><<<blocks, threads, 0, s>>>(a);
    else factor32_kernel<32, 16><<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t run_factor64(const FactorArgs& a, int max_flagged, cudaStream_t s)
{
    int blocks = max_flagged;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    return launch_dependent(factor64_kernel<kNT64>, dim3(blocks), dim3(kNT64), 0, s, a);
}

}  // namespace

cudaError_t launch_factor32(const vp_plan* p, const float2* H, int C, float2* U_out, float2* P_out,
                            uint8_t* ul_out, cudaStream_t s)
{
    return run_factor32(make_args(p, H, C, U_out, P_out, ul_out), s);
}

cudaError_t launch_factor64(const vp_plan* p, const float2* H, int C, float2* U_out, float2* P_out,
                            uint8_t* ul_out, cudaStream_t s)
{
    return run_factor64(make_args(p, H, C, U_out, P_out, ul_out), C, s);
}

cudaError_t launch_factor32_batch(const BatchProblem* probs, const int* ids, int count, int K, int M,
                                  int* nflag, int* flags, cudaStream_t s)
{
    FactorArgs a = FactorArgs();
    a.C = count;
    a.K = K;
    a.M = M;
    a.Mp = M;            // the batch table has lambda = 0
    a.kappa_thr = 0.f;   // per problem, read from the table
    a.probs = probs;
    a.ids = ids;
    a.nflag_in = nflag;
    a.nflag = nflag;
    a.flags = flags;
    return run_factor32(a, s);
}

cudaError_t launch_factor64_batch(const BatchProblem* probs, const int* nflag, const int* flags, int max_flagged,
                                  cudaStream_t s)
{
    FactorArgs a = FactorArgs();
    a.probs = probs;
    a.nflag_in = nflag;
    a.flags = const_cast<int*>(flags);
    return run_factor64(a, max_flagged, s);
}

}  // namespace vp
