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
//   U <- U (2I - R U) in FP64, then P = H^H U^H U as a hi/lo FP32 pair.
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
    int C, K, M;
    float kappa_thr;
    DeviceState d;
    float2* U_out;
    float2* P_out;
    uint8_t* ul_out;
};

template <int MT>
struct Smem32 {
    float2 refl[kMaxK][MT];    // Householder vector of step t (zero above row t)
    float2 ru[kMaxK][kMaxK];   // ru[t][j]: entry of row t of R' in the column of user j
    float2 rl[kMaxK][kMaxK];   // R, level order
    float2 uu[kMaxK][kMaxK];   // U = R^-1, level order
    float2 phi[kMaxK];         // phase of R'_tt
    float beta[kMaxK];
    float rdiag[kMaxK];        // |R'_tt|
    int piv[kMaxK];            // user pivoted at step t
};

__device__ __forceinline__ void write_channel_outputs_zero(const FactorArgs& a, int c, int j)
{
    const int K = a.K, M = a.M;
    if (j < K) {
        for (int k = 0; k < K; ++k) {
            a.d.utp[((size_t)c * K + j) * K + k] = make_float4(0.f, 0.f, 0.f, 0.f);
            a.d.utc[((size_t)c * K + j) * K + k] = make_float2(0.f, 0.f);
            if (a.U_out) a.U_out[((size_t)c * K + j) * K + k] = make_float2(0.f, 0.f);
        }
        for (int m = 0; m < M; ++m) {
            a.d.pt[((size_t)c * K + j) * M + m] = make_float2(0.f, 0.f);
            a.d.ptlo[((size_t)c * K + j) * M + m] = make_float2(0.f, 0.f);
            if (a.P_out) a.P_out[((size_t)c * M + m) * K + j] = make_float2(0.f, 0.f);
        }
        a.d.w[(size_t)c * K + j] = 0.f;
        a.d.ul[(size_t)c * K + j] = (uint8_t)j;
        if (a.ul_out) a.ul_out[(size_t)c * K + j] = (uint8_t)j;
    }
}

// sigma_max(A)^2 of an upper-triangular K x K matrix held in shared memory,
// by power iteration on A^H A (a lower bound that converges from below). Every
// lane of the warp calls it; lane j < K holds component j of the iterate.
__device__ float power_sigma2(const float2 (*A)[kMaxK], int K, int j)
{
    const bool act = j < K;
    float2 v = make_float2(act ? 1.f + 0.0625f * (float)j : 0.f, 0.f);
    float lam = 0.f;
    for (int it = 0; it < 6; ++it) {
        float2 w = make_float2(0.f, 0.f);                       // w = A v
        for (int k = 0; k < K; ++k) {
            const float2 vk = make_float2(__shfl_sync(kFull, v.x, k, kLanes), __shfl_sync(kFull, v.y, k, kLanes));
            if (act && k >= j) w = cfma(A[j][k], vk, w);
        }
        float2 z = make_float2(0.f, 0.f);                       // z = A^H w
        for (int i = 0; i < K; ++i) {
            const float2 wi = make_float2(__shfl_sync(kFull, w.x, i, kLanes), __shfl_sync(kFull, w.y, i, kLanes));
            if (act && i <= j) z = cfma(make_float2(A[i][j].x, -A[i][j].y), wi, z);
        }
        float nw = cabs2(w), nv = cabs2(v), nz = cabs2(z);
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) {
            nw += __shfl_xor_sync(kFull, nw, off, kLanes);
            nv += __shfl_xor_sync(kFull, nv, off, kLanes);
            nz += __shfl_xor_sync(kFull, nz, off, kLanes);
        }
        lam = nw / nv;                                          // Rayleigh quotient of A^H A
        const float sc = rsqrtf(nz);
        v = make_float2(z.x * sc, z.y * sc);
    }
    return lam;
}

template <int MT>
__global__ void __launch_bounds__(kLanes * kChPerBlock32) factor32_kernel(FactorArgs a)
{
    __shared__ Smem32<MT> smem[kChPerBlock32];
    const int slot = threadIdx.x / kLanes;
    const int j = threadIdx.x % kLanes;
    const int hw = (threadIdx.x >> 4) & 1;                 // half of the warp
    const unsigned hmask = 0xFFFFu << (16 * hw);
    const int c = blockIdx.x * kChPerBlock32 + slot;
    const bool valid = c < a.C;
    const int K = a.K, M = a.M;
    const bool act = j < K;
    Smem32<MT>& sm = smem[slot];

    // column j of A = H^H
    float2 av[MT];
    bool finite = true;
#pragma unroll
    for (int m = 0; m < MT; ++m) {
        float2 h = make_float2(0.f, 0.f);
        if (valid && act && m < M) h = a.H[((size_t)c * K + j) * M + m];
        finite = finite && isfinite(h.x) && isfinite(h.y);
        av[m] = make_float2(h.x, -h.y);
    }
    const bool nonfinite = (__ballot_sync(kFull, !finite) & hmask) != 0u;
    if (nonfinite) {
#pragma unroll
        for (int m = 0; m < MT; ++m) av[m] = make_float2(0.f, 0.f);
    }

    bool placed = !act;
    bool degenerate = false;
#pragma unroll
    for (int t = 0; t < MT; ++t) {
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
#pragma unroll
            for (int m = t; m < MT; ++m) {
                vv[m].x = __shfl_sync(kFull, vv[m].x, p, kLanes);
                vv[m].y = __shfl_sync(kFull, vv[m].y, p, kLanes);
            }
            beta = __shfl_sync(kFull, beta, p, kLanes);
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
    const float kappa = power_sigma2(sm.rl, K, j) * power_sigma2(sm.uu, K, j);
    const bool degen = (__ballot_sync(kFull, degenerate) & hmask) != 0u;
    const bool to64 = !nonfinite && (degen || !(kappa <= a.kappa_thr));
    if (!valid) return;

    if (nonfinite) {
        write_channel_outputs_zero(a, c, j);
        if (j == 0) a.d.st[c] = (uint8_t)VP_CH_NONFINITE;
        return;
    }
    if (to64) {
        if (j == 0) {
            const int idx = atomicAdd(a.d.nflag, 1);
            a.d.flags[idx] = c;
            a.d.st[c] = (uint8_t)VP_CH_FP64;
        }
        return;
    }

    if (act) {
        const int i = j;
        const float rii = sm.rl[i][i].x;
        const float uii = sm.uu[i][i].x;
        a.d.w[(size_t)c * K + i] = uii * uii;
        const uint8_t ui = (uint8_t)sm.piv[K - 1 - i];
        a.d.ul[(size_t)c * K + i] = ui;
        if (a.ul_out) a.ul_out[(size_t)c * K + i] = ui;
        for (int k = 0; k < K; ++k) {
            float2 u = sm.uu[i][k];
            float2 ut = (k > i) ? make_float2(u.x * rii, u.y * rii)
                                : (k == i ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f));
            a.d.utp[((size_t)c * K + i) * K + k] = make_float4(ut.x, ut.y, ut.y, ut.x);
            a.d.utc[((size_t)c * K + k) * K + i] = ut;
            if (a.U_out) a.U_out[((size_t)c * K + i) * K + k] = u;
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
        for (int t = MT - 1; t >= 0; --t) {
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
            if (m < M) {
                a.d.pt[((size_t)c * K + u) * M + m] = z[m];
                a.d.ptlo[((size_t)c * K + u) * M + m] = make_float2(0.f, 0.f);
                if (a.P_out) a.P_out[((size_t)c * M + m) * K + u] = z[m];
            }
        }
    }
    if (j == 0) a.d.st[c] = 0;
}

// ---------------------------------------------------------------------------
// FP64 path for the flagged channels: one 256-thread block per channel,
// thread (r, q) <-> matrix entry (r, q). GB300's FP64 rate is low, so FP64 is
// kept to the pivoted Cholesky of the Gram matrix, U = R^-1 and one Newton
// step; the Gram matrix and P are accumulated in compensated FP32 (exact
// products of the FP32 inputs, ~48-bit sums).

struct Smem64 {
    float2 h[kMaxK][kMaxM];      // H rows (user order)
    double2 s[kMaxK][kMaxK];     // Gram / Schur complement, lower triangle (user index); later A = U2^H U2
    double2 lc[kMaxK][kMaxK];    // lc[t][j]: column of R at level t, by user j; later the substitution sums
    double2 r[kMaxK][kMaxK];     // R, level order; later E = I - R U
    double2 u[kMaxK][kMaxK];     // U = R^-1
    double2 u2[kMaxK][kMaxK];    // U after one Newton step
    float2 ahi[kMaxK][kMaxK];    // A = U2^H U2 split into FP32 hi + lo
    float2 alo[kMaxK][kMaxK];
    double2 pc[kMaxK];           // pivot column / R_tt of the current step
    double rd[kMaxK];
    double rinv[kMaxK];          // 1 / R_mm
    int uol[kMaxK];
    double dmax;
    double pivv;
    int piv;
};

__device__ __forceinline__ double2 s_at(const Smem64& sm, int i, int j)   // Schur entry (i, j) from the lower triangle
{
    return i >= j ? sm.s[i][j] : zconj(sm.s[j][i]);
}

__global__ void __launch_bounds__(256) factor64_kernel(FactorArgs a)
{
    __shared__ Smem64 sm;
    const int tid = threadIdx.x;
    const int r = tid >> 4, q = tid & 15;
    const int K = a.K, M = a.M;
    const int nflag = *a.d.nflag;

    for (int slot = blockIdx.x; slot < nflag; slot += gridDim.x) {
        const int c = a.d.flags[slot];
        for (int i = tid; i < K * M; i += blockDim.x) sm.h[i / M][i % M] = a.H[(size_t)c * K * M + i];
        __syncthreads();
        // Gram, lower triangle: G_rq = sum_m h_rm conj(h_qm), compensated FP32 -> FP64
        if (r < K && q <= r) {
            float re = 0.f, ree = 0.f, im = 0.f, ime = 0.f;
            for (int m = 0; m < M; ++m) {
                const float2 x = sm.h[r][m], y = sm.h[q][m];
                dot2_acc(x.x, y.x, re, ree);
                dot2_acc(x.y, y.y, re, ree);
                dot2_acc(x.y, y.x, im, ime);
                dot2_acc(-x.x, y.y, im, ime);
            }
            sm.s[r][q] = make_double2((double)re + (double)ree, (double)im + (double)ime);
        }
        __syncthreads();
        if (tid == 0) {
            double dm = 0.0;
            for (int j = 0; j < K; ++j) dm = fmax(dm, sm.s[j][j].x);
            sm.dmax = dm;
        }

        // pivoted reverse Cholesky: at level t (from K-1 down) the remaining user
        // with the smallest Schur diagonal (ties: lowest user) becomes the pivot
        unsigned remm = (1u << K) - 1u;
        bool singular = false;
        for (int t = K - 1; t >= 0 && !singular; --t) {
            __syncthreads();
            if (tid < 32) {
                double key = (tid < K && ((remm >> tid) & 1u)) ? sm.s[tid][tid].x : INFINITY;
                int kj = tid;
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) {
                    const double ok = __shfl_xor_sync(kFull, key, off);
                    const int oj = __shfl_xor_sync(kFull, kj, off);
                    if (ok < key || (ok == key && oj < kj)) { key = ok; kj = oj; }
                }
                if (tid == 0) { sm.piv = kj; sm.pivv = key; }
            }
            __syncthreads();
            const int p = sm.piv;
            const double pv = sm.pivv;
            if (!(pv > 1e-12 * sm.dmax)) { singular = true; break; }   // uniform: every thread reads the same values
            const double rt = sqrt(pv);
            const double irt = 1.0 / rt;
            remm &= ~(1u << p);
            if (tid < K) {
                double2 v = make_double2(0.0, 0.0);
                if ((remm >> tid) & 1u) {
                    const double2 sp = s_at(sm, tid, p);
                    v = make_double2(sp.x * irt, sp.y * irt);
                }
                sm.pc[tid] = v;
                sm.lc[t][tid] = v;
            }
            if (tid == 0) { sm.rd[t] = rt; sm.uol[t] = p; }
            __syncthreads();
            if (r < K && q <= r && ((remm >> r) & 1u) && ((remm >> q) & 1u)) {
                const double2 pr = zmul(sm.pc[r], zconj(sm.pc[q]));
                sm.s[r][q].x -= pr.x;
                sm.s[r][q].y -= pr.y;
            }
        }
        __syncthreads();

        if (!singular) {
            // R in level order
            if (r < K && q < K)
                sm.r[r][q] = (q > r) ? sm.lc[q][sm.uol[r]] : (q == r ? make_double2(sm.rd[r], 0.0) : make_double2(0.0, 0.0));
            if (tid < K) sm.rinv[tid] = 1.0 / sm.rd[tid];
            __syncthreads();
            // U = R^-1 by rows from the bottom: U_i. = (e_i - sum_{m>i} R_im U_m.) / R_ii
            if (r < K && q < K) sm.lc[r][q] = make_double2(0.0, 0.0);
            __syncthreads();
            for (int m = K - 1; m >= 0; --m) {
                if (tid < K) {
                    const int k = tid;
                    const double2 acc = sm.lc[m][k];
                    const double ri = sm.rinv[m];
                    sm.u[m][k] = (k < m) ? make_double2(0.0, 0.0)
                                         : make_double2(((k == m ? 1.0 : 0.0) - acc.x) * ri, -acc.y * ri);
                }
                __syncthreads();
                if (r < m && q < K && q >= m) sm.lc[r][q] = zfma(sm.r[r][m], sm.u[m][q], sm.lc[r][q]);
                __syncthreads();
            }
            // one Newton step: E = I - R U, U2 = U + U E (upper triangular)
            double2 e = make_double2(0.0, 0.0);
            if (r < K && q < K && q >= r) {
                e = make_double2(r == q ? 1.0 : 0.0, 0.0);
                for (int m = r; m <= q; ++m) {
                    const double2 pr = zmul(sm.r[r][m], sm.u[m][q]);
                    e.x -= pr.x;
                    e.y -= pr.y;
                }
            }
            __syncthreads();
            if (r < K && q < K) sm.r[r][q] = e;
            __syncthreads();
            if (r < K && q < K) {
                double2 v = make_double2(0.0, 0.0);
                if (q >= r) {
                    v = sm.u[r][q];
                    for (int m = r; m <= q; ++m) v = zfma(sm.u[r][m], sm.r[m][q], v);
                }
                sm.u2[r][q] = v;
            }
            __syncthreads();
            // A = U2^H U2 (Hermitian), as an FP32 hi + lo pair
            if (r < K && q < K) {
                double2 v = make_double2(0.0, 0.0);
                const int mx = r < q ? r : q;
                for (int m = 0; m <= mx; ++m) v = zfma(zconj(sm.u2[m][r]), sm.u2[m][q], v);
                const float hx = (float)v.x, hy = (float)v.y;
                sm.ahi[r][q] = make_float2(hx, hy);
                sm.alo[r][q] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
            }
            __syncthreads();
            // outputs: row r of U~, w_r, user of level r
            if (r < K && q < K) {
                const double urr = sm.u2[r][r].x;
                const double2 uv = sm.u2[r][q];
                const float2 ut = (q > r) ? make_float2((float)(uv.x / urr), (float)(uv.y / urr))
                                          : (q == r ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f));
                a.d.utp[((size_t)c * K + r) * K + q] = make_float4(ut.x, ut.y, ut.y, ut.x);
                a.d.utc[((size_t)c * K + q) * K + r] = ut;
                if (a.U_out) a.U_out[((size_t)c * K + r) * K + q] = make_float2((float)uv.x, (float)uv.y);
                if (q == 0) {
                    a.d.w[(size_t)c * K + r] = (float)(urr * urr);
                    a.d.ul[(size_t)c * K + r] = (uint8_t)sm.uol[r];
                    if (a.ul_out) a.ul_out[(size_t)c * K + r] = (uint8_t)sm.uol[r];
                }
            }
            // P_level[m][k] = sum_j conj(H_perm[j][m]) A[j][k], compensated FP32 with A = hi + lo
            for (int e2 = tid; e2 < M * K; e2 += blockDim.x) {
                const int m = e2 / K, k = e2 % K;
                float re = 0.f, ree = 0.f, im = 0.f, ime = 0.f;
                for (int j = 0; j < K; ++j) {
                    const float2 hv = sm.h[sm.uol[j]][m];
                    const float ahx = sm.ahi[j][k].x, ahy = sm.ahi[j][k].y;
                    const float alx = sm.alo[j][k].x, aly = sm.alo[j][k].y;
                    // conj(h) * a = (h.x a.x + h.y a.y) + i (h.x a.y - h.y a.x)
                    dot2_acc(hv.x, ahx, re, ree);
                    dot2_acc(hv.y, ahy, re, ree);
                    dot2_acc(hv.x, ahy, im, ime);
                    dot2_acc(-hv.y, ahx, im, ime);
                    ree = fmaf(hv.x, alx, fmaf(hv.y, aly, ree));
                    ime = fmaf(hv.x, aly, fmaf(-hv.y, alx, ime));
                }
                const float2 hi = make_float2(__fadd_rn(re, ree), __fadd_rn(im, ime));
                const float2 lo = make_float2(__fsub_rn(ree, __fsub_rn(hi.x, re)), __fsub_rn(ime, __fsub_rn(hi.y, im)));
                const int uk = sm.uol[k];
                a.d.pt[((size_t)c * K + uk) * M + m] = hi;
                a.d.ptlo[((size_t)c * K + uk) * M + m] = lo;
                if (a.P_out) a.P_out[((size_t)c * M + m) * K + uk] = hi;
            }
            if (tid == 0) a.d.st[c] = (uint8_t)VP_CH_FP64;
        } else {
            if (tid < 16) write_channel_outputs_zero(a, c, tid);
            if (tid == 0) a.d.st[c] = (uint8_t)(VP_CH_FP64 | VP_CH_SINGULAR);
        }
        __syncthreads();
    }
}

FactorArgs make_args(const vp_plan* p, const float2* H, int C, float2* U_out, float2* P_out, uint8_t* ul_out)
{
    FactorArgs a;
    a.H = H;
    a.C = C;
    a.K = p->K;
    a.M = p->M;
    a.kappa_thr = p->kappa_thr;
    a.d = p->d;
    a.U_out = U_out;
    a.P_out = P_out;
    a.ul_out = ul_out;
    return a;
}

}  // namespace

cudaError_t launch_factor32(const vp_plan* p, const float2* H, int C, float2* U_out, float2* P_out,
                            uint8_t* ul_out, cudaStream_t s)
{
    const FactorArgs a = make_args(p, H, C, U_out, P_out, ul_out);
    const int blocks = (C + kChPerBlock32 - 1) / kChPerBlock32;
    const int threads = kLanes * kChPerBlock32;
    if (p->M <= 4) factor32_kernel<4><<<blocks, threads, 0, s>>>(a);
    else if (p->M <= 8) factor32_kernel<8><<<blocks, threads, 0, s>>>(a);
    else factor32_kernel<16><<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_factor64(const vp_plan* p, const float2* H, int C, float2* U_out, float2* P_out,
                            uint8_t* ul_out, cudaStream_t s)
{
    const FactorArgs a = make_args(p, H, C, U_out, P_out, ul_out);
    int blocks = C < 152 * 8 ? C : 152 * 8;
    factor64_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vp
