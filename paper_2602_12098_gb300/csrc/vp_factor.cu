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
// factor64_kernel: channels whose kappa_hat = max R_ll^2 / min R_ll^2 passes
//   the plan threshold are redone in FP64: Gram matrix, pivoted reverse
//   Cholesky with the same min-pivot rule, U = R^-1 plus one Newton step
//   U <- U (2I - R U), and P = H^H U^H U.
//
// Outputs per channel (level order unless noted): U~ = U_lk / U_ll (unit
// upper), w_l = U_ll^2, the user of each level, and P^T in user order.
#include "vp_internal.cuh"

namespace vp {
namespace {

constexpr int kLanes = 16;        // lanes per channel
constexpr int kChPerBlock32 = 4;  // FP32 kernel: 64 threads
constexpr int kChPerBlock64 = 2;  // FP64 kernel: 32 threads
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

    // kappa_hat = (max R_ll / min R_ll)^2 and the FP64 decision
    float rmax = act ? sm.rdiag[j] : 0.f;
    float rmin = act ? sm.rdiag[j] : INFINITY;
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
        rmax = fmaxf(rmax, __shfl_xor_sync(kFull, rmax, off, kLanes));
        rmin = fminf(rmin, __shfl_xor_sync(kFull, rmin, off, kLanes));
    }
    const bool degen = (__ballot_sync(kFull, degenerate) & hmask) != 0u;
    const float ratio = rmax / rmin;
    const float kappa = ratio * ratio;
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
    __syncwarp(hmask);

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
    __syncwarp(hmask);

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
// FP64 path for the flagged channels.

struct Smem64 {
    float2 h[kMaxK][kMaxM];
    double2 s[kMaxK][kMaxK];     // Schur complement (user index); later the refined U
    double2 lc[kMaxK][kMaxK];    // lc[t][j] = S[j][p] / R_tt at level t; later E and A
    double2 r[kMaxK][kMaxK];     // R, level order
    double2 u[kMaxK][kMaxK];     // U = R^-1
    double rd[kMaxK];
    int uol[kMaxK];
};

__global__ void __launch_bounds__(kLanes * kChPerBlock64) factor64_kernel(FactorArgs a)
{
    __shared__ Smem64 smem[kChPerBlock64];
    const int half = threadIdx.x / kLanes;
    const int j = threadIdx.x % kLanes;
    Smem64& sm = smem[half];
    const int K = a.K, M = a.M;
    const int nflag = *a.d.nflag;

    for (int base = blockIdx.x * kChPerBlock64; base < nflag; base += gridDim.x * kChPerBlock64) {
        const int slot = base + half;
        const bool on = slot < nflag;
        const int c = on ? a.d.flags[slot] : 0;

        if (on && j < K)
            for (int m = 0; m < M; ++m) sm.h[j][m] = a.H[((size_t)c * K + j) * M + m];
        __syncwarp(kFull);
        if (on && j < K) {
            for (int i = 0; i < K; ++i) {
                double2 acc = make_double2(0.0, 0.0);
                for (int m = 0; m < M; ++m) {
                    const float2 x = sm.h[j][m], y = sm.h[i][m];
                    acc = zfma(make_double2(x.x, x.y), make_double2(y.x, -(double)y.y), acc);
                }
                sm.s[j][i] = acc;
            }
        }
        __syncwarp(kFull);

        double dmax = (on && j < K) ? sm.s[j][j].x : 0.0;
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) dmax = fmax(dmax, __shfl_xor_sync(kFull, dmax, off, kLanes));

        unsigned remm = (1u << K) - 1u;
        bool singular = false;
        for (int t = K - 1; t >= 0; --t) {
            // every lane of both halves runs every step (shuffles use the full mask)
            double key = (on && !singular && ((remm >> j) & 1u)) ? sm.s[j][j].x : INFINITY;
            int kj = j;
#pragma unroll
            for (int off = 8; off >= 1; off >>= 1) {
                const double ok = __shfl_xor_sync(kFull, key, off, kLanes);
                const int oj = __shfl_xor_sync(kFull, kj, off, kLanes);
                if (ok < key || (ok == key && oj < kj)) { key = ok; kj = oj; }
            }
            const int p = kj;
            if (!(key > 1e-12 * dmax)) singular = true;             // uniform within the half
            const double rt = sqrt(key);
            remm &= ~(1u << p);
            if (!singular && j == p) { sm.rd[t] = rt; sm.uol[t] = p; }
            if (on && !singular && ((remm >> j) & 1u)) {
                const double2 v = sm.s[j][p];
                sm.lc[t][j] = make_double2(v.x / rt, v.y / rt);
            }
            __syncwarp(kFull);
            if (on && !singular && ((remm >> j) & 1u)) {
                const double2 lj = sm.lc[t][j];
                for (int i = 0; i < K; ++i) {
                    if ((remm >> i) & 1u) {
                        const double2 li = sm.lc[t][i];
                        const double2 pr = zmul(lj, zconj(li));
                        sm.s[j][i].x -= pr.x;
                        sm.s[j][i].y -= pr.y;
                    }
                }
            }
            __syncwarp(kFull);
        }
        // the two halves may disagree on `singular`; each handles its own channel
        const bool good = on && !singular;

        if (good && j < K) {
            const int i = j;
            const int ui = sm.uol[i];
            for (int k = 0; k < K; ++k)
                sm.r[i][k] = (k > i) ? sm.lc[k][ui] : (k == i ? make_double2(sm.rd[i], 0.0) : make_double2(0.0, 0.0));
        }
        __syncwarp(kFull);
        if (good && j < K) {                      // U = R^-1 (column j)
            const int k = j;
            sm.u[k][k] = make_double2(1.0 / sm.r[k][k].x, 0.0);
            for (int i = k - 1; i >= 0; --i) {
                double2 s = make_double2(0.0, 0.0);
                for (int m = i + 1; m <= k; ++m) s = zfma(sm.r[i][m], sm.u[m][k], s);
                sm.u[i][k] = make_double2(-s.x / sm.r[i][i].x, -s.y / sm.r[i][i].x);
            }
            for (int i = k + 1; i < K; ++i) sm.u[i][k] = make_double2(0.0, 0.0);
        }
        __syncwarp(kFull);
        if (good && j < K) {                      // E = I - R U (column j), into lc
            const int k = j;
            for (int i = 0; i < K; ++i) {
                double2 s = make_double2(i == k ? 1.0 : 0.0, 0.0);
                for (int m = i; m <= k; ++m) {
                    const double2 pr = zmul(sm.r[i][m], sm.u[m][k]);
                    s.x -= pr.x;
                    s.y -= pr.y;
                }
                sm.lc[i][k] = (i <= k) ? s : make_double2(0.0, 0.0);
            }
        }
        __syncwarp(kFull);
        if (good && j < K) {                      // U2 = U + U E (Newton step), into s
            const int k = j;
            for (int i = 0; i < K; ++i) {
                double2 s = sm.u[i][k];
                for (int m = i; m <= k; ++m) s = zfma(sm.u[i][m], sm.lc[m][k], s);
                sm.s[i][k] = (i <= k) ? s : make_double2(0.0, 0.0);
            }
        }
        __syncwarp(kFull);
        if (good && j < K) {                      // A = U2^H U2 (column j), into lc
            const int k = j;
            for (int i = 0; i < K; ++i) {
                double2 s = make_double2(0.0, 0.0);
                const int mx = i < k ? i : k;
                for (int m = 0; m <= mx; ++m) s = zfma(zconj(sm.s[m][i]), sm.s[m][k], s);
                sm.lc[i][k] = s;
            }
        }
        __syncwarp(kFull);
        if (good && j < K) {
            const int i = j;                      // row i of U~, w_i, user of level i
            const double uii = sm.s[i][i].x;
            a.d.w[(size_t)c * K + i] = (float)(uii * uii);
            const uint8_t ui = (uint8_t)sm.uol[i];
            a.d.ul[(size_t)c * K + i] = ui;
            if (a.ul_out) a.ul_out[(size_t)c * K + i] = ui;
            for (int k = 0; k < K; ++k) {
                const double2 u = sm.s[i][k];
                const float2 ut = (k > i) ? make_float2((float)(u.x / uii), (float)(u.y / uii))
                                          : (k == i ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f));
                a.d.utp[((size_t)c * K + i) * K + k] = make_float4(ut.x, ut.y, ut.y, ut.x);
                a.d.utc[((size_t)c * K + k) * K + i] = ut;
                if (a.U_out) a.U_out[((size_t)c * K + i) * K + k] = make_float2((float)u.x, (float)u.y);
            }
            // P_level[:, k=j] = H_perm^H A[:, k]; stored under user uol[k]
            const int k = j;
            const int uk = sm.uol[k];
            for (int m = 0; m < M; ++m) {
                double2 s = make_double2(0.0, 0.0);
                for (int q = 0; q < K; ++q) {
                    const float2 hv = sm.h[sm.uol[q]][m];
                    s = zfma(make_double2(hv.x, -(double)hv.y), sm.lc[q][k], s);
                }
                const float2 pv = make_float2((float)s.x, (float)s.y);
                a.d.pt[((size_t)c * K + uk) * M + m] = pv;
                a.d.ptlo[((size_t)c * K + uk) * M + m] =
                    make_float2((float)(s.x - (double)pv.x), (float)(s.y - (double)pv.y));
                if (a.P_out) a.P_out[((size_t)c * M + m) * K + uk] = pv;
            }
        }
        if (on && !good) {
            write_channel_outputs_zero(a, c, j);
        }
        if (on && j == 0) a.d.st[c] = (uint8_t)(VP_CH_FP64 | (good ? 0u : VP_CH_SINGULAR));
        __syncwarp(kFull);
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
    int blocks = (C + kChPerBlock64 - 1) / kChPerBlock64;
    if (blocks > 152 * 16) blocks = 152 * 16;
    factor64_kernel<<<blocks, kLanes * kChPerBlock64, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vp
