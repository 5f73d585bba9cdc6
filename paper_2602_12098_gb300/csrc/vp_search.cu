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
// one packed FP32 add per complex term from a per-block table of -U~_ml t,
// and t_l is the p_l-th nearest point of {-1,0,1}+j{-1,0,1} to r'_l (DEMAP),
// ties to the smaller (Re t, Im t).
// The PED grows by w_l tau^2 |r'_l - t_l|^2.
// The zero perturbation is candidate 0; the warp's (PED, index) minimum wins
// (ties: lower index). w = P u with u = s + tau l, gamma = ||w||^2 and x = the
// antenna rows of w / sqrt(gamma) (with lambda > 0, P has K more rows: the
// regularisation part of Alg. 2's w, which counts in gamma but is not sent),
// the product P u formed with exact products and compensated sums.
//
// Fixed-point form (FIX, Section IV's 16-bit datapath with F fractional
// bits): the entries of U~ are rounded to multiples of 2^-F (halves to even)
// and saturated to +-32767 2^-F; the starting residual b' = (s + U~ s) / tau
// is formed from those words and rounded once, and every column update
// saturates. Words, the sum of two of them, and b' before its rounding
// (odd integers <= 15 times words: numerators below 2^24 units of 2^-F for
// K <= 16) are all exact in FP32, so the FMAs perform the integer arithmetic
// exactly; DEMAP then works on dyadic points with the tie shift scaled to
// the word (below).
#include "vp_internal.cuh"
#include "vp_select.cuh"

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
    int Mp;          // rows of P kept (M, or M + K with lambda > 0)
    float tau, inv_tau;
    DeviceState d;
    // batch mode (probs != null): block i works on problem ids[i] of the table;
    // KM, NP give the shared-memory layout (the launch's largest K*M and n)
    const BatchProblem* probs;
    const int* ids;
    int KM, NP;
    int demap;       // VP_DEMAP_* (plan launches)
    int frac;        // fractional bits of the fixed-point search (0: floating point)
    int tcp;         // 1: w = P u on the tensor cores (plan launches, exact DEMAP, floating point)
};

// One level of the descent for a lane's candidate: DEMAP selection of the
// digit's point around r'_lv, PED update, the chosen t recorded as a 4-bit
// code, and the column update r'_m -= U~_m,lv t for m < lv.
template <int KT, bool LUT, bool FIX>
__device__ __forceinline__ void level_step(int lv, const float2* ctab, const float* wv, uint32_t cw0, uint32_t cw1,
                                           uint32_t mq0, uint32_t mq1, const uint64_t* lut, const FixP& fx,
                                           float2 (&r)[KT], float& ped, uint32_t& lc0, uint32_t& lc1)
{
    const int sh = 4 * (lv & 7);
    const uint32_t cwl = (lv < 8) ? cw0 : cw1;
    const float cx = r[lv].x, cy = r[lv].y;
    int tr, ti;
    if (LUT) {
        select_lut(cx, cy, (int)(cwl >> sh) & 15, lut, tr, ti);
    } else {
        const int mql = (int)(((lv < 8) ? mq0 : mq1) >> sh) & 15;
        if (FIX) select_point<false>(cx, cy, cwl, sh, mql, tr, ti, fx.epsx, fx.epsy);
        else select_point<true>(cx, cy, cwl, sh, mql, tr, ti, kEpsX, kEpsY);
    }
    // point code (tr + 1) | (ti + 1) << 2, written as a sum, and recorded by an
    // add (the level's nibble is still zero): both fuse into multiply-adds
    const int kd = tr + 4 * ti + 5;
    const uint32_t dig = (uint32_t)kd << sh;
    if (lv < 8) lc0 += dig; else lc1 += dig;
    const float2* col = ctab + ct_off(lv) + kd * ct_stride(lv);
    const float2 d = __fadd2_rn(r[lv], col[lv]);                 // r'_lv - t
    ped = fmaf(wv[lv], fmaf(d.x, d.x, d.y * d.y), ped);
    if (lv > 0) {
#pragma unroll
        for (int m = 0; m < KT; ++m) {
            if (m < lv) {
                r[m] = __fadd2_rn(r[m], col[m]);
                if (FIX) {
                    r[m].x = fminf(fmaxf(r[m].x, -fx.lim), fx.lim);
                    r[m].y = fminf(fmaxf(r[m].y, -fx.lim), fx.lim);
                }
            }
        }
    }
}

// One level's term of y = P u with P = ph + pl (hi + lo pair, user order):
// exact products and compensated sums (u holds small integers, so P u keeps
// ~48 bits before the final rounding).
__device__ __forceinline__ void py_acc(const float2* pt, const float2* ptl, int idx, float ur, float ui, float& yr,
                                       float& yre, float& yi, float& yie)
{
    const float2 ph = pt[idx], pl = ptl[idx];
    dot2_acc(ph.x, ur, yr, yre);
    dot2_acc(-ph.y, ui, yr, yre);
    dot2_acc(ph.x, ui, yi, yie);
    dot2_acc(ph.y, ur, yi, yie);
    yre = fmaf(pl.x, ur, fmaf(-pl.y, ui, yre));
    yie = fmaf(pl.x, ui, fmaf(pl.y, ur, yie));
}

// y = P u, gamma = ||y||^2 and x = the antenna rows / sqrt(gamma) for two
// vectors at once: half-warp hf takes vector hf ? vB : vA (Mp <= 16 rows);
// upk holds u, lanes 0-15 by level for vA and lanes 16-31 for vB.
__device__ __forceinline__ void pair_rows_out(const float2* pt, const float2* ptl, const int* ulv, float2 upk, int K,
                                              int M, int Mp, int vA, int vB, int v1, float2* xo, float* go)
{
    const int lane = threadIdx.x & 31;
    const int hf = lane >> 4, m = lane & 15;
    const int vh = hf ? vB : vA;
    const bool on = vh < v1 && m < Mp;
    float yr = 0.f, yre = 0.f, yi = 0.f, yie = 0.f;
    for (int lv = 0; lv < K; ++lv) {
        const float ur = __shfl_sync(kFull, upk.x, lv + 16 * hf), ui = __shfl_sync(kFull, upk.y, lv + 16 * hf);
        if (on) py_acc(pt, ptl, ulv[lv] * Mp + m, ur, ui, yr, yre, yi, yie);
    }
    const float2 y = make_float2(__fadd_rn(yr, yre), __fadd_rn(yi, yie));
    float g = on ? cabs2(y) : 0.f;              // ||w||^2 over all rows (Alg. 2's d)
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) g += __shfl_xor_sync(kFull, g, o);
    const float rs = __frsqrt_rn(g);
    if (vh < v1 && m < M) xo[(size_t)vh * M + m] = make_float2(y.x * rs, y.y * rs);
    if (vh < v1 && m == 0) go[vh] = g;
    __syncwarp(kFull);
}

// ---------------------------------------------------------------------------
// w = P u on the tensor cores (Eqs. 24-25, the PV block of Section IV-B), for
// a round of up to kTcCols data vectors of one channel, by the whole block.
//
// In real form W = A V with A = [[Re P, -Im P], [Im P, Re P]] (2Mp x 2K, user
// order) and V = [Re u; Im u] (2K x vectors). u holds small integers
// (|Re u|, |Im u| <= 47), exact in TF32. P = ph + pl is split, per complex
// row m, into three pieces on the grids 2^(E_m - 10), 2^(E_m - 21) and
// 2^(E_m - 32), where 2^E_m bounds the row's largest component (the
// error-free splitting of Ozaki et al. for exact matrix products): each piece
// is an integer of at most 11 bits times its grid, exact in TF32, so every
// product is exact, and every partial sum of a piece's product (at most 32
// terms of at most 2^16 grid units) stays below 2^22 grid units, so the FP32
// accumulation of the tensor cores is exact as well. The three exact piece
// products are added by one error-free addition; the split keeps P to 2^-33
// of its row's largest entry, below the FP32 rounding of P itself.
// mma.sync m16n8k8 (TF32 in, FP32 accumulate): a warp per 16 x 8 output
// tile. The pieces are staged row-major in shared memory with row stride
// 2K + 4 floats (the 8 rows x 4 columns a fragment reads fall on distinct
// banks), V as [2K][24] floats (conflict-free for the B fragment).
constexpr int kTcCols = 16;     // vectors per round
constexpr int kTcVs = 24;       // row stride of V and W (floats)

__host__ __device__ inline int tc_pad16(int x) { return (x + 15) & ~15; }
__host__ __device__ inline int tc_pad8(int x) { return (x + 7) & ~7; }

// Bytes of the round's work area (pieces, V, W, row exponents).
__host__ __device__ inline int tc_area_bytes(int K, int Mp)
{
    const int mp2 = tc_pad16(2 * Mp), k2 = tc_pad8(2 * K);
    return 4 * (3 * mp2 * (k2 + 4) + k2 * kTcVs + mp2 * kTcVs + 32);
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One round: vectors v0r .. v0r + nv - 1 of the channel, their u (level
// order) in ust[col][level]. Every thread of the block calls it, after the
// round's searches. Writes x (antenna rows of w / sqrt(gamma)) and gamma.
__device__ void tc_round(const float2* __restrict__ pt, const float2* __restrict__ ptl, const int* ulv,
                         const float2* ust, int KT, int K, int M, int Mp, int v0r, int nv, float* area, float2* xo,
                         float* go)
{
    const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31, NW = nthr >> 5;
    const int mp2 = tc_pad16(2 * Mp), k2 = tc_pad8(2 * K), as = k2 + 4;
    float* Ap = area;                                  // [3][mp2][as]
    float* V = Ap + 3 * mp2 * as;                      // [k2][kTcVs]
    float* W = V + k2 * kTcVs;                         // [mp2][kTcVs]
    int* Es = reinterpret_cast<int*>(W + mp2 * kTcVs); // [Mp] row exponents
    __syncthreads();                                   // the round's searches are done; area is free
    for (int m = tid; m < Mp; m += nthr) {
        float mx = 0.f;
        for (int k = 0; k < K; ++k) {
            const float2 z = pt[k * Mp + m];
            mx = fmaxf(mx, fmaxf(fabsf(z.x), fabsf(z.y)));
        }
        int e = 0;
        frexpf(mx, &e);                                // mx < 2^e
        Es[m] = e;
    }
    for (int i = tid; i < k2 * kTcCols; i += nthr) {   // V: Re u over the users, then Im u
        const int kr = i / kTcCols, col = i - kr * kTcCols;
        float v = 0.f;
        if (col < nv && kr < 2 * K) {
            const int usr = kr < K ? kr : kr - K;
            int lev = 0;
            for (int l = 0; l < K; ++l) lev = ulv[l] == usr ? l : lev;
            const float2 u = ust[col * KT + lev];
            v = kr < K ? u.x : u.y;
        }
        V[kr * kTcVs + col] = v;
    }
    __syncthreads();
    for (int i = tid; i < mp2 * k2; i += nthr) {       // the three pieces of A
        const int R = i / k2, C = i - R * k2;
        float p1 = 0.f, p2 = 0.f, p3 = 0.f;
        if (R < 2 * Mp && C < 2 * K) {
            const int pr = R >= Mp, m = R - pr * Mp, pc = C >= K, k = C - pc * K;
            const float2 zh = pt[k * Mp + m], zl = ptl[k * Mp + m];
            float vh, vl;                               // [[Re, -Im], [Im, Re]]
            if (pr == pc) { vh = zh.x; vl = zl.x; }
            else if (pc) { vh = -zh.y; vl = -zl.y; }
            else { vh = zh.y; vl = zl.y; }
            const int E = Es[m];
            const float t = ldexpf(vh, 10 - E);        // |t| < 2^10, exact scaling
            p1 = rintf(t);
            float r = __fadd_rn(__fsub_rn(t, p1), ldexpf(vl, 10 - E)) * 2048.f;
            p2 = rintf(r);
            r = __fsub_rn(r, p2) * 2048.f;
            p3 = rintf(r);
        }
        Ap[R * as + C] = p1;
        Ap[mp2 * as + R * as + C] = p2;
        Ap[2 * mp2 * as + R * as + C] = p3;
    }
    __syncthreads();
    const int g = lane >> 2, t4 = lane & 3;
    const int ntile = nv > 8 ? 2 : 1, ntiles = (mp2 >> 4) * ntile;
    for (int tile = warp; tile < ntiles; tile += NW) {
        const int mt = tile / ntile, nt = tile - mt * ntile;
        float acc[3][4] = {};
        for (int ks = 0; ks < (k2 >> 3); ++ks) {
            const uint32_t b0 = __float_as_uint(V[(8 * ks + t4) * kTcVs + 8 * nt + g]);
            const uint32_t b1 = __float_as_uint(V[(8 * ks + t4 + 4) * kTcVs + 8 * nt + g]);
#pragma unroll
            for (int pc = 0; pc < 3; ++pc) {
                const float* A = Ap + pc * mp2 * as + (16 * mt + g) * as + 8 * ks + t4;
                mma_tf32(acc[pc], __float_as_uint(A[0]), __float_as_uint(A[8 * as]), __float_as_uint(A[4]),
                         __float_as_uint(A[8 * as + 4]), b0, b1);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {                   // c0..c3: rows g, g, g+8, g+8; columns 2 t4, 2 t4 + 1
            const int R = 16 * mt + g + (e >> 1) * 8, col = 8 * nt + 2 * t4 + (e & 1);
            if (R < 2 * Mp) {
                const int m = R >= Mp ? R - Mp : R, E = Es[m];
                const float x1 = ldexpf(acc[0][e], E - 10), x2 = ldexpf(acc[1][e], E - 21), x3 = ldexpf(acc[2][e], E - 32);
                float sh, sl;
                two_sum(x1, x2, sh, sl);
                W[R * kTcVs + col] = __fadd_rn(sh, __fadd_rn(sl, x3));
            }
        }
    }
    __syncthreads();
    for (int col = warp; col < nv; col += NW) {         // gamma = ||w||^2 over all rows, x = antenna rows / sqrt
        float gsum = 0.f;
        for (int R = lane; R < 2 * Mp; R += 32) gsum += W[R * kTcVs + col] * W[R * kTcVs + col];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
        const float rs = __frsqrt_rn(gsum);
        const int v = v0r + col;
        if (lane < M) xo[(size_t)v * M + lane] = make_float2(W[lane * kTcVs + col] * rs, W[(lane + Mp) * kTcVs + col] * rs);
        if (lane == 0) go[v] = gsum;
    }
    __syncthreads();                                   // the area and ust are reused by the next round
}

__host__ __device__ inline int take16(int& o, int bytes)
{
    const int r = o;
    o += (bytes + 15) & ~15;
    return r;
}


// Shared-memory layout of one search block (byte offsets, 16-byte aligned).
// The paths' codes and meta words are staged as well, unless gp (the block
// reads them in place from global memory, once per 32-path chunk; tc = meta
// = -1): the launch chooses gp when staging them would leave fewer than four
// blocks on an SM, the register limit of the launch bounds.
constexpr int kSearchSmemBudget = 57344;   // (228 KB per SM) / 4 - 1 KB reserved per block

struct SearchSmem {
    int ctab, utc, pt, ptl, ust, bvec, scr, tmq, pcode, lut, scrl, scrp, wv, ulv, tc, meta, total;
};

// tcp: the tensor-core product (u of a round staged in ust; the prefix-state
// area scr doubles as its work area after each round, sized for MPL rows of
// P), else the CUDA-core one (P staged in pt / ptl).
__host__ __device__ inline SearchSmem search_smem(int KT, int KM, int NP, int NW, bool gp, bool tcp = false, int MPL = 0)
{
    SearchSmem s;
    int o = 0;
    s.ctab = take16(o, 8 * ct_size(KT));
    s.utc = take16(o, 8 * KT * KT);
    s.pt = tcp ? -1 : take16(o, 8 * KM);
    s.ptl = tcp ? -1 : take16(o, 8 * KM);
    s.ust = tcp ? take16(o, 8 * kTcCols * KT) : -1;
    s.bvec = take16(o, 8 * NW * KT);
    s.scr = take16(o, tcp ? max(8 * NW * KT * kMaxPrefix, tc_area_bytes(KT, MPL)) : 8 * NW * KT * kMaxPrefix);
    s.tc = gp ? -1 : take16(o, 8 * NP);
    s.tmq = take16(o, 8 * n_chunks(NP));
    s.pcode = take16(o, 8 * kMaxPrefix);
    s.scrl = take16(o, 8 * NW * kMaxPrefix);
    s.scrp = take16(o, 4 * NW * kMaxPrefix);
    s.wv = take16(o, 4 * KT);
    s.ulv = take16(o, 4 * KT);
    s.meta = gp ? -1 : take16(o, 4 * NP);
    s.lut = take16(o, 8 * 72);
    s.total = o;
    return s;
}

// Per channel (block): path selection left the paths in evaluation order
// with their MoP rank (for tie-breaking) and shared-prefix index, the
// distinct prefixes of the top T <= 3 levels (<= 32 of them) and the digit
// maxima. Per vector the prefixes are evaluated once, one lane each, and
// their residuals, PED and chosen points stored in shared memory; every path
// then continues from its prefix's state through the remaining levels. The
// arithmetic per path is the same as a full descent, so results are
// identical; the shared levels are the ones with the most column updates.
template <int KT, bool BATCH, bool LUT, bool FIX, bool GP, bool TC>
__device__ __forceinline__ void search_block(const SearchArgs& a, int c, unsigned char* smraw)
{
    const int NW = blockDim.x >> 5;
    int K, M, Mp, n, nch, m_qam;
    float tau, inv_tau;
    int v0, v1;
    ChanState cs;
    const uint8_t* sym;
    float2* xo;
    int8_t* lo;
    float* go;
    if (BATCH) {
        const BatchProblem& p = a.probs[a.ids[c]];
        K = p.K; M = p.M; Mp = p.M; n = p.n; nch = n_chunks(p.n); m_qam = p.m_qam;
        tau = p.tau; inv_tau = 1.0f / p.tau;
        v0 = 0; v1 = p.S;
        cs = chan_state(p);
        sym = p.sym; xo = p.x; lo = p.l; go = p.gamma;
        if (threadIdx.x == 0 && p.status) p.status[0] = p.st[0];
    } else {
        K = a.K; M = a.M; Mp = a.Mp; n = a.n; nch = a.nch; m_qam = a.m_qam;
        tau = a.tau; inv_tau = a.inv_tau;
        if (a.off) {
            v0 = min(max(a.off[c], 0), a.n_vec);
            v1 = min(max(a.off[c + 1], v0), a.n_vec);
        } else {
            v0 = c * a.S;
            v1 = v0 + a.S;
        }
        cs = chan_state(a.d, (size_t)c, K, Mp, n);
        sym = a.sym; xo = a.x; lo = a.l; go = a.gamma;
    }
    const int KM = BATCH ? a.KM : K * Mp, NP = BATCH ? a.NP : n;
    const SearchSmem L = search_smem(KT, KM, NP, NW, GP, TC, Mp);
    float2* ctab = reinterpret_cast<float2*>(smraw + L.ctab);      // column table
    float2* utc = reinterpret_cast<float2*>(smraw + L.utc);        // [KT][KT]
    float2* pt = TC ? nullptr : reinterpret_cast<float2*>(smraw + L.pt);     // [K][M] leading part of P^T
    float2* ptl = TC ? nullptr : reinterpret_cast<float2*>(smraw + L.ptl);   // [K][M] trailing part
    float2* ust = TC ? reinterpret_cast<float2*>(smraw + L.ust) : nullptr;   // [kTcCols][KT] u of a round
    float2* bvec = reinterpret_cast<float2*>(smraw + L.bvec);      // [NW][KT]
    float2* scr_all = reinterpret_cast<float2*>(smraw + L.scr);    // [NW][KT][32] prefix residuals
    // [n] codes in evaluation order and their MoP rank | prefix << 16 (staged unless GP)
    uint64_t* tc = GP ? nullptr : reinterpret_cast<uint64_t*>(smraw + L.tc);
    uint32_t* meta = GP ? nullptr : reinterpret_cast<uint32_t*>(smraw + L.meta);
    uint64_t* tmq = reinterpret_cast<uint64_t*>(smraw + L.tmq);    // [nch] chunk digit maxima, evaluation order
    uint64_t* pcode = reinterpret_cast<uint64_t*>(smraw + L.pcode);// [32] a code of each prefix
    uint2* scrl_all = reinterpret_cast<uint2*>(smraw + L.scrl);    // [NW][32] prefix chosen points
    float* scrp_all = reinterpret_cast<float*>(smraw + L.scrp);    // [NW][32] prefix PED
    float* wv = reinterpret_cast<float*>(smraw + L.wv);            // [KT]
    int* ulv = reinterpret_cast<int*>(smraw + L.ulv);              // [KT]
    uint64_t* lut = reinterpret_cast<uint64_t*>(smraw + L.lut);    // [72] region lists (LUT DEMAP)
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

    const FixP fx = fix_params(FIX ? a.frac : 0);
    for (int i = threadIdx.x; i < KT * KT; i += blockDim.x) {
        const int r = i / KT, q = i % KT;
        const bool in = r < K && q < K;
        float2 uc = in ? cs.utc[r * K + q] : make_float2(0.f, 0.f);
        if (FIX) uc = make_float2(qword(uc.x, fx), qword(uc.y, fx));
        utc[i] = uc;
    }
    build_ctab<FIX>(ctab, cs.utp, K, fx);
    if (!TC) {
        for (int i = threadIdx.x; i < K * Mp; i += blockDim.x) {
            pt[i] = cs.pt[i];
            ptl[i] = cs.ptlo[i];
        }
    }
    // evaluation order, shared prefixes and chunk digit maxima (from path selection)
    if (!GP) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            tc[i] = cs.ecode[i];
            meta[i] = cs.emeta[i];
        }
    }
    for (int i = threadIdx.x; i < nch; i += blockDim.x) tmq[i] = cs.maxq[i];
    for (int i = threadIdx.x; i < kMaxPrefix; i += blockDim.x) pcode[i] = cs.pcode[i];
    for (int i = threadIdx.x; i < KT; i += blockDim.x) {
        wv[i] = i < K ? cs.w[i] * tau * tau : 0.f;   // w_l tau^2
        ulv[i] = i < K ? (int)cs.ul[i] : 0;
    }
    const int4 hdr = cs.phdr[0];
    const int T = (K == KT) ? hdr.x : 0;   // shared top levels (0 when K does not fill the tile)
    const int NPF = T > 0 ? hdr.y : 1;
    const uint64_t amq = (uint64_t)(uint32_t)hdr.z | ((uint64_t)(uint32_t)hdr.w << 32);
    if (T == 0 && threadIdx.x == 0) pcode[0] = 0ull;
    if (LUT) build_lut(lut);
    __syncthreads();

    float2* bw = bvec + warp * KT;
    float2* scr = scr_all + warp * KT * kMaxPrefix;
    float* scrp = scrp_all + warp * kMaxPrefix;
    uint2* scrl = scrl_all + warp * kMaxPrefix;
    const int KB = K - T;   // levels evaluated per path
    // One data vector on the warp: b', the shared prefixes, every path, the
    // (PED, rank) argmin against the zero candidate; writes l and returns u =
    // s + tau l in level order (lane k <-> level k, lanes >= K zero).
    auto search_vec = [&](int vh) -> float2 {
            // symbols in level order (lane k <-> level k) and b_k = s_k + sum_{m>k} U~_km s_m
            float2 s = make_float2(0.f, 0.f);
            if (lane < K) s = qam_point((int)sym[(size_t)vh * K + ulv[lane]], m_qam);
            float2 b = s;
            for (int m = 1; m < K; ++m) {
                const float2 sm = make_float2(__shfl_sync(kFull, s.x, m), __shfl_sync(kFull, s.y, m));
                if (lane < m) b = cfma(utc[m * KT + lane], sm, b);
            }
            // residuals are kept in units of tau: r' = r / tau is the effective point of Eq. (17)
            b = make_float2(b.x * inv_tau, b.y * inv_tau);
            if (FIX) b = make_float2(qword(b.x, fx), qword(b.y, fx));
            if (lane < KT) bw[lane] = (lane < K) ? b : make_float2(0.f, 0.f);
            float g0 = (lane < K) ? wv[lane] * cabs2(b) : 0.f;     // zero candidate: ||U s||^2
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) g0 += __shfl_xor_sync(kFull, g0, o);
            __syncwarp(kFull);

            // shared top levels, one lane per prefix (T = 0: lane 0 stores the root state)
            {
                const uint64_t code = lane < NPF ? pcode[lane] : 0ull;
                const uint32_t cw0 = (uint32_t)code, cw1 = (uint32_t)(code >> 32);
                float2 r[KT];
#pragma unroll
                for (int m = 0; m < KT; ++m) r[m] = bw[m];
                float ped = 0.f;
                uint32_t lc0 = 0, lc1 = 0;
                constexpr int kLo = KT >= 8 ? KT - kSplitMax : KT;   // no shared levels for small tiles
#pragma unroll
                for (int lv = KT - 1; lv >= kLo; --lv) {
                    if (lv >= KT - T)
                        level_step<KT, LUT, FIX>(lv, ctab, wv, cw0, cw1, (uint32_t)amq, (uint32_t)(amq >> 32), lut, fx,
                                                 r, ped, lc0, lc1);
                }
                if (lane < NPF) {
#pragma unroll
                    for (int m = 0; m < KT; ++m)
                        if (m < KB) scr[m * kMaxPrefix + lane] = r[m];
                    scrp[lane] = ped;
                    scrl[lane] = make_uint2(lc0, lc1);
                }
            }
            __syncwarp(kFull);

            float bp = INFINITY;
            int brk = 0x7fffffff;
            uint32_t blc0 = 0, blc1 = 0;
            for (int ch = 0; ch < nch; ++ch) {
                const int jp = ch * 32 + lane;
                const bool vld = jp < n;
                const uint64_t code = !vld ? 0ull : (GP ? __ldg(cs.ecode + jp) : tc[jp]);
                const uint32_t cw0 = (uint32_t)code, cw1 = (uint32_t)(code >> 32);
                const uint32_t mt = !vld ? 0u : (GP ? __ldg(cs.emeta + jp) : meta[jp]);
                const int rk = vld ? (int)(mt & 0xffffu) : 0x7fffffff;
                const int p = (int)(mt >> 16);
                const uint64_t mq = tmq[ch];
                float2 r[KT];
#pragma unroll
                for (int m = 0; m < KT; ++m) r[m] = (m < KB) ? scr[m * kMaxPrefix + p] : make_float2(0.f, 0.f);
                float ped = scrp[p];
                const uint2 lcp = scrl[p];
                uint32_t lc0 = lcp.x, lc1 = lcp.y;
#pragma unroll
                for (int lv = KT - 1; lv >= 0; --lv) {
                    if (lv < KB)
                        level_step<KT, LUT, FIX>(lv, ctab, wv, cw0, cw1, (uint32_t)mq, (uint32_t)(mq >> 32), lut, fx,
                                                 r, ped, lc0, lc1);
                }
                if (vld && (ped < bp || (ped == bp && rk < brk))) { bp = ped; brk = rk; blc0 = lc0; blc1 = lc1; }
            }
            // (PED, rank) minimum over the warp; candidate index = rank + 1
            float wbp = bp;
            int wbr = brk;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const float obp = __shfl_xor_sync(kFull, wbp, o);
                const int obr = __shfl_xor_sync(kFull, wbr, o);
                if (obp < wbp || (obp == wbp && obr < wbr)) { wbp = obp; wbr = obr; }
            }
            const bool zero_wins = !(wbp < g0);
            const unsigned who = __ballot_sync(kFull, bp == wbp && brk == wbr);
            const int src = (zero_wins || who == 0u) ? 0 : (__ffs(who) - 1);
            uint32_t w0 = __shfl_sync(kFull, blc0, src), w1 = __shfl_sync(kFull, blc1, src);
            if (zero_wins) { w0 = 0x55555555u; w1 = 0x55555555u; }

            // l (user order) and u = s + tau l = s - tau t in level order
            float2 u = make_float2(0.f, 0.f);
            if (lane < K) {
                const int nib = (int)(((lane < 8 ? w0 : w1) >> (4 * (lane & 7))) & 15u);
                const int tr = (nib & 3) - 1, ti = (nib >> 2) - 1;
                u = make_float2(s.x - (float)tr * tau, s.y - (float)ti * tau);
                const int usr = ulv[lane];
                lo[((size_t)vh * K + usr) * 2] = (int8_t)(-tr);
                lo[((size_t)vh * K + usr) * 2 + 1] = (int8_t)(-ti);
            }
            return u;
    };

    if constexpr (TC) {
        // rounds of kTcCols vectors: the warp searches v, v + NW, ... of the
        // round, then the block forms w = P u for the round (tc_round)
        for (int r0 = v0; r0 < v1; r0 += kTcCols) {
            const int rend = min(r0 + kTcCols, v1);
#pragma unroll 1
            for (int vh = r0 + warp; vh < rend; vh += NW) {
                const float2 u = search_vec(vh);
                if (lane < KT) ust[(vh - r0) * KT + lane] = u;
                __syncwarp(kFull);
            }
            tc_round(cs.pt, cs.ptlo, ulv, ust, KT, K, M, Mp, r0, rend - r0, reinterpret_cast<float*>(smraw + L.scr), xo,
                     go);
        }
    } else {
        // The warp takes its vectors in pairs (v, v + NW): both are searched in
        // turn, then one pass forms y = P u for both, one half-warp each (when
        // the Mp rows fit 16 lanes; else each vector gets a whole-warp pass).
        const bool pair_rows = Mp <= 16;
        for (int v = v0 + warp; v < v1; v += 2 * NW) {
            float2 upk = make_float2(0.f, 0.f);   // u of the pair: lanes 0-15 levels of v, lanes 16-31 of v + NW
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const int vh = v + h * NW;
                if (vh >= v1) break;
                const float2 u = search_vec(vh);
                if (pair_rows) {
                    const float ux = __shfl_sync(kFull, u.x, lane & 15), uy = __shfl_sync(kFull, u.y, lane & 15);
                    if ((lane >> 4) == h) upk = make_float2(ux, uy);
                    __syncwarp(kFull);
                    continue;
                }
                // y = P u with P = pt + ptl, all Mp rows on the warp
                float yr = 0.f, yre = 0.f, yi = 0.f, yie = 0.f;
                for (int lv = 0; lv < K; ++lv) {
                    const float ur = __shfl_sync(kFull, u.x, lv), ui = __shfl_sync(kFull, u.y, lv);
                    if (lane < Mp) py_acc(pt, ptl, ulv[lv] * Mp + lane, ur, ui, yr, yre, yi, yie);
                }
                const float2 y = make_float2(__fadd_rn(yr, yre), __fadd_rn(yi, yie));
                float g = (lane < Mp) ? cabs2(y) : 0.f;     // ||w||^2 over all rows (Alg. 2's d)
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) g += __shfl_xor_sync(kFull, g, o);
                const float rs = __frsqrt_rn(g);
                if (lane < M) xo[(size_t)vh * M + lane] = make_float2(y.x * rs, y.y * rs);
                if (lane == 0) go[vh] = g;
                __syncwarp(kFull);
            }
            if (pair_rows) pair_rows_out(pt, ptl, ulv, upk, K, M, Mp, v, v + NW, v1, xo, go);
        }
    }
}

template <int KT, bool BATCH, bool LUT, bool FIX, bool GP, bool TC>
__global__ void __launch_bounds__(224, 4) search_kernel(SearchArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_wait();                                // paths and factors of the kernels before
    search_block<KT, BATCH, LUT, FIX, GP, TC>(a, blockIdx.x, smraw);
    pdl_trigger();
}

// One problem of a persistent launch, as its own function (each K tile keeps
// the register allocation of its plain kernel; the call is once per problem).
template <int KT, bool GP>
__device__ __noinline__ void search_item(const SearchArgs& a, int c, unsigned char* smraw)
{
    search_block<KT, true, false, false, GP, false>(a, c, smraw);
}

// Uneven batches in one persistent launch: resident blocks take problems
// from a device counter in the order of a.ids (heaviest first, all K tiles
// mixed), each with the search body of its K tile; the shared-memory layout
// of every tile fits the launch's (sized for the largest). GP16: the 16-level
// tile reads the path codes in place.
template <bool GP16>
__global__ void __launch_bounds__(224, 4) search_persist_kernel(SearchArgs a, int* counter)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int item;
    pdl_wait();
    pdl_trigger();
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(counter, 1);
        __syncthreads();
        const int c = item;
        __syncthreads();                     // every thread has read the item (and left the last one's smem)
        if (c >= a.C) break;
        switch (search_tile(a.probs[a.ids[c]].K)) {
        case 2: search_item<2, false>(a, c, smraw); break;
        case 4: search_item<4, false>(a, c, smraw); break;
        case 8: search_item<8, false>(a, c, smraw); break;
        case 12: search_item<12, false>(a, c, smraw); break;
        default: search_item<16, GP16>(a, c, smraw); break;
        }
    }
}

// Shared-memory layout of the one-pass search (byte offsets, 16-byte aligned).
struct SmallSmem {
    int ctab, utc, pt, ptl, tc, meta, wv, ulv, bw, sv, g0, wins, total;
};

__host__ __device__ inline SmallSmem small_smem(int KT, int KM, int NW, int G)
{
    SmallSmem s;
    int o = 0;
    s.ctab = take16(o, 8 * ct_size(KT));
    s.utc = take16(o, 8 * KT * KT);
    s.pt = take16(o, 8 * KM);
    s.ptl = take16(o, 8 * KM);
    s.tc = take16(o, 8 * 32);
    s.meta = take16(o, 4 * 32);
    s.wv = take16(o, 4 * KT);
    s.ulv = take16(o, 4 * KT);
    s.bw = take16(o, 8 * NW * G * KT);
    s.sv = take16(o, 8 * NW * G * KT);
    s.g0 = take16(o, 4 * NW * G);
    s.wins = take16(o, 8 * NW * G);
    s.total = o;
    return s;
}

// The search for path budgets of one pass (n <= 32 / G): G data vectors per
// warp, P = 32 / G lanes each (lane g P + p: vector g, path p), so that small
// budgets keep the lanes busy. The arithmetic per path and the (PED, rank)
// argmin are those of search_kernel, which shares no levels when n <= 32,
// and y = P u takes the same paired half-warp pass: the outputs are the same.
template <int KT, int G>
__global__ void __launch_bounds__(224, 4) search_small_kernel(SearchArgs a)
{
    constexpr int P = 32 / G;
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_wait();
    pdl_trigger();
    const int NW = blockDim.x >> 5;
    const int c = blockIdx.x;
    const int K = a.K, M = a.M, Mp = a.Mp, n = a.n, m_qam = a.m_qam;
    const float tau = a.tau, inv_tau = a.inv_tau;
    int v0, v1;
    if (a.off) {
        v0 = min(max(a.off[c], 0), a.n_vec);
        v1 = min(max(a.off[c + 1], v0), a.n_vec);
    } else {
        v0 = c * a.S;
        v1 = v0 + a.S;
    }
    const ChanState cs = chan_state(a.d, (size_t)c, K, Mp, n);
    const uint8_t* sym = a.sym;
    float2* xo = a.x;
    int8_t* lo = a.l;
    float* go = a.gamma;
    const SmallSmem L = small_smem(KT, K * Mp, NW, G);
    float2* ctab = reinterpret_cast<float2*>(smraw + L.ctab);      // column table
    float2* utc = reinterpret_cast<float2*>(smraw + L.utc);        // [KT][KT]
    float2* pt = reinterpret_cast<float2*>(smraw + L.pt);          // [K][Mp]
    float2* ptl = reinterpret_cast<float2*>(smraw + L.ptl);
    uint64_t* tc = reinterpret_cast<uint64_t*>(smraw + L.tc);      // [n] codes
    uint32_t* meta = reinterpret_cast<uint32_t*>(smraw + L.meta);  // [n] MoP rank
    float* wv = reinterpret_cast<float*>(smraw + L.wv);            // [KT]
    int* ulv = reinterpret_cast<int*>(smraw + L.ulv);              // [KT]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* bw = reinterpret_cast<float2*>(smraw + L.bw) + warp * G * KT;   // [G][KT] b' of the warp's vectors
    float2* sv = reinterpret_cast<float2*>(smraw + L.sv) + warp * G * KT;   // [G][KT] their symbols
    float* g0s = reinterpret_cast<float*>(smraw + L.g0) + warp * G;         // [G] zero candidates
    uint2* wins = reinterpret_cast<uint2*>(smraw + L.wins) + warp * G;      // [G] chosen points

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
        utc[i] = in ? cs.utc[r * K + q] : make_float2(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < K * Mp; i += blockDim.x) {
        pt[i] = cs.pt[i];
        ptl[i] = cs.ptlo[i];
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tc[i] = cs.ecode[i];
        meta[i] = cs.emeta[i];
    }
    for (int i = threadIdx.x; i < KT; i += blockDim.x) {
        wv[i] = i < K ? cs.w[i] * tau * tau : 0.f;   // w_l tau^2
        ulv[i] = i < K ? (int)cs.ul[i] : 0;
    }
    const uint64_t mq = cs.maxq[0];                   // one chunk: digit maxima of all paths
    const FixP fx = FixP();
    build_ctab<false>(ctab, cs.utp, K, fx);
    __syncthreads();

    const int g = lane / P, p = lane % P;
    for (int vb = v0 + warp * G; vb < v1; vb += NW * G) {
        // b' and the zero candidate of each vector (lane k <-> level k)
#pragma unroll 1
        for (int h = 0; h < G; ++h) {
            const int vh = vb + h;
            if (vh >= v1) break;
            float2 s = make_float2(0.f, 0.f);
            if (lane < K) s = qam_point((int)sym[(size_t)vh * K + ulv[lane]], m_qam);
            float2 b = s;
            for (int m = 1; m < K; ++m) {
                const float2 sm = make_float2(__shfl_sync(kFull, s.x, m), __shfl_sync(kFull, s.y, m));
                if (lane < m) b = cfma(utc[m * KT + lane], sm, b);
            }
            b = make_float2(b.x * inv_tau, b.y * inv_tau);
            if (lane < KT) {
                bw[h * KT + lane] = (lane < K) ? b : make_float2(0.f, 0.f);
                sv[h * KT + lane] = s;
            }
            float g0 = (lane < K) ? wv[lane] * cabs2(b) : 0.f;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) g0 += __shfl_xor_sync(kFull, g0, o);
            if (lane == 0) g0s[h] = g0;
        }
        __syncwarp(kFull);

        // every path of every vector: lane (g, p)
        const int vg = vb + g;
        const bool vld = vg < v1 && p < n;
        const uint64_t code = vld ? tc[p] : 0ull;
        const uint32_t cw0 = (uint32_t)code, cw1 = (uint32_t)(code >> 32);
        const int rk = vld ? (int)(meta[p] & 0xffffu) : 0x7fffffff;
        float2 r[KT];
#pragma unroll
        for (int m = 0; m < KT; ++m) r[m] = bw[g * KT + m];
        float ped = 0.f;
        uint32_t lc0 = 0, lc1 = 0;
#pragma unroll
        for (int lv = KT - 1; lv >= 0; --lv) {
            if (lv < K)
                level_step<KT, false, false>(lv, ctab, wv, cw0, cw1, (uint32_t)mq, (uint32_t)(mq >> 32), nullptr, fx,
                                             r, ped, lc0, lc1);
        }
        const float bp = vld ? ped : INFINITY;
        const int brk = rk;
        float wbp = bp;
        int wbr = brk;
#pragma unroll
        for (int o = P / 2; o >= 1; o >>= 1) {
            const float obp = __shfl_xor_sync(kFull, wbp, o);
            const int obr = __shfl_xor_sync(kFull, wbr, o);
            if (obp < wbp || (obp == wbp && obr < wbr)) { wbp = obp; wbr = obr; }
        }
        const bool zero_wins = !(wbp < g0s[g]);
        const unsigned gmask = (P == 32) ? kFull : (((1u << P) - 1u) << (g * P));
        const unsigned who = __ballot_sync(kFull, bp == wbp && brk == wbr) & gmask;
        const int src = (zero_wins || who == 0u) ? g * P : (__ffs(who) - 1);
        uint32_t w0 = __shfl_sync(kFull, lc0, src), w1 = __shfl_sync(kFull, lc1, src);
        if (zero_wins) { w0 = 0x55555555u; w1 = 0x55555555u; }
        if (p == 0) wins[g] = make_uint2(w0, w1);
        __syncwarp(kFull);

        // l, u and y = P u, two vectors per pass
#pragma unroll 1
        for (int h0 = 0; h0 < G; h0 += 2) {
            if (vb + h0 >= v1) break;
            float2 upk = make_float2(0.f, 0.f);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int h = h0 + hh, vh = vb + h;
                if (vh >= v1) break;
                const uint2 wn = wins[h];
                float2 u = make_float2(0.f, 0.f);
                if (lane < K) {
                    const int nib = (int)(((lane < 8 ? wn.x : wn.y) >> (4 * (lane & 7))) & 15u);
                    const int tr = (nib & 3) - 1, ti = (nib >> 2) - 1;
                    const float2 s = sv[h * KT + lane];
                    u = make_float2(s.x - (float)tr * tau, s.y - (float)ti * tau);
                    const int usr = ulv[lane];
                    lo[((size_t)vh * K + usr) * 2] = (int8_t)(-tr);
                    lo[((size_t)vh * K + usr) * 2 + 1] = (int8_t)(-ti);
                }
                const float ux = __shfl_sync(kFull, u.x, lane & 15), uy = __shfl_sync(kFull, u.y, lane & 15);
                if ((lane >> 4) == hh) upk = make_float2(ux, uy);
            }
            pair_rows_out(pt, ptl, ulv, upk, K, M, Mp, vb + h0, vb + h0 + 1, v1, xo, go);
        }
    }
}

template <int KT, int G>
cudaError_t launch_small(const SearchArgs& a, int C, int per, cudaStream_t s)
{
    int nw = (per + G - 1) / G;
    nw = nw < 1 ? 1 : (nw > 7 ? 7 : nw);
    const size_t sh = (size_t)small_smem(KT, a.K * a.Mp, nw, G).total;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(search_small_kernel<KT, G>), sh);
    if (e != cudaSuccess) return e;
    return launch_dependent(search_small_kernel<KT, G>, dim3(C), dim3(nw * 32), sh, s, a);
}

template <int KT>
cudaError_t launch_small_kt(const SearchArgs& a, int C, int per, cudaStream_t s)
{
    if (a.n <= 4) return launch_small<KT, 8>(a, C, per, s);
    if (a.n <= 8) return launch_small<KT, 4>(a, C, per, s);
    return launch_small<KT, 2>(a, C, per, s);
}

template <int KT, bool BATCH, bool LUT, bool FIX, bool GP, bool TC = false>
cudaError_t launch_one(const SearchArgs& a, int C, int threads, int KM, int NP, cudaStream_t s)
{
    const size_t sh = (size_t)search_smem(KT, KM, NP, threads / 32, GP, TC, a.Mp).total;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(search_kernel<KT, BATCH, LUT, FIX, GP, TC>), sh);
    if (e != cudaSuccess) return e;
    return launch_dependent(search_kernel<KT, BATCH, LUT, FIX, GP, TC>, dim3(C), dim3(threads), sh, s, a);
}

// Paths read in place (GP) where staging them would cost occupancy: only the
// 16-level tile can get there (n up to 1024, or P with the K rows of
// lambda > 0), and only its plain and batch forms have the GP variant; the
// study variants keep the staged layout with fewer blocks per SM.
template <int KT, bool BATCH, bool LUT, bool FIX>
cudaError_t launch_gp(const SearchArgs& a, int C, int threads, int KM, int NP, cudaStream_t s)
{
    if constexpr (KT == 16 && !LUT && !FIX) {
        if (search_smem(KT, KM, NP, threads / 32, false).total > kSearchSmemBudget)
            return launch_one<KT, BATCH, LUT, FIX, true>(a, C, threads, KM, NP, s);
    }
    return launch_one<KT, BATCH, LUT, FIX, false>(a, C, threads, KM, NP, s);
}

template <int KT>
cudaError_t launch_kt(const SearchArgs& a, int C, int threads, cudaStream_t s)
{
    const int KM = a.probs ? a.KM : a.K * a.Mp, NP = a.probs ? a.NP : a.n;
    if (a.probs) return launch_gp<KT, true, false, false>(a, C, threads, KM, NP, s);
    if (a.frac > 0) return launch_gp<KT, false, false, true>(a, C, threads, KM, NP, s);
    if (a.demap == VP_DEMAP_LUT) return launch_gp<KT, false, true, false>(a, C, threads, KM, NP, s);
    if (a.tcp) {
        if (search_smem(KT, KM, NP, threads / 32, false, true, a.Mp).total > kSearchSmemBudget)
            return launch_one<KT, false, false, false, true, true>(a, C, threads, KM, NP, s);
        return launch_one<KT, false, false, false, false, true>(a, C, threads, KM, NP, s);
    }
    return launch_gp<KT, false, false, false>(a, C, threads, KM, NP, s);
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
    a.Mp = p_rows(p);
    a.demap = p->demap;
    a.frac = p->frac_bits;
    a.tcp = (p->tensor_product && p->demap == VP_DEMAP_EXACT && p->frac_bits == 0) ? 1 : 0;
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
    // budgets of 16 paths or fewer: several vectors per warp (same results)
    if (a.n <= 16 && a.Mp <= 16 && a.demap == VP_DEMAP_EXACT && a.frac == 0 && !a.tcp && per >= 2) {
        if (K <= 2) return launch_small_kt<2>(a, p->C, per, s);
        if (K <= 4) return launch_small_kt<4>(a, p->C, per, s);
        if (K <= 8) return launch_small_kt<8>(a, p->C, per, s);
        if (K <= 12) return launch_small_kt<12>(a, p->C, per, s);
        return launch_small_kt<16>(a, p->C, per, s);
    }
    if (K <= 2) return launch_kt<2>(a, p->C, threads, s);
    if (K <= 4) return launch_kt<4>(a, p->C, threads, s);
    if (K <= 8) return launch_kt<8>(a, p->C, threads, s);
    if (K <= 12) return launch_kt<12>(a, p->C, threads, s);
    return launch_kt<16>(a, p->C, threads, s);
}

cudaError_t launch_search_persist(const BatchProblem* probs, const int* ids, int count, int km_max, int n_max,
                                  int s_max, int* counter, cudaStream_t s, int nw_set, int blocks_per_sm, int stage16)
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
    if (nw_set >= 1 && nw_set <= 7) nw = nw_set;
    // the 16-level tile stages its path codes (stage16 = 1), reads them in
    // place (2), or decides by the budget of four blocks per SM (0)
    bool gp16 = search_smem(16, km_max, n_max, nw, false).total > kSearchSmemBudget;
    if (stage16 == 1) gp16 = false;
    if (stage16 == 2) gp16 = true;
    int sh = search_smem(16, km_max, n_max, nw, gp16).total;
    for (int kt : {2, 4, 8, 12}) sh = max(sh, search_smem(kt, km_max, n_max, nw, false).total);
    const void* fn = gp16 ? reinterpret_cast<const void*>(search_persist_kernel<true>)
                          : reinterpret_cast<const void*>(search_persist_kernel<false>);
    cudaError_t e = allow_dynamic_smem(fn, (size_t)sh);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nw * 32, (size_t)sh)) != cudaSuccess) return e;
    if (blocks_per_sm >= 1 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    int grid = sms * (per_sm < 1 ? 1 : per_sm);
    if (grid > count) grid = count;
    if (grid < 1) return cudaSuccess;
    if (gp16) search_persist_kernel<true><<<grid, nw * 32, sh, s>>>(a, counter);
    else search_persist_kernel<false><<<grid, nw * 32, sh, s>>>(a, counter);
    return cudaGetLastError();
}

cudaError_t launch_search_batch(const BatchProblem* probs, const int* ids, int count, int KT, int km_max,
                                int n_max, int s_max, cudaStream_t s, int nw_set)
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
    if (nw_set >= 1 && nw_set <= 7) nw = nw_set;
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
