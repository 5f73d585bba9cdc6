// DEMAP selection and the column table shared by the search kernels (GPU
// side only; never included by the oracle). Section III-A-2 and Alg. 2:
// the p_l-th nearest point of the bounded alphabet {-1,0,1}+j{-1,0,1} around
// the effective point of Eq. (17), and the column updates of the descent.
#pragma once

#include "vp_internal.cuh"

namespace vp {
namespace {

// Fixed-point parameters of a launch: the word scale 2^F and its inverse, the
// saturation bound 32767 2^-F and the DEMAP tie shift.
struct FixP {
    float scale, inv_scale, lim, epsx, epsy;
};

__device__ __forceinline__ FixP fix_params(int F)
{
    FixP f;
    f.scale = __int_as_float((127 + F) << 23);
    f.inv_scale = __int_as_float((127 - F) << 23);
    f.lim = 32767.f * f.inv_scale;
    f.epsx = __int_as_float((127 - F - 2) << 23);    // 2^-(F+2)
    f.epsy = __int_as_float((127 - F - 4) << 23);    // 2^-(F+4)
    return f;
}

// a real value as a word: round half to even, saturate
__device__ __forceinline__ float qword(float v, const FixP& f)
{
    return fminf(fmaxf(rintf(v * f.scale), -32767.f), 32767.f) * f.inv_scale;
}

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
// Per axis the points in increasing distance are n_0, n_1, n_2, and their
// squared distances exceed that of n_0 by 0, D1 = |1 - 2|x||,
// D2 = max(1 + 2|x|, 4|x|). The 9
// points form a 3x3 table of sums Dx_i + Dy_j (cell (i, j) = (n_i(x), n_j(y))).
// Against the origin cell the 8 others are
//   A=(1,0): D1x  B=(0,1): D1y  C=(2,0): D2x  D=(0,2): D2y  E=(1,1): D1x+D1y
//   F=(1,2): D1x+D2y  G=(2,1): D2x+D1y  H=(2,2): largest,
// and every pair not ordered by the table's structure is one of
//   f0 A<B, f1 C<B, f2 A<D, f3 C<D, f4 E<C, f5 E<D, f6 F<C, f7 G<D, f8 F<G,
// so the rank of each cell is a short sum of these bits.
//
// In the fixed-point search every centre is a multiple of 2^-F and may reach
// 32767 2^-F, where 2^-23 is below the spacing of floats; there the shift is
// (2^-(F+2), 2^-(F+4)): distinct squared distances of such centres differ by
// at least 2^(1-F), the shift moves a difference by at most 1.25 2^-F, and it
// still orders ties by (tr, ti) since eps_x > 2 eps_y. The shifted centre and
// every gap below keep <= 21 significant bits, so all of it is exact in FP32.
constexpr float kEpsX = 0x1p-23f;
constexpr float kEpsY = 0x1p-25f;
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

// Cell (ci | cj << 2) of rank q at the shifted point (px, py) for a warp whose
// largest q at this level (`mq`, uniform) is >= 1; the branch on mq picks the
// cheapest form that is exact for every lane. Out of line on purpose: the
// level bodies are unrolled 16 times, and keeping these rarer branches out
// of them keeps the kernel's hot code within the instruction cache (inlined,
// the search ran 9% slower on GB300).
__device__ __noinline__ int select_cell(float px, float py, int q, int mq)
{
    const float D1x = gap1(px), D1y = gap1(py);
    const bool f0 = D1x < D1y;                                        // rank 1: A (step in x) or B
    int ci, cj;
    if (mq == 1) {
        ci = (q == 1 && f0) ? 1 : 0;
        cj = (q == 1 && !f0) ? 1 : 0;
    } else {
        const float D2x = gap2(px), D2y = gap2(py);
        if (mq == 2) {
            const bool g = f0 ? (D1y < D2x) : (D1x < D2y);            // rank 2: the other of A/B, or C / D
            const int c2i = f0 ? (g ? 0 : 2) : (g ? 1 : 0);
            const int c2j = f0 ? (g ? 1 : 0) : (g ? 0 : 2);
            ci = q == 0 ? 0 : (q == 1 ? (f0 ? 1 : 0) : c2i);
            cj = q == 0 ? 0 : (q == 1 ? (f0 ? 0 : 1) : c2j);
        } else {
            rank_cell(D1x, D2x, D1y, D2y, q, ci, cj);
            if (q == 0) { ci = 0; cj = 0; }
        }
    }
    return ci | (cj << 2);
}

// Nearest-point thresholds of the exact DEMAP: comparing x - 2^-23 with
// +-1/2 (the tie shift above) is the same as comparing x with 1/2 + 2^-23
// and -1/2 + 2^-23; for y - 2^-25 (rounded) the equivalent thresholds are
// 1/2 + 2^-24 and -1/2 + 2^-25 (checked for every float in [-2.5, -0.2] and
// [0.2, 2.5]; outside, both sides agree trivially). The nearest point then
// needs no shifted coordinates.
constexpr float kT1x = 0.5f + 0x1p-23f, kT2x = -0.5f + 0x1p-23f;
constexpr float kT1y = 0.5f + 0x1p-24f, kT2y = -0.5f + 0x1p-25f;

// t for the digit of this level (4 bits at `sh` of the code word cw) at the
// effective point (cx, cy); `mq` = the warp's largest digit at this level
// (uniform): 0 needs only the nearest point, and the digit is read only
// otherwise. The cells are chosen per axis among n0 (the clamped rounding),
// s - n0 and -s, s = +1 for x > 0 else -1 (the three points of {-1, 0, 1}
// sum to zero). SHIFTED: the exact float DEMAP with the tie shift (kEpsX,
// kEpsY) folded into the nearest-point thresholds; otherwise the shift
// (epsx, epsy) of the fixed-point search.
template <bool SHIFTED>
__device__ __forceinline__ void select_point(float cx, float cy, uint32_t cw, int sh, int mq, int& tr, int& ti,
                                             float epsx, float epsy)
{
    int n0x, n0y;
    if (SHIFTED) {
        n0x = (cx > kT1x) - (cx <= kT2x);
        n0y = (cy > kT1y) - (cy <= kT2y);
    } else {
        const float qx = cx - epsx, qy = cy - epsy;
        n0x = (qx > 0.5f) - (qx <= -0.5f);
        n0y = (qy > 0.5f) - (qy <= -0.5f);
    }
    if (mq == 0) {
        tr = n0x;
        ti = n0y;
        return;
    }
    const int q = (int)(cw >> sh) & 15;
    const float px = cx - epsx, py = cy - epsy;
    const int cc = select_cell(px, py, q, mq);
    const int ci = cc & 3, cj = cc >> 2;
    const int sx = px > 0.f ? 1 : -1, sy = py > 0.f ? 1 : -1;
    tr = ci == 0 ? n0x : (ci == 1 ? sx - n0x : -sx);
    ti = cj == 0 ? n0y : (cj == 1 ? sy - n0y : -sy);
}

// Region-LUT DEMAP: nearest alphabet point n0 (clamped rounding, halves to
// the smaller value) and the octant of d = c - n0 pick one of 72 regions; the
// region's list (9 alphabet indices, 4 bits each) is the exact distance order
// from the octant centroid, built once per block by build_lut.
__device__ __forceinline__ void select_lut(float cx, float cy, int q, const uint64_t* lut, int& tr, int& ti)
{
    const int nx = (cx > 0.5f) - (cx <= -0.5f), ny = (cy > 0.5f) - (cy <= -0.5f);
    const float dx = cx - (float)nx, dy = cy - (float)ny;
    const int oct = (dx > 0.f) | ((dy > 0.f) << 1) | ((fabsf(dx) > fabsf(dy)) << 2);
    const int a = (int)(lut[((nx + 1) * 3 + (ny + 1)) * 8 + oct] >> (4 * q)) & 15;
    tr = ((a * 11) >> 5) - 1;                        // a / 3 for a <= 8
    ti = a - 3 * (tr + 1) - 1;
}

// The 72 region lists: distances from the octant centroid n0 + (+-1/3, +-1/6)
// (|d.re| > |d.im|) or n0 + (+-1/6, +-1/3), compared exactly in sixths, ties to
// the smaller alphabet index a = 3 (tr + 1) + (ti + 1).
__device__ void build_lut(uint64_t* lut)
{
    for (int rg = threadIdx.x; rg < 72; rg += blockDim.x) {
        const int cell = rg >> 3, oct = rg & 7;
        const int cx = 6 * (cell / 3 - 1) + ((oct & 1) ? 1 : -1) * ((oct & 4) ? 2 : 1);
        const int cy = 6 * (cell % 3 - 1) + ((oct & 2) ? 1 : -1) * ((oct & 4) ? 1 : 2);
        int key[9];
        for (int a = 0; a < 9; ++a) {
            const int ex = 6 * (a / 3 - 1) - cx, ey = 6 * (a % 3 - 1) - cy;
            key[a] = (ex * ex + ey * ey) * 16 + a;          // distance, then index
        }
        uint64_t word = 0;
        for (int q = 0; q < 9; ++q) {                       // q-th smallest key
            int best = 0x7fffffff;
            for (int a = 0; a < 9; ++a) {
                int rankless = 0;
                for (int b = 0; b < 9; ++b) rankless += key[b] < key[a];
                if (rankless == q) best = a;
            }
            word |= (uint64_t)best << (4 * q);
        }
        lut[rg] = word;
    }
}

// Column table of the descent. The column update r'_m -= U~_m,lv t has only
// nine possible right-hand sides per (m, lv), one per alphabet point t, so
// each block tabulates them once: entry (lv, k, m) = -U~_m,lv t for the 4-bit
// point code k = (Re t + 1) | (Im t + 1) << 2 (the code recorded for the
// path; 0..10, 3 and 7 unused) and m < lv, and entry (lv, k, lv) = -t itself
// (for the PED's r'_lv - t). A lane's update is then one shared load and one
// packed add per row, the load's address depending on its own t. Row stride
// (lv + 1) | 1 (odd, in float2 units): the nine codes of a warp then fall on
// distinct bank pairs (k * stride mod 16 differs for distinct k < 16).
__host__ __device__ constexpr int ct_stride(int lv) { return (lv + 1) | 1; }
__host__ __device__ constexpr int ct_off(int lv)
{
    int o = 0;
    for (int j = 0; j < lv; ++j) o += 11 * ct_stride(j);
    return o;
}
__host__ __device__ constexpr int ct_size(int KT) { return ct_off(KT); }   // float2 entries, levels 0..KT-1

// Fills the block's column table from U~ as (re, im, im, re)-packed float4
// [K][K] (level order): one pass over U~, a thread per entry above the
// diagonal writing its nine codes, then the points -t at m = lv. Only those
// entries are ever read (valid codes, m <= lv < K). FIX rounds the entries of
// U~ to words first, so a table entry (the sum of two words) is exact.
template <bool FIX>
__device__ void build_ctab(float2* ctab, const float4* utp_g, int K, const FixP& fx)
{
    for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
        const int m = i / K, lv = i - m * K;
        if (m >= lv) continue;
        float4 u = utp_g[i];
        if (FIX) u = make_float4(qword(u.x, fx), qword(u.y, fx), qword(u.z, fx), qword(u.w, fx));
        float2* e = ctab + ct_off(lv) + m;
        const int st = ct_stride(lv);
#pragma unroll
        for (int a = 0; a < 9; ++a) {                  // alphabet point a = 3 (tr + 1) + (ti + 1)
            const float tr = (float)(a / 3 - 1), ti = (float)(a % 3 - 1);
            const int k = (a / 3) | ((a % 3) << 2);
            e[k * st] = make_float2(fmaf(u.z, ti, -tr * u.x), fmaf(u.w, -ti, -tr * u.y));
        }
    }
    for (int i = threadIdx.x; i < 9 * K; i += blockDim.x) {   // -t itself, at m = lv
        const int lv = i / 9, a = i - 9 * lv;
        const int k = (a / 3) | ((a % 3) << 2);
        ctab[ct_off(lv) + k * ct_stride(lv) + lv] = make_float2((float)(1 - a / 3), (float)(1 - a % 3));
    }
}

}  // namespace
}  // namespace vp
