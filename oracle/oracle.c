/*
 * FP64 CPU oracle of the ViPer NL-COMM vector-perturbation precoder.
 *
 * TEST INFRASTRUCTURE ONLY: slow, plain and written to be checked against the
 * paper by eye. Nothing here is shared with the CUDA library; only the tests,
 * the smoke check and the benchmark's CPU-baseline / reference legs load it.
 *
 * Every function cites the part of the paper it restates. Readings of points
 * where the paper is silent or garbled are marked "Reading:".
 *
 * Parity pins: every function below is pinned by the CPU test-suite
 * (tests/test_oracle_*.py) against brute force, closed forms, textbook
 * routines or hand-derived golden values. The one exception is the rate
 * comparison with the paper's own BER/SER curves, which the paper prints
 * only as images: that part is "parity unpinned".
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

static cplx ld(const double* p, int i) { return p[2 * i] + I * p[2 * i + 1]; }
static void st(double* p, int i, cplx z) { p[2 * i] = creal(z); p[2 * i + 1] = cimag(z); }

/* ------------------------------------------------------------------------ */
/* QAM constellation (Section II). Reading: odd-integer grid with spacing 2,
 * index -> point as documented in oracle.h; tau = 2*sqrt(qam) is the usual
 * perturbation interval for this grid (the paper fixes tau per QAM order
 * without printing it). */
void orc_qam_point(int qam, int idx, double* re, double* im)
{
    int m = 1;
    while (m * m < qam) m++;
    *re = 2.0 * (idx % m) - (m - 1);
    *im = 2.0 * (idx / m) - (m - 1);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (ISRQD) on Hbar = [H lambda*I] (Section III-A-1), followed by
 * the index reversal of Section IV-B.
 *
 * Alg. 1 works on the rows of Qbar (initialised to Hbar). At position i it
 * takes the remaining row with the smallest squared norm, swaps it into
 * place, sets Rbar_ii to that norm's square root and projects it out of all
 * later rows, which gives a LOWER-triangular Rbar in pick order
 * (Hbar_perm = Rbar * Qbar).
 * Readings:
 *  - the pseudocode never divides q_i by Rbar_ii although the norm update
 *    norm_j -= |Rbar_ji|^2 needs unit q_i: q_i is normalised here;
 *  - "argmin over j = 1..N_R" is read as over the rows not yet picked, ties
 *    going to the smallest original user index;
 *  - the squared norms are recomputed from the rows at every step (the
 *    quantity the pseudocode's downdate tracks), to keep FP64 accuracy for
 *    ill-conditioned H;
 *  - the index reversal of Section IV-B maps pick position i to tree level
 *    K-1-i, giving an upper-triangular R with the first-picked (weakest) row
 *    at the last level, which the tree search visits first. */
int orc_isrqd(int K, int M, const double* H, double lambda,
              int* user_of_level, double* R, double* Qbar)
{
    const int Mq = M + K;
    cplx* Q = (cplx*)calloc((size_t)K * Mq, sizeof(cplx));   /* rows in pick order */
    cplx* L = (cplx*)calloc((size_t)K * K, sizeof(cplx));    /* lower, pick order  */
    int* perm = (int*)malloc(sizeof(int) * K);
    double* nrm = (double*)malloc(sizeof(double) * K);
    int rc = 0;

    for (int j = 0; j < K; j++) {
        for (int m = 0; m < M; m++) Q[j * Mq + m] = ld(H, j * M + m);
        Q[j * Mq + M + j] = lambda;
        perm[j] = j;
    }
    for (int j = 0; j < K * M; j++)
        if (!isfinite(H[2 * j]) || !isfinite(H[2 * j + 1])) rc = ORC_STATUS_NONFINITE;

    double nmax = 0.0;
    for (int j = 0; j < K && rc == 0; j++) {
        double s = 0.0;
        for (int m = 0; m < Mq; m++) s += creal(Q[j * Mq + m] * conj(Q[j * Mq + m]));
        if (s > nmax) nmax = s;
    }

    for (int i = 0; i < K && rc == 0; i++) {
        for (int j = i; j < K; j++) {
            double s = 0.0;
            for (int m = 0; m < Mq; m++) s += creal(Q[j * Mq + m] * conj(Q[j * Mq + m]));
            nrm[j] = s;
        }
        int p = i;
        for (int j = i + 1; j < K; j++)
            if (nrm[j] < nrm[p] || (nrm[j] == nrm[p] && perm[j] < perm[p])) p = j;
        if (p != i) {
            for (int m = 0; m < Mq; m++) { cplx t = Q[i * Mq + m]; Q[i * Mq + m] = Q[p * Mq + m]; Q[p * Mq + m] = t; }
            for (int k = 0; k < i; k++) { cplx t = L[i * K + k]; L[i * K + k] = L[p * K + k]; L[p * K + k] = t; }
            int tp = perm[i]; perm[i] = perm[p]; perm[p] = tp;
            double tn = nrm[i]; nrm[i] = nrm[p]; nrm[p] = tn;
        }
        if (!(nrm[i] > 1e-12 * nmax)) { rc = ORC_STATUS_SINGULAR; break; }
        double rii = sqrt(nrm[i]);
        L[i * K + i] = rii;
        for (int m = 0; m < Mq; m++) Q[i * Mq + m] /= rii;
        for (int j = i + 1; j < K; j++) {
            cplx r = 0.0;                      /* Rbar_ji = q_j . q_i^H */
            for (int m = 0; m < Mq; m++) r += Q[j * Mq + m] * conj(Q[i * Mq + m]);
            L[j * K + i] = r;
            for (int m = 0; m < Mq; m++) Q[j * Mq + m] -= r * Q[i * Mq + m];
        }
    }

    if (rc == 0) {
        /* index reversal: level l <-> pick position K-1-l */
        for (int l = 0; l < K; l++) {
            user_of_level[l] = perm[K - 1 - l];
            for (int k = 0; k < K; k++)
                st(R, l * K + k, (k >= l) ? L[(K - 1 - l) * K + (K - 1 - k)] : 0.0);
            for (int m = 0; m < Mq; m++) st(Qbar, l * Mq + m, Q[(K - 1 - l) * Mq + m]);
        }
    }
    free(Q); free(L); free(perm); free(nrm);
    return rc;
}

/* Rtilde = R^-1 (Section III-A-1: the inverse factor the search uses). Plain
 * back substitution, column by column: R X = I, X upper. */
void orc_tri_inv_upper(int K, const double* R, double* Rt)
{
    for (int i = 0; i < K * K; i++) { Rt[2 * i] = 0.0; Rt[2 * i + 1] = 0.0; }
    for (int k = 0; k < K; k++) {
        st(Rt, k * K + k, 1.0 / ld(R, k * K + k));
        for (int i = k - 1; i >= 0; i--) {
            cplx s = 0.0;
            for (int m = i + 1; m <= k; m++) s += ld(R, i * K + m) * ld(Rt, m * K + k);
            st(Rt, i * K + k, -s / ld(R, i * K + i));
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Metric of Promise K-Best (Section III-A-2, Eq. mop and the K-Best text
 * that follows it): levels 1..K in turn, every survivor expanded into its 9
 * children, the n smallest partial MoPs kept. Reading: ties in the partial
 * metric go to the smaller path code (lexicographic, level K first); with
 * this total order the n survivors are exactly the n smallest full-length
 * vectors whatever the level order. */
typedef struct { double m; uint64_t c; } mop_entry;

static int mop_cmp(const void* a, const void* b)
{
    const mop_entry* x = (const mop_entry*)a;
    const mop_entry* y = (const mop_entry*)b;
    if (x->m < y->m) return -1;
    if (x->m > y->m) return 1;
    if (x->c < y->c) return -1;
    if (x->c > y->c) return 1;
    return 0;
}

int orc_mop_kbest(int K, const double* w, int n, uint64_t* codes, double* metric)
{
    if (K < 1 || K > 16 || n < 1) return -1;
    mop_entry* surv = (mop_entry*)malloc(sizeof(mop_entry) * (size_t)n);
    mop_entry* kids = (mop_entry*)malloc(sizeof(mop_entry) * (size_t)n * 9);
    int ns = 1;
    surv[0].m = 0.0; surv[0].c = 0;
    for (int l = 0; l < K; l++) {
        int nk = 0;
        for (int s = 0; s < ns; s++)
            for (int p = 0; p < 9; p++) {          /* child with p_l - 1 = p */
                kids[nk].m = surv[s].m + w[l] * (double)p;
                kids[nk].c = surv[s].c | ((uint64_t)p << (4 * l));
                nk++;
            }
        qsort(kids, (size_t)nk, sizeof(mop_entry), mop_cmp);
        ns = nk < n ? nk : n;
        memcpy(surv, kids, sizeof(mop_entry) * (size_t)ns);
    }
    for (int s = 0; s < ns; s++) {
        codes[s] = surv[s].c;
        if (metric) metric[s] = surv[s].m;
    }
    free(surv); free(kids);
    return ns;
}

/* ------------------------------------------------------------------------ */
/* DEMAP ranking (Alg. 2 and the LUT paragraph before it): the p-th element
 * of the neighbour ordering around s_hat. Reading: the exact ordering by
 * squared Euclidean distance, ties to the smaller alphabet index
 * a = 3*(Re t + 1) + (Im t + 1). */
void orc_rank9(double sr, double si, int order[9])
{
    double d[9];
    for (int a = 0; a < 9; a++) {
        double tr = a / 3 - 1, ti = a % 3 - 1;
        d[a] = (tr - sr) * (tr - sr) + (ti - si) * (ti - si);
        order[a] = a;
    }
    for (int i = 1; i < 9; i++) {               /* insertion sort on (d, a) */
        int a = order[i], j = i - 1;
        while (j >= 0 && (d[order[j]] > d[a] || (d[order[j]] == d[a] && order[j] > a))) {
            order[j + 1] = order[j];
            j--;
        }
        order[j + 1] = a;
    }
}

/* Region-LUT DEMAP (Section III-A-2: the effective point's position relative
 * to its nearest lattice point addresses a table of neighbour orders). Reading:
 * the nearest alphabet point n0 (clamped rounding, halves to the smaller
 * value) and the octant of d = s_hat - n0 (sign of d.re, sign of d.im,
 * |d.re| > |d.im|) select one of 9 x 8 regions; the region's list is the
 * exact distance order of the 9 alphabet points seen from the octant's
 * centroid n0 + (+-1/3, +-1/6) (x-dominant) or n0 + (+-1/6, +-1/3), ties to the
 * smaller alphabet index. Distances are compared exactly in sixths. */
static int lut_region(double sr, double si)
{
    const int nr = (sr > 0.5) - (sr <= -0.5), ni = (si > 0.5) - (si <= -0.5);
    const double dr = sr - nr, di = si - ni;
    const int oct = (dr > 0.0) | ((di > 0.0) << 1) | ((fabs(dr) > fabs(di)) << 2);
    return ((nr + 1) * 3 + (ni + 1)) * 8 + oct;
}

void orc_lut_order(int region, int order[9])
{
    const int cell = region / 8, oct = region % 8;
    const int nr = cell / 3 - 1, ni = cell % 3 - 1;
    const int big = 2, small = 1;                 /* centroid offsets in sixths */
    const int xr = (oct >> 2) ? big : small, xi = (oct >> 2) ? small : big;
    const int pr = 6 * nr + ((oct & 1) ? xr : -xr), pi = 6 * ni + ((oct & 2) ? xi : -xi);
    long d[9];
    for (int a = 0; a < 9; a++) {
        const int tr = a / 3 - 1, ti = a % 3 - 1;
        d[a] = (long)(6 * tr - pr) * (6 * tr - pr) + (long)(6 * ti - pi) * (6 * ti - pi);
        order[a] = a;
    }
    for (int i = 1; i < 9; i++) {                 /* insertion sort on (d, a) */
        int a = order[i], j = i - 1;
        while (j >= 0 && (d[order[j]] > d[a] || (d[order[j]] == d[a] && order[j] > a))) {
            order[j + 1] = order[j];
            j--;
        }
        order[j + 1] = a;
    }
}

void orc_rank9_lut(double sr, double si, int order[9]) { orc_lut_order(lut_region(sr, si), order); }

/* ------------------------------------------------------------------------ */
/* Parallel post-processing of Alg. 2 for one data vector:
 *   for every candidate k: t^(k) = DEMAP(p^(k)), level K first, with the
 *   effective point s_hat_l of Eq. (17); w^(k) = Qbar^H Rtilde (v - tau t^(k));
 *   d^(k) = ||w^(k)||^2; then k* = argmin d^(k), gamma = d^(k*),
 *   v_precoded = w^(k*) / sqrt(gamma) (P_T = 1).
 * Reading (from the problem statement, not the paper): the zero perturbation
 * is candidate 0 ahead of the n MoP paths, and argmin ties go to the lower
 * candidate index. */
void orc_search_vector(int K, int M, const double* Rt, const double* Qbar, int Mq,
                       const double* v_level, double tau, int n, const uint64_t* codes,
                       int* t_level, double* gamma, double* x, int* best, double* d_all)
{
    orc_search_vector_demap(K, M, Rt, Qbar, Mq, v_level, tau, n, codes, 0, t_level, gamma, x, best, d_all);
}

void orc_search_vector_demap(int K, int M, const double* Rt, const double* Qbar, int Mq,
                             const double* v_level, double tau, int n, const uint64_t* codes, int demap,
                             int* t_level, double* gamma, double* x, int* best, double* d_all)
{
    int* t = (int*)malloc(sizeof(int) * 2 * K);
    int* tbest = (int*)calloc((size_t)2 * K, sizeof(int));
    cplx* z = (cplx*)malloc(sizeof(cplx) * K);
    cplx* w = (cplx*)malloc(sizeof(cplx) * Mq);
    cplx* wbest = (cplx*)calloc((size_t)Mq, sizeof(cplx));
    double dbest = INFINITY;
    int kbest = -1;

    for (int cand = 0; cand <= n; cand++) {
        if (cand == 0) {
            for (int i = 0; i < 2 * K; i++) t[i] = 0;
        } else {
            uint64_t code = codes[cand - 1];
            for (int l = K - 1; l >= 0; l--) {
                /* Eq. (17): s_hat_l = (s~_l - sum_{k>l} Rt_lk tau t_k) / (Rt_ll tau),
                 * s~ = Rtilde v */
                cplx num = 0.0;
                for (int m = l; m < K; m++) num += ld(Rt, l * K + m) * ld(v_level, m);
                for (int m = l + 1; m < K; m++)
                    num -= ld(Rt, l * K + m) * tau * (t[2 * m] + I * t[2 * m + 1]);
                cplx sh = num / (ld(Rt, l * K + l) * tau);
                int order[9];
                if (demap) orc_rank9_lut(creal(sh), cimag(sh), order);
                else orc_rank9(creal(sh), cimag(sh), order);
                int q = (int)((code >> (4 * l)) & 15u);
                int a = order[q];
                t[2 * l] = a / 3 - 1;
                t[2 * l + 1] = a % 3 - 1;
            }
        }
        for (int l = 0; l < K; l++) {           /* z = Rtilde (v - tau t) */
            cplx s = 0.0;
            for (int m = l; m < K; m++)
                s += ld(Rt, l * K + m) * (ld(v_level, m) - tau * (t[2 * m] + I * t[2 * m + 1]));
            z[l] = s;
        }
        double d = 0.0;                         /* w = Qbar^H z, d = ||w||^2 */
        for (int c = 0; c < Mq; c++) {
            cplx s = 0.0;
            for (int l = 0; l < K; l++) s += conj(ld(Qbar, l * Mq + c)) * z[l];
            w[c] = s;
            d += creal(s * conj(s));
        }
        if (d_all) d_all[cand] = d;
        if (d < dbest) {
            dbest = d;
            kbest = cand;
            memcpy(tbest, t, sizeof(int) * 2 * K);
            memcpy(wbest, w, sizeof(cplx) * Mq);
        }
    }
    memcpy(t_level, tbest, sizeof(int) * 2 * K);
    *gamma = dbest;
    *best = kbest;
    double sc = 1.0 / sqrt(dbest);
    for (int c = 0; c < M; c++) st(x, c, wbest[c] * sc);
    free(t); free(tbest); free(z); free(w); free(wbest);
}

/* ------------------------------------------------------------------------ */
/* Fixed-point form of the search (the accelerator's datapath of Section IV:
 * signed words of `word` bits, `frac` of them fractional; the paper keeps 16
 * bits and studies 8..13 fractional bits). Reading: the quantities held in
 * that format are the ones the descent updates, the level residuals in units
 * of tau, r'_m = (s_m + sum_{k>m} Ut_mk (s_k - tau t_k)) / tau, and the
 * normalised entries Ut_mk = Rt_mk / Rt_mm they are updated with. Each word
 * is the nearest multiple of 2^-frac (halves to even), saturated to
 * +-(2^(word-1) - 1) 2^-frac per real component. The entries are rounded
 * first; the starting residual b'_m = (s_m + sum_{k>m} Utq_mk s_k) / tau is
 * formed from them with a wide accumulator (exact: small odd integers times
 * words) and rounded once; every column update r'_m <- r'_m - Utq_ml t_l
 * saturates (exact integer arithmetic).
 * DEMAP ranks the quantised point; the PED sum_l |Rt_ll|^2 tau^2 |r'_l - t_l|^2
 * and the argmin are exact, and gamma and x are computed exactly for the chosen
 * t. */
static double qfix(double v, double scale, double lim)
{
    double q = nearbyint(v * scale);           /* round-half-even in the default mode */
    if (q > lim) q = lim;
    if (q < -lim) q = -lim;
    return q / scale;
}

static double clampd(double v, double lim) { return v > lim ? lim : (v < -lim ? -lim : v); }

void orc_search_vector_fixed(int K, int M, const double* Rt, const double* Qbar, int Mq,
                             const double* v_level, double tau, int n, const uint64_t* codes, int demap,
                             int frac, int word, int* t_level, double* gamma, double* x, int* best)
{
    const double scale = ldexp(1.0, frac), ilim = ldexp(1.0, word - 1) - 1.0, lim = ilim / scale;
    cplx* ut = (cplx*)malloc(sizeof(cplx) * K * K);
    cplx* b = (cplx*)malloc(sizeof(cplx) * K);
    cplx* r = (cplx*)malloc(sizeof(cplx) * K);
    double* wt = (double*)malloc(sizeof(double) * K);
    int* t = (int*)malloc(sizeof(int) * 2 * K);
    int* tbest = (int*)calloc((size_t)2 * K, sizeof(int));
    for (int m = 0; m < K; m++) {
        const cplx d = ld(Rt, m * K + m);
        wt[m] = creal(d * conj(d)) * tau * tau;
        cplx acc = ld(v_level, m);
        for (int k = m + 1; k < K; k++) {
            const cplx u = ld(Rt, m * K + k) / d;
            ut[m * K + k] = qfix(creal(u), scale, ilim) + I * qfix(cimag(u), scale, ilim);
            acc += ut[m * K + k] * ld(v_level, k);
        }
        acc /= tau;
        b[m] = qfix(creal(acc), scale, ilim) + I * qfix(cimag(acc), scale, ilim);
    }
    double pbest = 0.0;                        /* candidate 0: t = 0 */
    for (int m = 0; m < K; m++) pbest += wt[m] * creal(b[m] * conj(b[m]));
    int kbest = 0;
    for (int cand = 1; cand <= n; cand++) {
        const uint64_t code = codes[cand - 1];
        for (int m = 0; m < K; m++) r[m] = b[m];
        double ped = 0.0;
        for (int l = K - 1; l >= 0; l--) {
            int order[9];
            if (demap) orc_rank9_lut(creal(r[l]), cimag(r[l]), order);
            else orc_rank9(creal(r[l]), cimag(r[l]), order);
            const int a = order[(int)((code >> (4 * l)) & 15u)];
            const int tr = a / 3 - 1, ti = a % 3 - 1;
            t[2 * l] = tr;
            t[2 * l + 1] = ti;
            const cplx e = r[l] - (tr + I * ti);
            ped += wt[l] * creal(e * conj(e));
            for (int m = 0; m < l; m++) {
                const cplx v = r[m] - ut[m * K + l] * (tr + I * ti);
                r[m] = clampd(creal(v), lim) + I * clampd(cimag(v), lim);
            }
        }
        if (ped < pbest) {
            pbest = ped;
            kbest = cand;
            memcpy(tbest, t, sizeof(int) * 2 * K);
        }
    }
    /* gamma and x for the chosen perturbation: w = Qbar^H Rt (v - tau t) */
    cplx* z = (cplx*)malloc(sizeof(cplx) * K);
    for (int l = 0; l < K; l++) {
        cplx s = 0.0;
        for (int m = l; m < K; m++)
            s += ld(Rt, l * K + m) * (ld(v_level, m) - tau * (tbest[2 * m] + I * tbest[2 * m + 1]));
        z[l] = s;
    }
    double d = 0.0;
    cplx* w = (cplx*)malloc(sizeof(cplx) * Mq);
    for (int c = 0; c < Mq; c++) {
        cplx s = 0.0;
        for (int l = 0; l < K; l++) s += conj(ld(Qbar, l * Mq + c)) * z[l];
        w[c] = s;
        d += creal(s * conj(s));
    }
    *gamma = d;
    *best = kbest;
    memcpy(t_level, tbest, sizeof(int) * 2 * K);
    for (int c = 0; c < M; c++) st(x, c, w[c] / sqrt(d));
    free(ut); free(b); free(r); free(wt); free(t); free(tbest); free(z); free(w);
}

/* ------------------------------------------------------------------------ */
/* Whole pipeline over channels x vectors (Alg. 2 end to end). lambda > 0 is
 * the Tikhonov-regularised form: Hbar = [H lambda*I], Qbar has M+K columns,
 * and x is the first M entries of w / sqrt(gamma) with gamma = ||w||^2. */
static void precode_channel(int K, int M, int qam, double tau, double lambda, int demap, int frac,
                            int word, int n_paths,
                            const float* Hc, int v0, int v1, const uint8_t* sym_idx,
                            double* x, int8_t* l, double* gamma, int32_t* best, uint8_t* status)
{
    const int Mq = M + K;
    double* H = (double*)malloc(sizeof(double) * 2 * K * M);
    double* R = (double*)malloc(sizeof(double) * 2 * K * K);
    double* Rt = (double*)malloc(sizeof(double) * 2 * K * K);
    double* Q = (double*)malloc(sizeof(double) * 2 * K * Mq);
    double* wgt = (double*)malloc(sizeof(double) * K);
    double* v = (double*)malloc(sizeof(double) * 2 * K);
    int* ul = (int*)malloc(sizeof(int) * K);
    int* t = (int*)malloc(sizeof(int) * 2 * K);
    uint64_t* codes = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n_paths);

    for (int i = 0; i < 2 * K * M; i++) H[i] = (double)Hc[i];
    int rc = orc_isrqd(K, M, H, lambda, ul, R, Q);
    *status = (uint8_t)rc;
    int np = 0;
    if (rc == 0) {
        orc_tri_inv_upper(K, R, Rt);
        for (int i = 0; i < K; i++) {           /* |Rtilde_ll|^2 */
            cplx d = ld(Rt, i * K + i);
            wgt[i] = creal(d * conj(d));
        }
        np = orc_mop_kbest(K, wgt, n_paths, codes, NULL);
    }
    for (int vi = v0; vi < v1; vi++) {
        double* xv = x + (size_t)vi * 2 * M;
        int8_t* lv = l + (size_t)vi * 2 * K;
        if (rc != 0) {
            memset(xv, 0, sizeof(double) * 2 * M);
            memset(lv, 0, (size_t)2 * K);
            gamma[vi] = 0.0;
            best[vi] = -1;
            continue;
        }
        for (int lev = 0; lev < K; lev++)
            orc_qam_point(qam, sym_idx[(size_t)vi * K + ul[lev]], &v[2 * lev], &v[2 * lev + 1]);
        int kb;
        if (frac > 0)
            orc_search_vector_fixed(K, M, Rt, Q, Mq, v, tau, np, codes, demap, frac, word, t, &gamma[vi], xv, &kb);
        else orc_search_vector_demap(K, M, Rt, Q, Mq, v, tau, np, codes, demap, t, &gamma[vi], xv, &kb, NULL);
        best[vi] = kb;
        for (int lev = 0; lev < K; lev++) {     /* l = -t, back to user order */
            lv[2 * ul[lev]] = (int8_t)(-t[2 * lev]);
            lv[2 * ul[lev] + 1] = (int8_t)(-t[2 * lev + 1]);
        }
    }
    free(H); free(R); free(Rt); free(Q); free(wgt); free(v); free(ul); free(t); free(codes);
}

int orc_precode_batch(int K, int M, int qam, double tau, double lambda, int demap, int frac, int word,
                      int n_paths, int C,
                      const float* H, const int32_t* vec_off, const uint8_t* sym_idx,
                      double* x, int8_t* l, double* gamma, int32_t* best,
                      uint8_t* status, int nthreads)
{
    if (K < 1 || K > 16 || M < 1 || n_paths < 1 || C < 0 || !(lambda >= 0.0)) return -1;
    if (M < K && lambda == 0.0) return -1;   /* H H^H is singular without the regularisation */
    if (frac < 0 || (frac > 0 && (word < 2 || word > 53 || frac > 52))) return -1;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int c = 0; c < C; c++)
        precode_channel(K, M, qam, tau, lambda, demap, frac, word, n_paths, H + (size_t)c * 2 * K * M,
                        vec_off[c], vec_off[c + 1], sym_idx, x, l, gamma, best, &status[c]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact references over the bounded alphabet (Eq. qrse with t in
 * {-1,0,1}^K + j{-1,0,1}^K). */
static double gamma_of(int K, const double* Rt, const double* v, double tau, const int* t)
{
    double g = 0.0;
    for (int l = 0; l < K; l++) {
        cplx s = 0.0;
        for (int m = l; m < K; m++)
            s += ld(Rt, l * K + m) * (ld(v, m) - tau * (t[2 * m] + I * t[2 * m + 1]));
        g += creal(s * conj(s));
    }
    return g;
}

double orc_brute_min(int K, const double* Rt, const double* v_level, double tau, int* t_level)
{
    long total = 1;
    for (int i = 0; i < K; i++) total *= 9;
    int* t = (int*)malloc(sizeof(int) * 2 * K);
    double gbest = INFINITY;
    for (long e = 0; e < total; e++) {
        long r = e;
        for (int l = 0; l < K; l++) {
            int a = (int)(r % 9);
            r /= 9;
            t[2 * l] = a / 3 - 1;
            t[2 * l + 1] = a % 3 - 1;
        }
        double g = gamma_of(K, Rt, v_level, tau, t);
        if (g < gbest) { gbest = g; memcpy(t_level, t, sizeof(int) * 2 * K); }
    }
    free(t);
    return gbest;
}

/* Schnorr-Euchner depth-first enumeration with radius pruning: PED
 * recursion of Section II-B from level K down, children in increasing
 * distance from s_hat_l (Eq. 17). */
typedef struct {
    int K;
    const double* Rt;
    const double* v;
    double tau;
    int* t;
    int* tbest;
    double best;
} se_state;

static void se_rec(se_state* S, int l, double ped)
{
    const int K = S->K;
    cplx num = 0.0;
    for (int m = l; m < K; m++) num += ld(S->Rt, l * K + m) * ld(S->v, m);
    for (int m = l + 1; m < K; m++)
        num -= ld(S->Rt, l * K + m) * S->tau * (S->t[2 * m] + I * S->t[2 * m + 1]);
    cplx rll = ld(S->Rt, l * K + l);
    cplx sh = num / (rll * S->tau);
    double wl = creal(rll * conj(rll)) * S->tau * S->tau;
    int order[9];
    orc_rank9(creal(sh), cimag(sh), order);
    for (int q = 0; q < 9; q++) {
        int a = order[q];
        double tr = a / 3 - 1, ti = a % 3 - 1;
        double inc = wl * ((creal(sh) - tr) * (creal(sh) - tr) + (cimag(sh) - ti) * (cimag(sh) - ti));
        double p2 = ped + inc;
        if (p2 >= S->best) break;               /* children come in increasing PED */
        S->t[2 * l] = (int)tr;
        S->t[2 * l + 1] = (int)ti;
        if (l == 0) {
            S->best = p2;
            memcpy(S->tbest, S->t, sizeof(int) * 2 * K);
        } else {
            se_rec(S, l - 1, p2);
        }
    }
}

double orc_sphere_min(int K, const double* Rt, const double* v_level, double tau, int* t_level)
{
    se_state S;
    S.K = K; S.Rt = Rt; S.v = v_level; S.tau = tau;
    S.t = (int*)calloc((size_t)2 * K, sizeof(int));
    S.tbest = (int*)calloc((size_t)2 * K, sizeof(int));
    S.best = INFINITY;
    se_rec(&S, K - 1, 0.0);
    memcpy(t_level, S.tbest, sizeof(int) * 2 * K);
    free(S.t); free(S.tbest);
    return S.best;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
