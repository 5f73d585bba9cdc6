/*
 * FP64 CPU oracle of the ViPer NL-COMM vector-perturbation (VP) precoder.
 *
 * TEST INFRASTRUCTURE ONLY. This code is the slow, plain reference that the
 * CUDA path is checked against. It shares no code, header, table or helper
 * with the CUDA library; only tests/, __graft_entry__.smoke() and bench.py
 * (its cpu_baseline leg and its "reference" arm) may load it. The product
 * path never calls it.
 *
 * Conventions.
 *   - Complex arrays are interleaved (re, im) doubles, row-major.
 *   - K users (paper N_R), M AP antennas (paper N_T), lambda = 0 unless given.
 *   - "Level" l = 0..K-1 is the paper's tree level l+1. The tree search runs
 *     from level K (index K-1) down to level 1 (index 0), as in the PED
 *     recursion of Section II-B.
 *   - The paper's perturbation t and the returned l are related by l = -t, so
 *     v - tau*t = s + tau*l (Eq. se / Alg. 2).
 *   - Perturbation alphabet (B = 1, Section III-A-2): the 9 points
 *     {-1,0,1} + j{-1,0,1}; point index a = 3*(Re t + 1) + (Im t + 1).
 *   - A path code packs p_l - 1 (0..8) in 4 bits per level, level index l at
 *     bits [4l, 4l+4). Codes compare as integers in lexicographic order with
 *     level K most significant.
 *
 * Readings of the paper that this oracle takes (each one is listed in the
 * design notes): see the comment on each function.
 */
#ifndef VP_ORACLE_H
#define VP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status bits of a channel (shared meaning with the GPU path, separate code). */
#define ORC_STATUS_NONFINITE 1 /* H holds a NaN or Inf */
#define ORC_STATUS_SINGULAR  2 /* a pivot norm fell to <= 1e-12 of the largest row norm */

/* QAM point of symbol index idx for a square qam-point constellation with
 * odd-integer coordinates (spacing 2): with m = sqrt(qam),
 * Re = 2*(idx mod m) - (m-1), Im = 2*floor(idx/m) - (m-1).
 * Section II (QAM symbols v); the index-to-point map is a reading. */
void orc_qam_point(int qam, int idx, double* re, double* im);

/* Algorithm 1 (ISRQD), min-norm-first sorted RQ of Hbar = [H  lambda*I]
 * by modified Gram-Schmidt on the rows, then the index reversal of
 * Section IV-B so that the first row picked sits at tree level K.
 *   H          K x M complex (row-major)
 *   lambda     Tikhonov parameter (0 gives the plain sorted RQ of H)
 * Outputs, all in LEVEL order:
 *   user_of_level[l]  which row of H sits at level l
 *   R                 K x K upper triangular, positive real diagonal
 *   Qbar              K x (M+K): row l is the orthonormal row of level l
 *                     (the last K columns are the lambda*I extension)
 * H_perm_bar = R * Qbar, where H_perm_bar's row l is [H[user_of_level[l]], lambda e_user].
 * Returns 0, ORC_STATUS_NONFINITE or ORC_STATUS_SINGULAR. */
int orc_isrqd(int K, int M, const double* H, double lambda,
              int* user_of_level, double* R, double* Qbar);

/* Rtilde = R^-1 for an upper-triangular R (back substitution). */
void orc_tri_inv_upper(int K, const double* R, double* Rt);

/* Metric of Promise (Eq. mop) K-Best path pre-selection (Section III-A-2):
 * breadth-first over levels 1..K, expanding every survivor into its 9
 * children and keeping the n smallest partial metrics
 * sum_l w[l]*(p_l - 1), ties by path code. The survivors of the last level
 * are returned sorted by (metric, code).
 *   w       K weights |Rtilde_ll|^2 in level order
 *   n       requested number of paths (1 <= n)
 * Returns the number of paths written (min(n, 9^K)), or -1 on bad input. */
int orc_mop_kbest(int K, const double* w, int n, uint64_t* codes, double* metric);

/* The 9 alphabet indices ordered by (|s_hat - t|^2, a) ascending: element
 * p-1 is the p-th nearest perturbation symbol to s_hat (DEMAP of Alg. 2,
 * exact-ranking reading of the neighbour ordering). */
void orc_rank9(double sr, double si, int order[9]);

/* Region-LUT DEMAP, the paper's table-driven alternative (Section III-A-2,
 * "DEMAP" of Alg. 2). Reading: region = nearest alphabet point n0 (3 x 3) x
 * octant of s_hat - n0 (signs, |re| > |im|), 72 regions; each region's list is
 * the exact distance order from the octant centroid n0 + (+-1/3, +-1/6) or
 * n0 + (+-1/6, +-1/3), ties to the smaller alphabet index.
 *   orc_lut_order   the list of region r (0..71): r = ((n0r+1)*3 + n0i+1)*8 +
 *                   [d.re > 0] + 2 [d.im > 0] + 4 [|d.re| > |d.im|]
 *   orc_rank9_lut   the list for the effective point (sr, si) */
void orc_lut_order(int region, int order[9]);
void orc_rank9_lut(double sr, double si, int order[9]);

/* Parallel post-processing of Alg. 2 for one data vector, plus the zero
 * perturbation as candidate 0.
 *   Rt           K x K upper, level order (Rtilde)
 *   Qbar, Mq     K x Mq orthonormal rows, level order (Mq = M or M+K)
 *   M            number of transmit antennas; x gets the first M entries of w
 *   v_level      K complex QAM symbols already in level order
 *   codes, n     MoP paths (candidate k+1 is codes[k])
 * Outputs:
 *   t_level      K pairs (int) of the winning perturbation, level order
 *   gamma        d^(k*) = ||w^(k*)||^2
 *   x            M complex: w^(k*) / sqrt(gamma)  (P_T = 1)
 *   best         k* (0 = zero perturbation, k+1 = codes[k])
 *   d_all        optional (may be NULL): n+1 candidate metrics d^(k) */
void orc_search_vector(int K, int M, const double* Rt, const double* Qbar, int Mq,
                       const double* v_level, double tau, int n, const uint64_t* codes,
                       int* t_level, double* gamma, double* x, int* best, double* d_all);
/* The same with the DEMAP chosen: demap 0 = exact ranking, 1 = region LUT. */
void orc_search_vector_demap(int K, int M, const double* Rt, const double* Qbar, int Mq,
                             const double* v_level, double tau, int n, const uint64_t* codes, int demap,
                             int* t_level, double* gamma, double* x, int* best, double* d_all);

/* Fixed-point search (Section IV's datapath: signed `word`-bit values with
 * `frac` fractional bits; the accelerator uses 16 bits). The level residuals
 * in units of tau and the normalised entries Rt_mk / Rt_mm are rounded half to
 * even to multiples of 2^-frac and saturated to +-(2^(word-1) - 1) 2^-frac (the
 * starting residuals formed from the rounded entries and rounded once), the
 * residual updates saturate at every level, DEMAP (demap 0 exact, 1 region
 * LUT) ranks the quantised point; the PEDs, the argmin, gamma and x are
 * exact. */
void orc_search_vector_fixed(int K, int M, const double* Rt, const double* Qbar, int Mq,
                             const double* v_level, double tau, int n, const uint64_t* codes, int demap,
                             int frac, int word, int* t_level, double* gamma, double* x, int* best);

/* Whole pipeline over a batch of channels, as the GPU library computes it.
 *   lambda     Tikhonov parameter of Alg. 2 "Regularize & factorize"
 *              (0: the plain sorted RQ, needs M >= K); with lambda > 0,
 *              gamma = ||w||^2 over all M+K entries of w = Qbar^H Rt (v - tau t)
 *              and x = the first M entries of w / sqrt(gamma)
 *   demap      0: exact ranking (orc_rank9); 1: region LUT (orc_rank9_lut)
 *   frac, word 0: floating-point search; frac > 0: the fixed-point search
 *              (orc_search_vector_fixed) with `word`-bit values (2..53),
 *              `frac` (1..52) of them fractional
 *   H          complex64 [C][K][M] as float pairs (the GPU's own input)
 *   vec_off    [C+1] vector ranges per channel (channel c owns vectors
 *              vec_off[c] .. vec_off[c+1]-1)
 *   sym_idx    [V][K] QAM indices in user order
 * Outputs per vector v: x [V][M] complex (double pairs), l [V][K] int8 pairs
 * in user order, gamma [V], best [V]; per channel: status [C].
 * Channels whose status is nonzero get zero outputs.
 * nthreads > 1 runs channels in parallel (OpenMP), when built with it. */
int orc_precode_batch(int K, int M, int qam, double tau, double lambda, int demap, int frac, int word,
                      int n_paths, int C,
                      const float* H, const int32_t* vec_off, const uint8_t* sym_idx,
                      double* x, int8_t* l, double* gamma, int32_t* best,
                      uint8_t* status, int nthreads);

/* Exhaustive minimum of ||Rt (v - tau t)||^2 over all 9^K bounded
 * perturbations (K <= 8). Ties keep the first in enumeration order.
 * Returns gamma_min; writes t_level. */
double orc_brute_min(int K, const double* Rt, const double* v_level, double tau, int* t_level);

/* Schnorr-Euchner depth-first sphere encoder over the same bounded alphabet:
 * the exact minimum, children visited in increasing PED. Returns gamma_min. */
double orc_sphere_min(int K, const double* Rt, const double* v_level, double tau, int* t_level);

/* Number of OpenMP threads the batch routine would use (1 without OpenMP). */
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
