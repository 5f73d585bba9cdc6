/*
 * libvp -- vector-perturbation (VP) precoding on one GB300 GPU (sm_103a).
 *
 * The library implements the data-parallel hot path of ViPer NL-COMM
 * (Thomas, Katsaros, Jayawardena, Nikitopoulos, "ViPer NL-COMM: Making
 * Vector Perturbation Precoding Practical", arXiv 2602.12098):
 *
 *   per channel (Alg. 2 "Regularize & factorize", lambda = 0, and
 *   "Most Promising Perturbation Vector Identification"):
 *     - the min-norm-first sorted RQ of H (Alg. 1 with the index reversal of
 *       Section IV-B), H_perm = R Q, so (H H^H)^-1 = U^H U with U = R^-1
 *       upper triangular (Eq. viper_rq1);
 *     - the n_paths position vectors with the smallest Metric of Promise
 *       (Eq. mop) by K-Best;
 *   per data vector (Alg. 2 "Parallel post-processing"):
 *     - every candidate path descends the K tree levels from level K, with
 *       per-level interference cancellation and the p_l-th nearest Gaussian
 *       integer around the effective point of Eq. (17) (DEMAP);
 *     - the candidate with the smallest gamma = ||U (s + tau l)||^2 wins,
 *       the zero perturbation being candidate 0 (ties: lower index);
 *     - x = H^H (H H^H)^-1 (s + tau l) / sqrt(gamma)   (v_precoded, P_T = 1).
 *
 * Notation: K users (paper N_R), M AP antennas (paper N_T), s the QAM
 * symbol vector (paper v), l = -t the perturbation (paper t), tau the
 * perturbation interval. A "level" l = 0..K-1 is the paper's tree level l+1.
 *
 * Memory. Every array argument is caller-owned DEVICE memory unless marked
 * HOST. Complex numbers are interleaved (re, im) float pairs (complex64),
 * row-major. The plan owns only its resident per-channel state (factor,
 * paths, precoding matrix) and frees it in vp_plan_destroy.
 *
 * Streams. `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream). Calls enqueue work and return without synchronising,
 * except where noted. Stream order holds as usual: work the caller enqueues
 * before a call is complete before the call's kernels read their inputs,
 * and work enqueued after a call starts after the call's kernels end. (The
 * library's own kernels after the first of vp_factorize use programmatic
 * dependent launch, which only lets their launch overlap the end of the
 * kernel before them.)
 *
 * Errors. Argument errors are returned synchronously and nothing is
 * enqueued. Launch failures return VP_ERR_CUDA. Per-channel numerical
 * problems are reported in the `status` byte array (VP_CH_* bits); the
 * outputs of such a channel are zero. No call aborts or traps.
 *
 * Threading. A plan is used by one host thread at a time. Different plans
 * are independent.
 */
#ifndef VP_H
#define VP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vp_plan vp_plan;

typedef enum {
    VP_OK = 0,
    VP_ERR_INVALID_ARG = 1,    /* a size, pointer or parameter is out of range */
    VP_ERR_CUDA = 2,           /* a CUDA runtime call or kernel launch failed */
    VP_ERR_OOM = 3,            /* device allocation failed */
    VP_ERR_TIMEOUT = 4,        /* a bounded device wait gave up */
    VP_ERR_NOT_FACTORIZED = 5, /* vp_precode before vp_factorize, or for more channels */
    VP_ERR_CAPACITY = 6        /* the request exceeds fixed storage: vp_precode_noalloc's array or a server pool */
} vp_status;

/* Per-channel status bits (the `status` output of vp_factorize). */
#define VP_CH_NONFINITE 1u  /* H holds NaN or Inf; the channel's outputs are zero */
#define VP_CH_SINGULAR  2u  /* a pivot fell below 1e-12 of the largest row norm^2 (rank deficient) */
#define VP_CH_FP64      4u  /* kappa_hat exceeded the plan's threshold: factorised in FP64 */

/* Largest supported sizes. */
#define VP_MAX_K 16
#define VP_MAX_M 16
#define VP_MAX_PATHS 1024

/*
 * Create a plan for one problem shape: the inputs of Alg. 2 other than the
 * channel and the symbols (the user count N_R = K, the antenna count N_T = M,
 * the QAM order of the symbols v, the number of most promising perturbation
 * vectors, and the perturbation interval tau of Section II-B).
 *   K        users, 1 <= K <= VP_MAX_K
 *   M        antennas, 1 <= M <= VP_MAX_M; K > M (overloaded) needs lambda > 0
 *            (vp_plan_set_lambda) before vp_factorize
 *   qam      4, 16, 64 or 256; QAM index i maps to the odd-integer point
 *            (2(i mod m) - (m-1)) + j(2 floor(i/m) - (m-1)), m = sqrt(qam)
 *   n_paths  candidate paths, 1 <= n_paths <= min(9^K, VP_MAX_PATHS)
 *   tau      perturbation interval > 0; pass 0 for the default 2*sqrt(qam)
 *   out      HOST: receives the plan
 * The FP64 fix-up threshold starts at kappa_hat > 1e4 (vp_plan_set_fp64_threshold).
 * Allocates nothing on the device yet. Returns VP_ERR_INVALID_ARG on bad sizes.
 */
vp_status vp_plan_create(int K, int M, int qam, int n_paths, float tau, vp_plan** out);

/* Channels whose kappa_hat = sigma_max(R)^2 sigma_max(U)^2, each largest
 * singular value estimated by six power iterations on the FP32 factor (a
 * lower bound on cond(H H^H) that is tight in practice), exceeds
 * `kappa_hat` are re-factorised in FP64 on the GPU
 * (pivoted Cholesky of the FP64 Gram matrix and one Newton refinement of
 * U). 0 sends every channel to FP64; +inf none. Negative or NaN is invalid. */
vp_status vp_plan_set_fp64_threshold(vp_plan* plan, float kappa_hat);

/*
 * Tikhonov regularisation of Alg. 2 "Regularize & factorize": the factor is
 * the sorted RQ of Hbar = [H  lambda*I] (Section III-A-1), so
 * (H H^H + lambda^2 I)^-1 = U^H U and P = H^H (H H^H + lambda^2 I)^-1 (RZF).
 * The paper takes lambda = sigma / E|s_l| (noise standard deviation over the
 * mean symbol magnitude). With lambda > 0, gamma = ||w||^2 over all M + K
 * entries of Alg. 2's w = Qbar^H U (s + tau l) and x is its first M entries
 * over sqrt(gamma), so ||x|| < 1. 0 (the default) is the plain sorted RQ.
 * Negative or non-finite is invalid. Resident channels are dropped: call
 * vp_factorize again. (The uneven-batch entry points use lambda = 0.)
 */
vp_status vp_plan_set_lambda(vp_plan* plan, float lambda);

/*
 * DEMAP of Alg. 2 (the p_l-th point around the effective point of Eq. 17):
 *   VP_DEMAP_EXACT  exact ranking by distance, ties to the smaller alphabet
 *                   index (the default)
 *   VP_DEMAP_LUT    the region lookup of Section III-A-2: the nearest alphabet
 *                   point (3 x 3) and the octant of the offset from it select
 *                   one of 72 stored orders, each the exact order seen from
 *                   the octant's centroid (n0 + (+-1/3, +-1/6) or
 *                   n0 + (+-1/6, +-1/3)). An approximation: a path's point can
 *                   differ from the exact ranking's away from the centroid.
 * Takes effect at the next vp_precode. Other values are invalid.
 */
typedef enum { VP_DEMAP_EXACT = 0, VP_DEMAP_LUT = 1 } vp_demap;
vp_status vp_plan_set_demap(vp_plan* plan, int demap);

/*
 * Fixed-point search (Section IV, Precision and Numerical Accuracy: signed
 * 16-bit words, the number of fractional bits studied from 8 to 13).
 *   frac_bits  0: the floating-point search (the default);
 *              1..15: the descent holds the level residuals in units of tau
 *              (the effective points of Eq. 17) and the normalised factor
 *              entries U~_mk = U_mk / U_mm as 16-bit words with frac_bits
 *              fractional bits: each is rounded to the nearest multiple of
 *              2^-frac_bits (halves to even) and saturated to
 *              +-32767 2^-frac_bits, every column update saturates the same
 *              way, and DEMAP ranks the quantised point exactly (ties to the
 *              smaller alphabet index). The PEDs are summed in FP32; l, gamma
 *              and x are then computed for the chosen perturbation exactly as
 *              in the floating-point search.
 * The 16-bit arithmetic is carried out exactly in FP32 registers (every word
 * and every sum of two words is representable). Only with VP_DEMAP_EXACT:
 * frac_bits > 0 with the LUT DEMAP (set in either order) is invalid, as is a
 * value outside 0..15. Takes effect at the next vp_precode.
 */
vp_status vp_plan_set_fixed_point(vp_plan* plan, int frac_bits);

/*
 * Where vp_precode forms the output w = P u (Eqs. 24-25, the PV block of
 * Section IV-B; P = H^H (H H^H)^-1, u = s + tau l, exact small integers):
 *   0  CUDA cores (the default): exact products and compensated sums, per
 *      data vector;
 *   1  tensor cores: per channel and round of 16 data vectors, one TF32
 *      matrix product (mma.sync m16n8k8) of the real form [[Re P, -Im P],
 *      [Im P, Re P]] with P split into three 11-bit pieces on per-row grids,
 *      so that every product and partial sum is exact, then one error-free
 *      addition of the three (P kept to 2^-33 of its row's largest entry).
 * Both agree to FP32 rounding; the search and l are the same. Applies to
 * the exact floating-point search (not the region LUT or fixed-point
 * variants, which use the CUDA-core form). Takes effect at the next
 * vp_precode. Other values are invalid.
 */
vp_status vp_plan_set_tensor_product(vp_plan* plan, int enable);

/* Free the plan and its device state. Synchronises the device first so that
 * no enqueued work still reads the state. NULL is accepted. */
vp_status vp_plan_destroy(vp_plan* plan);

/*
 * Factorise C channels and select their candidate paths (Alg. 1, Eq. mop,
 * K-Best); the results stay resident in the plan for the vp_precode calls
 * that follow (one slot: the 14 symbols share the channel).
 *   H       complex64 [C][K][M], H[c][k][m] = channel from antenna m to user k
 *   C       number of channels, C >= 1 (the plan grows its state as needed)
 *   U       optional (may be NULL): complex64 [C][K][K], the upper factor
 *           U = R^-1 in LEVEL order ((H_perm H_perm^H)^-1 = U^H U)
 *   P       optional (may be NULL): complex64 [C][M][K], the precoding
 *           matrix P = H^H (H H^H + lambda^2 I)^-1 in USER order
 *           (x = P u / sqrt(gamma))
 *   user_of_level  optional (may be NULL): uint8 [C][K], the user at each level
 *   status  optional (may be NULL): uint8 [C], VP_CH_* bits per channel
 * Growing the plan allocates device memory (cudaMalloc) and synchronises.
 * Returns VP_ERR_INVALID_ARG for K > M with lambda = 0.
 */
vp_status vp_factorize(vp_plan* plan, const void* H, int C, void* U, void* P,
                       uint8_t* user_of_level, uint8_t* status, void* stream);

/*
 * Precode data vectors against the channels of the last vp_factorize: Alg. 2
 * "Parallel post-processing". For each vector every candidate path descends
 * the levels from level K; at level l the DEMAP point is the p_l-th nearest
 * of the bounded alphabet to the effective point of Eq. (17), the partial
 * distance grows as in the PED recursion of Section II-B, and the candidate
 * with the smallest d^(k) = ||w^(k)||^2 gives x = w^(k*) / sqrt(d^(k*))
 * (Eqs. 24-25 with P_T = 1). The zero perturbation competes as candidate 0.
 *   sym_idx      uint8 [V][K], QAM indices in USER order
 *   S            vectors per channel when vec_offsets is NULL (V = C*S,
 *                vector v belongs to channel v / S)
 *   vec_offsets  optional int32 [C+1]: channel c owns vectors
 *                vec_offsets[c] .. vec_offsets[c+1]-1 (non-decreasing,
 *                vec_offsets[0] = 0); then S is ignored and V = n_vec
 *   n_vec        number of vectors V (must equal C*S when vec_offsets is NULL)
 *   x            complex64 [V][M] precoded vectors, ||x|| = 1 (< 1 with lambda > 0)
 *   l            int8 [V][K][2] perturbation (re, im) in USER order, entries in {-1,0,1}
 *   gamma        float [V], gamma = ||U (s + tau l)||^2 = ||w||^2 of the chosen candidate
 * Returns VP_ERR_NOT_FACTORIZED if no channels are resident.
 */
vp_status vp_precode(vp_plan* plan, const uint8_t* sym_idx, int S, const int32_t* vec_offsets,
                     int n_vec, void* x, int8_t* l, float* gamma, void* stream);

/*
 * Copy the resident candidate paths of the last vp_factorize.
 *   codes  uint64 [C][n_paths]: path k of channel c, rank order (smallest
 *          Metric of Promise first, ties by code); 4 bits per level
 *          (p_l - 1 at bits 4l..4l+3)
 */
vp_status vp_get_paths(vp_plan* plan, uint64_t* codes, void* stream);

/*
 * One whole slot from HOST buffers: copies H and sym_idx to the device,
 * runs vp_factorize and vp_precode (S vectors per channel), returns x, l and
 * gamma, and waits for the stream. Outputs in page-locked, mapped memory
 * (cudaHostAlloc, or cudaHostRegister with cudaHostRegisterMapped) are
 * written by the search kernel in place (on Grace systems over NVLink-C2C);
 * others are copied back. Host buffers should be pinned for asynchronous
 * copies; pageable memory works but copies synchronously.
 *   H_host      HOST complex64 [C][K][M]
 *   sym_host    HOST uint8 [C*S][K]
 *   x_host      HOST complex64 [C*S][M]
 *   l_host      HOST int8 [C*S][K][2] (may be NULL)
 *   gamma_host  HOST float [C*S] (may be NULL)
 * The plan keeps device staging buffers for these copies.
 */
vp_status vp_run_slot_host(vp_plan* plan, const void* H_host, int C, const uint8_t* sym_host,
                           int S, void* x_host, int8_t* l_host, float* gamma_host, void* stream);

/*
 * One slot like vp_factorize + vp_precode (S symbols per channel), without
 * allocating anything. The paper has no counterpart. It serves callers that
 * cannot let a library call cudaMalloc: real-time slot loops, where
 * cudaMalloc may synchronise the device and take unbounded time inside a
 * slot's deadline; processes whose device memory is reserved up front by
 * another framework's allocator; hosts that only hand this library device
 * buffers. The per-channel state that a plan keeps
 * in cudaMalloc'd memory lives instead in one static device array of
 * vp_noalloc_capacity_bytes() bytes (8 MiB); vp_noalloc_max_channels(plan)
 * gives the largest C that fits for the plan's shape. Every GPU that loads
 * the library holds that array until the process exits.
 *   plan     supplies the parameters only (K, M, qam, n_paths, tau, FP64
 *            threshold); its own device state is neither used nor allocated
 *   H        complex64 [C][K][M]; sym_idx uint8 [C*S][K] (vector v -> channel v / S)
 *   x, l, gamma  as vp_precode; status optional uint8 [C] as vp_factorize
 * Returns VP_ERR_CAPACITY when C channels of this shape do not fit
 * (C > vp_noalloc_max_channels(plan)), and VP_ERR_INVALID_ARG when C * S
 * exceeds INT_MAX, with nothing enqueued. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture. All calls share the one array, which keeps
 * the last call's contents: calls whose work overlaps on the GPU (different
 * streams, or several host threads) race on it, so serialise them.
 */
vp_status vp_precode_noalloc(const vp_plan* plan, const void* H, int C, const uint8_t* sym_idx, int S,
                             void* x, int8_t* l, float* gamma, uint8_t* status, void* stream);

/* Size in bytes of the static device array behind vp_precode_noalloc. */
size_t vp_noalloc_capacity_bytes(void);

/* Largest channel count C that vp_precode_noalloc accepts for the plan's
 * shape (K, M, n_paths, lambda): the per-channel state of C channels, each
 * piece 256-byte aligned, fits vp_noalloc_capacity_bytes(). Host only; 0 for
 * a null plan. */
int vp_noalloc_max_channels(const vp_plan* plan);

/*
 * Uneven batches: many independent problems of different shape in a few
 * launches (the paper's many-users / many-cells setting, where every
 * subcarrier or cell brings its own K x M channel, QAM order and path budget).
 * A problem is one channel and its S data vectors; it goes through the same
 * steps as vp_factorize + vp_precode (Alg. 1, Eq. mop, Alg. 2). The limits of
 * each field are those of vp_plan_create.
 */
typedef struct {
    int K, M, qam, n_paths;
    float tau;               /* perturbation interval; 0 = 2 sqrt(qam) */
    int S;                   /* data vectors of this problem (>= 0) */
    const void* H;           /* complex64 [K][M] */
    const uint8_t* sym_idx;  /* uint8 [S][K], QAM indices in user order */
    void* x;                 /* complex64 [S][M] precoded vectors */
    int8_t* l;               /* int8 [S][K][2] perturbation, user order */
    float* gamma;            /* float [S] */
    uint8_t* status;         /* optional uint8 [1]: VP_CH_* bits of the channel */
} vp_problem_desc;

typedef struct vp_batch vp_batch;

/*
 * Plan an uneven batch (host only; nothing is allocated on the device).
 *   descs           HOST array [n_problems]; the device pointers it holds
 *                   are captured and must stay valid while the batch is used
 *   fp64_threshold  as vp_plan_set_fp64_threshold (1e4 is the default)
 * Problems are grouped by kernel shape: one factor launch per (K, M), one
 * path-selection launch per n_paths class (<= 16, 64, 256, 1024), one
 * search launch per K class (<= 2, 4, 8, 12, 16), heaviest problems first.
 * Returns VP_ERR_INVALID_ARG if any descriptor is out of range.
 */
vp_status vp_batch_create(const vp_problem_desc* descs, int n_problems, float fp64_threshold, vp_batch** out);

/* Device workspace the batch needs: its problem table and the per-channel
 * state (about 24 K^2 + 16 K M + 8 n_paths + 5 K bytes per problem). */
size_t vp_batch_workspace_bytes(const vp_batch* batch);

/*
 * Bind the batch to a caller-owned device workspace of at least
 * vp_batch_workspace_bytes bytes (16-byte aligned) and enqueue the upload of
 * its problem table there. The table is copied from the batch's host memory
 * (staged before the call returns). Call again after moving the workspace.
 */
vp_status vp_batch_bind(vp_batch* batch, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Run the whole batch: enqueue memsets and the kernel launches
 * (vp_batch_launch_count of them) on `stream`; no host synchronisation, no
 * allocation and no host-to-device copy. Inputs are read and outputs written
 * through the descriptors' pointers. Returns VP_ERR_NOT_FACTORIZED if the
 * batch was never bound.
 */
vp_status vp_batch_launch(vp_batch* batch, void* stream);

/* Kernel launches enqueued by one vp_batch_launch. */
int vp_batch_launch_count(const vp_batch* batch);

/*
 * How vp_batch_launch runs the search (Alg. 2's post-processing) of the
 * batch:
 *   0  (the default) one launch per K tile (2, 4, 8, 12, 16), heaviest
 *      first inside each;
 *   1  one persistent launch for all problems: resident blocks take
 *      problems from a device counter, heaviest first (S * n_paths * K^2),
 *      each with the search body of its K tile, so that tiles of different
 *      size fill each other's tails.
 * The outputs are the same. Factorisation and path selection run grouped
 * by (K, M) and by path-count class either way.
 */
vp_status vp_batch_set_persistent(vp_batch* batch, int persistent);

/*
 * Whether the launches of one stage (the factor launches per (K, M), the
 * path-selection launches per path class, the search launches per K tile)
 * run side by side: 1 (the default for a handle made by vp_batch_create)
 * puts group k > 0 of a stage on the batch's side stream k - 1, forked from
 * the caller's stream by an event and joined back before the next stage
 * (the groups touch disjoint problems; a CUDA graph capture of
 * vp_batch_launch takes the fork and join along); 0 enqueues every launch on
 * the caller's stream in order. The side streams (4) and their events are
 * created by vp_batch_bind on the current device and freed by
 * vp_batch_destroy; the outputs are the same either way. vp_precode_batch
 * uses 0. VP_ERR_INVALID_ARG for other values; VP_ERR_CUDA if the streams
 * cannot be created.
 */
vp_status vp_batch_set_concurrent(vp_batch* batch, int concurrent);

/*
 * Autotuner. Every path-selection and search launch of a batch (a "group")
 * has one mapping knob (0 is the built-in choice):
 *   path selection: the threads that work on one channel's path lists
 *     (32, 64, 128 or 256);
 *   search of one K tile: warps per block (1..7, the data vectors of a
 *     problem in flight at once);
 *   persistent search (stage 3): warps per block (bits 0-2, 0 or 1..7)
 *     | resident blocks per SM (bits 3-5: 0 = as many as fit, 1..4: the
 *     problems in flight per SM) | staging of the 16-level tile's path codes
 *     (bits 6-7: 0 by the shared-memory budget, 1 staged in shared memory,
 *     2 read in place from global memory).
 * The knobs change how the work maps to lanes, blocks and memory, never the
 * arithmetic: the outputs are the same for every setting. Groups of the
 * search form not in use (see vp_batch_set_persistent) are not timed.
 *
 * vp_batch_autotune runs the bound batch once, then times each group alone
 * under every candidate (reps launches each, CUDA events on `stream`) and
 * keeps the fastest. It synchronises the host with the stream (not for use
 * inside a stream capture) and leaves the outputs of a full launch behind.
 * Returns VP_ERR_NOT_FACTORIZED if the batch is not bound, VP_ERR_INVALID_ARG
 * for reps outside 1..100.
 */
vp_status vp_batch_autotune(vp_batch* batch, int reps, void* stream);

/* The knob of each group (launch order): writes min(count, max_knobs) values
 * to the HOST array `knobs` (may be NULL) and returns count (-1 for NULL). */
int vp_batch_get_tuning(const vp_batch* batch, int* knobs, int max_knobs);

/* Set every group's knob (e.g. from a cache of earlier vp_batch_autotune
 * results); n_knobs must equal the group count and each value must be one
 * of the candidates above or 0, else VP_ERR_INVALID_ARG and nothing changes. */
vp_status vp_batch_set_tuning(vp_batch* batch, const int* knobs, int n_knobs);

/* Shape of each group, for keying a tuning cache: 6 ints per group in the
 * HOST array `info` (stage 0 factor / 1 paths / 2 search of one K tile /
 * 3 persistent search, problem count, K (factor) or K tile (stage 2) else 0,
 * M (factor) else 0, largest n_paths, largest S); returns the group count
 * (-1 for NULL). */
int vp_batch_group_info(const vp_batch* batch, int* info, int max_groups);

/* Free the batch (host memory only; the workspace stays the caller's). */
vp_status vp_batch_destroy(vp_batch* batch);

/*
 * One-shot form: vp_batch_create (threshold 1e4) + vp_batch_bind +
 * vp_batch_launch + vp_batch_destroy. `workspace_bytes` must be at least
 * vp_precode_batch_workspace_bytes(descs, n_problems).
 */
vp_status vp_precode_batch(const vp_problem_desc* descs, int n_problems, size_t workspace_bytes, void* workspace,
                           void* stream);

/* Workspace of vp_precode_batch for these descriptors (0 if any is invalid). */
size_t vp_precode_batch_workspace_bytes(const vp_problem_desc* descs, int n_problems);

/*
 * Serving: a job server that runs whole slots (jobs) as they arrive, on
 * several CUDA streams ("lanes") at once, with admission by device memory.
 * The paper's accelerator streams one cell's slot through its pipeline; a
 * GPU serving many cells instead admits each arriving job as soon as a lane
 * and the job's per-channel state fit, so that jobs that arrive while others
 * run overlap with them on the device. Each job is one slot of one plan
 * shape: vp_factorize + vp_precode over C channels and S symbols per channel
 * (the same kernels, so a job's outputs do not depend on what runs beside it).
 *
 * Memory. vp_server_create reserves one device pool (one cudaMalloc); a job
 * holds a piece of it, its per-channel state (about 24 K^2 + 16 K Mp +
 * 20 n_paths + 5 K + 300 bytes per channel, Mp = M or M + K with lambda > 0), from
 * admission until the server sees it finished. Inputs and outputs stay
 * caller-owned device memory.
 *
 * Admission is first come, first served: the oldest waiting job is admitted
 * when a lane is idle and its state fits in the pool (first fit); a job that
 * does not fit waits, and the jobs behind it wait too. A job that could never
 * fit (larger than the whole pool) is refused at submission.
 *
 * Progress happens inside vp_server_submit, vp_server_poll and
 * vp_server_drain (no background thread): each retires the jobs whose last
 * kernel has finished (frees their state and lane) and admits waiting jobs.
 * The calls may come from different host threads (they take the server's
 * lock).
 *
 * Time. Job times are device times in milliseconds since the last
 * vp_server_reset_clock (one event on lane 0, waited for by the host before
 * that call returns), from the events recorded on the job's lane before its
 * first and after its last kernel. The same call zeroes a host clock when the
 * wait returns (used by vp_server_replay and by the fake server), so host
 * times read at most that wait's latency behind device times.
 *
 * The server serves the paper's per-slot precoding (Alg. 2 on every
 * subcarrier of a slot) for several cells or slots whose jobs arrive
 * independently; the paper's accelerator processes one stream of slots.
 */
typedef struct vp_server vp_server;

typedef struct {
    int K, M, qam, n_paths;  /* as vp_plan_create */
    float tau;               /* 0 = 2 sqrt(qam) */
    float lambda;            /* as vp_plan_set_lambda (0 = plain sorted RQ) */
    float fp64_threshold;    /* as vp_plan_set_fp64_threshold; 0 = the default 1e4 */
    int demap;               /* vp_demap */
    int frac_bits;           /* as vp_plan_set_fixed_point */
    int C, S;                /* channels (>= 1), data vectors per channel (>= 0) */
    const void* H;           /* complex64 [C][K][M] */
    const uint8_t* sym_idx;  /* uint8 [C*S][K] (vector v -> channel v / S) */
    void* x;                 /* complex64 [C*S][M] */
    int8_t* l;               /* int8 [C*S][K][2] */
    float* gamma;            /* float [C*S] */
    uint8_t* status;         /* optional uint8 [C] */
    void* ready_event;       /* optional cudaEvent_t the job's lane waits for
                                before reading H and sym_idx (NULL: the inputs
                                are ready when vp_server_submit is called) */
} vp_job_desc;

typedef struct {
    int64_t id;        /* as returned by vp_server_submit */
    int status;        /* VP_OK, or VP_ERR_CUDA if a launch failed */
    float admit_ms;    /* device time of admission (its first kernel enqueued after) */
    float end_ms;      /* device time when its last kernel finished */
    int rank;          /* priority rank of its stream under VP_SERVE_AGE_PRIORITY
                          (0 = highest), else 0 */
} vp_job_done;

/* Admission policies (vp_server_set_policy). */
typedef enum {
    VP_SERVE_FCFS = 0,          /* every lane at the default stream priority */
    VP_SERVE_AGE_PRIORITY = 1   /* a job's kernels outrank those of the jobs
                                   admitted after it while it runs */
} vp_serve_policy;

typedef struct {
    int lanes, queued, in_flight, max_in_flight;
    int64_t submitted, completed;
    size_t pool_bytes, pool_used, pool_high_water;
} vp_server_stats;

/*
 * Create a server on the current device.
 *   pool_bytes  device memory for the admitted jobs' state (>= 1 MiB)
 *   lanes       CUDA streams, 1..32; at most that many jobs run at once
 * Returns VP_ERR_INVALID_ARG for out-of-range arguments, VP_ERR_OOM if the
 * pool cannot be allocated.
 */
vp_status vp_server_create(size_t pool_bytes, int lanes, vp_server** out);

/*
 * A server with the same admission, pool accounting and reporting, whose
 * jobs run on a host clock instead of the GPU: nothing is allocated on or
 * sent to a device, and a job occupies its lane and pool piece for C
 * microseconds (its channel count) from admission; job times are host
 * milliseconds since vp_server_reset_clock. For testing and studying the
 * scheduling without a GPU. Arguments as vp_server_create.
 */
vp_status vp_server_create_fake(size_t pool_bytes, int lanes, vp_server** out);

/*
 * Queue a job (the descriptor is copied; the device buffers it points to
 * must stay valid until the job is reported done) and admit what fits.
 * Writes the job's id (1, 2, ...). VP_ERR_INVALID_ARG: a field out of range
 * (the limits of vp_plan_create and the plan setters); VP_ERR_CAPACITY: the
 * job's state is larger than the whole pool. Nothing is queued then.
 */
vp_status vp_server_submit(vp_server* srv, const vp_job_desc* job, int64_t* id);

/*
 * Retire finished jobs and admit waiting ones; never blocks on the GPU.
 * Writes up to `max_done` finished jobs (oldest first) to the HOST array
 * `done` and their number to *n_done; jobs not written are reported by the
 * next call.
 */
vp_status vp_server_poll(vp_server* srv, vp_job_done* done, int max_done, int* n_done);

/*
 * Wait until every submitted job has finished (admitting waiting jobs as
 * lanes and memory free up), or until `timeout_s` seconds have passed
 * (VP_ERR_TIMEOUT; the jobs keep running). Finished jobs are still reported
 * by vp_server_poll.
 */
vp_status vp_server_drain(vp_server* srv, double timeout_s);

/* Set the zero of the job times (see Time above). */
vp_status vp_server_reset_clock(vp_server* srv);

/*
 * Choose how admitted jobs share the GPU; only while no job is waiting or
 * running (else VP_ERR_INVALID_ARG). Admission order stays first come, first
 * served under both policies.
 *   VP_SERVE_FCFS          (default) all lanes at one stream priority: the
 *                          running jobs' blocks share the SMs as the block
 *                          scheduler picks them.
 *   VP_SERVE_AGE_PRIORITY  each lane gets one stream per CUDA stream-priority
 *                          level (cudaDeviceGetStreamPriorityRange); a job
 *                          admitted while others run takes the level below the
 *                          youngest running job's, one admitted to an idle
 *                          server the highest, so that older jobs' pending
 *                          blocks are scheduled first (earliest deadline first
 *                          when every job has the same relative deadline).
 *                          Once the levels run out, later jobs share the
 *                          lowest. A fake server models 6 levels.
 * VP_ERR_CUDA if the streams cannot be created (the policy stays FCFS).
 */
vp_status vp_server_set_policy(vp_server* srv, int policy);

/*
 * Open-loop replay of a job trace, for measuring the server under a given
 * arrival process without the caller's own dispatch delay. The server must be
 * idle (no job waiting or running; else VP_ERR_INVALID_ARG). Resets the clock
 * (vp_server_reset_clock), then submits job i (HOST array `jobs`) as soon as
 * the host clock reaches arrival_ms[i] (HOST, milliseconds from the clock
 * zero, finite, non-decreasing), retiring and admitting jobs while it waits,
 * and returns when every job has finished or `timeout_s` seconds after the
 * last submission (VP_ERR_TIMEOUT; the jobs keep running and are reported by
 * vp_server_poll). Writes job i's record to done[i] (HOST, n records) and, if
 * `submit_ms` is not NULL, the host-clock time of its submission to
 * submit_ms[i]; submit_ms[i] - arrival_ms[i] is the replay's own dispatch lag.
 * The host clock reads at most the clock-zero wait's latency behind the device
 * clock, so end_ms - arrival_ms over-states a job's latency by at most that.
 * Every descriptor is checked before anything is submitted (the errors of
 * vp_server_submit). The records of this replay's jobs are not reported by
 * vp_server_poll.
 */
vp_status vp_server_replay(vp_server* srv, const vp_job_desc* jobs, const double* arrival_ms, int n,
                           double timeout_s, vp_job_done* done, double* submit_ms);

/* Counters of the server (HOST struct). */
vp_status vp_server_get_stats(vp_server* srv, vp_server_stats* out);

/* Wait for every lane, then free the pool, streams and events. NULL is
 * accepted. Jobs still waiting for admission are dropped. */
vp_status vp_server_destroy(vp_server* srv);

/* Number of kernel launches the last vp_factorize / vp_precode /
 * vp_run_slot_host call enqueued (copies and memsets not counted). */
int vp_last_launch_count(const vp_plan* plan);

/* Human-readable name of a status code (static string). */
const char* vp_status_string(vp_status s);

#ifdef __cplusplus
}
#endif
#endif /* VP_H */
