// Uneven batches: many independent problems (one channel and its data
// vectors each) of different K x M, QAM order, path budget and tau, run by
// the same kernels as a plan, in a few grouped launches.
//
// Grouping. The factor kernel keeps two channels in one warp (16 lanes each)
// and loops over K and M with shuffles, so one launch holds one (K, M). Path
// selection sizes its shared lists by n_paths: one launch per class
// n <= 16, 64, 256, 1024. The search is templated on a K tile: one launch
// per K <= 2, 4, 8, 12, 16. Inside a launch the problems run heaviest first
// (S * n * K^2), so the long blocks start early and the short ones fill the
// tail. The FP64 fix-up runs once over the channels all factor launches
// flagged. The launches of one stage touch disjoint problems, so by default
// they run side by side on the batch's own streams (the latency-bound factor
// launches and the launch tails overlap), each stage joined before the next.
//
// Workspace (caller-owned device memory): the problem table, the three
// launch orders, the FP64 list and every problem's resident state.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "vp_internal.cuh"

struct vp_batch {
    struct Group {
        int stage;   // 0 factor, 1 paths, 2 search of one K tile, 3 the persistent search of all problems
        int start, count;
        int K, M, KT, n_max, km_max, s_max;
        // tuned mapping (0 = built in): paths = threads per channel; search of
        // a K tile = warps per block; persistent search = warps per block
        // (bits 0-2) | resident blocks per SM (bits 3-5) | staging of the
        // 16-level tile's path codes, 1 shared memory 2 in place (bits 6-7)
        int knob = 0;
    };
    std::vector<vp_problem_desc> descs;
    std::vector<vp::BatchProblem> table;   // device pointers filled in by bind
    std::vector<int> ids;                  // [4][n]: factor, paths, search order per K tile, search order
    std::vector<size_t> state_off;         // per problem, from the state base
    std::vector<Group> groups;
    float kappa_thr = 1e4f;
    // the search stage in one persistent launch over all problems (heaviest
    // first, all K tiles: the stage-3 group), or one launch per K tile (the
    // default: faster on GB300 for the 20,000-problem mix, 4.82 vs 5.05 ms)
    int persistent = 0;
    // the launches of one stage (they touch disjoint problems) run side by
    // side: group k > 0 of a stage on side stream k - 1, forked from and
    // joined back to the caller's stream by events (graph-capturable); off,
    // every launch goes to the caller's stream in order
    int concurrent = 1;
    std::vector<cudaStream_t> side;        // created by vp_batch_bind
    std::vector<cudaEvent_t> joins;        // one per side stream, plus the fork event last
    int km_all = 0, n_all = 0, s_all = 0;
    size_t off_table = 0, off_ids = 0, off_nflag = 0, off_flags = 0, off_state = 0, bytes = 0;
    unsigned char* ws = nullptr;
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Per-problem state, in the order phdr, utp, utc, pt, ptlo, paths, maxq,
// ecode, pcode, emeta, w, ul, st (16-byte parts first).
size_t state_bytes(int K, int M, int n)
{
    size_t b = 16 + 16 * (size_t)K * K;
    b += 8 * (size_t)K * K + 16 * (size_t)K * M + 8 * (size_t)n + 8 * (size_t)vp::n_chunks(n);
    b += 8 * (size_t)n + 8 * (size_t)vp::kMaxPrefix + 4 * (size_t)n;
    b += 4 * (size_t)K + (size_t)K + 1;
    return align_up(b, 16);
}

bool desc_ok(const vp_problem_desc& d)
{
    if (!vp::shape_ok(d.K, d.M, d.qam, d.n_paths, d.tau) || d.S < 0 || !d.H) return false;
    if (d.S > 0 && (!d.sym_idx || !d.x || !d.l || !d.gamma)) return false;
    return true;
}

int k_tile(int K) { return K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : K <= 12 ? 12 : 16; }
int n_class(int n) { return n <= 16 ? 16 : n <= 64 ? 64 : n <= 256 ? 256 : 1024; }

vp_status plan_batch(const vp_problem_desc* descs, int n, float thr, vp_batch* b)
{
    b->descs.assign(descs, descs + n);
    b->kappa_thr = thr;
    const size_t N = (size_t)n;
    b->ids.assign(4 * N, 0);
    b->state_off.assign(N, 0);
    size_t st = 0;
    for (size_t i = 0; i < N; ++i) {
        b->state_off[i] = st;
        st += state_bytes(descs[i].K, descs[i].M, descs[i].n_paths);
    }
    auto cost = [&](int i) {
        const vp_problem_desc& d = descs[i];
        return (double)d.S * d.n_paths * d.K * d.K + 1.0;
    };
    std::vector<int> idx(N);
    for (size_t i = 0; i < N; ++i) idx[i] = (int)i;

    // stage 0: factor, grouped by (K, M)
    std::vector<int> o = idx;
    std::stable_sort(o.begin(), o.end(), [&](int a, int c) {
        if (descs[a].K != descs[c].K) return descs[a].K > descs[c].K;
        return descs[a].M > descs[c].M;
    });
    for (size_t i = 0; i < N;) {
        size_t j = i;
        while (j < N && descs[o[j]].K == descs[o[i]].K && descs[o[j]].M == descs[o[i]].M) ++j;
        vp_batch::Group g = {0, (int)i, (int)(j - i), descs[o[i]].K, descs[o[i]].M, 0, 0, 0, 0};
        b->groups.push_back(g);
        i = j;
    }
    std::copy(o.begin(), o.end(), b->ids.begin());

    // stage 1: paths, grouped by n class, heaviest first inside
    o = idx;
    std::stable_sort(o.begin(), o.end(), [&](int a, int c) {
        const int ca = n_class(descs[a].n_paths), cc = n_class(descs[c].n_paths);
        if (ca != cc) return ca > cc;
        return (long long)descs[a].n_paths * descs[a].K > (long long)descs[c].n_paths * descs[c].K;
    });
    for (size_t i = 0; i < N;) {
        size_t j = i;
        int nmax = 0;
        while (j < N && n_class(descs[o[j]].n_paths) == n_class(descs[o[i]].n_paths)) {
            nmax = std::max(nmax, descs[o[j]].n_paths);
            ++j;
        }
        vp_batch::Group g = {1, (int)i, (int)(j - i), 0, 0, 0, nmax, 0, 0};
        b->groups.push_back(g);
        i = j;
    }
    std::copy(o.begin(), o.end(), b->ids.begin() + N);

    // stage 2: search, grouped by K tile, heaviest first inside
    o = idx;
    std::stable_sort(o.begin(), o.end(), [&](int a, int c) {
        const int ta = k_tile(descs[a].K), tc = k_tile(descs[c].K);
        if (ta != tc) return ta > tc;
        return cost(a) > cost(c);
    });
    for (size_t i = 0; i < N;) {
        size_t j = i;
        int nmax = 0, km = 0, smax = 0;
        while (j < N && k_tile(descs[o[j]].K) == k_tile(descs[o[i]].K)) {
            const vp_problem_desc& d = descs[o[j]];
            nmax = std::max(nmax, d.n_paths);
            km = std::max(km, d.K * d.M);
            smax = std::max(smax, d.S);
            ++j;
        }
        vp_batch::Group g = {2, (int)i, (int)(j - i), 0, 0, k_tile(descs[o[i]].K), nmax, km, smax};
        b->groups.push_back(g);
        i = j;
    }
    std::copy(o.begin(), o.end(), b->ids.begin() + 2 * N);

    // the persistent search: heaviest first over all problems
    o = idx;
    std::stable_sort(o.begin(), o.end(), [&](int a, int c) { return cost(a) > cost(c); });
    std::copy(o.begin(), o.end(), b->ids.begin() + 3 * N);
    for (size_t i = 0; i < N; ++i) {
        b->km_all = std::max(b->km_all, descs[i].K * descs[i].M);
        b->n_all = std::max(b->n_all, descs[i].n_paths);
        b->s_all = std::max(b->s_all, descs[i].S);
    }
    {
        vp_batch::Group g = {3, 0, (int)N, 0, 0, 0, b->n_all, b->km_all, b->s_all};
        b->groups.push_back(g);
    }

    b->off_table = 0;
    b->off_ids = align_up(sizeof(vp::BatchProblem) * N, 256);
    b->off_nflag = b->off_ids + align_up(sizeof(int) * 4 * N, 256);
    b->off_flags = b->off_nflag + 256;
    b->off_state = b->off_flags + align_up(sizeof(int) * N, 256);
    b->bytes = b->off_state + st;
    return VP_OK;
}

void fill_table(vp_batch* b)
{
    const size_t N = b->descs.size();
    b->table.resize(N);
    unsigned char* base = b->ws + b->off_state;
    for (size_t i = 0; i < N; ++i) {
        const vp_problem_desc& d = b->descs[i];
        vp::BatchProblem& p = b->table[i];
        const int K = d.K, M = d.M, n = d.n_paths;
        unsigned char* q = base + b->state_off[i];
        p.phdr = reinterpret_cast<int4*>(q);
        q += 16;
        p.utp = reinterpret_cast<float4*>(q);
        q += 16 * (size_t)K * K;
        p.utc = reinterpret_cast<float2*>(q);
        q += 8 * (size_t)K * K;
        p.pt = reinterpret_cast<float2*>(q);
        q += 8 * (size_t)K * M;
        p.ptlo = reinterpret_cast<float2*>(q);
        q += 8 * (size_t)K * M;
        p.paths = reinterpret_cast<uint64_t*>(q);
        q += 8 * (size_t)n;
        p.maxq = reinterpret_cast<uint64_t*>(q);
        q += 8 * (size_t)vp::n_chunks(n);
        p.ecode = reinterpret_cast<uint64_t*>(q);
        q += 8 * (size_t)n;
        p.pcode = reinterpret_cast<uint64_t*>(q);
        q += 8 * (size_t)vp::kMaxPrefix;
        p.emeta = reinterpret_cast<uint32_t*>(q);
        q += 4 * (size_t)n;
        p.w = reinterpret_cast<float*>(q);
        q += 4 * (size_t)K;
        p.ul = q;
        q += K;
        p.st = q;
        p.H = static_cast<const float2*>(d.H);
        p.sym = d.sym_idx;
        p.x = static_cast<float2*>(d.x);
        p.l = d.l;
        p.gamma = d.gamma;
        p.status = d.status;
        p.K = K;
        p.M = M;
        p.n = n;
        p.m_qam = vp::qam_side(d.qam);
        p.S = d.S;
        p.tau = (d.tau == 0.f) ? 2.0f * std::sqrt((float)d.qam) : d.tau;
        p.kappa_thr = b->kappa_thr;
        p.pad_ = 0;
    }
}

constexpr int kSideStreams = 4;

// Streams and events of the concurrent mode, created once (at bind, before
// any stream capture) on the current device.
bool make_side_streams(vp_batch* b)
{
    if (!b->side.empty()) return true;
    for (int i = 0; i < kSideStreams; ++i) {
        cudaStream_t q = nullptr;
        if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) break;
        b->side.push_back(q);
    }
    for (int i = 0; (int)b->side.size() == kSideStreams && i <= kSideStreams; ++i) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) break;
        b->joins.push_back(e);
    }
    if ((int)b->side.size() == kSideStreams && (int)b->joins.size() == kSideStreams + 1) return true;
    cudaGetLastError();
    for (cudaStream_t q : b->side) cudaStreamDestroy(q);
    for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
    b->side.clear();
    b->joins.clear();
    return false;
}

// Launches every group of one stage: in order on `s`, or (concurrent mode)
// the k-th group on side stream k - 1 after a fork event on `s`, then `s`
// waits for every side stream it used.
template <class F>
cudaError_t launch_stage(const vp_batch* b, int stage, cudaStream_t s, F&& launch)
{
    const bool conc = b->concurrent && !b->side.empty();
    cudaEvent_t fork = conc ? b->joins[kSideStreams] : nullptr;
    int k = 0;
    cudaError_t e = cudaSuccess;
    for (const vp_batch::Group& g : b->groups) {
        if (g.stage != stage) continue;
        cudaStream_t q = s;
        if (conc && k > 0) {
            q = b->side[(k - 1) % kSideStreams];
            if (k == 1 && (e = cudaEventRecord(fork, s)) != cudaSuccess) return e;
            if (k <= kSideStreams && (e = cudaStreamWaitEvent(q, fork, 0)) != cudaSuccess) return e;
        }
        if ((e = launch(g, q)) != cudaSuccess) return e;
        ++k;
    }
    for (int i = 0; conc && i < k - 1 && i < kSideStreams; ++i) {
        if ((e = cudaEventRecord(b->joins[i], b->side[i])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, b->joins[i], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One search group: a K tile's launch (stage 2), or the persistent launch of
// every problem (stage 3, its counter reset first).
cudaError_t launch_search_group(const vp_batch* b, const vp_batch::Group& g, cudaStream_t s)
{
    const int N = (int)b->descs.size();
    const vp::BatchProblem* probs = reinterpret_cast<const vp::BatchProblem*>(b->ws + b->off_table);
    const int* ids = reinterpret_cast<const int*>(b->ws + b->off_ids);
    if (g.stage == 2)
        return vp::launch_search_batch(probs, ids + 2 * N + g.start, g.count, g.KT, g.km_max, g.n_max, g.s_max, s,
                                       g.knob);
    int* counter = reinterpret_cast<int*>(b->ws + b->off_nflag) + 1;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    return vp::launch_search_persist(probs, ids + 3 * N, g.count, g.km_max, g.n_max, g.s_max, counter, s,
                                     g.knob & 7, (g.knob >> 3) & 7, (g.knob >> 6) & 3);
}

}  // namespace

extern "C" {

vp_status vp_batch_create(const vp_problem_desc* descs, int n_problems, float fp64_threshold, vp_batch** out)
{
    if (!out) return VP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!descs || n_problems < 1 || std::isnan(fp64_threshold) || fp64_threshold < 0.f) return VP_ERR_INVALID_ARG;
    for (int i = 0; i < n_problems; ++i)
        if (!desc_ok(descs[i])) return VP_ERR_INVALID_ARG;
    vp_batch* b = new (std::nothrow) vp_batch();
    if (!b) return VP_ERR_OOM;
    try {
        plan_batch(descs, n_problems, fp64_threshold, b);
    } catch (...) {
        delete b;
        return VP_ERR_OOM;
    }
    *out = b;
    return VP_OK;
}

size_t vp_batch_workspace_bytes(const vp_batch* b) { return b ? b->bytes : 0; }

vp_status vp_batch_bind(vp_batch* b, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!b || !workspace || workspace_bytes < b->bytes || (reinterpret_cast<uintptr_t>(workspace) & 15u))
        return VP_ERR_INVALID_ARG;
    b->ws = static_cast<unsigned char*>(workspace);
    try {
        fill_table(b);
    } catch (...) {
        b->ws = nullptr;
        return VP_ERR_OOM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t N = b->descs.size();
    if (b->concurrent && !make_side_streams(b)) b->concurrent = 0;   // no side streams: one stream in order
    if (cudaMemcpyAsync(b->ws + b->off_table, b->table.data(), sizeof(vp::BatchProblem) * N, cudaMemcpyHostToDevice,
                        s) != cudaSuccess ||
        cudaMemcpyAsync(b->ws + b->off_ids, b->ids.data(), sizeof(int) * 4 * N, cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
        b->ws = nullptr;
        return VP_ERR_CUDA;
    }
    return VP_OK;
}

vp_status vp_batch_launch(vp_batch* b, void* stream)
{
    if (!b) return VP_ERR_INVALID_ARG;
    if (!b->ws) return VP_ERR_NOT_FACTORIZED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int N = (int)b->descs.size();
    const vp::BatchProblem* probs = reinterpret_cast<const vp::BatchProblem*>(b->ws + b->off_table);
    const int* ids = reinterpret_cast<const int*>(b->ws + b->off_ids);
    int* nflag = reinterpret_cast<int*>(b->ws + b->off_nflag);
    int* flags = reinterpret_cast<int*>(b->ws + b->off_flags);
    if (cudaMemsetAsync(nflag, 0, sizeof(int), s) != cudaSuccess) return VP_ERR_CUDA;
    if (launch_stage(b, 0, s, [&](const vp_batch::Group& g, cudaStream_t q) {
            return vp::launch_factor32_batch(probs, ids + g.start, g.count, g.K, g.M, nflag, flags, q);
        }) != cudaSuccess)
        return VP_ERR_CUDA;
    if (vp::launch_factor64_batch(probs, nflag, flags, N, s) != cudaSuccess) return VP_ERR_CUDA;
    if (launch_stage(b, 1, s, [&](const vp_batch::Group& g, cudaStream_t q) {
            return vp::launch_pathsel_batch(probs, ids + N + g.start, g.count, g.n_max, q, g.knob);
        }) != cudaSuccess)
        return VP_ERR_CUDA;
    if (launch_stage(b, b->persistent ? 3 : 2, s, [&](const vp_batch::Group& g, cudaStream_t q) {
            return launch_search_group(b, g, q);
        }) != cudaSuccess)
        return VP_ERR_CUDA;
    return VP_OK;
}

vp_status vp_batch_set_persistent(vp_batch* b, int persistent)
{
    if (!b || (persistent != 0 && persistent != 1)) return VP_ERR_INVALID_ARG;
    b->persistent = persistent;
    return VP_OK;
}

vp_status vp_batch_set_concurrent(vp_batch* b, int concurrent)
{
    if (!b || (concurrent != 0 && concurrent != 1)) return VP_ERR_INVALID_ARG;
    if (concurrent && b->ws && !make_side_streams(b)) return VP_ERR_CUDA;
    b->concurrent = concurrent;
    return VP_OK;
}

// The values a group's knob may take (0 = the built-in choice).
static bool knob_ok(int stage, int v)
{
    if (v == 0) return true;
    if (stage == 1) return v == 32 || v == 64 || v == 128 || v == 256;
    if (stage == 2) return v >= 1 && v <= 7;
    if (stage == 3) return v > 0 && v < 256 && ((v >> 3) & 7) <= 4 && ((v >> 6) & 3) <= 2;
    return false;
}

vp_status vp_batch_autotune(vp_batch* b, int reps, void* stream)
{
    if (!b || reps < 1 || reps > 100) return VP_ERR_INVALID_ARG;
    if (!b->ws) return VP_ERR_NOT_FACTORIZED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int N = (int)b->descs.size();
    const vp::BatchProblem* probs = reinterpret_cast<const vp::BatchProblem*>(b->ws + b->off_table);
    const int* ids = reinterpret_cast<const int*>(b->ws + b->off_ids);
    // one whole launch leaves every problem's factor and paths in place: a
    // path-selection or search group can then be rerun alone (same outputs)
    vp_status st = vp_batch_launch(b, stream);
    if (st != VP_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return VP_ERR_CUDA;
    }
    static const int kPaths[] = {32, 64, 128, 256};
    static const int kWarps[] = {4, 5, 6, 7};
    // persistent search: warps per block x resident blocks per SM x staging
    std::vector<int> kPersist;
    for (int nw : {0, 6, 7})
        for (int bps : {0, 2, 3})
            for (int stg : {0, 1, 2}) kPersist.push_back(nw | (bps << 3) | (stg << 6));
    st = VP_OK;
    for (vp_batch::Group& g : b->groups) {
        if (g.stage == 0 || g.stage == (b->persistent ? 2 : 3)) continue;
        std::vector<int> cand;
        if (g.stage == 1) cand.assign(kPaths, kPaths + 4);
        else if (g.stage == 2) cand.assign(kWarps, kWarps + 4);
        else cand = kPersist;
        float best = INFINITY;
        int best_v = 0;
        for (int ci = -1; ci < (int)cand.size() && st == VP_OK; ++ci) {
            const int v = ci < 0 ? 0 : cand[ci];
            float ms = 0.f;
            cudaError_t e = cudaEventRecord(e0, s);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                if (g.stage == 1) e = vp::launch_pathsel_batch(probs, ids + N + g.start, g.count, g.n_max, s, v);
                else {
                    vp_batch::Group gv = g;
                    gv.knob = v;
                    e = launch_search_group(b, gv, s);
                }
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                cudaGetLastError();
                st = VP_ERR_CUDA;
                break;
            }
            if (ms < best) { best = ms; best_v = v; }
        }
        g.knob = best_v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

int vp_batch_get_tuning(const vp_batch* b, int* knobs, int max_knobs)
{
    if (!b) return -1;
    const int n = (int)b->groups.size();
    for (int i = 0; i < n && i < max_knobs && knobs; ++i) knobs[i] = b->groups[i].knob;
    return n;
}

vp_status vp_batch_set_tuning(vp_batch* b, const int* knobs, int n_knobs)
{
    if (!b || !knobs || n_knobs != (int)b->groups.size()) return VP_ERR_INVALID_ARG;
    for (int i = 0; i < n_knobs; ++i)
        if (!knob_ok(b->groups[i].stage, knobs[i])) return VP_ERR_INVALID_ARG;
    for (int i = 0; i < n_knobs; ++i) b->groups[i].knob = knobs[i];
    return VP_OK;
}

int vp_batch_group_info(const vp_batch* b, int* info, int max_groups)
{
    if (!b) return -1;
    const int n = (int)b->groups.size();
    for (int i = 0; i < n && i < max_groups && info; ++i) {
        const vp_batch::Group& g = b->groups[i];
        int* o = info + 6 * i;
        o[0] = g.stage;
        o[1] = g.count;
        o[2] = g.stage == 0 ? g.K : (g.stage == 2 ? g.KT : 0);   // stage 3: every K tile
        o[3] = g.stage == 0 ? g.M : 0;
        o[4] = g.n_max;
        o[5] = g.s_max;
    }
    return n;
}

int vp_batch_launch_count(const vp_batch* b)
{
    if (!b) return 0;
    int n = 1;   // the FP64 fix-up
    for (const vp_batch::Group& g : b->groups)
        if (g.stage < 2 || g.stage == (b->persistent ? 3 : 2)) ++n;
    return n;
}

vp_status vp_batch_destroy(vp_batch* b)
{
    if (!b) return VP_OK;
    for (cudaStream_t q : b->side) {
        cudaStreamSynchronize(q);
        cudaStreamDestroy(q);
    }
    for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
    cudaGetLastError();
    delete b;
    return VP_OK;
}

size_t vp_precode_batch_workspace_bytes(const vp_problem_desc* descs, int n_problems)
{
    vp_batch* b = nullptr;
    if (vp_batch_create(descs, n_problems, 1e4f, &b) != VP_OK) return 0;
    const size_t bytes = b->bytes;
    vp_batch_destroy(b);
    return bytes;
}

vp_status vp_precode_batch(const vp_problem_desc* descs, int n_problems, size_t workspace_bytes, void* workspace,
                           void* stream)
{
    vp_batch* b = nullptr;
    vp_status st = vp_batch_create(descs, n_problems, 1e4f, &b);
    if (st != VP_OK) return st;
    b->concurrent = 0;   // one call, one stream: no side streams to create per call
    st = vp_batch_bind(b, workspace, workspace_bytes, stream);
    if (st == VP_OK) st = vp_batch_launch(b, stream);
    vp_batch_destroy(b);
    return st;
}

}  // extern "C"
