// Host side of the RAS / RASPEN library: the C ABI of include/ras.h, the
// decomposition (Sec. 4.2), the launch sequence of the RASPEN function
// (Alg. 3), GMRES, RASPEN (Alg. 2) and Newton_RAS (Alg. 1 with linear RAS).
// Every arithmetic step runs in the kernels of local.cu, solve.cu and
// residual.cu; this file orders launches, moves scalars and applies the stop
// rules.
//
// A handle holds one or more independent problems (a batch). All subdomains
// of all problems form one table, so every step of a RASPEN-function
// evaluation is one launch for the whole batch; global vectors are the
// concatenation of the problems' [y | p] planes (problem k at ProbDev.ofs),
// and GMRES runs the problems in lockstep with segmented reductions, one host
// synchronisation per Krylov step for the whole batch.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ras.h"
#include "ras_internal.cuh"

namespace ras {
static std::atomic<long long> g_launches{0};
// While a thread captures a graph its launches are counted here instead (a
// graph's kernels count when the graph runs).
static thread_local long long* t_capture_count = nullptr;
void count_launch() {
    if (t_capture_count) ++*t_capture_count;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace ras

using ras::LocalState;
using ras::NewtonParams;
using ras::ProbDev;
using ras::Seg;
using ras::SubDev;

struct ras_problem {
    int nprob = 0;
    std::vector<ras_problem_desc> desc;
    std::vector<int> sz;      // per problem: subdomains along x3 on the cube, 0 on the square
    ras_opts o{};
    cudaStream_t st = nullptr;
    int nsub = 0, maxm = 0;   // maxm: largest 2*bl of the narrow (register / streaming path) subdomains
    long long L = 0;          // length of a global vector (sum of 2 nn_k)
    long long Lsum = 0;       // sum of 2*wx*wy*wz
    long long Nsum = 0;       // sum of wx*wy*wz
    long long Gsum = 0;       // sum of bw*mp^2
    std::vector<SubDev> subs;
    std::vector<ProbDev> probs;
    std::vector<Seg> segs;
    std::vector<int> sub_first, sub_count;   // subdomains of each problem (contiguous)
    SubDev* d_subs = nullptr;
    ProbDev* d_probs = nullptr;
    Seg* d_segs = nullptr;
    int* d_lists = nullptr;                  // subdomain indices grouped by register-tile class
    std::vector<int> tile_off, tile_cnt;     // per tile class 2, 4, 6, 8, 10 (index tile/2 - 1)
    double* yd = nullptr;
    double* f = nullptr;
    double *cpool = nullptr, *dpool = nullptr, *Kpool = nullptr, *Ktpool = nullptr, *rpool = nullptr;
    double* coef = nullptr;
    void* gpool = nullptr;
    void* wpool = nullptr;
    int gprec = -1;
    LocalState* ls = nullptr;
    int* d_active = nullptr;
    int* d_err = nullptr;        // [0]: set by kernels whose bounded waits ran out; [1]: opts.wait_test
    int h_wait_test = 0;         // host copy of opts.wait_test (source of the copy into d_err[1])
    int* h_active = nullptr;     // pinned
    int* d_mask = nullptr;       // per-problem masks: row 0 [0, nprob) GMRES/JVP, row 1 outer loop
    double* d_pstart = nullptr;  // per-problem eps start of a RASPEN-function evaluation
    double *X = nullptr, *F = nullptr, *Dv = nullptr, *Ov = nullptr, *T1 = nullptr, *T2 = nullptr,
           *T3 = nullptr, *Z = nullptr;
    double* coefG = nullptr;
    double* partials = nullptr;
    int nbp = 0;                 // blocks per problem of the segmented kernels
    ras_tuning tune{{-1, -1, -1, -1, -1}, 0, ras::VEC_BLOCKS};   // launch shapes (ras_autotune)
    int sms = 0;                 // SMs of the device (0 until queried)
    bool own_factors = true;     // factors and coefficients in gpool / coef (else per subdomain pointers)
    ras_state last_state{};      // state at the end of the last outer solve (checkpoint)
    bool have_last = false;
    ras_state resume{};          // one-shot resume point for the next outer solve
    bool have_resume = false;
    int* d_order = nullptr;      // subdomain indices, largest factors first (solve kernels)
    int* d_ticket = nullptr;     // work counter of the persistent solve kernels
    std::vector<int> h_wide;     // wide-block subdomains (MAX_M < 2 bl <= MAX_MW)
    int* d_wide = nullptr;
    // block tables of the segmented kernels, one per mask row (0: GMRES/JVP,
    // 1: outer loop, 2: every problem), VEC_BLOCKS + nprob entries each
    int2* d_tab = nullptr;       // row 3: the GMRES cycle's table, built on the device from d_mask row 0
    int* d_nbps = nullptr;       // 4 rows of nprob block counts
    int* d_toff = nullptr;       // nprob + 1 ints: scratch of the device-built table
    int ntab[3] = {0, 0, 0};
    std::vector<int> last_mask[3];
    double* scal = nullptr;      // device scalars, 4 * 32 per problem
    double* h_scal = nullptr;    // pinned host scalars, same layout
    double* V = nullptr;
    int Vm = 0;
    bool jvp_ready = false;
    std::vector<int> last_its;
    // live kernel timing (ras_profile)
    struct ProfRec {
        int kind;
        cudaEvent_t a, b;
        double work;
    };
    bool prof_on = false;
    std::vector<ProfRec> prof_recs;
    // GMRES restart cycles: per-problem Arnoldi state on the device, and one
    // graph per operator kind with an IF node per Arnoldi step
    double *gm_H = nullptr, *gm_cs = nullptr, *gm_sn = nullptr, *gm_g = nullptr, *gm_target = nullptr;
    int *gm_its = nullptr, *gm_steps = nullptr, *gm_any = nullptr;
    int* h_any = nullptr;            // pinned
    bool use_graphs = true;
    unsigned long long gen = 1;      // bumped whenever a buffer, the layout, the options or the tuning change
    struct CycleGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        unsigned long long gen = 0;
        const double* V = nullptr;
        int m = 0;
        std::vector<long long> kps;                 // kernels per step
    };
    CycleGraph cg[3];                // by operator: 0 Jacobian action of Alg. 4, 1 global Jacobian, 2 with RAS
    // the RASPEN-function evaluation (Alg. 3: the local Newton sweeps of Alg. 1
    // in every subdomain) as one graph: init, a WHILE node over the sweep
    // steps, the factors at the local solutions and the prolongation
    struct SweepGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        unsigned long long gen = 0;
        const double* Fout = nullptr;
        int prec = -1;
        long long k_pre = 0, k_body = 0, k_post = 0;   // kernels of each part
    };
    SweepGraph sg;
    int* d_guard = nullptr;          // sweep steps taken + 1 (device)
    int* h_guard = nullptr;          // pinned
    cudaStream_t cap_st = nullptr;   // capture stream
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[RAS_K_COUNT] = {};
    long long prof_n[RAS_K_COUNT] = {};
    double prof_work[RAS_K_COUNT] = {};
    std::vector<std::pair<void*, size_t>> allocs;   // device allocations and their bytes
    size_t bytes = 0;
    std::vector<int> h_lists;                       // host copy of d_lists
    size_t cap_hscal = 0;                           // doubles in h_scal
    std::string err;
};

namespace {

constexpr int SS = ras::SEG_STRIDE;   // per-problem stride of scalar arrays

// NVTX range for tools (Nsight); costs a few nanoseconds when none is attached.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};
constexpr int NTILE = 5;              // register tiles 2, 4, 6, 8, 10
static_assert(NTILE == RAS_NTILE, "tile classes of the header");
static_assert(ras::VEC_BLOCKS == RAS_VEC_BLOCKS_MAX, "vector-kernel grid of the header");

int fail(ras_problem* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(h, RAS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(expr)                 \
    do {                          \
        int r_ = (expr);          \
        if (r_ < 0) return r_;    \
    } while (0)

void prof_flush(ras_problem* h) {
    for (auto& r : h->prof_recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            h->prof_ms[r.kind] += ms;
            h->prof_n[r.kind] += 1;
            h->prof_work[r.kind] += r.work;
        }
        h->ev_pool.push_back(r.a);
        h->ev_pool.push_back(r.b);
    }
    h->prof_recs.clear();
    cudaGetLastError();
}

cudaEvent_t prof_event(ras_problem* h) {
    if (h->ev_pool.empty()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
}

// Launch through `fn`; with profiling on, bracket it with events on the stream.
template <class Fn>
cudaError_t timed(ras_problem* h, int kind, double work, Fn fn) {
    if (!h->prof_on) return fn();
    cudaEvent_t a = prof_event(h), b = prof_event(h);
    if (!a || !b) return fn();
    cudaEventRecord(a, h->st);
    const cudaError_t e = fn();
    cudaEventRecord(b, h->st);
    h->prof_recs.push_back({kind, a, b, work});
    return e;
}

template <class T>
int dalloc(ras_problem* h, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(h, RAS_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    h->allocs.emplace_back((void*)*p, count * sizeof(T));
    h->bytes += count * sizeof(T);
    ++h->gen;
    return RAS_OK;
}

void dfree(ras_problem* h, void* p) {
    if (!p) return;
    ++h->gen;
    for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it) {
        if (it->first == p) {
            h->bytes -= it->second;
            h->allocs.erase(it);
            break;
        }
    }
    cudaFree(p);
}

size_t dcap(const ras_problem* h, const void* p) {
    for (const auto& a : h->allocs)
        if (a.first == p) return a.second;
    return 0;
}

// *p holds at least count elements afterwards (contents not kept on growth).
template <class T>
int ensure(ras_problem* h, T** p, size_t count) {
    if (count == 0) count = 1;
    if (*p && dcap(h, *p) >= count * sizeof(T)) return RAS_OK;
    dfree(h, *p);
    *p = nullptr;
    return dalloc(h, p, count);
}

// Balanced split of range(n) into s blocks, the first (n mod s) one node larger.
std::vector<std::pair<int, int>> split_blocks(int n, int s) {
    std::vector<std::pair<int, int>> out;
    int start = 0;
    for (int k = 0; k < s; ++k) {
        const int size = n / s + (k < n % s ? 1 : 0);
        out.emplace_back(start, start + size);
        start += size;
    }
    return out;
}

int validate_opts(ras_problem* h, const ras_opts& o) {
    if (!(o.tol > 0) || !(o.inner_tol > 0) || !(o.sigma >= 1.0) || !(o.eps0 > 0) || !(o.gamma > 0) ||
        !(o.gamma <= 1.0) || !(o.eps_min > 0) || !(o.eps0 >= o.eps_min) || o.kmax_outer_raspen < 0 ||
        o.kmax_outer_newton < 0 || o.kmax_inner < 0 || o.max_halvings < 0 || o.gmres_restart < 1 ||
        o.gmres_restart > 30 || o.gmres_maxit < 1 || !(o.gmres_rtol > 0) || !(o.floor_factor >= 0) ||
        (o.precision != RAS_FP64 && o.precision != RAS_MIXED) || o.ir_max < 0 || !(o.ir_rtol >= 0) ||
        !std::isfinite(o.kappa) || o.jvp_ir < 0 || o.jvp_ir > 8 || o.wait_test < 0 || o.wait_test > 1)
        return fail(h, RAS_EINVAL,
                    "invalid options (need tol, inner_tol, eps0, gamma, eps_min > 0, eps0 >= eps_min, "
                    "gamma <= 1, sigma >= 1, 1 <= gmres_restart <= 30, precision RAS_FP64|RAS_MIXED)");
    return RAS_OK;
}

NewtonParams inner_params(const ras_opts& o) {
    NewtonParams np{};
    np.eps_min = o.eps_min;
    np.gamma = o.gamma;
    np.sigma = o.sigma;
    np.tol = o.inner_tol;
    np.floor_factor = o.floor_factor;
    np.ir_rtol = o.ir_rtol;
    np.kmax = o.kmax_inner;
    np.max_halvings = o.max_halvings;
    np.ir_max = (o.precision == RAS_MIXED) ? o.ir_max : 0;
    return np;
}

int alloc_factor_pools(ras_problem* h) {
    const int prec = h->o.precision;
    const size_t es = (prec == RAS_MIXED) ? sizeof(float) : sizeof(double);
    char* g = static_cast<char*>(h->gpool);
    char* w = static_cast<char*>(h->wpool);
    if (h->own_factors) {
        TRY(ensure(h, &g, (size_t)h->Gsum * es));
        h->gpool = g;
    }
    TRY(ensure(h, &w, (size_t)h->Lsum * es));
    h->wpool = w;
    h->gprec = prec;
    return RAS_OK;
}

int sync(ras_problem* h) {
    CK(cudaStreamSynchronize(h->st));
    if (h->prof_on && h->prof_recs.size() > 2048) prof_flush(h);
    return RAS_OK;
}

// Copy opts.wait_test into d_err[1], where the streamed solves read it.
int push_wait_test(ras_problem* h) {
    if (!h->d_err) return RAS_OK;
    h->h_wait_test = h->o.wait_test;
    CK(cudaMemcpyAsync(h->d_err + 1, &h->h_wait_test, sizeof(int), cudaMemcpyHostToDevice, h->st));
    return RAS_OK;
}

// RAS_ETIMEOUT if a kernel reported that a bounded wait ran out (then clears it).
int check_err(ras_problem* h) {
    int v = 0;
    CK(cudaMemcpyAsync(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (v != 0) {
        CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->st));
        CK(cudaStreamSynchronize(h->st));
        return fail(h, RAS_ETIMEOUT, "a device-side wait exceeded its limit");
    }
    return RAS_OK;
}

// A device-side failure found after the solve (a bounded wait that ran out):
// the call's stats carry the same status as its return value.
int check_err_stats(ras_problem* h, ras_stats* stats, int count) {
    const int e = check_err(h);
    if (e != RAS_OK && stats)
        for (int k = 0; k < count; ++k) stats[k].status = e;
    return e;
}

size_t prec_bytes(const ras_problem* h) { return h->o.precision == RAS_MIXED ? sizeof(float) : sizeof(double); }

// Algorithmic work of a factorisation: 16 bl^3 bw flops per subdomain (block-
// tridiagonal Gauss-Jordan = no-fill band LU count; bl nodes per block row,
// bw block rows). With `ls`: only active
// subdomains, or (skip_skipped) all but those of non-participating problems.
double factor_flops(const ras_problem* h, const std::vector<LocalState>* ls, bool skip_skipped) {
    double w = 0.0;
    for (int i = 0; i < h->nsub; ++i) {
        if (ls && !skip_skipped && !(*ls)[i].active) continue;
        if (ls && skip_skipped && (*ls)[i].status == ras::ST_SKIP) continue;
        const double bl = h->subs[i].bl, bw = h->subs[i].bw;
        w += 16.0 * bl * bl * bl * bw;
    }
    return w;
}

// Bytes of one two-pass block solve over the factors of the problems in mask.
double solve_bytes(const ras_problem* h, const std::vector<int>* mask) {
    double b = 0.0;
    for (int i = 0; i < h->nsub; ++i) {
        const SubDev& s = h->subs[i];
        if (mask && !(*mask)[s.prob]) continue;
        b += 2.0 * (double)s.bw * s.mp * s.mp * (double)prec_bytes(h);
    }
    return b;
}

long long plane(const ras_problem* h, int p) { return h->probs[p].nn; }

double resid_bytes(const ras_problem* h) { return (h->f ? 48.0 : 40.0) * (double)plane(h, 0); }

// Block table of row `row`: tune.vec_blocks blocks spread over the problems with
// m[p] != 0 in proportion to their segment lengths (at least one each, and
// no more than one per 512 elements).
int build_grid(ras_problem* h, int row, const std::vector<int>& m) {
    if (h->last_mask[row] == m) return RAS_OK;
    const int P = h->nprob, cap = ras::VEC_BLOCKS + P;
    double tot = 0.0;
    for (int p = 0; p < P; ++p)
        if (m[p]) tot += (double)h->segs[p].len;
    std::vector<int> nbps(P, 0);
    std::vector<int2> tab;
    for (int p = 0; p < P; ++p) {
        if (!m[p]) continue;
        const double len = (double)h->segs[p].len;
        const int most = (int)std::max(1.0, std::ceil(len / 512.0));
        const int vb = h->tune.vec_blocks;
        int nb = (int)std::floor(vb * len / tot + 0.5);
        nb = std::max(1, std::min(nb, std::min(most, vb)));
        nbps[p] = nb;
        for (int b = 0; b < nb; ++b) tab.push_back(make_int2(p, b));
    }
    if ((int)tab.size() > cap) return fail(h, RAS_EINVAL, "block table overflow");
    CK(cudaMemcpyAsync(h->d_nbps + row * P, nbps.data(), P * sizeof(int), cudaMemcpyHostToDevice, h->st));
    if (!tab.empty())
        CK(cudaMemcpyAsync(h->d_tab + (size_t)row * cap, tab.data(), tab.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, h->st));
    h->ntab[row] = (int)tab.size();
    h->last_mask[row] = m;
    return RAS_OK;
}

ras::SegGrid seg_grid(const ras_problem* h, int row) {
    ras::SegGrid g;
    g.tab = h->d_tab + (size_t)row * (ras::VEC_BLOCKS + h->nprob);
    g.nbps = h->d_nbps + row * h->nprob;
    g.nblocks = h->ntab[row];
    return g;
}

// The GMRES cycle's table (row 3): every entry launched, unused ones idle.
ras::SegGrid cycle_grid(const ras_problem* h) {
    ras::SegGrid g;
    const int cap = ras::VEC_BLOCKS + h->nprob;
    g.tab = h->d_tab + (size_t)3 * cap;
    g.nbps = h->d_nbps + 3 * h->nprob;
    g.nblocks = cap;
    return g;
}

// Rebuild row 3 on the device for the problems flagged in d_mask row 0.
int cycle_table(ras_problem* h) {
    const int cap = ras::VEC_BLOCKS + h->nprob;
    CK(timed(h, RAS_K_OTHER, 0.0, [&] {
        return ras::launch_seg_table(h->st, h->nprob, h->d_mask, h->d_segs, h->tune.vec_blocks, cap,
                                     h->d_tab + (size_t)3 * cap, h->d_nbps + 3 * h->nprob, h->d_toff);
    }));
    return RAS_OK;
}

int set_mask(ras_problem* h, int row, const std::vector<int>& m) {
    CK(cudaMemcpyAsync(h->d_mask + row * h->nprob, m.data(), h->nprob * sizeof(int), cudaMemcpyHostToDevice,
                       h->st));
    return build_grid(h, row, m);
}

// Per-problem squared norms of the segments of v (problems of mask row
// `row`), into h->scal[p * SS] (device) and h->h_scal[p * SS] (host).
int seg_norms2(ras_problem* h, const double* v, int row) {
    const int P = h->nprob;
    const ras::SegGrid g = seg_grid(h, row);
    double len = 0.0;
    for (int p = 0; p < P; ++p)
        if (h->last_mask[row][p]) len += 8.0 * h->segs[p].len;
    CK(timed(h, RAS_K_KRYLOV, len, [&] {
        return ras::launch_seg_dot(h->st, g, h->d_segs, v, h->L, 1, v, h->partials);
    }));
    CK(timed(h, RAS_K_OTHER, 0.0,
             [&] { return ras::launch_seg_reduce(h->st, P, g.nbps, 1, h->partials, h->scal); }));
    CK(cudaMemcpyAsync(h->h_scal, h->scal, (size_t)P * SS * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    return sync(h);
}

// ||F(x + alpha d, eps)|| and the rounding-floor norm (problem 0); writes F if given.
int residual_norm(ras_problem* h, const double* x, const double* d, double alpha, double eps, double* Fout,
                  double& nrm, double& flr) {
    const long long N = plane(h, 0);
    CK(timed(h, RAS_K_RESIDUAL, resid_bytes(h), [&] {
        return ras::launch_residual_global(h->st, h->probs[0], x, x + N, d, d ? d + N : nullptr, alpha, eps, Fout,
                                           Fout ? Fout + N : nullptr, h->partials, 1);
    }));
    CK(timed(h, RAS_K_OTHER, 0.0,
             [&] { return ras::launch_reduce_partials(h->st, h->partials, ras::VEC_BLOCKS, 2, h->scal); }));
    CK(cudaMemcpyAsync(h->h_scal, h->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    nrm = std::sqrt(h->h_scal[0]);
    flr = std::sqrt(h->h_scal[1]);
    return RAS_OK;
}

int copy_in(ras_problem* h, double* dst, int p, const double* y, const double* pp) {
    const long long N = plane(h, p), o = h->probs[p].ofs;
    CK(cudaMemcpyAsync(dst + o, y, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(dst + o + N, pp, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    return RAS_OK;
}

int copy_out(ras_problem* h, const double* src, int p, double* y, double* pp) {
    const long long N = plane(h, p), o = h->probs[p].ofs;
    if (y) CK(cudaMemcpyAsync(y, src + o, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (pp) CK(cudaMemcpyAsync(pp, src + o + N, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    return RAS_OK;
}

void stats_clear(ras_stats* s, int count) {
    if (!s) return;
    std::memset(s, 0, sizeof(ras_stats) * count);
}

// Factorisation of the wide-block subdomains (none: nothing launched).
template <typename T>
cudaError_t launch_factor_wide(ras_problem* h, int only_active) {
    return ras::launch_local_factor_big<T>(h->st, (int)h->h_wide.size(), h->d_wide, h->d_subs, h->d_probs, h->X,
                                           h->ls, h->cpool, h->coef, (T*)h->gpool, only_active);
}

// Factorisation launches: FP32 one per register-tile class, FP64 one, and
// one for the wide-block subdomains.
template <typename T>
// nwork: most subdomains that factorise in this sweep (the active count, or
// every subdomain); up to tune.factor_wide_max of a class (default: one per
// SM) the 1024-thread kernel is used.
int launch_factor(ras_problem* h, int only_active, double flops, int nwork) {
    if (sizeof(T) == sizeof(float)) {
        if (h->sms == 0) {
            int dev = 0;
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
        }
        bool first = true;   // the profile books the flops on the first launch of the sweep
        for (int c = 0; c < NTILE; ++c) {
            if (h->tile_cnt[c] == 0) continue;
            const int thr = h->tune.factor_wide_max[c] < 0 ? h->sms : h->tune.factor_wide_max[c];
            const int wide = std::min(nwork, h->tile_cnt[c]) <= thr ? 1 : 0;
            CK(timed(h, RAS_K_FACTOR, first ? flops : 0.0, [&] {
                return ras::launch_local_factor_f32(h->st, 2 * (c + 1), h->tile_cnt[c], h->d_lists + h->tile_off[c],
                                                    h->d_subs, h->d_probs, h->X, h->ls, h->cpool, h->coef,
                                                    (float*)h->gpool, only_active, wide);
            }));
            first = false;
        }
        if (!h->h_wide.empty())
            CK(timed(h, RAS_K_FACTOR, first ? flops : 0.0, [&] { return launch_factor_wide<T>(h, only_active); }));
        return RAS_OK;
    }
    CK(timed(h, RAS_K_FACTOR, flops, [&] {
        cudaError_t e = cudaSuccess;
        if (h->maxm > 0)
            e = ras::launch_local_factor<T>(h->st, h->nsub, h->maxm, h->d_subs, h->d_probs, h->X, h->ls, h->cpool,
                                            h->coef, (T*)h->gpool, only_active);
        if (e == cudaSuccess) e = launch_factor_wide<T>(h, only_active);
        return e;
    }));
    return RAS_OK;
}

// Sweep-step factorisation for a graph: both FP32 kernels of every class,
// the device's active count choosing which one works (the rule of
// launch_factor).
template <typename T>
int launch_factor_sel(ras_problem* h) {
    if (sizeof(T) == sizeof(float)) {
        for (int c = 0; c < NTILE; ++c) {
            if (h->tile_cnt[c] == 0) continue;
            const int thr = h->tune.factor_wide_max[c] < 0 ? h->sms : h->tune.factor_wide_max[c];
            for (int wide = 0; wide < 2; ++wide)
                CK(ras::launch_local_factor_f32(h->st, 2 * (c + 1), h->tile_cnt[c], h->d_lists + h->tile_off[c],
                                                h->d_subs, h->d_probs, h->X, h->ls, h->cpool, h->coef,
                                                (float*)h->gpool, 1, wide, ras::FactorSel{h->d_active, thr}));
        }
        CK(launch_factor_wide<T>(h, 1));
        return RAS_OK;
    }
    if (h->maxm > 0)
        CK(ras::launch_local_factor<T>(h->st, h->nsub, h->maxm, h->d_subs, h->d_probs, h->X, h->ls, h->cpool,
                                       h->coef, (T*)h->gpool, 1));
    CK(launch_factor_wide<T>(h, 1));
    return RAS_OK;
}

// Capture what fn enqueues on h->st into a new graph (*out); *count: the
// kernels it launched.
template <class Fn>
int capture_graph(ras_problem* h, Fn fn, cudaGraph_t* out, long long* count) {
    *out = nullptr;
    CK(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeRelaxed));
    const cudaStream_t saved = h->st;
    long long c = 0;
    h->st = h->cap_st;
    ras::t_capture_count = &c;
    const int rc = fn();
    ras::t_capture_count = nullptr;
    h->st = saved;
    const cudaError_t e = cudaStreamEndCapture(h->cap_st, out);
    *count = c;
    if (rc < 0) {
        if (*out) cudaGraphDestroy(*out);
        *out = nullptr;
        cudaGetLastError();
        return rc;
    }
    if (e != cudaSuccess) return fail(h, RAS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    return RAS_OK;
}

void destroy_sweep_graph(ras_problem::SweepGraph& G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G = ras_problem::SweepGraph{};
}

// The evaluation as one graph: [init] -> [condition] -> WHILE { factor
// (device choice of kernel), direction, line search, condition } ->
// [factors at x^(i), prolongation into Fout]. The condition is the host
// loop's: active subdomains left and at most kmax_inner + 2 steps.
template <typename T>
int build_sweep_graph(ras_problem* h, double* Fout, const NewtonParams& np) {
    auto& G = h->sg;
    destroy_sweep_graph(G);
    if (!h->cap_st) CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    CK(cudaGraphCreate(&G.graph, 0));
    T* gp = (T*)h->gpool;
    T* wp = (T*)h->wpool;
    const int limit = h->o.kmax_inner + 1;
    int rc = RAS_OK;
    cudaGraph_t part = nullptr;
    cudaGraphNode_t n_pre = nullptr, n_c0 = nullptr, n_w = nullptr, n_post = nullptr;
    cudaGraphConditionalHandle w{};
    cudaError_t e = cudaGraphConditionalHandleCreate(&w, G.graph, 0u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) rc = fail(h, RAS_ECUDA, std::string("graph: ") + cudaGetErrorString(e));
    if (rc == RAS_OK)
        rc = capture_graph(h, [&]() -> int {
            CK(cudaMemsetAsync(h->d_active, 0, sizeof(int), h->st));
            CK(ras::launch_local_init(h->st, h->nsub, h->d_subs, h->d_probs, h->X, h->ls, h->d_pstart, np, h->cpool,
                                      h->Kpool, h->d_active));
            return RAS_OK;
        }, &part, &G.k_pre);
    if (rc == RAS_OK) {
        e = cudaGraphAddChildGraphNode(&n_pre, G.graph, nullptr, 0, part);
        cudaGraphDestroy(part);
        part = nullptr;
        if (e == cudaSuccess)
            e = ras::add_sweep_cond_node(G.graph, n_pre, w, h->d_active, h->d_guard, limit, 1, &n_c0);
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = w;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (e == cudaSuccess) e = cudaGraphAddNode(&n_w, G.graph, &n_c0, nullptr, 1, &cp);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(h->cap_st, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) rc = fail(h, RAS_ECUDA, std::string("graph: ") + cudaGetErrorString(e));
        if (rc == RAS_OK) {
            const cudaStream_t saved = h->st;
            long long c = 0;
            h->st = h->cap_st;
            ras::t_capture_count = &c;
            rc = [&]() -> int {
                TRY(launch_factor_sel<T>(h));
                CK(ras::launch_local_direction<T>(h->st, h->nsub, h->tune.solve_ctas_per_sm, h->d_subs, h->d_probs,
                                                  h->ls, np, h->coef, gp, h->Kpool, h->dpool, h->rpool, wp, h->d_err,
                                                  h->d_order, h->d_ticket));
                CK(ras::launch_local_direction_wide<T>(h->st, (int)h->h_wide.size(), h->d_wide, h->d_subs,
                                                       h->d_probs, h->ls, np, h->coef, gp, h->Kpool, h->dpool,
                                                       h->rpool, wp, h->d_err));
                CK(cudaMemsetAsync(h->d_active, 0, sizeof(int), h->st));
                CK(ras::launch_local_linesearch(h->st, h->nsub, h->d_subs, h->d_probs, h->X, h->ls, np, h->cpool,
                                                h->dpool, h->Kpool, h->Ktpool, h->d_active));
                CK(ras::launch_sweep_cond(h->st, w, h->d_active, h->d_guard, limit, 0));
                return RAS_OK;
            }();
            ras::t_capture_count = nullptr;
            h->st = saved;
            cudaGraph_t body = nullptr;
            e = cudaStreamEndCapture(h->cap_st, &body);
            if (rc == RAS_OK && e != cudaSuccess)
                rc = fail(h, RAS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            G.k_body = c;
        }
    }
    if (rc == RAS_OK)
        rc = capture_graph(h, [&]() -> int {
            TRY(launch_factor<T>(h, 0, 0.0, h->nsub));
            CK(ras::launch_local_prolong(h->st, h->nsub, h->d_subs, h->d_probs, h->ls, h->cpool, Fout));
            return RAS_OK;
        }, &part, &G.k_post);
    if (rc == RAS_OK) {
        e = cudaGraphAddChildGraphNode(&n_post, G.graph, &n_w, 1, part);
        cudaGraphDestroy(part);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, G.graph, 0);
        if (e != cudaSuccess) rc = fail(h, RAS_ECUDA, std::string("graph: ") + cudaGetErrorString(e));
    }
    cudaGetLastError();
    if (rc != RAS_OK) {
        destroy_sweep_graph(G);
        return rc;
    }
    G.gen = h->gen;
    G.Fout = Fout;
    G.prec = h->o.precision;
    return RAS_OK;
}

int evaluation_results(ras_problem* h, const std::vector<double>& pstart, ras_stats* stats);

// --------------------------------------------------------------- Alg. 3
// RASPEN function of the problems with pstart[p] > 0 (eps at which their
// local solves start); per-problem counters into stats[p] (may be null).
template <typename T>
int ras_apply_T(ras_problem* h, const std::vector<double>& pstart, double* Fout, ras_stats* stats) {
    Range range("ras: RASPEN function (local Newton solves)");
    const NewtonParams np = inner_params(h->o);
    T* gp = (T*)h->gpool;
    T* wp = (T*)h->wpool;
    CK(cudaMemcpyAsync(h->d_pstart, pstart.data(), h->nprob * sizeof(double), cudaMemcpyHostToDevice, h->st));
    if (h->use_graphs && !h->prof_on) {
        // the whole evaluation as one graph launch (profiled runs take the loop below)
        if (h->sms == 0) {
            int dev = 0;
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
        }
        TRY(ensure(h, &h->d_guard, (size_t)1));
        if (!h->h_guard && cudaMallocHost((void**)&h->h_guard, sizeof(int)) != cudaSuccess) {
            h->h_guard = nullptr;
            return fail(h, RAS_ENOMEM, "pinned host allocation failed");
        }
        auto& G = h->sg;
        if (!G.exec || G.gen != h->gen || G.Fout != Fout || G.prec != h->o.precision)
            TRY(build_sweep_graph<T>(h, Fout, np));
        CK(cudaGraphLaunch(G.exec, h->st));
        CK(cudaMemcpyAsync(h->h_guard, h->d_guard, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        TRY(sync(h));
        ras::add_launches(G.k_pre + 1 + (long long)std::max(0, *h->h_guard - 1) * G.k_body + G.k_post);
        return evaluation_results(h, pstart, stats);
    }
    CK(cudaMemsetAsync(h->d_active, 0, sizeof(int), h->st));
    CK(timed(h, RAS_K_INIT, 0.0, [&] {
        return ras::launch_local_init(h->st, h->nsub, h->d_subs, h->d_probs, h->X, h->ls, h->d_pstart, np,
                                      h->cpool, h->Kpool, h->d_active);
    }));
    CK(cudaMemcpyAsync(h->h_active, h->d_active, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    std::vector<LocalState> before, after;
    auto read_ls = [&](std::vector<LocalState>& v) -> int {
        v.resize(h->nsub);
        CK(cudaMemcpyAsync(v.data(), h->ls, h->nsub * sizeof(LocalState), cudaMemcpyDeviceToHost, h->st));
        return sync(h);
    };
    int guard = 0;
    while (*h->h_active > 0 && guard++ <= h->o.kmax_inner + 1) {
        double fl = 0.0;
        if (h->prof_on) {
            TRY(read_ls(before));
            fl = factor_flops(h, &before, false);
        }
        TRY(launch_factor<T>(h, 1, fl, *h->h_active));
        CK(timed(h, RAS_K_DIRECTION, 0.0, [&] {
            cudaError_t e = ras::launch_local_direction<T>(h->st, h->nsub, h->tune.solve_ctas_per_sm, h->d_subs,
                                                           h->d_probs, h->ls, np, h->coef, gp, h->Kpool, h->dpool,
                                                           h->rpool, wp, h->d_err, h->d_order, h->d_ticket);
            if (e == cudaSuccess)
                e = ras::launch_local_direction_wide<T>(h->st, (int)h->h_wide.size(), h->d_wide, h->d_subs,
                                                        h->d_probs, h->ls, np, h->coef, gp, h->Kpool, h->dpool,
                                                        h->rpool, wp, h->d_err);
            return e;
        }));
        const size_t dir_rec = h->prof_recs.size();
        CK(cudaMemsetAsync(h->d_active, 0, sizeof(int), h->st));
        CK(timed(h, RAS_K_LINESEARCH, 0.0, [&] {
            return ras::launch_local_linesearch(h->st, h->nsub, h->d_subs, h->d_probs, h->X, h->ls, np, h->cpool,
                                                h->dpool, h->Kpool, h->Ktpool, h->d_active);
        }));
        CK(cudaMemcpyAsync(h->h_active, h->d_active, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        TRY(sync(h));
        if (h->prof_on && dir_rec >= 1 && dir_rec <= h->prof_recs.size()) {
            TRY(read_ls(after));
            double bytes = 0.0;
            for (int i = 0; i < h->nsub; ++i) {
                const double mp = h->subs[i].mp;
                bytes += (after[i].solves - before[i].solves) * 2.0 * mp * mp * h->subs[i].bw * sizeof(T);
            }
            h->prof_recs[dir_rec - 1].work = bytes;
        }
    }
    // factors at x^(i) = x + P_i C_i(x) for the Jacobian action (Alg. 4)
    double fl_all = 0.0;
    if (h->prof_on) {
        TRY(read_ls(before));
        fl_all = factor_flops(h, &before, true);
    }
    TRY(launch_factor<T>(h, 0, fl_all, h->nsub));
    CK(timed(h, RAS_K_OTHER, 0.0, [&] {
        return ras::launch_local_prolong(h->st, h->nsub, h->d_subs, h->d_probs, h->ls, h->cpool, Fout);
    }));
    return evaluation_results(h, pstart, stats);
}

// Local states after an evaluation: counters into stats, the local
// iteration counts, and the first local failure.
int evaluation_results(ras_problem* h, const std::vector<double>& pstart, ras_stats* stats) {
    std::vector<LocalState> ls(h->nsub);
    CK(cudaMemcpyAsync(ls.data(), h->ls, h->nsub * sizeof(LocalState), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    int worst = RAS_OK;
    h->last_its.assign(h->nsub, 0);
    std::vector<int> itmax(h->nprob, 0), fails(h->nprob, 0), halv(h->nprob, 0), exh(h->nprob, 0);
    std::vector<long long> itsum(h->nprob, 0);
    for (int i = 0; i < h->nsub; ++i) {
        const int p = h->subs[i].prob;
        if (ls[i].status == ras::ST_SKIP) continue;
        h->last_its[i] = ls[i].k;
        itmax[p] = std::max(itmax[p], ls[i].k);
        itsum[p] += ls[i].k;
        halv[p] += ls[i].halvings;
        exh[p] += ls[i].exhausted;
        if (ls[i].status < 0) {
            ++fails[p];
            // Alg. 1 stopped at kmax_inner returns its iterate: the
            // evaluation goes on with it (counted in local_failures); a
            // non-finite residual or a singular block ends it
            if (ls[i].status != ras::ST_ENOCONV) worst = std::min(worst, ls[i].status);
        }
    }
    h->jvp_ready = (worst >= 0);
    if (stats) {
        for (int p = 0; p < h->nprob; ++p) {
            if (!(pstart[p] > 0)) continue;
            ras_stats& s = stats[p];
            s.evaluations += 1;
            s.inner_its_max += itmax[p];
            s.inner_its_sum += itsum[p];
            s.halvings += halv[p];
            s.exhausted += exh[p];
            s.local_failures += fails[p];
            s.eps_final = h->o.eps_min;
        }
    }
    if (worst < 0) {
        int nf = 0;
        for (int v : fails) nf += v;
        return fail(h, worst, "local Newton solve failed in " + std::to_string(nf) + " subdomain(s)");
    }
    return RAS_OK;
}

int ras_apply_internal(ras_problem* h, const std::vector<double>& pstart, double* Fout, ras_stats* stats) {
    TRY(alloc_factor_pools(h));
    if (h->o.precision == RAS_MIXED) return ras_apply_T<float>(h, pstart, Fout, stats);
    return ras_apply_T<double>(h, pstart, Fout, stats);
}

// Alg. 4 for the problems flagged in `mask` (device copy: d_mask row 0), or all.
int jvp_internal(ras_problem* h, const double* D, double* O, const std::vector<int>* mask) {
    const int nir = (h->o.precision == RAS_MIXED) ? h->o.jvp_ir : 0;
    const int* dm = mask ? h->d_mask : nullptr;
    CK(timed(h, RAS_K_JVP, solve_bytes(h, mask) * (1 + nir), [&] {
        const int nw = (int)h->h_wide.size();
        cudaError_t e;
        if (h->o.precision == RAS_MIXED) {
            e = ras::launch_local_jvp<float>(h->st, h->nsub, h->tune.solve_ctas_per_sm, h->d_subs, h->d_probs,
                                             (const float*)h->gpool, (float*)h->wpool, h->coef, h->dpool, h->rpool,
                                             h->Ktpool, nir, D, O, dm, h->d_err, h->d_order, h->d_ticket);
            if (e == cudaSuccess)
                e = ras::launch_local_jvp_wide<float>(h->st, nw, h->d_wide, h->d_subs, h->d_probs,
                                                      (const float*)h->gpool, (float*)h->wpool, h->coef, h->dpool,
                                                      h->rpool, h->Ktpool, nir, D, O, dm, h->d_err);
            return e;
        }
        e = ras::launch_local_jvp<double>(h->st, h->nsub, h->tune.solve_ctas_per_sm, h->d_subs, h->d_probs,
                                          (const double*)h->gpool, (double*)h->wpool, h->coef, h->dpool, h->rpool,
                                          h->Ktpool, 0, D, O, dm, h->d_err, h->d_order, h->d_ticket);
        if (e == cudaSuccess)
            e = ras::launch_local_jvp_wide<double>(h->st, nw, h->d_wide, h->d_subs, h->d_probs,
                                                   (const double*)h->gpool, (double*)h->wpool, h->coef, h->dpool,
                                                   h->rpool, h->Ktpool, 0, D, O, dm, h->d_err);
        return e;
    }));
    return RAS_OK;
}

// Factorise R_i F'(x, eps) P_i for every subdomain (x = h->X, c = 0).
int factor_at(ras_problem* h, double eps) {
    TRY(alloc_factor_pools(h));
    std::vector<LocalState> ls(h->nsub);
    for (auto& s : ls) {
        std::memset(&s, 0, sizeof(s));
        s.eps = eps;
        s.active = 1;
    }
    CK(cudaMemsetAsync(h->cpool, 0, h->Lsum * sizeof(double), h->st));
    CK(cudaMemcpyAsync(h->ls, ls.data(), h->nsub * sizeof(LocalState), cudaMemcpyHostToDevice, h->st));
    if (h->o.precision == RAS_MIXED) {
        TRY(launch_factor<float>(h, 0, factor_flops(h, nullptr, false), h->nsub));
    } else {
        TRY(launch_factor<double>(h, 0, factor_flops(h, nullptr, false), h->nsub));
    }
    CK(cudaMemcpyAsync(ls.data(), h->ls, h->nsub * sizeof(LocalState), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    h->jvp_ready = false;
    for (auto& s : ls)
        if (s.status < 0) return fail(h, s.status, "singular local Jacobian");
    return RAS_OK;
}

int precond_internal(ras_problem* h, const double* R, double* Zo) {
    CK(timed(h, RAS_K_PRECOND, solve_bytes(h, nullptr), [&] {
        const int nw = (int)h->h_wide.size();
        cudaError_t e;
        if (h->o.precision == RAS_MIXED) {
            e = ras::launch_local_precond<float>(h->st, h->nsub, h->tune.solve_ctas_per_sm, h->d_subs, h->d_probs,
                                                 (const float*)h->gpool, (float*)h->wpool, R, Zo, h->d_err,
                                                 h->d_order, h->d_ticket);
            if (e == cudaSuccess)
                e = ras::launch_local_precond_wide<float>(h->st, nw, h->d_wide, h->d_subs, h->d_probs,
                                                          (const float*)h->gpool, (float*)h->wpool, R, Zo, h->d_err);
            return e;
        }
        e = ras::launch_local_precond<double>(h->st, h->nsub, h->tune.solve_ctas_per_sm, h->d_subs, h->d_probs,
                                              (const double*)h->gpool, (double*)h->wpool, R, Zo, h->d_err,
                                              h->d_order, h->d_ticket);
        if (e == cudaSuccess)
            e = ras::launch_local_precond_wide<double>(h->st, nw, h->d_wide, h->d_subs, h->d_probs,
                                                       (const double*)h->gpool, (double*)h->wpool, R, Zo, h->d_err);
        return e;
    }));
    return RAS_OK;
}

// --------------------------------------------------------------- GMRES
// Restarted GMRES(m) for every problem p with part[p] != 0, in lockstep:
// CGS2 Arnoldi with segmented (per-problem) reductions, Givens rotations and
// stop tests on the device, x0 = 0, right preconditioning when `prec`.
// A(in, out, mask) and M(in, out, mask) act on the problems flagged in
// d_mask row 0, which the Givens kernel keeps equal to the problems still
// iterating. The host reads each restart cycle once (back-substitution and
// update); the cycle itself is one graph launch or a step-by-step loop.
// Resumable GMRES for the serving loop: per problem, `fresh` starts from
// x = 0 and sets its stop target from ||b||; otherwise x holds the iterate of
// earlier cycles and `target` the target set then. At most max_cycles restart
// cycles run; `pending` reports the problems still iterating. Restart cycles
// only carry x, so a solve split over calls is the same sequence of cycles.
struct GmresResume {
    std::vector<int> fresh;
    std::vector<double> target;
    int max_cycles = 1;
    std::vector<int> pending;
};

// Arnoldi step j of a GMRES(m) cycle for the problems flagged in d_mask row
// 0 (the device flags that the Givens kernel clears): the operator
// (w = A v_j, or A M v_j), two CGS passes against v_0 .. v_j, the norm, the
// Givens update of the Hessenberg column and the stop test (device state
// gm_*), and v_{j+1} = w / ||w||. Only enqueues work: nothing reads the host,
// so the same sequence runs step by step or captured in a graph. The
// segmented kernels use the cycle's table (row 3), which is rebuilt on the
// device for the problems still iterating after every Givens update.
template <class Aop, class Mop>
int enqueue_step(ras_problem* h, int j, bool prec, Aop& A, Mop& M, const std::vector<int>& cyc, double seglen) {
    const int P = h->nprob, m = h->o.gmres_restart;
    const long long L = h->L;
    double* V = h->V;
    double* vj = V + (long long)j * L;
    double* w = V + (long long)(j + 1) * L;
    if (prec) {
        TRY(M(vj, h->Z, cyc));
        TRY(A(h->Z, w, cyc));
    } else {
        TRY(A(vj, w, cyc));
    }
    const ras::SegGrid gr = cycle_grid(h);
    const double dbytes = 8.0 * seglen * (j + 2), abytes = 8.0 * seglen * (j + 3);
    double* h1 = h->scal;
    double* h2 = h->scal + (size_t)P * SS;
    double* n2 = h->scal + (size_t)2 * P * SS;
    CK(timed(h, RAS_K_KRYLOV, dbytes,
             [&] { return ras::launch_seg_dot(h->st, gr, h->d_segs, V, L, j + 1, w, h->partials); }));
    CK(timed(h, RAS_K_OTHER, 0.0, [&] { return ras::launch_seg_reduce(h->st, P, gr.nbps, j + 1, h->partials, h1); }));
    CK(timed(h, RAS_K_KRYLOV, abytes,
             [&] { return ras::launch_seg_axpy(h->st, gr, h->d_segs, V, L, j + 1, h1, -1.0, w); }));
    CK(timed(h, RAS_K_KRYLOV, dbytes,
             [&] { return ras::launch_seg_dot(h->st, gr, h->d_segs, V, L, j + 1, w, h->partials); }));
    CK(timed(h, RAS_K_OTHER, 0.0, [&] { return ras::launch_seg_reduce(h->st, P, gr.nbps, j + 1, h->partials, h2); }));
    CK(timed(h, RAS_K_KRYLOV, abytes,
             [&] { return ras::launch_seg_axpy(h->st, gr, h->d_segs, V, L, j + 1, h2, -1.0, w); }));
    CK(timed(h, RAS_K_KRYLOV, 8.0 * seglen,
             [&] { return ras::launch_seg_dot(h->st, gr, h->d_segs, w, L, 1, w, h->partials); }));
    CK(timed(h, RAS_K_OTHER, 0.0, [&] { return ras::launch_seg_reduce(h->st, P, gr.nbps, 1, h->partials, n2); }));
    CK(timed(h, RAS_K_OTHER, 0.0, [&] {
        return ras::launch_gmres_givens(h->st, P, m, j, h->d_mask, h1, h2, n2, h->gm_H, h->gm_cs, h->gm_sn, h->gm_g,
                                        h->gm_its, h->gm_steps, h->gm_target, h->o.gmres_maxit, h->gm_any);
    }));
    TRY(cycle_table(h));
    CK(timed(h, RAS_K_KRYLOV, 16.0 * seglen,
             [&] { return ras::launch_seg_scale(h->st, gr, h->d_segs, w, n2, 1.0, w); }));
    return RAS_OK;
}

void destroy_cycle_graph(ras_problem::CycleGraph& G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G = ras_problem::CycleGraph{};
}

// One GMRES(m) cycle as a graph: for j = 0 .. m-1 an IF node holding Arnoldi
// step j (captured from enqueue_step), its condition set by a one-thread
// kernel after step j-1 from the flag the Givens kernel leaves (step 0 always
// runs). A cycle that stops after k steps runs k bodies and skips the rest.
template <class Aop, class Mop>
int build_cycle_graph(ras_problem* h, int op, bool prec, Aop& A, Mop& M, const std::vector<int>& cyc,
                      double seglen) {
    auto& G = h->cg[op];
    destroy_cycle_graph(G);
    const int m = h->o.gmres_restart;
    if (!h->cap_st) CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    CK(cudaGraphCreate(&G.graph, 0));
    std::vector<cudaGraphConditionalHandle> cond(m);
    for (int j = 0; j < m; ++j)
        CK(cudaGraphConditionalHandleCreate(&cond[j], G.graph, j == 0 ? 1u : 0u, cudaGraphCondAssignDefault));
    G.kps.assign(m, 0);
    cudaGraphNode_t prev = nullptr;
    const cudaStream_t saved = h->st;
    int rc = RAS_OK;
    for (int j = 0; j < m && rc == RAS_OK; ++j) {
        cudaError_t e = cudaSuccess;
        if (j > 0) {
            cudaGraphNode_t sc = nullptr;
            e = ras::add_set_conditional_node(G.graph, prev, cond[j], h->gm_any, &sc);
            prev = sc;
        }
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond[j];
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, G.graph, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &cp);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(h->cap_st, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            rc = fail(h, RAS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            break;
        }
        long long count = 0;
        h->st = h->cap_st;
        ras::t_capture_count = &count;
        rc = enqueue_step(h, j, prec, A, M, cyc, seglen);
        ras::t_capture_count = nullptr;
        h->st = saved;
        cudaGraph_t body = nullptr;
        e = cudaStreamEndCapture(h->cap_st, &body);
        if (rc == RAS_OK && e != cudaSuccess)
            rc = fail(h, RAS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        G.kps[j] = count;
        prev = node;
    }
    if (rc == RAS_OK) {
        const cudaError_t e = cudaGraphInstantiate(&G.exec, G.graph, 0);
        if (e != cudaSuccess) rc = fail(h, RAS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    cudaGetLastError();
    if (rc != RAS_OK) {
        destroy_cycle_graph(G);
        return rc;
    }
    G.gen = h->gen;
    G.V = h->V;
    G.m = m;
    return RAS_OK;
}

// Run the Arnoldi steps of one cycle (device state set up by the caller):
// as one graph launch, or step by step with a read of the flag after each
// (always so while profiling: per-kernel events cannot sit inside the
// conditional bodies of a graph). *ran: the graph that ran, else nullptr.
template <class Aop, class Mop>
int run_cycle(ras_problem* h, int op, bool prec, Aop& A, Mop& M, const std::vector<int>& cyc, double seglen,
              ras_problem::CycleGraph** ran) {
    const int m = h->o.gmres_restart;
    *ran = nullptr;
    if (h->use_graphs && !h->prof_on) {
        auto& G = h->cg[op];
        if (!G.exec || G.gen != h->gen || G.V != h->V || G.m != m)
            TRY(build_cycle_graph(h, op, prec, A, M, cyc, seglen));
        CK(cudaGraphLaunch(G.exec, h->st));
        *ran = &G;
        return RAS_OK;
    }
    for (int j = 0; j < m; ++j) {
        TRY(enqueue_step(h, j, prec, A, M, cyc, seglen));
        CK(cudaMemcpyAsync(h->h_any, h->gm_any, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        TRY(sync(h));
        if (!*h->h_any) break;
    }
    return RAS_OK;
}

// After a graph launch that ran `steps` Arnoldi steps: count its kernels.
void account_graph(const ras_problem::CycleGraph& G, int steps) {
    long long n = (long long)G.m - 1;   // condition kernels
    for (int j = 0; j < steps; ++j) n += G.kps[j];
    ras::add_launches(n);
}

// GMRES(m) (CGS2, Givens) for the problems with part[p], in lockstep, with
// right preconditioning when prec. its: steps taken (cumulative when
// resuming), conv: converged to rtol * ||b||. op: operator kind (the cycle
// graph of each kind is kept on the handle).
template <class Aop, class Mop>
int gmres(ras_problem* h, int op, Aop A, Mop M, bool prec, const double* b, double* x, const std::vector<int>& part,
          std::vector<int>& its, std::vector<int>& conv, GmresResume* res = nullptr) {
    Range range("ras: GMRES");
    const int P = h->nprob, m = h->o.gmres_restart, maxit = h->o.gmres_maxit;
    const long long L = h->L;
    const double rtol = h->o.gmres_rtol;
    const double* V_before = h->V;
    TRY(ensure(h, &h->V, (size_t)(m + 1) * L));
    if (h->V != V_before)   // basis vectors past a problem's last step must stay finite
        CK(cudaMemsetAsync(h->V, 0, (size_t)(m + 1) * L * sizeof(double), h->st));
    h->Vm = m;
    double* V = h->V;
    TRY(ensure(h, &h->gm_H, (size_t)P * (m + 1) * m));
    TRY(ensure(h, &h->gm_cs, (size_t)P * m));
    TRY(ensure(h, &h->gm_sn, (size_t)P * m));
    TRY(ensure(h, &h->gm_g, (size_t)P * (m + 1)));
    TRY(ensure(h, &h->gm_target, (size_t)P));
    TRY(ensure(h, &h->gm_its, (size_t)P));
    TRY(ensure(h, &h->gm_steps, (size_t)P));
    TRY(ensure(h, &h->gm_any, (size_t)1));
    if (!h->h_any && cudaMallocHost((void**)&h->h_any, sizeof(int)) != cudaSuccess) {
        h->h_any = nullptr;
        return fail(h, RAS_ENOMEM, "pinned host allocation failed");
    }
    double* r = h->T2;
    double* upd = h->T3;
    if (!res) its.assign(P, 0);
    its.resize(P, 0);
    conv.assign(P, 0);
    std::vector<int> act(P, 0), cyc(P, 0), steps(P, 0), cont(P, 0);
    std::vector<double> target(P, 0.0), beta(P, 0.0);
    if (!res) {
        CK(cudaMemsetAsync(x, 0, L * sizeof(double), h->st));
    } else {
        for (int p = 0; p < P; ++p) {
            if (part[p] && res->fresh[p])
                CK(cudaMemsetAsync(x + h->segs[p].ofs, 0, h->segs[p].len * sizeof(double), h->st));
            cont[p] = part[p] && !res->fresh[p];
        }
        res->pending.assign(P, 0);
        res->target.resize(P, 0.0);
    }
    TRY(set_mask(h, 0, part));
    TRY(seg_norms2(h, b, 0));
    for (int p = 0; p < P; ++p) {
        if (!part[p]) continue;
        const double bn = std::sqrt(h->h_scal[p * SS]);
        if (cont[p]) {
            target[p] = res->target[p];
            act[p] = 1;
            continue;
        }
        target[p] = rtol * bn;
        if (res) res->target[p] = target[p];
        if (bn == 0.0) conv[p] = 1;
        else act[p] = 1;
    }
    CK(cudaMemcpyAsync(r, b, L * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    double seglen = 0.0;
    for (int p = 0; p < P; ++p) seglen += (double)h->segs[p].len;
    if (std::any_of(cont.begin(), cont.end(), [](int v) { return v != 0; })) {
        // resumed problems: r = b - A x from the iterate of the earlier cycles
        TRY(set_mask(h, 0, cont));
        TRY(A(x, r, cont));
        CK(timed(h, RAS_K_KRYLOV, 24.0 * seglen, [&] {
            return ras::launch_seg_add_scaled(h->st, seg_grid(h, 0), h->d_segs, b, r, -1.0, r);
        }));
    }
    std::vector<double> H((size_t)P * (m + 1) * m), g((size_t)P * (m + 1)), y((size_t)P * SS, 0.0);
    for (int cycle = 0;; ++cycle) {
        // true residual norms of the problems still iterating
        TRY(set_mask(h, 0, act));
        TRY(seg_norms2(h, r, 0));
        bool any = false;
        for (int p = 0; p < P; ++p) {
            if (!act[p]) continue;
            beta[p] = std::sqrt(h->h_scal[p * SS]);
            if (beta[p] <= target[p] || its[p] >= maxit) {
                conv[p] = beta[p] <= target[p];
                act[p] = 0;
            } else {
                any = true;
            }
        }
        if (!any) return RAS_OK;
        if (res && cycle >= res->max_cycles) {
            res->pending = act;
            return RAS_OK;
        }
        cyc = act;
        TRY(set_mask(h, 0, cyc));
        // V_0 = r / beta (device-side, from the squared norms in h->scal)
        CK(timed(h, RAS_K_KRYLOV, 16.0 * seglen, [&] {
            return ras::launch_seg_scale(h->st, seg_grid(h, 0), h->d_segs, r, h->scal, 1.0, V);
        }));
        // device state of the cycle: g = beta e_1, step counters, targets
        std::fill(g.begin(), g.end(), 0.0);
        for (int p = 0; p < P; ++p) {
            g[(size_t)p * (m + 1)] = beta[p];
            steps[p] = 0;
        }
        CK(cudaMemcpyAsync(h->gm_g, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
        CK(cudaMemcpyAsync(h->gm_its, its.data(), (size_t)P * sizeof(int), cudaMemcpyHostToDevice, h->st));
        CK(cudaMemcpyAsync(h->gm_target, target.data(), (size_t)P * sizeof(double), cudaMemcpyHostToDevice, h->st));
        CK(cudaMemsetAsync(h->gm_steps, 0, (size_t)P * sizeof(int), h->st));
        TRY(cycle_table(h));
        ras_problem::CycleGraph* ran = nullptr;
        TRY(run_cycle(h, op, prec, A, M, cyc, seglen, &ran));
        CK(cudaMemcpyAsync(H.data(), h->gm_H, H.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpyAsync(g.data(), h->gm_g, g.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpyAsync(its.data(), h->gm_its, (size_t)P * sizeof(int), cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpyAsync(steps.data(), h->gm_steps, (size_t)P * sizeof(int), cudaMemcpyDeviceToHost, h->st));
        TRY(sync(h));
        if (ran) account_graph(*ran, *std::max_element(steps.begin(), steps.end()));
        // x += M (V y) for the problems that took steps in this cycle
        int maxsteps = 0;
        std::vector<int> took(P, 0);
        std::fill(y.begin(), y.end(), 0.0);
        for (int p = 0; p < P; ++p) {
            if (steps[p] == 0) continue;
            took[p] = 1;
            maxsteps = std::max(maxsteps, steps[p]);
            const double* Hp = H.data() + (size_t)p * (m + 1) * m;
            const double* gp = g.data() + (size_t)p * (m + 1);
            double* yp = y.data() + (size_t)p * SS;
            for (int i = steps[p] - 1; i >= 0; --i) {
                double s = gp[i];
                for (int k = i + 1; k < steps[p]; ++k) s -= Hp[i * m + k] * yp[k];
                yp[i] = s / Hp[i * m + i];
            }
        }
        if (maxsteps == 0) return RAS_OK;
        double* ycoef = h->scal + (size_t)3 * P * SS;
        CK(cudaMemcpyAsync(ycoef, y.data(), (size_t)P * SS * sizeof(double), cudaMemcpyHostToDevice, h->st));
        TRY(set_mask(h, 0, took));
        CK(cudaMemsetAsync(upd, 0, L * sizeof(double), h->st));
        CK(timed(h, RAS_K_KRYLOV, 8.0 * seglen * (maxsteps + 2), [&] {
            return ras::launch_seg_axpy(h->st, seg_grid(h, 0), h->d_segs, V, L, maxsteps, ycoef, 1.0, upd);
        }));
        const double* add = upd;
        if (prec) {
            TRY(M(upd, h->Z, took));
            add = h->Z;
        }
        CK(timed(h, RAS_K_KRYLOV, 24.0 * seglen, [&] {
            return ras::launch_seg_add_scaled(h->st, seg_grid(h, 0), h->d_segs, x, add, 1.0, x);
        }));
        // r = b - A x for the problems still iterating
        if (std::none_of(act.begin(), act.end(), [](int v) { return v != 0; })) return RAS_OK;
        TRY(set_mask(h, 0, act));
        TRY(A(x, r, act));
        CK(timed(h, RAS_K_KRYLOV, 24.0 * seglen, [&] {
            return ras::launch_seg_add_scaled(h->st, seg_grid(h, 0), h->d_segs, b, r, -1.0, r);
        }));
    }
}

// --------------------------------------------------------------- Alg. 2
// RASPEN for every problem of the handle, in lockstep: a problem leaves the
// loop when its own stop test holds (or at kmax).
int raspen_internal(ras_problem* h, ras_stats* s) {
    Range range("ras: RASPEN solve");
    const int P = h->nprob;
    const ras_opts& o = h->o;
    const bool resumed = (P == 1 && h->have_resume);
    const ras_state rs = h->resume;
    h->have_resume = false;
    if (resumed && rs.method != RAS_METHOD_RASPEN) return fail(h, RAS_ESTATE, "the state belongs to another method");
    std::vector<double> pstart(P, (resumed && rs.k > 0) ? o.eps_min : o.eps0);
    int rc = ras_apply_internal(h, pstart, h->F, s);
    if (rc < 0) return rc;
    std::vector<int> all(P, 1), need(P, 0), k(P, resumed ? rs.k : 0), its, conv;
    std::vector<double> nrm(P), stop(P), res0(P);
    TRY(set_mask(h, 1, all));
    TRY(seg_norms2(h, h->F, 1));
    for (int p = 0; p < P; ++p) {
        nrm[p] = std::sqrt(h->h_scal[p * SS]);
        stop[p] = resumed ? rs.stop : std::max(o.tol, o.tol * nrm[p]);
        res0[p] = resumed ? rs.res0 : nrm[p];
        if (s) s[p].res0 = res0[p];
    }
    double seglen = 0.0;
    for (auto& sg : h->segs) seglen += (double)sg.len;
    // the JVP runs for the problems GMRES is still iterating (d_mask row 0)
    auto A = [&](const double* in, double* out, const std::vector<int>& mask) {
        return jvp_internal(h, in, out, &mask);
    };
    auto M = [&](const double*, double*, const std::vector<int>&) { return RAS_OK; };
    for (;;) {
        bool any = false;
        for (int p = 0; p < P; ++p) {
            need[p] = (nrm[p] > stop[p] && k[p] < o.kmax_outer_raspen) ? 1 : 0;
            any = any || need[p];
        }
        if (!any) break;
        TRY(set_mask(h, 1, need));
        CK(timed(h, RAS_K_KRYLOV, 16.0 * seglen, [&] {
            return ras::launch_seg_scale(h->st, seg_grid(h, 1), h->d_segs, h->F, nullptr, -1.0, h->T1);
        }));
        TRY(gmres(h, 0, A, M, false, h->T1, h->Dv, need, its, conv));
        CK(timed(h, RAS_K_KRYLOV, 24.0 * seglen, [&] {
            return ras::launch_seg_add_scaled(h->st, seg_grid(h, 1), h->d_segs, h->X, h->Dv, 1.0, h->X);
        }));
        for (int p = 0; p < P; ++p) {
            if (need[p]) {
                k[p] += 1;
                if (s) s[p].gmres_its += its[p];
                pstart[p] = o.eps_min;
            } else {
                pstart[p] = 0.0;
            }
        }
        rc = ras_apply_internal(h, pstart, h->F, s);
        if (rc < 0) {
            for (int p = 0; p < P; ++p)
                if (s) s[p].outer_its = k[p];
            return rc;
        }
        TRY(seg_norms2(h, h->F, 1));
        for (int p = 0; p < P; ++p)
            if (need[p]) nrm[p] = std::sqrt(h->h_scal[p * SS]);
    }
    int worst = RAS_OK;
    for (int p = 0; p < P; ++p) {
        const int st = (nrm[p] <= stop[p]) ? RAS_OK : RAS_ENOCONV;
        if (s) {
            s[p].outer_its = k[p];
            s[p].res = nrm[p];
            s[p].status = st;
        }
        worst = std::min(worst, st);
    }
    if (P == 1) {
        h->last_state = ras_state{RAS_METHOD_RASPEN, k[0], k[0] > 0 ? o.eps_min : o.eps0, res0[0], stop[0]};
        h->have_last = true;
    }
    if (worst < 0) return fail(h, worst, "RASPEN reached kmax_outer_raspen");
    return RAS_OK;
}

// ------------------------------------------------------- Newton_RAS / Newton
// Alg. 1 on the global system F_eps(x) = 0; its Newton systems are solved by
// GMRES, right-preconditioned by the linear RAS preconditioner at x (prec:
// Newton_RAS) or unpreconditioned (the paper's Newton baseline). With
// eps0 > eps_min the continuation makes them Newton_RAS,eps / Newton_eps.
int newton_internal(ras_problem* h, ras_stats* s, bool prec) {
    Range range(prec ? "ras: Newton_RAS solve" : "ras: Newton solve");
    const long long N = plane(h, 0);
    const ras_opts& o = h->o;
    const double seglen = (double)h->segs[0].len;
    const int method = prec ? RAS_METHOD_NEWTON_RAS : RAS_METHOD_NEWTON;
    const bool resumed = h->have_resume;
    const ras_state rs = h->resume;
    h->have_resume = false;
    if (resumed && rs.method != method) return fail(h, RAS_ESTATE, "the state belongs to another method");
    double eps = resumed ? rs.eps : o.eps0, nrm, flr;
    TRY(residual_norm(h, h->X, nullptr, 0.0, eps, h->F, nrm, flr));
    const double stop = resumed ? rs.stop : std::max(o.tol, o.tol * nrm);
    const double res0 = resumed ? rs.res0 : nrm;
    if (s) s->res0 = res0;
    int k = resumed ? rs.k : 0, status = RAS_OK;
    std::vector<int> one(1, 1), its, conv;
    auto A = [&](const double* in, double* out, const std::vector<int>&) -> int {
        CK(timed(h, RAS_K_OTHER, 56.0 * N, [&] {
            return ras::launch_jacvec_global(h->st, h->probs[0], h->coefG, in, in + N, out, out + N);
        }));
        return RAS_OK;
    };
    auto M = [&](const double* in, double* out, const std::vector<int>&) {
        return prec ? precond_internal(h, in, out) : RAS_OK;
    };
    for (;;) {
        if (!std::isfinite(nrm)) { status = RAS_ENONFINITE; break; }
        if (eps == o.eps_min) {
            if (nrm <= stop) { status = RAS_OK; break; }
            if (nrm <= o.floor_factor * 1.1102230246251565e-16 * flr) { status = RAS_OK_FLOOR; break; }
        }
        if (k >= o.kmax_outer_newton) { status = RAS_ENOCONV; break; }
        if (prec) TRY(factor_at(h, eps));
        CK(timed(h, RAS_K_OTHER, 40.0 * N, [&] {
            return ras::launch_coef_global(h->st, h->probs[0], h->X, h->X + N, eps, h->coefG);
        }));
        CK(timed(h, RAS_K_KRYLOV, 16.0 * seglen, [&] {
            return ras::launch_seg_scale(h->st, seg_grid(h, 2), h->d_segs, h->F, nullptr, -1.0, h->T1);
        }));
        TRY(gmres(h, prec ? 2 : 1, A, M, prec, h->T1, h->Dv, one, its, conv));
        if (s) s->gmres_its += its[0];
        double alpha = 1.0, nt = 0.0, ft = 0.0;
        int hh = 0;
        for (;;) {
            TRY(residual_norm(h, h->X, h->Dv, alpha, eps, h->Ov, nt, ft));
            if (nt <= o.sigma * nrm || hh == o.max_halvings) break;
            alpha *= 0.5;
            ++hh;
        }
        if (s) {
            s->halvings += hh;
            if (!(nt <= o.sigma * nrm)) s->exhausted += 1;
        }
        CK(timed(h, RAS_K_KRYLOV, 24.0 * seglen, [&] {
            return ras::launch_seg_add_scaled(h->st, seg_grid(h, 2), h->d_segs, h->X, h->Dv, alpha, h->X);
        }));
        const double en = ras::next_eps(eps, o.gamma, o.eps_min);
        if (en == eps) {
            std::swap(h->F, h->Ov);
            nrm = nt;
            flr = ft;
        } else {
            TRY(residual_norm(h, h->X, nullptr, 0.0, en, h->F, nrm, flr));
        }
        eps = en;
        ++k;
    }
    if (s) {
        s->outer_its = k;
        s->res = nrm;
        s->status = status;
        s->eps_final = eps;
    }
    h->last_state = ras_state{method, k, eps, res0, stop};
    h->have_last = true;
    if (status < 0) return fail(h, status, prec ? "Newton_RAS stopped without convergence"
                                                : "Newton stopped without convergence");
    return status;
}

int newton_ras_internal(ras_problem* h, ras_stats* s) { return newton_internal(h, s, true); }

// ------------------------------------------------------------ launch shapes
// Rebuild the block tables of the segmented kernels for the current
// tune.vec_blocks, each row for the problems it was last built for.
int rebuild_grids(ras_problem* h) {
    for (int row = 0; row < 3; ++row) {
        if (h->last_mask[row].empty()) continue;
        const std::vector<int> m = h->last_mask[row];
        h->last_mask[row].clear();
        TRY(build_grid(h, row, m));
    }
    return RAS_OK;
}

// Mean device time (ms) of one fn() over `reps` calls after one untimed call,
// from CUDA events on the handle's stream.
template <class Fn>
int time_launches(ras_problem* h, int reps, Fn fn, double& ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    cudaError_t e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(a, h->st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(b, h->st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    CK(e);
    ms = (double)t / reps;
    return RAS_OK;
}

// Index of the candidate to install: the default `d` unless another one is
// at least 2% faster (timing noise does not flip a choice).
int pick_faster(const std::vector<double>& ms, int d) {
    int best = d;
    for (int i = 0; i < (int)ms.size(); ++i)
        if (ms[i] < ms[best]) best = i;
    return ms[best] <= 0.98 * ms[d] ? best : d;
}

// FP32 factorisation: per tile class, both kernels at a ladder of subdomain
// counts (a prefix of the class's list, every listed subdomain factorised).
int tune_factor(ras_problem* h, ras_tune_report* rep, int* wide_max) {
    static const int ladder[] = {1, 8, 38, 76, 152, 304};
    for (int c = 0; c < NTILE; ++c) {
        wide_max[c] = -1;
        const int cnt = h->tile_cnt[c];
        if (cnt == 0) continue;
        std::vector<int> ks;
        for (int k : ladder)
            if (k < cnt) ks.push_back(k);
        ks.push_back(cnt);
        bool differs = false, run = true;
        int thr = 0;
        for (size_t i = 0; i < ks.size(); ++i) {
            std::vector<double> t(2, 0.0);
            for (int w = 0; w < 2; ++w) {
                TRY(time_launches(h, 3, [&] {
                    return ras::launch_local_factor_f32(h->st, 2 * (c + 1), ks[i], h->d_lists + h->tile_off[c],
                                                        h->d_subs, h->d_probs, h->X, h->ls, h->cpool, h->coef,
                                                        (float*)h->gpool, 0, w);
                }, t[w]));
            }
            rep->factor_count[c][i] = ks[i];
            rep->factor_ms[c][i][0] = t[0];
            rep->factor_ms[c][i][1] = t[1];
            const int def = ks[i] <= h->sms ? 1 : 0;      // the default rule's kernel
            const int use = pick_faster(t, def);
            differs = differs || use != def;
            if (run && use == 1) thr = ks[i];
            else run = false;
        }
        if (differs) wide_max[c] = thr;
    }
    return RAS_OK;
}

// Persistent local-solve kernels: one linear RAS application per CTAs-per-SM
// value that gives a different grid.
int tune_solve(ras_problem* h, ras_tune_report* rep, int& chosen) {
    const bool f32 = h->o.precision == RAS_MIXED;
    int fit = 0;
    CK(ras::solve_ctas_per_sm_max(f32, &fit));
    fit = std::max(1, std::min(fit, RAS_TUNE_MAX));
    std::vector<int> vals;
    std::vector<double> ms;
    int last_grid = -1;
    for (int c = 1; c <= fit; ++c) {
        const int grid = std::min(h->nsub, c * h->sms);
        if (grid == last_grid) break;                  // more CTAs than subdomains: same launch
        last_grid = grid;
        double t = 0.0;
        TRY(time_launches(h, 3, [&] {
            if (f32)
                return ras::launch_local_precond<float>(h->st, h->nsub, c, h->d_subs, h->d_probs,
                                                        (const float*)h->gpool, (float*)h->wpool, h->X, h->T1,
                                                        h->d_err, h->d_order, h->d_ticket);
            return ras::launch_local_precond<double>(h->st, h->nsub, c, h->d_subs, h->d_probs,
                                                     (const double*)h->gpool, (double*)h->wpool, h->X, h->T1,
                                                     h->d_err, h->d_order, h->d_ticket);
        }, t));
        TRY(check_err(h));
        rep->solve_ctas_per_sm[vals.size()] = c;
        rep->solve_ms[vals.size()] = t;
        vals.push_back(c);
        ms.push_back(t);
    }
    const int k = pick_faster(ms, (int)ms.size() - 1);  // default: as many as fit = the last grid
    chosen = k == (int)ms.size() - 1 ? 0 : vals[k];
    return RAS_OK;
}

// Segmented vector kernels: one CGS step (dot products against a 16-vector
// basis, their reduction, the AXPY) per block count, every problem taking part.
int tune_vectors(ras_problem* h, ras_tune_report* rep, int& chosen) {
    const int P = h->nprob, m = h->o.gmres_restart;
    const long long L = h->L;
    TRY(ensure(h, &h->V, (size_t)(m + 1) * L));
    h->Vm = m;
    const int nv = std::min(16, m);
    double* w = h->V + (long long)nv * L;
    CK(cudaMemsetAsync(h->V, 0, (size_t)(nv + 1) * L * sizeof(double), h->st));
    const int saved = h->tune.vec_blocks;
    std::vector<int> vals;
    std::vector<double> ms;
    int def = 0;
    for (int vb = 152; vb <= ras::VEC_BLOCKS; vb += 152) {
        h->tune.vec_blocks = vb;
        h->last_mask[0].clear();
        TRY(set_mask(h, 0, std::vector<int>(P, 1)));
        double t = 0.0;
        TRY(time_launches(h, 5, [&] {
            cudaError_t e = ras::launch_seg_dot(h->st, seg_grid(h, 0), h->d_segs, h->V, L, nv, w, h->partials);
            if (e == cudaSuccess) e = ras::launch_seg_reduce(h->st, P, seg_grid(h, 0).nbps, nv, h->partials, h->scal);
            if (e == cudaSuccess)
                e = ras::launch_seg_axpy(h->st, seg_grid(h, 0), h->d_segs, h->V, L, nv, h->scal, -1.0, w);
            return e;
        }, t));
        if (vb == ras::VEC_BLOCKS) def = (int)vals.size();
        rep->vec_blocks[vals.size()] = vb;
        rep->vec_ms[vals.size()] = t;
        vals.push_back(vb);
        ms.push_back(t);
    }
    h->tune.vec_blocks = saved;
    chosen = vals[pick_faster(ms, def)];
    return RAS_OK;
}

int validate_tuning(ras_problem* h, const ras_tuning& t) {
    for (int c = 0; c < NTILE; ++c)
        if (t.factor_wide_max[c] < -1) return fail(h, RAS_EINVAL, "factor_wide_max below -1");
    if (t.solve_ctas_per_sm < 0 || t.solve_ctas_per_sm > 64)
        return fail(h, RAS_EINVAL, "solve_ctas_per_sm outside 0..64");
    if (t.vec_blocks < 1 || t.vec_blocks > ras::VEC_BLOCKS)
        return fail(h, RAS_EINVAL, "vec_blocks outside 1..RAS_VEC_BLOCKS_MAX");
    return RAS_OK;
}

int install_tuning(ras_problem* h, const ras_tuning& t) {
    TRY(validate_tuning(h, t));
    h->tune = t;
    ++h->gen;
    TRY(rebuild_grids(h));
    return sync(h);
}

int autotune_internal(ras_problem* h, ras_tuning* chosen, ras_tune_report* rep) {
    Range range("ras: autotune");
    ras_tune_report local{};
    if (!rep) rep = &local;
    std::memset(rep, 0, sizeof(*rep));
    if (h->sms == 0) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const bool prof = h->prof_on;
    h->prof_on = false;
    ras_tuning t = h->tune;
    // every subdomain factorised at x = 0, eps = eps0 (the start of a solve)
    CK(cudaMemsetAsync(h->X, 0, (size_t)h->L * sizeof(double), h->st));
    int rc = factor_at(h, h->o.eps0);
    if (rc >= 0 && h->o.precision == RAS_MIXED) rc = tune_factor(h, rep, t.factor_wide_max);
    if (rc >= 0) rc = tune_solve(h, rep, t.solve_ctas_per_sm);
    if (rc >= 0) rc = tune_vectors(h, rep, t.vec_blocks);
    h->prof_on = prof;
    h->jvp_ready = false;
    TRY(rc);
    TRY(install_tuning(h, t));
    if (chosen) *chosen = h->tune;
    return RAS_OK;
}

int need_single(ras_problem* h) {
    if (h->nprob != 1) return fail(h, RAS_EINVAL, "this entry point takes a single-problem handle");
    return RAS_OK;
}

// ------------------------------------------------- the paper's model problem
// Dot product of two vectors of problem 0 (whole segment), read to the host.
int seg_dot_host(ras_problem* h, const double* a, const double* b, double& out) {
    const ras::SegGrid g = seg_grid(h, 2);
    CK(ras::launch_seg_dot(h->st, g, h->d_segs, a, h->L, 1, b, h->partials));
    CK(ras::launch_seg_reduce(h->st, 1, g.nbps, 1, h->partials, h->scal));
    CK(cudaMemcpyAsync(h->h_scal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    out = h->h_scal[0];
    return RAS_OK;
}

// F_y at (y + alpha d_y, p) into F (p-plane of F set to zero) and ||F_y||.
int state_residual(ras_problem* h, const double* x, const double* d, double alpha, double eps, double* F,
                   double& nrm) {
    const long long N = plane(h, 0);
    CK(ras::launch_residual_global(h->st, h->probs[0], x, x + N, d, d ? d + N : nullptr, alpha, eps, F, F + N,
                                   h->partials, 0));
    CK(cudaMemsetAsync(F + N, 0, N * sizeof(double), h->st));
    double s2 = 0.0;
    TRY(seg_dot_host(h, F, F, s2));
    nrm = std::sqrt(s2);
    return RAS_OK;
}

// Sec. 4: ybar solves the state equation F_y(ybar, pbar, eps) = 0 (damped
// Newton; each step by conjugate gradients on A + diag(phi'(y)), symmetric
// positive definite for increasing phi), then y_d = -A pbar - phi'(ybar) pbar
// + ybar, so that F(ybar, pbar, eps) = 0 with that y_d.
int manufacture_internal(ras_problem* h, const double* pbar, double eps, double* y_out, double* yd_out) {
    Range range("ras: manufactured solution");
    const long long N = plane(h, 0);
    const ras::SegGrid g = seg_grid(h, 2);
    double *X = h->X, *F = h->F, *D = h->Dv, *R = h->T1, *Pc = h->T2, *Q = h->T3;
    CK(cudaMemsetAsync(X, 0, N * sizeof(double), h->st));
    CK(cudaMemcpyAsync(X + N, pbar, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    double nrm = 0.0;
    TRY(state_residual(h, X, nullptr, 0.0, eps, F, nrm));
    const double nrm0 = nrm;
    constexpr double RTOL = 1e-14, CG_RTOL = 1e-10;
    for (int k = 0;; ++k) {
        if (!std::isfinite(nrm)) return fail(h, RAS_ENONFINITE, "state residual not finite");
        if (nrm <= RTOL * nrm0) break;
        if (k >= 100) return fail(h, RAS_ENOCONV, "state solve did not converge in 100 Newton steps");
        CK(ras::launch_coef_global(h->st, h->probs[0], X, X + N, eps, h->coefG));
        // conjugate gradients for (A + diag phi'(y)) d_y = -F_y; every vector's p-plane stays zero
        CK(cudaMemsetAsync(D, 0, 2 * N * sizeof(double), h->st));
        CK(ras::launch_seg_scale(h->st, g, h->d_segs, F, nullptr, -1.0, R));
        CK(cudaMemcpyAsync(Pc, R, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        double rr = 0.0;
        TRY(seg_dot_host(h, R, R, rr));
        const double rr0 = rr;
        for (int it = 0; it < 100000 && rr > CG_RTOL * CG_RTOL * rr0; ++it) {
            CK(ras::launch_jacvec_global(h->st, h->probs[0], h->coefG, Pc, Pc + N, Q, Q + N));
            CK(cudaMemsetAsync(Q + N, 0, N * sizeof(double), h->st));
            double pq = 0.0;
            TRY(seg_dot_host(h, Pc, Q, pq));
            if (!(pq > 0.0)) return fail(h, RAS_ENONFINITE, "state Jacobian not positive definite");
            const double a = rr / pq;
            CK(ras::launch_seg_add_scaled(h->st, g, h->d_segs, D, Pc, a, D));
            CK(ras::launch_seg_add_scaled(h->st, g, h->d_segs, R, Q, -a, R));
            double rn = 0.0;
            TRY(seg_dot_host(h, R, R, rn));
            const double b = rn / rr;
            rr = rn;
            CK(ras::launch_seg_add_scaled(h->st, g, h->d_segs, R, Pc, b, Pc));
        }
        // backtracking on ||F_y||
        double alpha = 1.0;
        bool moved = false;
        for (int hh = 0; hh < 40; ++hh) {
            double nt = 0.0;
            TRY(state_residual(h, X, D, alpha, eps, h->Ov, nt));
            if (nt <= (1.0 - 1e-4 * alpha) * nrm) {
                CK(ras::launch_seg_add_scaled(h->st, g, h->d_segs, X, D, alpha, X));
                CK(cudaMemcpyAsync(F, h->Ov, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
                nrm = nt;
                moved = true;
                break;
            }
            alpha *= 0.5;
        }
        if (!moved) {
            if (nrm <= 1e-9 * nrm0) break;   // rounding level
            return fail(h, RAS_ENOCONV, "state solve stalled");
        }
    }
    // y_d = -(A pbar + phi'(ybar) pbar - ybar): minus F_p at y_d = 0
    CK(cudaMemsetAsync(h->yd, 0, N * sizeof(double), h->st));
    CK(ras::launch_residual_global(h->st, h->probs[0], X, X + N, nullptr, nullptr, 0.0, eps, F, F + N, h->partials,
                                   0));
    CK(ras::launch_seg_scale(h->st, g, h->d_segs, F, nullptr, -1.0, R));
    CK(cudaMemcpyAsync(h->yd, R + N, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (y_out) CK(cudaMemcpyAsync(y_out, X, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (yd_out) CK(cudaMemcpyAsync(yd_out, h->yd, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    h->jvp_ready = false;
    return sync(h);
}


}  // namespace

// ===================================================================== C ABI
extern "C" {

int ras_default_opts(ras_opts* o) {
    if (!o) return RAS_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-10;
    o->inner_tol = 1e-8;
    o->sigma = 1.1;
    o->eps0 = 1.0;
    o->gamma = 0.2;
    o->eps_min = 1e-6;
    o->kmax_outer_raspen = 50;
    o->kmax_outer_newton = 200;
    o->kmax_inner = 100;
    o->max_halvings = 20;
    o->gmres_restart = 30;
    o->gmres_maxit = 1000;
    o->gmres_rtol = 1e-8;
    o->floor_factor = 16.0;
    o->precision = RAS_FP64;
    o->ir_max = 6;
    o->ir_rtol = 1e-12;
    o->kappa = 0.1;
    o->jvp_ir = 2;
    o->wait_test = 0;
    return RAS_OK;
}

namespace {

bool desc_valid(const ras_problem_desc& d) {
    return d.n >= 2 && d.sx >= 1 && d.sy >= 1 && d.sx <= d.n && d.sy <= d.n && d.overlap >= 0 && d.phi >= 0 &&
           d.phi <= 2 && d.nu > 0 && d.mu > 0 && std::isfinite(d.nu) && std::isfinite(d.mu);
}

// Host-side layout of a set of problems: problem and subdomain descriptors,
// segment offsets of the global vectors, offsets into the local pools and
// the register-tile classes. The y_d / f pointers are set by the caller.
int build_layout(ras_problem* h, int count, const ras_problem_desc* pd, const int* sz = nullptr) {
    h->nprob = count;
    h->desc.assign(pd, pd + count);
    h->sz.assign(count, 0);
    if (sz) h->sz.assign(sz, sz + count);
    h->probs.clear();
    h->segs.clear();
    h->subs.clear();
    h->sub_first.clear();
    h->sub_count.clear();
    h->maxm = 0;
    h->h_wide.clear();
    int maxm_all = 0;
    long long voff = 0, noff = 0, goff = 0, vec = 0;
    for (int p = 0; p < count; ++p) {
        const ras_problem_desc& d = pd[p];
        const int n = d.n;
        const bool cube = h->sz[p] > 0;
        ProbDev P{};
        P.n = n;
        P.nz = cube ? n : 1;
        P.nn = (long long)n * n * P.nz;
        P.phi = d.phi;
        P.h = 1.0 / (n + 1);
        P.beta = 1.0 / (P.h * P.h);
        P.diag = (cube ? 6.0 : 4.0) * P.beta;
        P.nu = d.nu;
        P.mu = d.mu;
        P.kappa = h->o.kappa;
        P.ofs = vec;
        h->probs.push_back(P);
        h->segs.push_back(Seg{vec, 2 * P.nn});
        h->sub_first.push_back((int)h->subs.size());
        const auto bx = split_blocks(n, d.sx), by = split_blocks(n, d.sy);
        const auto bz = cube ? split_blocks(n, h->sz[p]) : std::vector<std::pair<int, int>>{{0, 1}};
        for (int k = 0; k < (int)bz.size(); ++k) {
            for (int j = 0; j < d.sy; ++j) {
                for (int i = 0; i < d.sx; ++i) {
                    SubDev s{};
                    s.prob = p;
                    s.ox0 = bx[i].first; s.owx = bx[i].second - bx[i].first;
                    s.oy0 = by[j].first; s.owy = by[j].second - by[j].first;
                    s.oz0 = bz[k].first; s.owz = bz[k].second - bz[k].first;
                    s.x0 = std::max(0, s.ox0 - d.overlap);
                    s.y0 = std::max(0, s.oy0 - d.overlap);
                    s.wx = std::min(n, bx[i].second + d.overlap) - s.x0;
                    s.wy = std::min(n, by[j].second + d.overlap) - s.y0;
                    if (cube) {
                        s.z0 = std::max(0, s.oz0 - d.overlap);
                        s.wz = std::min(n, bz[k].second + d.overlap) - s.z0;
                        s.bl = s.wx * s.wy;
                        s.bw = s.wz;
                    } else {
                        s.z0 = 0;
                        s.wz = 1;
                        s.bl = s.wx;
                        s.bw = s.wy;
                    }
                    s.mp = ((2 * s.bl + 31) / 32) * 32;
                    s.voff = voff; s.noff = noff; s.goff = goff;
                    voff += 2LL * s.wx * s.wy * s.wz;
                    noff += (long long)s.wx * s.wy * s.wz;
                    // wide blocks: one scratch block after the bw factor blocks
                    goff += (long long)(s.bw + (s.mp > ras::MAX_M ? 1 : 0)) * s.mp * s.mp;
                    maxm_all = std::max(maxm_all, 2 * s.bl);
                    if (s.mp > ras::MAX_M) h->h_wide.push_back((int)h->subs.size());
                    else h->maxm = std::max(h->maxm, 2 * s.bl);
                    h->subs.push_back(s);
                }
            }
        }
        h->sub_count.push_back((int)h->subs.size() - h->sub_first.back());
        vec += 2 * P.nn;
    }
    if (maxm_all > ras::MAX_MW)
        return fail(h, RAS_EINVAL,
                    "a local block row has more than 512 unknowns (2 wx > 512; on the cube 2 wx wy > 512)");
    h->nsub = (int)h->subs.size();
    h->Lsum = voff; h->Nsum = noff; h->Gsum = goff; h->L = vec;
    // register-tile classes of the FP32 factorisation: tile = mp / 16
    h->h_lists.clear();
    h->tile_off.assign(NTILE, 0);
    h->tile_cnt.assign(NTILE, 0);
    for (int c = 0; c < NTILE; ++c) {
        h->tile_off[c] = (int)h->h_lists.size();
        for (int i = 0; i < h->nsub; ++i)
            if (h->subs[i].mp / 32 - 1 == c) h->h_lists.push_back(i);
        h->tile_cnt[c] = (int)h->h_lists.size() - h->tile_off[c];
    }
    h->nbp = std::max(8, ras::VEC_BLOCKS / count);
    h->jvp_ready = false;
    for (int r = 0; r < 3; ++r) {
        h->last_mask[r].clear();
        h->ntab[r] = 0;
    }
    return RAS_OK;
}

// Device buffers for the current layout (grown, never shrunk; contents of a
// grown buffer are not kept). own_data: the handle stores y_d and f itself.
int ensure_pools(ras_problem* h, bool own_data) {
    const int count = h->nprob;
    long long nn_tot = 0;
    bool any_f = false;
    for (int p = 0; p < count; ++p) {
        nn_tot += plane(h, p);
        any_f = any_f || h->desc[p].f != nullptr;
    }
    if (own_data) {
        TRY(ensure(h, &h->yd, nn_tot));
        if (any_f) TRY(ensure(h, &h->f, nn_tot));
    }
    TRY(ensure(h, &h->d_subs, h->nsub));
    TRY(ensure(h, &h->d_probs, count));
    TRY(ensure(h, &h->d_segs, count));
    TRY(ensure(h, &h->d_lists, std::max<size_t>(1, h->h_lists.size())));
    TRY(ensure(h, &h->d_order, h->nsub));
    TRY(ensure(h, &h->d_wide, std::max<size_t>(1, h->h_wide.size())));
    TRY(ensure(h, &h->d_ticket, 1));
    for (double** q : {&h->cpool, &h->dpool, &h->Kpool, &h->Ktpool, &h->rpool}) TRY(ensure(h, q, h->Lsum));
    if (h->own_factors) TRY(ensure(h, &h->coef, 3 * h->Nsum));
    TRY(ensure(h, &h->ls, h->nsub));
    TRY(ensure(h, &h->d_active, 1));
    if (!h->d_err) {
        TRY(dalloc(h, &h->d_err, 2));
        CK(cudaMemsetAsync(h->d_err, 0, 2 * sizeof(int), h->st));
    }
    TRY(push_wait_test(h));
    TRY(ensure(h, &h->d_mask, 2 * count));
    TRY(ensure(h, &h->d_tab, (size_t)4 * (ras::VEC_BLOCKS + count)));
    TRY(ensure(h, &h->d_nbps, (size_t)4 * count));
    TRY(ensure(h, &h->d_toff, (size_t)count + 1));
    TRY(ensure(h, &h->d_pstart, count));
    for (double** q : {&h->X, &h->F, &h->Dv, &h->Ov, &h->T1, &h->T2, &h->T3, &h->Z}) TRY(ensure(h, q, h->L));
    if (count == 1) TRY(ensure(h, &h->coefG, 3 * nn_tot));
    TRY(ensure(h, &h->partials, (size_t)count * SS * std::max(h->nbp, (int)ras::VEC_BLOCKS)));
    TRY(ensure(h, &h->scal, (size_t)4 * count * SS));
    TRY(alloc_factor_pools(h));
    if (!h->h_active) {
        if (cudaMallocHost((void**)&h->h_active, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, RAS_ENOMEM, "pinned host allocation failed");
        }
    }
    const size_t ns = (size_t)4 * count * SS;
    if (h->cap_hscal < ns) {
        if (h->h_scal) cudaFreeHost(h->h_scal);
        h->h_scal = nullptr;
        h->cap_hscal = 0;
        if (cudaMallocHost((void**)&h->h_scal, ns * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, RAS_ENOMEM, "pinned host allocation failed");
        }
        h->cap_hscal = ns;
    }
    return RAS_OK;
}

// Absolute factor / coefficient pointers of every subdomain into the
// handle's own pools (handles whose factors live elsewhere set them first).
void fill_pointers(ras_problem* h) {
    const size_t es = (h->o.precision == RAS_MIXED) ? sizeof(float) : sizeof(double);
    for (auto& sd : h->subs) {
        sd.gptr = static_cast<char*>(h->gpool) + sd.goff * es;
        sd.cptr = h->coef + 3 * sd.noff;
    }
}

int upload_layout(ras_problem* h) {
    ++h->gen;
    if (h->own_factors) fill_pointers(h);
    TRY(build_grid(h, 2, std::vector<int>(h->nprob, 1)));
    // solve order: largest factor (bw * mp^2) first, ties by index
    std::vector<int> order(h->nsub);
    for (int k = 0; k < h->nsub; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)h->subs[a].bw * h->subs[a].mp * h->subs[a].mp >
               (long long)h->subs[b].bw * h->subs[b].mp * h->subs[b].mp;
    });
    CK(cudaMemcpyAsync(h->d_order, order.data(), h->nsub * sizeof(int), cudaMemcpyHostToDevice, h->st));
    if (!h->h_wide.empty())
        CK(cudaMemcpyAsync(h->d_wide, h->h_wide.data(), h->h_wide.size() * sizeof(int), cudaMemcpyHostToDevice,
                           h->st));
    TRY(sync(h));
    CK(cudaMemcpyAsync(h->d_subs, h->subs.data(), h->nsub * sizeof(SubDev), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->d_probs, h->probs.data(), h->nprob * sizeof(ProbDev), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->d_segs, h->segs.data(), h->nprob * sizeof(Seg), cudaMemcpyHostToDevice, h->st));
    if (!h->h_lists.empty())
        CK(cudaMemcpyAsync(h->d_lists, h->h_lists.data(), h->h_lists.size() * sizeof(int), cudaMemcpyHostToDevice,
                           h->st));
    return RAS_OK;
}

// A handle for `count` problems; sz (null: all on the square) gives per
// problem the subdomains along x3 of a cube problem, 0 for the square.
int create_internal(int count, const ras_problem_desc* pd, const int* sz, const ras_opts* o, void* stream,
                    ras_problem** out) {
    if (!out) return RAS_EINVAL;
    *out = nullptr;
    if (count < 1 || count > 4096 || !pd) return RAS_EINVAL;
    for (int p = 0; p < count; ++p)
        if (!desc_valid(pd[p]) || !pd[p].y_d) return RAS_EINVAL;
    ras_problem* h = new ras_problem();
    if (o) h->o = *o;
    else ras_default_opts(&h->o);
    h->st = (cudaStream_t)stream;
    int rc = validate_opts(h, h->o);
    if (rc == RAS_OK) rc = build_layout(h, count, pd, sz);
    if (rc == RAS_OK) rc = ensure_pools(h, true);
    if (rc != RAS_OK) {
        ras_destroy(h);
        return rc;
    }
    // y_d and f of problem p at the plane offset sum_{q<p} nn_q
    long long poff = 0;
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < count && e == cudaSuccess; ++p) {
        const long long N = plane(h, p);
        h->probs[p].yd = h->yd + poff;
        h->probs[p].f = pd[p].f ? h->f + poff : nullptr;
        e = cudaMemcpyAsync(h->yd + poff, pd[p].y_d, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
        if (e == cudaSuccess && pd[p].f)
            e = cudaMemcpyAsync(h->f + poff, pd[p].f, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
        poff += N;
    }
    if (e == cudaSuccess && upload_layout(h) != RAS_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ras_destroy(h);
        return RAS_ECUDA;
    }
    *out = h;
    return RAS_OK;
}

}  // namespace

int ras_batch_create(int count, const ras_problem_desc* pd, const ras_opts* o, void* stream, ras_problem** out) {
    return create_internal(count, pd, nullptr, o, stream, out);
}

int ras_create3(int n, int sx, int sy, int sz, int overlap, int phi, double nu, double mu, const double* y_d,
                const double* f, const ras_opts* o, void* stream, ras_problem** out) {
    if (out) *out = nullptr;
    if (sz < 1 || sz > n) return RAS_EINVAL;
    ras_problem_desc d{};
    d.n = n; d.sx = sx; d.sy = sy; d.overlap = overlap; d.phi = phi; d.nu = nu; d.mu = mu;
    d.y_d = y_d; d.f = f;
    return create_internal(1, &d, &sz, o, stream, out);
}

int ras_problem_dim(const ras_problem* h) {
    if (!h) return RAS_EINVAL;
    return h->probs[0].nz > 1 ? 3 : 2;
}

int ras_create(int n, int sx, int sy, int overlap, int phi, double nu, double mu, const double* y_d,
               const double* f, const ras_opts* o, void* stream, ras_problem** out) {
    ras_problem_desc d{};
    d.n = n; d.sx = sx; d.sy = sy; d.overlap = overlap; d.phi = phi; d.nu = nu; d.mu = mu;
    d.y_d = y_d; d.f = f;
    return ras_batch_create(1, &d, o, stream, out);
}

int ras_problem_count(const ras_problem* h) { return h ? h->nprob : RAS_EINVAL; }

int ras_set_eps(ras_problem* h, double eps_min) {
    if (!h) return RAS_EINVAL;
    if (!(eps_min > 0) || !std::isfinite(eps_min)) return fail(h, RAS_EINVAL, "eps_min must be > 0");
    h->o.eps_min = eps_min;
    if (h->o.eps0 < eps_min) h->o.eps0 = eps_min;
    h->jvp_ready = false;
    return RAS_OK;
}

int ras_set_opts(ras_problem* h, const ras_opts* o) {
    if (!h || !o) return RAS_EINVAL;
    TRY(validate_opts(h, *o));
    {
        // only the failure-path test switch changed: the factors stay valid
        ras_opts t = *o;
        t.wait_test = h->o.wait_test;
        if (std::memcmp(&t, &h->o, sizeof(ras_opts)) == 0) {
            h->o.wait_test = o->wait_test;
            TRY(push_wait_test(h));
            TRY(sync(h));
            return RAS_OK;
        }
    }
    const bool kappa_changed = (o->kappa != h->o.kappa);
    h->o = *o;
    h->jvp_ready = false;
    ++h->gen;
    TRY(push_wait_test(h));
    TRY(alloc_factor_pools(h));
    if (h->own_factors) {
        fill_pointers(h);
        CK(cudaMemcpyAsync(h->d_subs, h->subs.data(), h->nsub * sizeof(SubDev), cudaMemcpyHostToDevice, h->st));
    }
    if (kappa_changed) {
        for (auto& P : h->probs) P.kappa = o->kappa;
        CK(cudaMemcpyAsync(h->d_probs, h->probs.data(), h->nprob * sizeof(ProbDev), cudaMemcpyHostToDevice, h->st));
    }
    TRY(sync(h));
    return RAS_OK;
}

int ras_set_data(ras_problem* h, const double* y_d, const double* f) {
    if (!h || !y_d) return RAS_EINVAL;
    TRY(need_single(h));
    const long long N = plane(h, 0);
    CK(cudaMemcpyAsync(h->yd, y_d, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (f) {
        if (!h->f) TRY(dalloc(h, &h->f, N));
        CK(cudaMemcpyAsync(h->f, f, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    }
    if ((f != nullptr) != (h->probs[0].f != nullptr)) {
        h->probs[0].f = f ? h->f : nullptr;
        CK(cudaMemcpyAsync(h->d_probs, h->probs.data(), sizeof(ProbDev), cudaMemcpyHostToDevice, h->st));
    }
    h->jvp_ready = false;
    return sync(h);
}

int ras_residual(ras_problem* h, const double* y, const double* p, double eps, double* Fy, double* Fp,
                 double* norm_host) {
    if (!h || !y || !p || !(eps > 0)) return RAS_EINVAL;
    TRY(need_single(h));
    CK(timed(h, RAS_K_RESIDUAL, resid_bytes(h), [&] {
        return ras::launch_residual_global(h->st, h->probs[0], y, p, nullptr, nullptr, 0.0, eps, Fy, Fp,
                                           h->partials, 0);
    }));
    CK(timed(h, RAS_K_OTHER, 0.0,
             [&] { return ras::launch_reduce_partials(h->st, h->partials, ras::VEC_BLOCKS, 2, h->scal); }));
    CK(cudaMemcpyAsync(h->h_scal, h->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    if (norm_host) *norm_host = std::sqrt(h->h_scal[0]);
    return RAS_OK;
}

int ras_apply(ras_problem* h, const double* y, const double* p, int continuation, double* Fy, double* Fp,
              ras_stats* stats) {
    if (!h || !y || !p || !Fy || !Fp) return RAS_EINVAL;
    TRY(need_single(h));
    stats_clear(stats, 1);
    TRY(copy_in(h, h->X, 0, y, p));
    const std::vector<double> pstart(1, continuation ? h->o.eps0 : h->o.eps_min);
    const int rc = ras_apply_internal(h, pstart, h->F, stats);
    if (rc == RAS_ECUDA) return rc;
    TRY(check_err_stats(h, stats, 1));
    TRY(copy_out(h, h->F, 0, Fy, Fp));
    TRY(sync(h));
    if (stats) stats->status = rc;
    return rc;
}

int ras_jvp(ras_problem* h, const double* dy, const double* dp, double* oy, double* op) {
    if (!h || !dy || !dp || !oy || !op) return RAS_EINVAL;
    TRY(need_single(h));
    if (!h->jvp_ready) return fail(h, RAS_ESTATE, "ras_jvp needs a successful ras_apply first");
    TRY(copy_in(h, h->Dv, 0, dy, dp));
    TRY(jvp_internal(h, h->Dv, h->Ov, nullptr));
    TRY(copy_out(h, h->Ov, 0, oy, op));
    TRY(sync(h));
    return check_err(h);
}

int ras_precondition(ras_problem* h, const double* y, const double* p, double eps, const double* ry,
                     const double* rp, double* zy, double* zp) {
    if (!h || !y || !p || !ry || !rp || !zy || !zp || !(eps > 0)) return RAS_EINVAL;
    TRY(need_single(h));
    TRY(copy_in(h, h->X, 0, y, p));
    TRY(factor_at(h, eps));
    TRY(copy_in(h, h->T1, 0, ry, rp));
    TRY(precond_internal(h, h->T1, h->Z));
    TRY(copy_out(h, h->Z, 0, zy, zp));
    TRY(sync(h));
    return check_err(h);
}

int ras_batch_raspen_solve(ras_problem* h, double* const* y, double* const* p, ras_stats* stats) {
    if (!h || !y || !p) return RAS_EINVAL;
    for (int k = 0; k < h->nprob; ++k)
        if (!y[k] || !p[k]) return RAS_EINVAL;
    stats_clear(stats, h->nprob);
    for (int k = 0; k < h->nprob; ++k) TRY(copy_in(h, h->X, k, y[k], p[k]));
    const int rc = raspen_internal(h, stats);
    if (rc == RAS_ECUDA) return rc;
    TRY(check_err_stats(h, stats, h->nprob));
    for (int k = 0; k < h->nprob; ++k) TRY(copy_out(h, h->X, k, y[k], p[k]));
    TRY(sync(h));
    return rc;
}

int ras_raspen_solve(ras_problem* h, double* y, double* p, ras_stats* stats) {
    if (!h || !y || !p) return RAS_EINVAL;
    TRY(need_single(h));
    return ras_batch_raspen_solve(h, &y, &p, stats);
}

int ras_newton_ras_solve(ras_problem* h, double* y, double* p, ras_stats* stats) {
    if (!h || !y || !p) return RAS_EINVAL;
    TRY(need_single(h));
    stats_clear(stats, 1);
    TRY(copy_in(h, h->X, 0, y, p));
    const int rc = newton_ras_internal(h, stats);
    if (rc == RAS_ECUDA) return rc;
    TRY(check_err_stats(h, stats, 1));
    TRY(copy_out(h, h->X, 0, y, p));
    TRY(sync(h));
    return rc;
}

int ras_newton_solve(ras_problem* h, double* y, double* p, ras_stats* stats) {
    if (!h || !y || !p) return RAS_EINVAL;
    TRY(need_single(h));
    stats_clear(stats, 1);
    TRY(copy_in(h, h->X, 0, y, p));
    const int rc = newton_internal(h, stats, false);
    if (rc == RAS_ECUDA) return rc;
    TRY(check_err_stats(h, stats, 1));
    TRY(copy_out(h, h->X, 0, y, p));
    TRY(sync(h));
    return rc;
}

int ras_get_state(const ras_problem* h, ras_state* state) {
    if (!h || !state) return RAS_EINVAL;
    if (h->nprob != 1 || !h->have_last) return RAS_ESTATE;
    *state = h->last_state;
    return RAS_OK;
}

int ras_set_state(ras_problem* h, const ras_state* st) {
    if (!h || !st) return RAS_EINVAL;
    TRY(need_single(h));
    if ((st->method != RAS_METHOD_RASPEN && st->method != RAS_METHOD_NEWTON_RAS &&
         st->method != RAS_METHOD_NEWTON) ||
        st->k < 0 || !(st->eps > 0) || !std::isfinite(st->eps) || !(st->res0 >= 0) || !std::isfinite(st->res0) ||
        !(st->stop > 0) || !std::isfinite(st->stop))
        return fail(h, RAS_EINVAL, "invalid state");
    h->resume = *st;
    h->have_resume = true;
    return RAS_OK;
}

int ras_autotune(ras_problem* h, ras_tuning* chosen, ras_tune_report* report) {
    if (!h) return RAS_EINVAL;
    return autotune_internal(h, chosen, report);
}

int ras_manufacture(ras_problem* h, const double* pbar, double eps, double* y_out, double* yd_out) {
    if (!h || !pbar || !(eps > 0) || !std::isfinite(eps)) return RAS_EINVAL;
    TRY(need_single(h));
    return manufacture_internal(h, pbar, eps, y_out, yd_out);
}

int ras_use_graphs(ras_problem* h, int enable) {
    if (!h) return RAS_EINVAL;
    h->use_graphs = enable != 0;
    return RAS_OK;
}

int ras_get_tuning(const ras_problem* h, ras_tuning* t) {
    if (!h || !t) return RAS_EINVAL;
    *t = h->tune;
    return RAS_OK;
}

int ras_set_tuning(ras_problem* h, const ras_tuning* t) {
    if (!h || !t) return RAS_EINVAL;
    return install_tuning(h, *t);
}

int ras_solve_host(ras_problem* h, int method, const double* y_d_host, double* y_host, double* p_host,
                   ras_stats* stats) {
    if (!h || !y_host || !p_host ||
        (method != RAS_METHOD_RASPEN && method != RAS_METHOD_NEWTON_RAS && method != RAS_METHOD_NEWTON))
        return RAS_EINVAL;
    TRY(need_single(h));
    stats_clear(stats, 1);
    const long long N = plane(h, 0);
    const size_t nb = N * sizeof(double);
    if (y_d_host) CK(cudaMemcpyAsync(h->yd, y_d_host, nb, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->X, y_host, nb, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->X + N, p_host, nb, cudaMemcpyHostToDevice, h->st));
    h->jvp_ready = false;
    const int rc = (method == RAS_METHOD_RASPEN)       ? raspen_internal(h, stats)
                   : (method == RAS_METHOD_NEWTON_RAS) ? newton_internal(h, stats, true)
                                                       : newton_internal(h, stats, false);
    if (rc == RAS_ECUDA) return rc;
    TRY(check_err(h));
    CK(cudaMemcpyAsync(y_host, h->X, nb, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(p_host, h->X + N, nb, cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    return rc;
}

int ras_local_iterations(const ras_problem* h, int* its_host, int count) {
    if (!h || !its_host || count < 0) return RAS_EINVAL;
    const int k = std::min<int>(count, (int)h->last_its.size());
    for (int i = 0; i < k; ++i) its_host[i] = h->last_its[i];
    return k;
}

int ras_subdomain_count(const ras_problem* h) { return h ? h->nsub : RAS_EINVAL; }

size_t ras_device_bytes(const ras_problem* h) { return h ? h->bytes : 0; }

const char* ras_last_error(const ras_problem* h) {
    if (!h) return "null handle";
    return h->err.c_str();
}

void ras_destroy(ras_problem* h) {
    if (!h) return;
    cudaStreamSynchronize(h->st);
    prof_flush(h);
    for (auto& G : h->cg) destroy_cycle_graph(G);
    if (h->sg.exec) cudaGraphExecDestroy(h->sg.exec);
    if (h->sg.graph) cudaGraphDestroy(h->sg.graph);
    if (h->h_guard) cudaFreeHost(h->h_guard);
    if (h->cap_st) cudaStreamDestroy(h->cap_st);
    if (h->h_any) cudaFreeHost(h->h_any);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (auto& a : h->allocs) cudaFree(a.first);
    h->allocs.clear();
    if (h->h_active) cudaFreeHost(h->h_active);
    if (h->h_scal) cudaFreeHost(h->h_scal);
    delete h;
}

// ------------------------------------------------------------------ serving
// Continuous batching of RASPEN_eps solves (Alg. 2) with restart-cycle
// granularity. Every admitted request is in one of two phases:
//   evaluation - the RASPEN function at x_k (local Newton solves, with
//                eps-continuation for k = 0, at eps_min after), then the stop
//                test: finished, or on to GMRES with b = -F(x_k);
//   GMRES      - restart cycles of GMRES(m) on F'(x_k) d = b with the Jacobian
//                action of Alg. 4; when it stops, x_{k+1} = x_k + d and the
//                request returns to evaluation.
// A step runs one evaluation for every request in the evaluation phase and
// then one restart cycle (at most m Arnoldi steps) for every request in the
// GMRES phase, each group in shared launches. A hard request therefore holds
// the others back by at most one cycle, not by its whole GMRES solve. Each
// request follows the sequence of Alg. 2 (restart cycles only carry the
// iterate), so its result is that of the solve alone up to rounding.
//
// Each admitted request owns one stream-ordered allocation holding what must
// survive between steps: x_k = (y, p), y_d, f, the GMRES right-hand side and
// iterate, the Jacobian coefficients and the local factors at x^(i) (the
// Jacobian action of its GMRES cycles uses them). The batch workspace holds
// only per-step scratch and is laid out anew for the admitted set when it
// changes (buffers only grow). Admission is first come, first served while
// the estimate of request storage plus workspace stays within the budget.
struct ras_server {
    ras_problem* ws = nullptr;        // workspace of the requests in evaluation (stream st)
    ras_problem* wk = nullptr;        // workspace of the requests in GMRES (stream st2)
    size_t budget = 0;
    int max_active = 0;
    ras_opts o{};
    cudaStream_t st = nullptr;
    cudaStream_t st2 = nullptr;
    enum { EVAL = 0, KRYLOV = 1 };
    struct Req {
        long long id = 0;
        ras_problem_desc d{};
        std::vector<double> yd_h, f_h;   // staged host data until admission
        char* mem = nullptr;             // persistent storage (layout below)
        double *x = nullptr, *yd = nullptr, *f = nullptr, *gb = nullptr, *gx = nullptr, *coef = nullptr;
        char* fac = nullptr;
        size_t slot = 0, scratch = 0;    // admission estimate
        int phase = EVAL, k = 0, its = 0;
        bool failed = false, fresh = false;
        double stop = 0.0, target = 0.0;
        ras_stats stats{};
    };
    std::deque<Req*> pending;
    std::vector<Req*> active;            // every admitted request
    std::vector<Req*> finished;          // result kept until fetched
    std::vector<Req*> ev, kr;            // admitted requests by phase (layouts of ws / wk)
    bool dirty = true, dirty_k = true;
    bool use_graphs = false;             // CUDA graphs in the two workspaces (re-captured per relayout)
    long long next_id = 1;
    size_t slot_held = 0, scratch_active = 0, ws_cap = 0;
    std::string err;
};

namespace {

int sfail(ras_server* s, int code, const std::string& msg) {
    if (s) s->err = msg;
    return code;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Persistent storage of one request (bytes, 256-byte aligned parts):
// x (2N), y_d (N), f (N if given), b (2N), GMRES iterate (2N), coefficients
// (3 Nsum), factors (Gsum elements).
struct ReqLayout {
    size_t x, yd, f, gb, gx, coef, fac, total;
};

ReqLayout req_layout(const ras_problem& t, const ras_problem_desc& d, const ras_opts& o) {
    const size_t N = (size_t)d.n * d.n * sizeof(double);
    const size_t es = (o.precision == RAS_MIXED) ? sizeof(float) : sizeof(double);
    ReqLayout L{};
    size_t at = 0;
    L.x = at; at += align256(2 * N);
    L.yd = at; at += align256(N);
    L.f = at; at += d.f ? align256(N) : 0;
    L.gb = at; at += align256(2 * N);
    L.gx = at; at += align256(2 * N);
    L.coef = at; at += align256((size_t)3 * t.Nsum * sizeof(double));
    L.fac = at; at += align256((size_t)t.Gsum * es);
    L.total = at;
    return L;
}

// Device bytes a request needs: its persistent storage, and its share of the
// batch workspace (local pools, global and Krylov vectors, descriptors).
int request_bytes(const ras_problem_desc& d, const ras_opts& o, size_t& slot, size_t& scratch) {
    ras_problem tmp;
    tmp.o = o;
    if (build_layout(&tmp, 1, &d) != RAS_OK) return RAS_EINVAL;
    const size_t es = (o.precision == RAS_MIXED) ? sizeof(float) : sizeof(double);
    slot = req_layout(tmp, d, o).total;
    double b = 5.0 * tmp.Lsum * sizeof(double) + (double)tmp.Lsum * es +
               (double)tmp.nsub * (sizeof(LocalState) + sizeof(SubDev) + 3 * sizeof(int)) +
               (8.0 + o.gmres_restart + 1.0) * tmp.L * sizeof(double) + 3.0 * (double)d.n * d.n * sizeof(double) +
               (double)SS * ras::VEC_BLOCKS * sizeof(double) + 4.0 * SS * sizeof(double) +
               4.0 * (ras::VEC_BLOCKS + 1) * 2 * sizeof(int) + 8.0 * sizeof(int) +
               ((o.gmres_restart + 1.0) * (o.gmres_restart + 3.0) + 1.0) * sizeof(double) + 256.0;
    scratch = (size_t)b;
    return RAS_OK;
}

int server_relayout(ras_server* s, ras_problem*& h, cudaStream_t st, const std::vector<ras_server::Req*>& reqs) {
    if (!h) {
        h = new ras_problem();
        h->o = s->o;
        h->st = st;
        h->own_factors = false;
        h->use_graphs = s->use_graphs;
    }
    std::vector<ras_problem_desc> descs;
    for (auto* r : reqs) {
        ras_problem_desc d = r->d;
        d.y_d = r->yd;
        d.f = r->f;
        descs.push_back(d);
    }
    TRY(build_layout(h, (int)descs.size(), descs.data()));
    TRY(ensure_pools(h, false));
    const size_t es = (s->o.precision == RAS_MIXED) ? sizeof(float) : sizeof(double);
    for (int p = 0; p < h->nprob; ++p) {
        h->probs[p].yd = descs[p].y_d;
        h->probs[p].f = descs[p].f;
        auto* r = reqs[p];
        const SubDev& first = h->subs[h->sub_first[p]];
        for (int k = 0; k < h->sub_count[p]; ++k) {
            SubDev& sd = h->subs[h->sub_first[p] + k];
            sd.gptr = r->fac + (sd.goff - first.goff) * es;
            sd.cptr = r->coef + 3 * (sd.noff - first.noff);
        }
    }
    TRY(upload_layout(h));
    return RAS_OK;
}

int server_admit(ras_server* s) {
    while (!s->pending.empty() && (int)s->active.size() < s->max_active) {
        auto* r = s->pending.front();
        // each of the two workspaces serves part of the admitted set, so
        // neither needs more than the whole set's scratch
        const size_t cap = std::max(s->ws_cap, 2 * (s->scratch_active + r->scratch));
        if (cap + s->slot_held + r->slot > s->budget) break;   // first come, first served
        ras_problem tmp;
        tmp.o = s->o;
        if (build_layout(&tmp, 1, &r->d) != RAS_OK) return sfail(s, RAS_EINVAL, "invalid request layout");
        const ReqLayout L = req_layout(tmp, r->d, s->o);
        void* m = nullptr;
        if (cudaMallocAsync(&m, L.total, s->st) != cudaSuccess) {
            cudaGetLastError();
            break;   // retry at a later step
        }
        r->mem = static_cast<char*>(m);
        r->x = reinterpret_cast<double*>(r->mem + L.x);
        r->yd = reinterpret_cast<double*>(r->mem + L.yd);
        r->f = r->f_h.empty() ? nullptr : reinterpret_cast<double*>(r->mem + L.f);
        r->gb = reinterpret_cast<double*>(r->mem + L.gb);
        r->gx = reinterpret_cast<double*>(r->mem + L.gx);
        r->coef = reinterpret_cast<double*>(r->mem + L.coef);
        r->fac = r->mem + L.fac;
        const long long N = (long long)r->d.n * r->d.n;
        cudaError_t e = cudaMemsetAsync(r->x, 0, 2 * N * sizeof(double), s->st);   // x0 = 0
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->yd, r->yd_h.data(), N * sizeof(double), cudaMemcpyHostToDevice, s->st);
        if (e == cudaSuccess && r->f)
            e = cudaMemcpyAsync(r->f, r->f_h.data(), N * sizeof(double), cudaMemcpyHostToDevice, s->st);
        if (e != cudaSuccess) return sfail(s, RAS_ECUDA, std::string("admission copy: ") + cudaGetErrorString(e));
        r->phase = ras_server::EVAL;
        s->pending.pop_front();
        s->active.push_back(r);
        s->ev.push_back(r);
        s->slot_held += r->slot;
        s->scratch_active += r->scratch;
        s->ws_cap = cap;
        s->dirty = true;
    }
    return RAS_OK;
}

// The evaluation phase of requests `reqs` (workspace h): the RASPEN function
// at x_k and the stop test; those that go on store b = -F(x_k) and are marked
// for GMRES (done[p] = 0, go[p] = 1), the others are finished (done[p] = 1).
int server_eval(ras_server* s, ras_problem* h, const std::vector<ras_server::Req*>& reqs, std::vector<int>& done,
                std::vector<int>& go) {
    Range range("ras: server evaluations");
    const int P = h->nprob;
    const ras_opts& o = s->o;
    done.assign(P, 0);
    go.assign(P, 0);
    std::vector<double> pstart(P);
    std::vector<ras_stats> st(P);
    for (int p = 0; p < P; ++p) {
        auto* r = reqs[p];
        CK(cudaMemcpyAsync(h->X + h->probs[p].ofs, r->x, 2 * plane(h, p) * sizeof(double), cudaMemcpyDeviceToDevice,
                           h->st));
        st[p] = r->stats;
        pstart[p] = (r->k == 0) ? o.eps0 : o.eps_min;
    }
    const int rc = ras_apply_internal(h, pstart, h->F, st.data());
    if (rc == RAS_ECUDA || rc == RAS_ETIMEOUT) return rc;
    for (int p = 0; p < P; ++p) {
        if (st[p].local_failures > reqs[p]->stats.local_failures) reqs[p]->failed = true;
        reqs[p]->stats = st[p];
    }
    TRY(set_mask(h, 1, std::vector<int>(P, 1)));
    TRY(seg_norms2(h, h->F, 1));
    for (int p = 0; p < P; ++p) {
        auto* r = reqs[p];
        const double nrm = std::sqrt(h->h_scal[p * SS]);
        if (r->k == 0) {
            r->stop = std::max(o.tol, o.tol * nrm);
            r->stats.res0 = nrm;
        }
        r->stats.res = nrm;
        if (!r->failed && nrm > r->stop && r->k < o.kmax_outer_raspen) {
            go[p] = 1;
        } else {
            done[p] = 1;
            r->stats.outer_its = r->k;
            r->stats.status = r->failed ? RAS_ENOCONV : (nrm <= r->stop ? RAS_OK : RAS_ENOCONV);
        }
    }
    if (std::any_of(go.begin(), go.end(), [](int v) { return v != 0; })) {
        TRY(set_mask(h, 1, go));
        CK(timed(h, RAS_K_KRYLOV, 0.0, [&] {
            return ras::launch_seg_scale(h->st, seg_grid(h, 1), h->d_segs, h->F, nullptr, -1.0, h->T1);
        }));
        for (int p = 0; p < P; ++p)
            if (go[p])
                CK(cudaMemcpyAsync(reqs[p]->gb, h->T1 + h->probs[p].ofs, 2 * plane(h, p) * sizeof(double),
                                   cudaMemcpyDeviceToDevice, h->st));
    }
    return sync(h);
}

// One GMRES restart cycle for requests `reqs` (workspace h); those whose
// GMRES stopped take x_{k+1} = x_k + d (stopped[p] = 1).
int server_krylov(ras_server* s, ras_problem* h, const std::vector<ras_server::Req*>& reqs,
                  std::vector<int>& stopped) {
    Range range("ras: server GMRES cycles");
    const int P = h->nprob;
    stopped.assign(P, 0);
    GmresResume rs;
    rs.fresh.assign(P, 0);
    rs.target.assign(P, 0.0);
    rs.max_cycles = 1;
    std::vector<int> its(P, 0), conv, all(P, 1);
    for (int p = 0; p < P; ++p) {
        auto* r = reqs[p];
        const long long N = plane(h, p), ofs = h->probs[p].ofs;
        CK(cudaMemcpyAsync(h->X + ofs, r->x, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(h->T1 + ofs, r->gb, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        if (!r->fresh)
            CK(cudaMemcpyAsync(h->Dv + ofs, r->gx, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        rs.fresh[p] = r->fresh ? 1 : 0;
        rs.target[p] = r->target;
        its[p] = r->its;
    }
    auto A = [&](const double* in, double* out, const std::vector<int>& mask) {
        return jvp_internal(h, in, out, &mask);
    };
    auto M = [&](const double*, double*, const std::vector<int>&) { return RAS_OK; };
    TRY(gmres(h, 0, A, M, false, h->T1, h->Dv, all, its, conv, &rs));
    for (int p = 0; p < P; ++p) {
        auto* r = reqs[p];
        r->fresh = false;
        r->target = rs.target[p];
        r->its = its[p];
        if (!rs.pending[p]) stopped[p] = 1;
    }
    if (std::any_of(stopped.begin(), stopped.end(), [](int v) { return v != 0; })) {
        TRY(set_mask(h, 1, stopped));
        CK(timed(h, RAS_K_KRYLOV, 0.0, [&] {
            return ras::launch_seg_add_scaled(h->st, seg_grid(h, 1), h->d_segs, h->X, h->Dv, 1.0, h->X);
        }));
    }
    for (int p = 0; p < P; ++p) {
        auto* r = reqs[p];
        const long long N = plane(h, p), ofs = h->probs[p].ofs;
        if (stopped[p])
            CK(cudaMemcpyAsync(r->x, h->X + ofs, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        else
            CK(cudaMemcpyAsync(r->gx, h->Dv + ofs, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    }
    return sync(h);
}

// One step: the evaluations (workspace ws, stream st) and the GMRES cycles
// (workspace wk, stream st2) run at the same time on two host threads, then
// the requests change phase. A request entering GMRES runs its first cycle
// in the next step; one whose GMRES stopped is evaluated in the next step.
int server_step_active(ras_server* s) {
    Range range("ras: server step");
    if (s->dirty && !s->ev.empty()) TRY(server_relayout(s, s->ws, s->st, s->ev));
    if (s->dirty_k && !s->kr.empty()) TRY(server_relayout(s, s->wk, s->st2, s->kr));
    s->dirty = s->dirty_k = false;
    std::vector<int> done, go, stopped;
    int rk = RAS_OK, re = RAS_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return sfail(s, RAS_ECUDA, "cudaGetDevice failed");
    }
    std::thread worker;
    if (!s->kr.empty()) {
        worker = std::thread([&] {
            if (cudaSetDevice(dev) != cudaSuccess) {
                rk = RAS_ECUDA;
                return;
            }
            rk = server_krylov(s, s->wk, s->kr, stopped);
        });
    }
    if (!s->ev.empty()) re = server_eval(s, s->ws, s->ev, done, go);
    if (worker.joinable()) worker.join();
    if (re < 0) {
        if (s->ws) s->err = s->ws->err;
        return re;
    }
    if (rk < 0) {
        if (s->wk) s->err = s->wk->err;
        return rk;
    }
    std::vector<ras_server::Req*> ev2, kr2;
    for (size_t p = 0; p < s->kr.size(); ++p) {
        auto* r = s->kr[p];
        if (stopped[p]) {
            r->stats.gmres_its += r->its;
            r->k += 1;
            r->phase = ras_server::EVAL;
            ev2.push_back(r);
        } else {
            kr2.push_back(r);
        }
    }
    for (size_t p = 0; p < s->ev.size(); ++p) {
        auto* r = s->ev[p];
        if (done[p]) {
            s->finished.push_back(r);
            s->scratch_active -= r->scratch;
            s->active.erase(std::find(s->active.begin(), s->active.end(), r));
        } else if (go[p]) {
            r->phase = ras_server::KRYLOV;
            r->fresh = true;
            r->its = 0;
            kr2.push_back(r);
        }
    }
    // layouts change when a phase group changes
    s->dirty = !s->ev.empty() || !ev2.empty();
    s->dirty_k = (kr2.size() != s->kr.size()) || !std::equal(kr2.begin(), kr2.end(), s->kr.begin());
    s->ev.swap(ev2);
    s->kr.swap(kr2);
    return RAS_OK;
}

}  // namespace

int ras_server_create(size_t hbm_budget, int max_active, const ras_opts* o, void* stream, ras_server** out) {
    if (!out) return RAS_EINVAL;
    *out = nullptr;
    if (hbm_budget == 0 || max_active < 1 || max_active > 4096) return RAS_EINVAL;
    auto* s = new ras_server();
    if (o) s->o = *o;
    else ras_default_opts(&s->o);
    ras_problem probe;
    if (validate_opts(&probe, s->o) != RAS_OK) {
        delete s;
        return RAS_EINVAL;
    }
    s->budget = hbm_budget;
    s->max_active = max_active;
    s->st = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&s->st2, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return RAS_ECUDA;
    }
    *out = s;
    return RAS_OK;
}

int ras_server_request_bytes(const ras_problem_desc* d, const ras_opts* o, size_t* slot_bytes,
                             size_t* scratch_bytes) {
    if (!d || !desc_valid(*d)) return RAS_EINVAL;
    ras_opts oo;
    if (o) oo = *o;
    else ras_default_opts(&oo);
    size_t a = 0, b = 0;
    TRY(request_bytes(*d, oo, a, b));
    if (slot_bytes) *slot_bytes = a;
    if (scratch_bytes) *scratch_bytes = b;
    return RAS_OK;
}

int ras_server_submit(ras_server* s, const ras_problem_desc* d, long long* id) {
    if (!s || !d || !id || !desc_valid(*d) || !d->y_d) return RAS_EINVAL;
    auto* r = new ras_server::Req();
    r->d = *d;
    if (request_bytes(r->d, s->o, r->slot, r->scratch) != RAS_OK) {
        delete r;
        return sfail(s, RAS_EINVAL, "a subdomain is wider than 256 nodes (2 wx > 512)");
    }
    if (r->slot + 2 * r->scratch > s->budget) {
        delete r;
        return sfail(s, RAS_ENOMEM, "the request alone exceeds the HBM budget");
    }
    const size_t N = (size_t)d->n * d->n;
    r->yd_h.assign(d->y_d, d->y_d + N);
    if (d->f) r->f_h.assign(d->f, d->f + N);
    r->d.y_d = nullptr;
    r->d.f = r->f_h.empty() ? nullptr : d->f;   // only its presence matters for the layout
    r->id = s->next_id++;
    s->pending.push_back(r);
    *id = r->id;
    return RAS_OK;
}

int ras_server_step(ras_server* s, int* active, int* finished) {
    if (!s) return RAS_EINVAL;
    const size_t fin0 = s->finished.size();
    int rc = server_admit(s);
    if (rc == RAS_OK && !s->active.empty()) {
        // admission writes request storage on st; the GMRES stream waits for it
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(ev, s->st);
            cudaStreamWaitEvent(s->st2, ev, 0);
            cudaEventDestroy(ev);
        }
        rc = server_step_active(s);
    }
    if (active) *active = (int)s->active.size();
    if (finished) *finished = (int)(s->finished.size() - fin0);
    return rc;
}

int ras_server_counts(const ras_server* s, int* pending, int* active, int* finished) {
    if (!s) return RAS_EINVAL;
    if (pending) *pending = (int)s->pending.size();
    if (active) *active = (int)s->active.size();
    if (finished) *finished = (int)s->finished.size();
    return RAS_OK;
}

int ras_server_finished_ids(const ras_server* s, long long* ids, int cap) {
    if (!s || (cap > 0 && !ids)) return RAS_EINVAL;
    int k = 0;
    for (auto* r : s->finished) {
        if (k >= cap) break;
        ids[k++] = r->id;
    }
    return k;
}

int ras_server_fetch(ras_server* s, long long id, double* y_host, double* p_host, ras_stats* st) {
    if (!s) return RAS_EINVAL;
    for (auto it = s->finished.begin(); it != s->finished.end(); ++it) {
        ras_server::Req* r = *it;
        if (r->id != id) continue;
        const long long N = (long long)r->d.n * r->d.n;
        cudaError_t e = cudaSuccess;
        if (y_host) e = cudaMemcpyAsync(y_host, r->x, N * sizeof(double), cudaMemcpyDeviceToHost, s->st);
        if (e == cudaSuccess && p_host)
            e = cudaMemcpyAsync(p_host, r->x + N, N * sizeof(double), cudaMemcpyDeviceToHost, s->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
        if (e != cudaSuccess) return sfail(s, RAS_ECUDA, std::string("fetch: ") + cudaGetErrorString(e));
        if (st) *st = r->stats;
        cudaFreeAsync(r->mem, s->st);
        s->slot_held -= r->slot;
        s->finished.erase(it);
        const int status = r->stats.status;
        delete r;
        // an idle server gives its workspaces back
        if (s->active.empty() && s->pending.empty()) {
            cudaStreamSynchronize(s->st);
            if (s->ws) ras_destroy(s->ws);
            if (s->wk) ras_destroy(s->wk);
            s->ws = s->wk = nullptr;
            s->ws_cap = 0;
            s->dirty = s->dirty_k = true;
        }
        return status;
    }
    return sfail(s, RAS_EINVAL, "no finished request with this id");
}

int ras_server_use_graphs(ras_server* s, int enable) {
    if (!s) return RAS_EINVAL;
    s->use_graphs = enable != 0;
    if (s->ws) s->ws->use_graphs = s->use_graphs;
    if (s->wk) s->wk->use_graphs = s->use_graphs;
    return RAS_OK;
}

int ras_server_cancel(ras_server* s, long long id) {
    if (!s) return RAS_EINVAL;
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
        if ((*it)->id != id) continue;
        delete *it;
        s->pending.erase(it);
        return RAS_OK;
    }
    auto drop = [&](std::vector<ras_server::Req*>& v, bool admitted) -> bool {
        for (auto it = v.begin(); it != v.end(); ++it) {
            ras_server::Req* r = *it;
            if (r->id != id) continue;
            if (r->mem) cudaFreeAsync(r->mem, s->st);
            s->slot_held -= r->slot;
            if (admitted) {
                s->scratch_active -= r->scratch;
                s->dirty = true;
            }
            v.erase(it);
            delete r;
            return true;
        }
        return false;
    };
    for (auto* v : {&s->ev, &s->kr}) {
        for (auto it = v->begin(); it != v->end(); ++it) {
            if ((*it)->id != id) continue;
            v->erase(it);
            s->dirty = s->dirty_k = true;
            break;
        }
    }
    if (drop(s->active, true) || drop(s->finished, false)) return RAS_OK;
    return sfail(s, RAS_EINVAL, "no request with this id");
}

size_t ras_server_device_bytes(const ras_server* s) {
    if (!s) return 0;
    return (s->ws ? s->ws->bytes : 0) + (s->wk ? s->wk->bytes : 0) + s->slot_held;
}

const char* ras_server_last_error(const ras_server* s) {
    if (!s) return "null server";
    return s->err.c_str();
}

void ras_server_destroy(ras_server* s) {
    if (!s) return;
    cudaStreamSynchronize(s->st);
    for (auto* r : s->active) {
        if (r->mem) cudaFreeAsync(r->mem, s->st);
        delete r;
    }
    for (auto* r : s->finished) {
        if (r->mem) cudaFreeAsync(r->mem, s->st);
        delete r;
    }
    for (auto* r : s->pending) delete r;
    if (s->ws) ras_destroy(s->ws);
    if (s->wk) ras_destroy(s->wk);
    cudaStreamSynchronize(s->st);
    if (s->st2) {
        cudaStreamSynchronize(s->st2);
        cudaStreamDestroy(s->st2);
    }
    delete s;
}

long long ras_launch_count(void) { return ras::g_launches.load(); }

int ras_profile(ras_problem* h, int enable) {
    if (!h) return RAS_EINVAL;
    TRY(sync(h));
    prof_flush(h);
    for (int k = 0; k < RAS_K_COUNT; ++k) {
        h->prof_ms[k] = 0.0;
        h->prof_n[k] = 0;
        h->prof_work[k] = 0.0;
    }
    h->prof_on = enable != 0;
    return RAS_OK;
}

int ras_profile_read(ras_problem* h, int kind, double* ms, long long* launches, double* work) {
    if (!h || kind < 0 || kind >= RAS_K_COUNT) return RAS_EINVAL;
    TRY(sync(h));
    prof_flush(h);
    if (ms) *ms = h->prof_ms[kind];
    if (launches) *launches = h->prof_n[kind];
    if (work) *work = h->prof_work[kind];
    return RAS_OK;
}

}  // extern "C"
