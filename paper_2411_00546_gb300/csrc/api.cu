// Host side of the RAS / RASPEN library: the C ABI of include/ras.h, the
// decomposition (Sec. 4.2), the per-sweep launch sequence of Alg. 3, GMRES,
// RASPEN (Alg. 2) and Newton_RAS (Alg. 1 with linear RAS). Every arithmetic
// step runs in the kernels of local.cu and residual.cu; this file only
// orders launches, moves scalars and applies the stop rules.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ras.h"
#include "ras_internal.cuh"

namespace ras {
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace ras

using ras::LocalState;
using ras::NewtonParams;
using ras::ProbDev;
using ras::SubDev;

struct ras_problem {
    int n = 0, sx = 0, sy = 0, overlap = 0, phi = 0;
    double nu = 0.0, mu = 0.0;
    ras_opts o{};
    cudaStream_t st = nullptr;
    int nsub = 0, maxm = 0;
    long long N = 0;          // n*n
    long long Lsum = 0;       // sum of 2*wx*wy
    long long Nsum = 0;       // sum of wx*wy
    long long Gsum = 0;       // sum of wy*(2wx)^2
    std::vector<SubDev> subs;
    ProbDev prob{};
    SubDev* d_subs = nullptr;
    ProbDev* d_prob = nullptr;
    double* yd = nullptr;
    double* f = nullptr;
    double *cpool = nullptr, *dpool = nullptr, *Kpool = nullptr, *Ktpool = nullptr, *rpool = nullptr;
    double* coef = nullptr;
    void* gpool = nullptr;
    void* wpool = nullptr;
    int gprec = -1;
    LocalState* ls = nullptr;
    int* d_active = nullptr;
    int* d_err = nullptr;        // set by kernels whose bounded waits ran out
    int* h_active = nullptr;     // pinned
    double *X = nullptr, *F = nullptr, *Dv = nullptr, *Ov = nullptr, *T1 = nullptr, *T2 = nullptr,
           *T3 = nullptr, *Z = nullptr;
    double* coefG = nullptr;
    double* partials = nullptr;
    double* scal = nullptr;      // device scalars
    double* h_scal = nullptr;    // pinned host scalars
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
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[RAS_K_COUNT] = {};
    long long prof_n[RAS_K_COUNT] = {};
    double prof_work[RAS_K_COUNT] = {};
    std::vector<void*> allocs;
    size_t bytes = 0;
    std::string err;
};

namespace {

constexpr int NSCAL = 160;

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
    h->allocs.push_back((void*)*p);
    h->bytes += count * sizeof(T);
    return RAS_OK;
}

void dfree(ras_problem* h, void* p) {
    if (!p) return;
    auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
    if (it != h->allocs.end()) h->allocs.erase(it);
    cudaFree(p);
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
        !std::isfinite(o.kappa) || o.jvp_ir < 0 || o.jvp_ir > 8)
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
    if (h->gprec == prec) return RAS_OK;
    dfree(h, h->gpool);
    dfree(h, h->wpool);
    h->gpool = h->wpool = nullptr;
    const size_t es = (prec == RAS_MIXED) ? sizeof(float) : sizeof(double);
    char* g = nullptr;
    char* w = nullptr;
    TRY(dalloc(h, &g, (size_t)h->Gsum * es));
    TRY(dalloc(h, &w, (size_t)h->Lsum * es));
    h->gpool = g;
    h->wpool = w;
    h->gprec = prec;
    return RAS_OK;
}

int sync(ras_problem* h) {
    CK(cudaStreamSynchronize(h->st));
    if (h->prof_on && h->prof_recs.size() > 2048) prof_flush(h);
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

size_t prec_bytes(const ras_problem* h) { return h->o.precision == RAS_MIXED ? sizeof(float) : sizeof(double); }

// Algorithmic work of a factorisation of the subdomains with mask[i] != 0:
// 16 wx^3 wy flops each (block-tridiagonal Gauss-Jordan = no-fill band LU count).
double factor_flops(const ras_problem* h, const std::vector<LocalState>* ls) {
    double w = 0.0;
    for (int i = 0; i < h->nsub; ++i) {
        if (ls && !(*ls)[i].active) continue;
        const double wx = h->subs[i].wx, wy = h->subs[i].wy;
        w += 16.0 * wx * wx * wx * wy;
    }
    return w;
}

// Bytes of one two-pass block solve over every subdomain's factor.
double solve_bytes_all(const ras_problem* h) {
    return 2.0 * (double)h->Gsum * (double)prec_bytes(h);
}

double resid_bytes(const ras_problem* h) { return (h->f ? 48.0 : 40.0) * (double)h->N; }

// ||F(x + alpha d, eps)|| and the rounding-floor norm; writes F to Fout (2N) if given.
int residual_norm(ras_problem* h, const double* x, const double* d, double alpha, double eps,
                  double* Fout, double& nrm, double& flr) {
    const long long N = h->N;
    CK(timed(h, RAS_K_RESIDUAL, resid_bytes(h), [&] {
        return ras::launch_residual_global(h->st, h->prob, x, x + N, d, d ? d + N : nullptr, alpha, eps, Fout,
                                           Fout ? Fout + N : nullptr, h->partials);
    }));
    CK(timed(h, RAS_K_OTHER, 0.0, [&] { return ras::launch_reduce_partials(h->st, h->partials, ras::VEC_BLOCKS, 2, h->scal); }));
    CK(cudaMemcpyAsync(h->h_scal, h->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    nrm = std::sqrt(h->h_scal[0]);
    flr = std::sqrt(h->h_scal[1]);
    return RAS_OK;
}

// ||v||_2 of a global vector (2N), deterministic.
int vec_norm(ras_problem* h, const double* v, double& out) {
    const long long len = 2 * h->N;
    CK(timed(h, RAS_K_KRYLOV, 8.0 * len, [&] { return ras::launch_dot_multi(h->st, v, len, 1, v, len, h->partials); }));
    CK(timed(h, RAS_K_OTHER, 0.0, [&] { return ras::launch_reduce_partials(h->st, h->partials, ras::VEC_BLOCKS, 1, h->scal); }));
    CK(cudaMemcpyAsync(h->h_scal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    out = std::sqrt(h->h_scal[0]);
    return RAS_OK;
}

int copy_in(ras_problem* h, double* dst, const double* y, const double* p) {
    CK(cudaMemcpyAsync(dst, y, h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(dst + h->N, p, h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    return RAS_OK;
}

int copy_out(ras_problem* h, const double* src, double* y, double* p) {
    if (y) CK(cudaMemcpyAsync(y, src, h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (p) CK(cudaMemcpyAsync(p, src + h->N, h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    return RAS_OK;
}

void stats_clear(ras_stats* s) {
    if (!s) return;
    std::memset(s, 0, sizeof(*s));
}

// --------------------------------------------------------------- Alg. 3
template <typename T>
int ras_apply_T(ras_problem* h, int continuation, double* Fout, ras_stats* stats) {
    const NewtonParams np = inner_params(h->o);
    const double eps_start = continuation ? h->o.eps0 : h->o.eps_min;
    T* gp = (T*)h->gpool;
    T* wp = (T*)h->wpool;
    CK(cudaMemsetAsync(h->d_active, 0, sizeof(int), h->st));
    CK(timed(h, RAS_K_INIT, 0.0, [&] {
        return ras::launch_local_init(h->st, h->nsub, h->d_subs, h->d_prob, h->X, h->ls, eps_start, np, h->cpool,
                                      h->Kpool, h->d_active);
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
            fl = factor_flops(h, &before);
        }
        CK(timed(h, RAS_K_FACTOR, fl, [&] {
            return ras::launch_local_factor<T>(h->st, h->nsub, h->maxm, h->d_subs, h->d_prob, h->X, h->ls,
                                               h->cpool, h->coef, gp, 1);
        }));
        CK(timed(h, RAS_K_DIRECTION, 0.0, [&] {
            return ras::launch_local_direction<T>(h->st, h->nsub, h->maxm, h->d_subs, h->d_prob, h->ls, np,
                                                  h->coef, gp, h->Kpool, h->dpool, h->rpool, wp, h->d_err);
        }));
        const size_t dir_rec = h->prof_recs.size();
        CK(cudaMemsetAsync(h->d_active, 0, sizeof(int), h->st));
        CK(timed(h, RAS_K_LINESEARCH, 0.0, [&] {
            return ras::launch_local_linesearch(h->st, h->nsub, h->d_subs, h->d_prob, h->X, h->ls, np, h->cpool,
                                                h->dpool, h->Kpool, h->Ktpool, h->d_active);
        }));
        CK(cudaMemcpyAsync(h->h_active, h->d_active, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        TRY(sync(h));
        if (h->prof_on && dir_rec >= 1 && dir_rec <= h->prof_recs.size()) {
            TRY(read_ls(after));
            double bytes = 0.0;
            for (int i = 0; i < h->nsub; ++i) {
                const double m = 2.0 * h->subs[i].wx;
                bytes += (after[i].solves - before[i].solves) * 2.0 * m * m * h->subs[i].wy * sizeof(T);
            }
            h->prof_recs[dir_rec - 1].work = bytes;
        }
    }
    // factors at x^(i) = x + P_i C_i(x) for the Jacobian action (Alg. 4)
    CK(timed(h, RAS_K_FACTOR, factor_flops(h, nullptr), [&] {
        return ras::launch_local_factor<T>(h->st, h->nsub, h->maxm, h->d_subs, h->d_prob, h->X, h->ls, h->cpool,
                                           h->coef, gp, 0);
    }));
    CK(timed(h, RAS_K_OTHER, 0.0, [&] {
        return ras::launch_local_prolong(h->st, h->nsub, h->d_subs, h->d_prob, h->cpool, Fout);
    }));
    std::vector<LocalState> ls(h->nsub);
    CK(cudaMemcpyAsync(ls.data(), h->ls, h->nsub * sizeof(LocalState), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    int worst = RAS_OK;
    h->last_its.assign(h->nsub, 0);
    int itmax = 0, fails = 0, halv = 0, exh = 0;
    long long itsum = 0;
    for (int i = 0; i < h->nsub; ++i) {
        h->last_its[i] = ls[i].k;
        itmax = std::max(itmax, ls[i].k);
        itsum += ls[i].k;
        halv += ls[i].halvings;
        exh += ls[i].exhausted;
        if (ls[i].status < 0) {
            ++fails;
            worst = std::min(worst, ls[i].status);
        }
    }
    h->jvp_ready = (worst >= 0);
    if (stats) {
        stats->evaluations += 1;
        stats->inner_its_max += itmax;
        stats->inner_its_sum += itsum;
        stats->halvings += halv;
        stats->exhausted += exh;
        stats->local_failures += fails;
        stats->eps_final = h->o.eps_min;
    }
    if (worst < 0) return fail(h, worst, "local Newton solve failed in " + std::to_string(fails) + " subdomain(s)");
    return RAS_OK;
}

int ras_apply_internal(ras_problem* h, int continuation, double* Fout, ras_stats* stats) {
    TRY(alloc_factor_pools(h));
    if (h->o.precision == RAS_MIXED) return ras_apply_T<float>(h, continuation, Fout, stats);
    return ras_apply_T<double>(h, continuation, Fout, stats);
}

int jvp_internal(ras_problem* h, const double* D, double* O) {
    const int nir = (h->o.precision == RAS_MIXED) ? h->o.jvp_ir : 0;
    CK(timed(h, RAS_K_JVP, solve_bytes_all(h) * (1 + nir), [&] {
        if (h->o.precision == RAS_MIXED)
            return ras::launch_local_jvp<float>(h->st, h->nsub, h->maxm, h->d_subs, h->d_prob,
                                                (const float*)h->gpool, (float*)h->wpool, h->coef, h->dpool,
                                                h->rpool, h->Ktpool, nir, D, O, h->d_err);
        return ras::launch_local_jvp<double>(h->st, h->nsub, h->maxm, h->d_subs, h->d_prob,
                                             (const double*)h->gpool, (double*)h->wpool, h->coef, h->dpool,
                                             h->rpool, h->Ktpool, 0, D, O, h->d_err);
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
    CK(timed(h, RAS_K_FACTOR, factor_flops(h, nullptr), [&] {
        if (h->o.precision == RAS_MIXED)
            return ras::launch_local_factor<float>(h->st, h->nsub, h->maxm, h->d_subs, h->d_prob, h->X, h->ls,
                                                   h->cpool, h->coef, (float*)h->gpool, 0);
        return ras::launch_local_factor<double>(h->st, h->nsub, h->maxm, h->d_subs, h->d_prob, h->X, h->ls,
                                                h->cpool, h->coef, (double*)h->gpool, 0);
    }));
    CK(cudaMemcpyAsync(ls.data(), h->ls, h->nsub * sizeof(LocalState), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    h->jvp_ready = false;
    for (auto& s : ls)
        if (s.status < 0) return fail(h, s.status, "singular local Jacobian");
    return RAS_OK;
}

int precond_internal(ras_problem* h, const double* R, double* Zo) {
    CK(timed(h, RAS_K_PRECOND, solve_bytes_all(h), [&] {
        if (h->o.precision == RAS_MIXED)
            return ras::launch_local_precond<float>(h->st, h->nsub, h->maxm, h->d_subs, h->d_prob,
                                                    (const float*)h->gpool, (float*)h->wpool, R, Zo, h->d_err);
        return ras::launch_local_precond<double>(h->st, h->nsub, h->maxm, h->d_subs, h->d_prob,
                                                 (const double*)h->gpool, (double*)h->wpool, R, Zo, h->d_err);
    }));
    return RAS_OK;
}

// --------------------------------------------------------------- GMRES
// Restarted GMRES(m), CGS2 Arnoldi, Givens rotations, x0 = 0, right
// preconditioning when `prec` is true. A(in, out) and M(in, out) act on
// global vectors (2N). One host synchronisation per Krylov step.
template <class Aop, class Mop>
int gmres(ras_problem* h, Aop A, Mop M, bool prec, const double* b, double* x, int& its, bool& conv) {
    const long long len = 2 * h->N;
    const int m = h->o.gmres_restart;
    const double rtol = h->o.gmres_rtol;
    const int maxit = h->o.gmres_maxit;
    if (h->Vm < m) {
        dfree(h, h->V);
        h->V = nullptr;
        TRY(dalloc(h, &h->V, (size_t)(m + 1) * len));
        h->Vm = m;
    }
    double* V = h->V;
    double* r = h->T2;
    double* upd = h->T3;
    CK(cudaMemsetAsync(x, 0, len * sizeof(double), h->st));
    its = 0;
    conv = false;
    double bnorm;
    TRY(vec_norm(h, b, bnorm));
    if (bnorm == 0.0) {
        conv = true;
        return RAS_OK;
    }
    const double target = rtol * bnorm;
    CK(cudaMemcpyAsync(r, b, len * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    for (;;) {
        double beta;
        TRY(vec_norm(h, r, beta));
        if (beta <= target || its >= maxit) {
            conv = beta <= target;
            return RAS_OK;
        }
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        CK(timed(h, RAS_K_KRYLOV, 16.0 * len, [&] { return ras::launch_scale_copy(h->st, r, nullptr, nullptr, 1.0 / beta, V, len); }));
        int steps = 0;
        for (int j = 0; j < m; ++j) {
            double* vj = V + (long long)j * len;
            double* w = V + (long long)(j + 1) * len;
            if (prec) {
                TRY(M(vj, h->Z));
                TRY(A(h->Z, w));
            } else {
                TRY(A(vj, w));
            }
            // CGS2: two passes of classical Gram-Schmidt
            const double dbytes = 8.0 * len * (j + 2), abytes = 8.0 * len * (j + 3);
            CK(timed(h, RAS_K_KRYLOV, dbytes, [&] { return ras::launch_dot_multi(h->st, V, len, j + 1, w, len, h->partials); }));
            CK(timed(h, RAS_K_OTHER, 0.0, [&] { return ras::launch_reduce_partials(h->st, h->partials, ras::VEC_BLOCKS, j + 1, h->scal); }));
            CK(timed(h, RAS_K_KRYLOV, abytes, [&] { return ras::launch_axpy_multi(h->st, V, len, j + 1, h->scal, -1.0, w, len); }));
            CK(timed(h, RAS_K_KRYLOV, dbytes, [&] { return ras::launch_dot_multi(h->st, V, len, j + 1, w, len, h->partials); }));
            CK(timed(h, RAS_K_OTHER, 0.0, [&] { return ras::launch_reduce_partials(h->st, h->partials, ras::VEC_BLOCKS, j + 1, h->scal + 32); }));
            CK(timed(h, RAS_K_KRYLOV, abytes, [&] { return ras::launch_axpy_multi(h->st, V, len, j + 1, h->scal + 32, -1.0, w, len); }));
            CK(timed(h, RAS_K_KRYLOV, 8.0 * len, [&] { return ras::launch_dot_multi(h->st, w, len, 1, w, len, h->partials); }));
            CK(timed(h, RAS_K_OTHER, 0.0, [&] { return ras::launch_reduce_partials(h->st, h->partials, ras::VEC_BLOCKS, 1, h->scal + 64); }));
            CK(cudaMemcpyAsync(h->h_scal, h->scal, 65 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
            TRY(sync(h));
            for (int i = 0; i <= j; ++i) H[i * m + j] = h->h_scal[i] + h->h_scal[32 + i];
            const double hn = std::sqrt(h->h_scal[64]);
            H[(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                H[i * m + j] = t;
            }
            const double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
            cs[j] = H[j * m + j] / den;
            sn[j] = H[(j + 1) * m + j] / den;
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++its;
            steps = j + 1;
            if (hn == 0.0 || std::fabs(g[j + 1]) <= target || its >= maxit) break;
            CK(timed(h, RAS_K_KRYLOV, 16.0 * len, [&] { return ras::launch_scale_copy(h->st, w, nullptr, nullptr, 1.0 / hn, w, len); }));
        }
        for (int i = steps - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < steps; ++k) s -= H[i * m + k] * y[k];
            y[i] = s / H[i * m + i];
        }
        for (int i = 0; i < steps; ++i) h->h_scal[96 + i] = y[i];
        CK(cudaMemcpyAsync(h->scal + 96, h->h_scal + 96, steps * sizeof(double), cudaMemcpyHostToDevice, h->st));
        CK(cudaMemsetAsync(upd, 0, len * sizeof(double), h->st));
        CK(timed(h, RAS_K_KRYLOV, 8.0 * len * (steps + 2), [&] { return ras::launch_axpy_multi(h->st, V, len, steps, h->scal + 96, 1.0, upd, len); }));
        if (prec) {
            TRY(M(upd, h->Z));
            CK(timed(h, RAS_K_KRYLOV, 24.0 * len, [&] { return ras::launch_axpy(h->st, 1.0, h->Z, x, len); }));
        } else {
            CK(timed(h, RAS_K_KRYLOV, 24.0 * len, [&] { return ras::launch_axpy(h->st, 1.0, upd, x, len); }));
        }
        TRY(A(x, r));
        CK(timed(h, RAS_K_KRYLOV, 24.0 * len, [&] { return ras::launch_add_scaled(h->st, b, r, -1.0, r, len); }));
    }
}

// --------------------------------------------------------------- Alg. 2
int raspen_internal(ras_problem* h, ras_stats* s) {
    const long long len = 2 * h->N;
    int rc = ras_apply_internal(h, 1, h->F, s);
    if (rc < 0) return rc;
    double nrm;
    TRY(vec_norm(h, h->F, nrm));
    const double stop = std::max(h->o.tol, h->o.tol * nrm);
    if (s) s->res0 = nrm;
    int k = 0;
    auto A = [&](const double* in, double* out) { return jvp_internal(h, in, out); };
    auto M = [&](const double*, double*) { return RAS_OK; };
    while (nrm > stop && k < h->o.kmax_outer_raspen) {
        CK(timed(h, RAS_K_KRYLOV, 16.0 * len, [&] { return ras::launch_scale_copy(h->st, h->F, nullptr, nullptr, -1.0, h->T1, len); }));
        int its = 0;
        bool conv = false;
        TRY(gmres(h, A, M, false, h->T1, h->Dv, its, conv));
        if (s) s->gmres_its += its;
        CK(timed(h, RAS_K_KRYLOV, 24.0 * len, [&] { return ras::launch_axpy(h->st, 1.0, h->Dv, h->X, len); }));
        ++k;
        rc = ras_apply_internal(h, 0, h->F, s);
        if (rc < 0) {
            if (s) s->outer_its = k;
            return rc;
        }
        TRY(vec_norm(h, h->F, nrm));
    }
    if (s) {
        s->outer_its = k;
        s->res = nrm;
        s->status = (nrm <= stop) ? RAS_OK : RAS_ENOCONV;
    }
    if (!(nrm <= stop)) return fail(h, RAS_ENOCONV, "RASPEN reached kmax_outer_raspen");
    return RAS_OK;
}

// --------------------------------------------------------------- Newton_RAS
int newton_ras_internal(ras_problem* h, ras_stats* s) {
    const long long len = 2 * h->N;
    const ras_opts& o = h->o;
    double eps = o.eps0, nrm, flr;
    TRY(residual_norm(h, h->X, nullptr, 0.0, eps, h->F, nrm, flr));
    const double stop = std::max(o.tol, o.tol * nrm);
    if (s) s->res0 = nrm;
    int k = 0, status = RAS_OK;
    auto A = [&](const double* in, double* out) -> int {
        CK(timed(h, RAS_K_OTHER, 56.0 * h->N, [&] { return ras::launch_jacvec_global(h->st, h->prob, h->coefG, in, in + h->N, out, out + h->N); }));
        return RAS_OK;
    };
    auto M = [&](const double* in, double* out) { return precond_internal(h, in, out); };
    for (;;) {
        if (!std::isfinite(nrm)) { status = RAS_ENONFINITE; break; }
        if (eps == o.eps_min) {
            if (nrm <= stop) { status = RAS_OK; break; }
            if (nrm <= o.floor_factor * 1.1102230246251565e-16 * flr) { status = RAS_OK_FLOOR; break; }
        }
        if (k >= o.kmax_outer_newton) { status = RAS_ENOCONV; break; }
        TRY(factor_at(h, eps));
        CK(timed(h, RAS_K_OTHER, 40.0 * h->N, [&] { return ras::launch_coef_global(h->st, h->prob, h->X, h->X + h->N, eps, h->coefG); }));
        CK(timed(h, RAS_K_KRYLOV, 16.0 * len, [&] { return ras::launch_scale_copy(h->st, h->F, nullptr, nullptr, -1.0, h->T1, len); }));
        int its = 0;
        bool conv = false;
        TRY(gmres(h, A, M, true, h->T1, h->Dv, its, conv));
        if (s) s->gmres_its += its;
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
        CK(timed(h, RAS_K_KRYLOV, 24.0 * len, [&] { return ras::launch_add_scaled(h->st, h->X, h->Dv, alpha, h->X, len); }));
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
    if (status < 0) return fail(h, status, "Newton_RAS stopped without convergence");
    return status;
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
    o->jvp_ir = 1;
    o->reserved = 0;
    return RAS_OK;
}

int ras_create(int n, int sx, int sy, int overlap, int phi, double nu, double mu, const double* y_d,
               const double* f, const ras_opts* o, void* stream, ras_problem** out) {
    if (!out) return RAS_EINVAL;
    *out = nullptr;
    if (n < 2 || sx < 1 || sy < 1 || sx > n || sy > n || overlap < 0 || phi < 0 || phi > 2 || !(nu > 0) ||
        !(mu > 0) || !std::isfinite(nu) || !std::isfinite(mu) || !y_d)
        return RAS_EINVAL;
    ras_problem* h = new ras_problem();
    h->n = n; h->sx = sx; h->sy = sy; h->overlap = overlap; h->phi = phi; h->nu = nu; h->mu = mu;
    if (o) h->o = *o;
    else ras_default_opts(&h->o);
    h->st = (cudaStream_t)stream;
    int rc = validate_opts(h, h->o);
    if (rc < 0) { delete h; return rc; }
    h->N = (long long)n * n;
    const auto bx = split_blocks(n, sx), by = split_blocks(n, sy);
    long long voff = 0, noff = 0, goff = 0;
    for (int j = 0; j < sy; ++j) {
        for (int i = 0; i < sx; ++i) {
            SubDev s{};
            s.prob = 0;
            s.ox0 = bx[i].first; s.owx = bx[i].second - bx[i].first;
            s.oy0 = by[j].first; s.owy = by[j].second - by[j].first;
            s.x0 = std::max(0, s.ox0 - overlap);
            s.y0 = std::max(0, s.oy0 - overlap);
            s.wx = std::min(n, bx[i].second + overlap) - s.x0;
            s.wy = std::min(n, by[j].second + overlap) - s.y0;
            s.mp = ((2 * s.wx + 31) / 32) * 32;
            s.voff = voff; s.noff = noff; s.goff = goff;
            voff += 2LL * s.wx * s.wy;
            noff += (long long)s.wx * s.wy;
            goff += (long long)s.wy * s.mp * s.mp;
            h->maxm = std::max(h->maxm, 2 * s.wx);
            h->subs.push_back(s);
        }
    }
    if (h->maxm > ras::MAX_M) {
        delete h;
        return RAS_EINVAL;
    }
    h->nsub = (int)h->subs.size();
    h->Lsum = voff; h->Nsum = noff; h->Gsum = goff;
    const long long N = h->N;
    rc = RAS_OK;
    auto A = [&](int r) { if (rc == RAS_OK && r < 0) rc = r; };
    A(dalloc(h, &h->yd, N));
    A(dalloc(h, &h->d_subs, h->nsub));
    A(dalloc(h, &h->d_prob, 1));
    A(dalloc(h, &h->cpool, h->Lsum));
    A(dalloc(h, &h->dpool, h->Lsum));
    A(dalloc(h, &h->Kpool, h->Lsum));
    A(dalloc(h, &h->Ktpool, h->Lsum));
    A(dalloc(h, &h->rpool, h->Lsum));
    A(dalloc(h, &h->coef, 3 * h->Nsum));
    A(dalloc(h, &h->ls, h->nsub));
    A(dalloc(h, &h->d_active, 1));
    A(dalloc(h, &h->d_err, 1));
    for (double** p : {&h->X, &h->F, &h->Dv, &h->Ov, &h->T1, &h->T2, &h->T3, &h->Z}) A(dalloc(h, p, 2 * N));
    A(dalloc(h, &h->coefG, 3 * N));
    A(dalloc(h, &h->partials, (size_t)ras::VEC_BLOCKS * 32));
    A(dalloc(h, &h->scal, NSCAL));
    if (rc == RAS_OK && f) A(dalloc(h, &h->f, N));
    if (rc == RAS_OK) A(alloc_factor_pools(h));
    if (rc == RAS_OK) {
        if (cudaMallocHost((void**)&h->h_active, sizeof(int)) != cudaSuccess ||
            cudaMallocHost((void**)&h->h_scal, NSCAL * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            rc = RAS_ENOMEM;
        }
    }
    if (rc != RAS_OK) {
        ras_destroy(h);
        return rc;
    }
    h->prob.n = n;
    h->prob.phi = phi;
    h->prob.h = 1.0 / (n + 1);
    h->prob.beta = 1.0 / (h->prob.h * h->prob.h);
    h->prob.nu = nu;
    h->prob.mu = mu;
    h->prob.kappa = h->o.kappa;
    h->prob.yd = h->yd;
    h->prob.f = h->f;
    h->prob.ofs = 0;
    cudaError_t e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->yd, y_d, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess && f) e = cudaMemcpyAsync(h->f, f, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_subs, h->subs.data(), h->nsub * sizeof(SubDev), cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_prob, &h->prob, sizeof(ProbDev), cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        ras_destroy(h);
        return RAS_ECUDA;
    }
    *out = h;
    return RAS_OK;
}

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
    const bool kappa_changed = (o->kappa != h->o.kappa);
    h->o = *o;
    h->jvp_ready = false;
    TRY(alloc_factor_pools(h));
    if (kappa_changed) {
        h->prob.kappa = o->kappa;
        CK(cudaMemcpyAsync(h->d_prob, &h->prob, sizeof(ProbDev), cudaMemcpyHostToDevice, h->st));
        TRY(sync(h));
    }
    return RAS_OK;
}

int ras_set_data(ras_problem* h, const double* y_d, const double* f) {
    if (!h || !y_d) return RAS_EINVAL;
    CK(cudaMemcpyAsync(h->yd, y_d, h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (f) {
        if (!h->f) TRY(dalloc(h, &h->f, h->N));
        CK(cudaMemcpyAsync(h->f, f, h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    }
    if ((f != nullptr) != (h->prob.f != nullptr)) {
        h->prob.f = f ? h->f : nullptr;
        CK(cudaMemcpyAsync(h->d_prob, &h->prob, sizeof(ProbDev), cudaMemcpyHostToDevice, h->st));
    }
    h->jvp_ready = false;
    return sync(h);
}

int ras_residual(ras_problem* h, const double* y, const double* p, double eps, double* Fy, double* Fp,
                 double* norm_host) {
    if (!h || !y || !p || !(eps > 0)) return RAS_EINVAL;
    CK(ras::launch_residual_global(h->st, h->prob, y, p, nullptr, nullptr, 0.0, eps, Fy, Fp, h->partials));
    CK(ras::launch_reduce_partials(h->st, h->partials, ras::VEC_BLOCKS, 2, h->scal));
    CK(cudaMemcpyAsync(h->h_scal, h->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    TRY(sync(h));
    if (norm_host) *norm_host = std::sqrt(h->h_scal[0]);
    return RAS_OK;
}

int ras_apply(ras_problem* h, const double* y, const double* p, int continuation, double* Fy, double* Fp,
              ras_stats* stats) {
    if (!h || !y || !p || !Fy || !Fp) return RAS_EINVAL;
    stats_clear(stats);
    TRY(copy_in(h, h->X, y, p));
    const int rc = ras_apply_internal(h, continuation, h->F, stats);
    if (rc == RAS_ECUDA) return rc;
    TRY(check_err(h));
    TRY(copy_out(h, h->F, Fy, Fp));
    TRY(sync(h));
    if (stats) stats->status = rc;
    return rc;
}

int ras_jvp(ras_problem* h, const double* dy, const double* dp, double* oy, double* op) {
    if (!h || !dy || !dp || !oy || !op) return RAS_EINVAL;
    if (!h->jvp_ready) return fail(h, RAS_ESTATE, "ras_jvp needs a successful ras_apply first");
    TRY(copy_in(h, h->Dv, dy, dp));
    TRY(jvp_internal(h, h->Dv, h->Ov));
    TRY(copy_out(h, h->Ov, oy, op));
    TRY(sync(h));
    return check_err(h);
}

int ras_precondition(ras_problem* h, const double* y, const double* p, double eps, const double* ry,
                     const double* rp, double* zy, double* zp) {
    if (!h || !y || !p || !ry || !rp || !zy || !zp || !(eps > 0)) return RAS_EINVAL;
    TRY(copy_in(h, h->X, y, p));
    TRY(factor_at(h, eps));
    TRY(copy_in(h, h->T1, ry, rp));
    TRY(precond_internal(h, h->T1, h->Z));
    TRY(copy_out(h, h->Z, zy, zp));
    TRY(sync(h));
    return check_err(h);
}

int ras_raspen_solve(ras_problem* h, double* y, double* p, ras_stats* stats) {
    if (!h || !y || !p) return RAS_EINVAL;
    stats_clear(stats);
    TRY(copy_in(h, h->X, y, p));
    const int rc = raspen_internal(h, stats);
    if (rc == RAS_ECUDA) return rc;
    TRY(check_err(h));
    TRY(copy_out(h, h->X, y, p));
    TRY(sync(h));
    return rc;
}

int ras_newton_ras_solve(ras_problem* h, double* y, double* p, ras_stats* stats) {
    if (!h || !y || !p) return RAS_EINVAL;
    stats_clear(stats);
    TRY(copy_in(h, h->X, y, p));
    const int rc = newton_ras_internal(h, stats);
    if (rc == RAS_ECUDA) return rc;
    TRY(check_err(h));
    TRY(copy_out(h, h->X, y, p));
    TRY(sync(h));
    return rc;
}

int ras_solve_host(ras_problem* h, int method, const double* y_d_host, double* y_host, double* p_host,
                   ras_stats* stats) {
    if (!h || !y_host || !p_host || (method != RAS_METHOD_RASPEN && method != RAS_METHOD_NEWTON_RAS))
        return RAS_EINVAL;
    stats_clear(stats);
    const size_t nb = h->N * sizeof(double);
    if (y_d_host) CK(cudaMemcpyAsync(h->yd, y_d_host, nb, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->X, y_host, nb, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->X + h->N, p_host, nb, cudaMemcpyHostToDevice, h->st));
    h->jvp_ready = false;
    const int rc = (method == RAS_METHOD_RASPEN) ? raspen_internal(h, stats) : newton_ras_internal(h, stats);
    if (rc == RAS_ECUDA) return rc;
    TRY(check_err(h));
    CK(cudaMemcpyAsync(y_host, h->X, nb, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(p_host, h->X + h->N, nb, cudaMemcpyDeviceToHost, h->st));
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
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    prof_flush(h);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->h_active) cudaFreeHost(h->h_active);
    if (h->h_scal) cudaFreeHost(h->h_scal);
    delete h;
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
