// Internal declarations of the RAS / RASPEN CUDA library (sm_103a).
//
// Layout in HBM
//  * grid functions: nn = n*n (square) or n*n*n (cube) FP64, x1 index fastest,
//    then x2, then x3 (node (i, j, k) at [(k*n + j)*n + i], k = 0 on the
//    square); global Krylov vectors are planar [y-plane | p-plane], 2*nn.
//  * per subdomain i (box Omega_i of wx*wy*wz nodes at (x0, y0, z0), wz = 1
//    on the square):
//      local vectors: 2*wx*wy*wz FP64, interleaved (y, p) per node, nodes
//                     lexicographic with the x1 index fastest, at voff;
//      node arrays:   wx*wy*wz FP64 (Jacobian coefficients), at noff;
//      factors:       bw blocks G_j of mp^2 T (mp = 2*bl rounded up to 32,
//                     zero padded) at goff, where G_j is the inverse of the
//                     j-th Schur complement of the block-tridiagonal local
//                     Jacobian. A block row is one grid line of the box on the
//                     square (bl = wx nodes, bw = wy rows) and one plane of it
//                     on the cube (bl = wx*wy nodes, bw = wz planes): in both
//                     the rows couple to their neighbours by -beta I only.
//                     Each block is stored in the "packed" order of
//                     packed_index(): the streaming solve reads it as mp/32
//                     contiguous slabs, one per group of 32 rows, and thread t
//                     of a 256-thread CTA finds its share of every slab as
//                     contiguous 16-byte vectors. Wide blocks (MAX_M < 2*bl
//                     <= MAX_MW) are stored column-major instead: element
//                     (r, c) of G_j at c*mp + r, so that the threads of a
//                     CTA, one row each, read a column together.
//                     A wide-block subdomain has one more block after its bw
//                     factor blocks: the factorisation's scratch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ras {

constexpr int MAX_M = 160;          // max unknowns of a block row on the register / streaming path (2*bl)
constexpr int MAX_MW = 512;         // max unknowns of a block row on the wide-block path
constexpr int BIG_THREADS = 1024;   // threads of the wide-block factorisation kernel
constexpr int BIG_PANEL = 16;       // pivots per panel of the wide-block factorisation
constexpr int BIG_CLUSTER = 8;      // CTAs (one per SM) factorising one wide-block subdomain
constexpr int FACT_THREADS = 256;   // threads of the factorisation kernel
constexpr int LOC_THREADS = 256;    // threads of the per-subdomain kernels
constexpr int VEC_THREADS = 256;    // threads of the grid-stride vector kernels
constexpr int VEC_BLOCKS = 608;     // 4 x 152 SMs: fixed grid => fixed reduction order

struct ProbDev {
    int n;                // nodes per grid direction
    int nz;               // grid planes: 1 on the square, n on the cube
    int phi;
    int pad_;
    double h, beta, nu, mu, kappa;
    double diag;          // 2 d beta: diagonal of the (2d+1)-point stencil, d = 2 or 3
    long long nn;         // grid nodes, n*n*nz
    const double* yd;
    const double* f;      // nullptr means f = 0
    long long ofs;        // offset of this problem's y-plane in every global
                          // vector buffer; its p-plane follows at ofs + nn
};

struct SubDev {
    int prob;
    int x0, y0, z0, wx, wy, wz;         // Omega_i (z0 = 0, wz = 1 on the square)
    int ox0, oy0, oz0, owx, owy, owz;   // tilde Omega_i (owned nodes)
    int bl, bw;               // nodes per block row and block rows (wx, wy; wx*wy, wz on the cube)
    int mp;                   // 2*bl rounded up to a multiple of 32 (packed block size)
    int pad_;
    long long goff;           // factor offset (elements of T); bw blocks of mp*mp
    long long voff;           // local-vector offset (doubles), length 2*wx*wy*wz
    long long noff;           // node-array offset (doubles), length wx*wy*wz
    void* gptr;               // this subdomain's factor blocks (bw blocks of mp*mp T)
    double* cptr;             // its Jacobian coefficients (3 arrays of wx*wy*wz doubles)
};

// Local node q of a box -> (lx, ly, lz), x1 index fastest.
__host__ __device__ __forceinline__ void local_coords(const SubDev& s, int q, int& lx, int& ly, int& lz) {
    lx = q % s.wx;
    const int r = q / s.wx;
    ly = r % s.wy;
    lz = r / s.wy;
}

// Global index of grid node (i, j, k) (k = 0 on the square).
__host__ __device__ __forceinline__ long long grid_index(const ProbDev& P, int i, int j, int k) {
    return ((long long)k * P.n + j) * P.n + i;
}

// Is node cx of a block row an in-row stencil neighbour of node ix (the same
// field)? A block row is a grid line (wx = its length, cube = false) or a
// plane of wx-node lines (cube = true).
__host__ __device__ __forceinline__ bool row_neighbour(int ix, int cx, int wx, bool cube) {
    const int d = cx - ix;
    if (!cube) return d == 1 || d == -1;
    if (d == wx || d == -wx) return true;
    if (d == 1) return ix % wx != wx - 1;
    if (d == -1) return ix % wx != 0;
    return false;
}

// Segment of one problem inside a global vector buffer: [ofs, ofs + len).
struct Seg {
    long long ofs, len;
};

// State of Alg. 1 for one subdomain.
struct LocalState {
    double eps, nrm, nrm0, stop, flr;
    int k, status, active, halvings, exhausted, solves;   // solves: local solves done
};

struct NewtonParams {
    double eps_min, gamma, sigma, tol, floor_factor, ir_rtol;
    int kmax, max_halvings, ir_max, pad;
};

// Packed position of element (r, c) of an mp x mp block of T. Thread
// t = 8*rho + kappa (256 threads) owns rows rho + 32 s and the column chunk
// kappa (mp/8 columns); within slab s its chunk is nv = mp/8/VE vectors of 16
// bytes (VE = 16/sizeof(T)) at slab offsets (v*256 + t)*16.
template <typename T>
__host__ __device__ __forceinline__ long long packed_index(int r, int c, int mp) {
    constexpr int VE = 16 / (int)sizeof(T);
    const int cw = mp >> 3, nv = cw / VE;
    const int rho = r & 31, s = r >> 5;
    const int kappa = c / cw, cc = c - kappa * cw;
    const int v = cc / VE, l = cc - v * VE;
    const int t = (rho << 3) + kappa;
    const long long e = (long long)s * nv + v;
    return (e * 256 + t) * VE + l;
}

// Status values (same numbers as the public RAS_* codes).
constexpr int ST_OK = 0;
constexpr int ST_OK_FLOOR = 1;
constexpr int ST_ENOCONV = -3;
constexpr int ST_ESINGULAR = -5;
constexpr int ST_ENONFINITE = -6;
constexpr int ST_ETIMEOUT = -7;
constexpr int ST_SKIP = 2;        // subdomain of a problem not taking part in this evaluation

// ------------------------------------------------------------- pointwise math
// The reduced system (Sec. 3.3) uses the smoothed projection P_eps of Sec. 3.1
// only in two combinations: the control u = -(1/nu)(p + mu P_eps(-p/mu)) =
// -(mu/nu)(P_eps(x) - x) with x = -p/mu, and the Jacobian entry
// (1/nu)(1 - P_eps'(x)). Where |x| < 1 both are O(eps) differences of O(1)
// numbers; evaluated as printed they would lose a relative 2^-53/eps. Both are
// written here with every difference |s| - sqrt(s^2 + eps) replaced by
// -eps/(|s| + sqrt(s^2 + eps)) (the device of Lemma 5's quotient form), so
// they keep full relative accuracy. One division each; valid for |x| < 1e30.

// P_eps(x) - x = x (2 - a - b)/(a + b), a = sqrt((x+1)^2+eps), b = sqrt((x-1)^2+eps),
// 2 - a - b = 2(1 - max(1,|x|)) - eps/t1 - eps/t2, t1 = |x+1| + a, t2 = |x-1| + b.
__device__ __forceinline__ double P_eps_minus_id(double x, double eps) {
    const double s1 = x + 1.0, s2 = x - 1.0;
    const double a = sqrt(fma(s1, s1, eps)), b = sqrt(fma(s2, s2, eps));
    const double t1 = fabs(s1) + a, t2 = fabs(s2) + b;
    const double gap = 2.0 * (1.0 - fmax(1.0, fabs(x)));
    const double t12 = t1 * t2;
    return x * fma(gap, t12, -eps * (t1 + t2)) / ((a + b) * t12);
}

// 1 - P_eps'(x) = ((1 - g(x+1)) + (1 + g(x-1)))/2, g(s) = s/sqrt(s^2+eps):
// 1 - g(s1) = r1/a with r1 = eps/(a + s1) (s1 > 0) or a - s1 (s1 <= 0);
// 1 + g(s2) = r2/b with r2 = eps/(b - s2) (s2 < 0) or b + s2 (s2 >= 0).
__device__ __forceinline__ double one_minus_dP_eps(double x, double eps) {
    const double s1 = x + 1.0, s2 = x - 1.0;
    const double a = sqrt(fma(s1, s1, eps)), b = sqrt(fma(s2, s2, eps));
    double n1, d1, n2, d2;
    if (s1 > 0.0) { n1 = eps; d1 = a + s1; } else { n1 = a - s1; d1 = 1.0; }
    if (s2 < 0.0) { n2 = eps; d2 = b - s2; } else { n2 = b + s2; d2 = 1.0; }
    return 0.5 * fma(n1 * d2, b, n2 * d1 * a) / (d1 * d2 * a * b);
}

// phi, phi', phi'' of the three nonlinearities.
__device__ __forceinline__ void phi_eval(int kind, double kappa, double y,
                                         double& ph, double& d1, double& d2) {
    if (kind == 0) {
        double y2 = y * y;
        ph = y2 * y; d1 = 3.0 * y2; d2 = 6.0 * y;
    } else if (kind == 1) {
        double e = exp(y);
        ph = e; d1 = e; d2 = e;
    } else {
        double e = exp(kappa * y);
        ph = kappa * (y * y * y + e);
        d1 = kappa * (3.0 * y * y + kappa * e);
        d2 = kappa * (6.0 * y + kappa * kappa * e);
    }
}

// eps_{k+1} = max(gamma eps_k, eps_min), with a product within a relative 1e-9
// of eps_min taken as eps_min (the FP64 rounding of the geometric sequence).
__device__ __host__ __forceinline__ double next_eps(double eps, double gamma, double eps_min) {
    double e = gamma * eps;
    return (e <= eps_min * (1.0 + 1e-9)) ? eps_min : e;
}

// Deterministic block sum of two values (fixed tree over the threads).
template <int NT>
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
    const int t = threadIdx.x;
    red[t] = a;
    red[NT + t] = b;
    __syncthreads();
#pragma unroll
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (t < s) {
            red[t] += red[t + s];
            red[NT + t] += red[NT + t + s];
        }
        __syncthreads();
    }
    a = red[0];
    b = red[NT];
    __syncthreads();
}

template <int NT>
__device__ __forceinline__ double block_sum1(double a, double* red) {
    const int t = threadIdx.x;
    red[t] = a;
    __syncthreads();
#pragma unroll
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (t < s) red[t] += red[t + s];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

}  // namespace ras

// ------------------------------------------------------------- launchers
// Implemented in the .cu files; every launcher returns the cudaError_t of
// its launch and counts the launch.
namespace ras {
void count_launch();

// global (grid) kernels: residual.cu
cudaError_t launch_residual_global(cudaStream_t st, const ProbDev& P, const double* y, const double* p,
                                   const double* dy, const double* dp, double alpha, double eps,
                                   double* Fy, double* Fp, double* partials, int floor);
cudaError_t launch_reduce_partials(cudaStream_t st, const double* partials, int nparts, int nvals,
                                   double* out);
cudaError_t launch_coef_global(cudaStream_t st, const ProbDev& P, const double* y, const double* p,
                               double eps, double* coef);
cudaError_t launch_jacvec_global(cudaStream_t st, const ProbDev& P, const double* coef,
                                 const double* vy, const double* vp, double* oy, double* op);
cudaError_t launch_dot_multi(cudaStream_t st, const double* V, long long ld, int nv, const double* w,
                             long long len, double* partials);
cudaError_t launch_axpy_multi(cudaStream_t st, const double* V, long long ld, int nv, const double* h,
                              double sign, double* w, long long len);
cudaError_t launch_scale_copy(cudaStream_t st, const double* src, const double* num, const double* den,
                              double sign, double* dst, long long len);
cudaError_t launch_axpy(cudaStream_t st, double a, const double* x, double* y, long long len);
cudaError_t launch_add_scaled(cudaStream_t st, const double* x, const double* d, double alpha,
                              double* out, long long len);

// segmented (one segment per problem) Krylov kernels: residual.cu.
// Partials / results are laid out [problem][32] (32 = max vectors).
constexpr int SEG_STRIDE = 32;
// Blocks of the segmented kernels: block b works on problem tab[b].x as its
// tab[b].y-th of nbps[problem] blocks (problems left out have nbps = 0). The
// host spreads VEC_BLOCKS blocks over the taking-part problems in proportion
// to their segment lengths; partial sums use the stride VEC_BLOCKS.
// Entries with tab[b].x < 0 are unused (their blocks do nothing).
struct SegGrid {
    const int2* tab;
    const int* nbps;
    int nblocks;
};
cudaError_t launch_seg_dot(cudaStream_t st, SegGrid g, const Seg* segs, const double* V, long long ld, int nv,
                           const double* w, double* partials);
cudaError_t launch_seg_reduce(cudaStream_t st, int nprob, const int* nbps, int nv, const double* partials,
                              double* out);
cudaError_t launch_seg_axpy(cudaStream_t st, SegGrid g, const Seg* segs, const double* V, long long ld, int nv,
                            const double* h, double sign, double* w);
cudaError_t launch_seg_scale(cudaStream_t st, SegGrid g, const Seg* segs, const double* src, const double* n2,
                             double sign, double* dst);
cudaError_t launch_seg_add_scaled(cudaStream_t st, SegGrid g, const Seg* segs, const double* x, const double* d,
                                  double alpha, double* out);

// Block table of the problems p with act[p] built on the device (one CTA):
// the same split as the host's (vec_blocks blocks in proportion to the
// segment lengths, at least one and at most one per 512 elements each), in
// tab[0 .. cap) with unused entries (-1, 0), nbps[p] blocks per problem (0
// for the others); offs: nprob + 1 ints of scratch.
cudaError_t launch_seg_table(cudaStream_t st, int nprob, const int* act, const Seg* segs, int vec_blocks, int cap,
                             int2* tab, int* nbps, int* offs);

// Arnoldi step j of GMRES(m) for every problem p with act[p] (one CTA, one
// thread per problem): column j of the Hessenberg matrix H_p from the CGS2
// coefficients h1 + h2 ([problem][32]) and hn = sqrt(n2), the earlier Givens
// rotations applied to it, the new rotation (cs, sn) and the rotated
// right-hand side g_p; its[p] and steps[p] advance, and act[p] is cleared
// when hn = 0, |g_p[j+1]| <= target[p] or its[p] >= maxit. *any: some problem
// still iterates. Layouts: H [p][(m+1) m] row-major, cs/sn [p][m], g [p][m+1].
cudaError_t launch_gmres_givens(cudaStream_t st, int nprob, int m, int j, int* act, const double* h1,
                                const double* h2, const double* n2, double* H, double* cs, double* sn, double* g,
                                int* its, int* steps, const double* target, int maxit, int* any);
// Kernel node (in graph `g`, after `dep`) that sets conditional handle `c` to
// (*any != 0).
cudaError_t add_set_conditional_node(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle c,
                                     const int* any, cudaGraphNode_t* out);
void add_launches(long long n);   // kernels a graph launch ran (counted once at capture)

// per-subdomain kernels: local.cu. X, F, D, O, R, Z are global vector bases
// (problem k at ProbDev.ofs); pools are indexed by SubDev offsets.
cudaError_t launch_local_init(cudaStream_t st, int nsub, const SubDev* subs, const ProbDev* probs,
                              const double* X, LocalState* ls, const double* pstart, NewtonParams np,
                              double* cpool, double* Kpool, int* active_count);
// FP32 register-tile factorisation of the `count` subdomains in `list`
// (device indices; null = 0..count-1), all with packed size mp <= 16*tile.
// Device-side choice between the two FP32 factor kernels of a class: with
// nwork set, the 1024-thread kernel works when min(*nwork, count) <= thr and
// the 256-thread one otherwise (the other returns at once), so one graph can
// hold both launches. nwork null: the launched kernel always works.
struct FactorSel {
    const int* nwork;
    int thr;
};
// FP32 factorisation of one register-tile class (tile = mp / 16) over the
// `count` subdomains of `list`: 256-thread CTAs (two per SM) by default;
// wide != 0 selects 1024-thread CTAs (one per SM), faster when at most one
// CTA per SM has work.
cudaError_t launch_local_factor_f32(cudaStream_t st, int tile, int count, const int* list, const SubDev* subs,
                                    const ProbDev* probs, const double* X, LocalState* ls, const double* cpool,
                                    double* coef, float* gpool, int only_active, int wide,
                                    FactorSel sel = FactorSel{nullptr, 0});
// Loop condition of the local Newton sweep (Alg. 1 in every subdomain) as a
// graph WHILE node: c = (*active > 0 && g <= limit) with g the number of
// earlier evaluations (*guard, 0 when reset), which it then increments.
cudaError_t launch_sweep_cond(cudaStream_t st, cudaGraphConditionalHandle c, const int* active, int* guard,
                              int limit, int reset);
cudaError_t add_sweep_cond_node(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle c,
                                const int* active, int* guard, int limit, int reset, cudaGraphNode_t* out);
template <typename T>
cudaError_t launch_local_factor(cudaStream_t st, int nsub, int maxm, const SubDev* subs,
                                const ProbDev* probs, const double* X, LocalState* ls,
                                const double* cpool, double* coef, T* gpool, int only_active);
// Factorisation of the `count` wide-block subdomains in `list` (device
// indices, MAX_M < 2*bl <= MAX_MW): one cluster of BIG_CLUSTER 1024-thread
// CTAs each, the block in its own factor slot in HBM (blocked Gauss-Jordan
// with partial pivoting by implicit interchanges, panels of BIG_PANEL pivots,
// the columns split among the CTAs), G_j stored column-major. Each such
// subdomain has one scratch block after its bw factor blocks.
template <typename T>
cudaError_t launch_local_factor_big(cudaStream_t st, int count, const int* list, const SubDev* subs,
                                    const ProbDev* probs, const double* X, LocalState* ls, const double* cpool,
                                    double* coef, T* gpool, int only_active);
// The local-solve kernels (direction, Jacobian action, linear RAS) are
// persistent: the grid holds as many CTAs as fit at once, and each takes the
// next of the nsub positions of `order` (subdomain indices, largest factors
// first) from *ticket, which the launcher zeroes on the stream. ctas_per_sm
// caps the CTAs per SM (0: as many as fit).
template <typename T>
cudaError_t launch_local_direction(cudaStream_t st, int nsub, int ctas_per_sm, const SubDev* subs,
                                   const ProbDev* probs, LocalState* ls, NewtonParams np,
                                   const double* coef, const T* gpool, const double* Kpool,
                                   double* dpool, double* rpool, T* wpool, int* err, const int* order,
                                   int* ticket);
cudaError_t launch_local_linesearch(cudaStream_t st, int nsub, const SubDev* subs, const ProbDev* probs,
                                    const double* X, LocalState* ls, NewtonParams np, double* cpool,
                                    const double* dpool, double* Kpool, double* Ktpool,
                                    int* active_count);
cudaError_t launch_local_prolong(cudaStream_t st, int nsub, const SubDev* subs, const ProbDev* probs,
                                 const LocalState* ls, const double* cpool, double* F);
template <typename T>
cudaError_t launch_local_jvp(cudaStream_t st, int nsub, int ctas_per_sm, const SubDev* subs,
                             const ProbDev* probs, const T* gpool, T* wpool, const double* coef,
                             double* zpool, double* rpool, double* bpool, int nir, const double* D,
                             double* O, const int* pmask, int* err, const int* order, int* ticket);
template <typename T>
cudaError_t launch_local_precond(cudaStream_t st, int nsub, int ctas_per_sm, const SubDev* subs,
                                 const ProbDev* probs, const T* gpool, T* wpool, const double* R,
                                 double* Z, int* err, const int* order, int* ticket);
// The same three solves for the `count` wide-block subdomains of `list` (one
// 256-thread CTA each, the column-major factor blocks streamed by TMA as
// chunks of whole columns).
// The kernels above skip wide-block subdomains.
template <typename T>
cudaError_t launch_local_direction_wide(cudaStream_t st, int count, const int* list, const SubDev* subs,
                                        const ProbDev* probs, LocalState* ls, NewtonParams np,
                                        const double* coef, const T* gpool, const double* Kpool, double* dpool,
                                        double* rpool, T* wpool, int* err);
template <typename T>
cudaError_t launch_local_jvp_wide(cudaStream_t st, int count, const int* list, const SubDev* subs,
                                  const ProbDev* probs, const T* gpool, T* wpool, const double* coef,
                                  double* zpool, double* rpool, double* bpool, int nir, const double* D, double* O,
                                  const int* pmask, int* err);
template <typename T>
cudaError_t launch_local_precond_wide(cudaStream_t st, int count, const int* list, const SubDev* subs,
                                      const ProbDev* probs, const T* gpool, T* wpool, const double* R, double* Z,
                                      int* err);
cudaError_t solve_ctas_per_sm_max(bool f32, int* per_sm);
}  // namespace ras
