// Per-subdomain kernels of the nonlinear RAS sweep (Alg. 3), its Jacobian
// action (Alg. 4) and the linear RAS preconditioner (Newton_RAS).
//
// One CTA owns one subdomain i for the whole launch. The local problem is
//   K_i(c) = R_i F_eps(x + P_i c) = 0                          (Sec. 4.2)
// solved by Alg. 1 from c = 0. Its Jacobian J_i = R_i F'(x + P_i c) P_i in the
// interleaved (y, p) ordering, grouped by grid rows of Omega_i, is block
// tridiagonal: diagonal blocks D_j (one grid row, m = 2 wx unknowns) and
// off-diagonal blocks -beta I (the 5-point coupling between neighbouring rows,
// beta = 1/h^2, the same for both fields). Its block LU therefore only needs
//   S_0 = D_0,  S_j = D_j - beta^2 S_{j-1}^-1,
// and the factor stores G_j = S_j^-1, computed by Gauss-Jordan elimination
// with partial pivoting inside each block. A solve J z = b is
//   w_0 = b_0, w_j = b_j + beta G_{j-1} w_{j-1};
//   z_{W-1} = G_{W-1} w_{W-1}, z_j = G_j (w_j + beta z_{j+1}).
#include "ras_internal.cuh"

namespace ras {

namespace {

constexpr int NT = LOC_THREADS;
constexpr int NW = NT / 32;
constexpr double U_ROUND = 1.1102230246251565e-16;  // 2^-53

// Value of the local state at local node (lx, ly), field f:
// x + c + alpha d on Omega_i, x on the ring outside it, 0 outside the grid.
struct LocalView {
    const double* X;   // y-plane of this problem; p-plane at X + nn
    long long nn;
    int n, x0, y0, wx, wy;
    const double* c;
    const double* d;   // may be null
    double alpha;

    __device__ __forceinline__ double val(int lx, int ly, int f) const {
        const int gi = x0 + lx, gj = y0 + ly;
        if (gi < 0 || gi >= n || gj < 0 || gj >= n) return 0.0;
        double v = X[f * nn + (long long)gj * n + gi];
        if (lx >= 0 && lx < wx && ly >= 0 && ly < wy) {
            const int lq = 2 * (ly * wx + lx) + f;
            double cc = c[lq];
            if (d) cc = fma(alpha, d[lq], cc);
            v += cc;
        }
        return v;
    }
};

__device__ __forceinline__ LocalView make_view(const SubDev& s, const ProbDev& P, const double* X,
                                               const double* c, const double* d, double alpha) {
    LocalView V;
    V.X = X + P.ofs;
    V.nn = (long long)P.n * P.n;
    V.n = P.n;
    V.x0 = s.x0; V.y0 = s.y0; V.wx = s.wx; V.wy = s.wy;
    V.c = c; V.d = d; V.alpha = alpha;
    return V;
}

// K_i at the view's state and eps (residual F of Sec. 3.3 at the nodes of
// Omega_i). Writes the interleaved residual to `out` when non-null and
// returns (block-wide) its squared 2-norm and the squared norm of the
// nodewise |term| sums (rounding-floor estimate).
__device__ void local_residual(const LocalView& V, const ProbDev& P, double eps, double* out,
                               double& nrm2, double& flr2, double* red) {
    const int wx = V.wx, nn = wx * V.wy;
    const double beta = P.beta, inu = 1.0 / P.nu, mu = P.mu;
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nn; q += NT) {
        const int lx = q % wx, ly = q / wx;
        const long long g = (long long)(V.y0 + ly) * V.n + (V.x0 + lx);
        const double yc = V.val(lx, ly, 0), yw = V.val(lx - 1, ly, 0), ye = V.val(lx + 1, ly, 0);
        const double ys = V.val(lx, ly - 1, 0), yn = V.val(lx, ly + 1, 0);
        const double pc = V.val(lx, ly, 1), pw = V.val(lx - 1, ly, 1), pe = V.val(lx + 1, ly, 1);
        const double ps = V.val(lx, ly - 1, 1), pn = V.val(lx, ly + 1, 1);
        double ph, d1, d2;
        phi_eval(P.phi, P.kappa, yc, ph, d1, d2);
        const double fv = P.f ? P.f[g] : 0.0;
        const double pe_ = P_eps(-pc / mu, eps);
        const double Fy = beta * (4.0 * yc - yw - ye - ys - yn) + ph - fv + inu * (pc + mu * pe_);
        const double Fp = beta * (4.0 * pc - pw - pe - ps - pn) + d1 * pc - yc + P.yd[g];
        const double My = beta * (4.0 * fabs(yc) + fabs(yw) + fabs(ye) + fabs(ys) + fabs(yn)) + fabs(ph) +
                          fabs(fv) + inu * (fabs(pc) + mu * fabs(pe_));
        const double Mp = beta * (4.0 * fabs(pc) + fabs(pw) + fabs(pe) + fabs(ps) + fabs(pn)) +
                          fabs(d1 * pc) + fabs(yc) + fabs(P.yd[g]);
        if (out) {
            out[2 * q] = Fy;
            out[2 * q + 1] = Fp;
        }
        a += Fy * Fy + Fp * Fp;
        b += My * My + Mp * Mp;
    }
    block_sum2<NT>(a, b, red);
    nrm2 = a;
    flr2 = b;
}

// Stop / continue decision of Alg. 1 (stop tests applied at eps_min only).
__device__ __forceinline__ void decide(LocalState& L, const NewtonParams& np) {
    if (!isfinite(L.nrm)) {
        L.status = ST_ENONFINITE;
        L.active = 0;
        return;
    }
    if (L.eps == np.eps_min) {
        if (L.nrm <= L.stop) {
            L.status = ST_OK;
            L.active = 0;
            return;
        }
        if (L.nrm <= np.floor_factor * U_ROUND * L.flr) {
            L.status = ST_OK_FLOOR;
            L.active = 0;
            return;
        }
    }
    if (L.k >= np.kmax) {
        L.status = ST_ENOCONV;
        L.active = 0;
        return;
    }
    L.status = ST_OK;
    L.active = 1;
}

__global__ void __launch_bounds__(NT) k_local_init(int nsub, const SubDev* __restrict__ subs,
                                                   const ProbDev* __restrict__ probs, const double* X,
                                                   LocalState* ls, double eps_start, NewtonParams np,
                                                   double* cpool, double* Kpool, int* active_count) {
    __shared__ double red[2 * NT];
    const int i = blockIdx.x;
    if (i >= nsub) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const int L = 2 * s.wx * s.wy;
    double* c = cpool + s.voff;
    for (int q = threadIdx.x; q < L; q += NT) c[q] = 0.0;
    __syncthreads();
    const LocalView V = make_view(s, P, X, c, nullptr, 0.0);
    double n2, f2;
    local_residual(V, P, eps_start, Kpool + s.voff, n2, f2, red);
    if (threadIdx.x == 0) {
        LocalState st;
        st.eps = eps_start;
        st.nrm = sqrt(n2);
        st.nrm0 = st.nrm;
        st.stop = fmax(np.tol, np.tol * st.nrm);
        st.flr = sqrt(f2);
        st.k = 0;
        st.halvings = 0;
        st.exhausted = 0;
        st.solves = 0;
        decide(st, np);
        ls[i] = st;
        if (st.active) atomicAdd(active_count, 1);
    }
}

// ------------------------------------------------------------------ factor
// Dynamic shared memory: M (maxm x (maxm+1) T), pivot column (maxm T),
// perm, rinv, used (3 x maxm int).
template <typename T>
__global__ void __launch_bounds__(FACT_THREADS) k_local_factor(int nsub, int maxm,
                                                               const SubDev* __restrict__ subs,
                                                               const ProbDev* __restrict__ probs,
                                                               const double* X, LocalState* ls,
                                                               const double* cpool, double* coef,
                                                               T* gpool, int only_active) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int FW = FACT_THREADS / 32;
    const int i = blockIdx.x;
    if (i >= nsub) return;
    if (only_active && !ls[i].active) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const int m = 2 * s.wx, W = s.wy, nn = s.wx * s.wy, LD = maxm + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T* M = reinterpret_cast<T*>(smem_raw);
    T* colk = M + (size_t)maxm * LD;
    int* perm = reinterpret_cast<int*>(colk + maxm);
    int* rinv = perm + maxm;
    int* used = rinv + maxm;
    __shared__ int sh_r, sh_fail;
    __shared__ T sh_piv;

    const double eps = ls[i].eps;
    const double beta = P.beta, inu = 1.0 / P.nu, mu = P.mu;
    double* ca = coef + 3 * s.noff;
    double* cb = ca + nn;
    double* cc = cb + nn;
    {
        const double* c = cpool + s.voff;
        const LocalView V = make_view(s, P, X, c, nullptr, 0.0);
        for (int q = tid; q < nn; q += FACT_THREADS) {
            const int lx = q % s.wx, ly = q / s.wx;
            const double y = V.val(lx, ly, 0), p = V.val(lx, ly, 1);
            double ph, d1, d2;
            phi_eval(P.phi, P.kappa, y, ph, d1, d2);
            ca[q] = d1;
            cb[q] = inu * (1.0 - dP_eps(-p / mu, eps));
            cc[q] = d2 * p - 1.0;
        }
    }
    if (tid == 0) sh_fail = 0;
    __syncthreads();

    const T tbeta = (T)beta, tbeta2 = (T)(beta * beta), tdiag = (T)(4.0 * beta);
    T* G = gpool + s.goff;
    for (int j = 0; j < W; ++j) {
        // S_j = D_j - beta^2 G_{j-1}
        const T* Gp = G + (long long)(j > 0 ? j - 1 : 0) * m * m;
        for (int r = warp; r < m; r += FW) {
            const int ix = r >> 1, f = r & 1;
            const int q = j * s.wx + ix;
            for (int cidx = lane; cidx < m; cidx += 32) {
                const int cx = cidx >> 1, cf = cidx & 1;
                T v = (j > 0) ? -tbeta2 * Gp[r * m + cidx] : (T)0;
                if (cx == ix) {
                    if (cf == f) v += tdiag + (T)ca[q];
                    else if (f == 0) v += (T)cb[q];
                    else v += (T)cc[q];
                } else if (cf == f && (cx == ix - 1 || cx == ix + 1)) {
                    v -= tbeta;
                }
                M[r * LD + cidx] = v;
            }
        }
        for (int t = tid; t < m; t += FACT_THREADS) used[t] = 0;
        __syncthreads();

        // Gauss-Jordan inversion in place, pivot rows chosen by partial
        // pivoting (max |.| among unused rows, ties to the lowest row) and
        // never moved: afterwards M[r][c] = S^-1[rinv[r]][perm[c]].
        for (int k = 0; k < m; ++k) {
            if (warp == 0) {
                T best = (T)-1;
                int bi = 0x7fffffff;
                for (int r = lane; r < m; r += 32) {
                    if (!used[r]) {
                        const T v = fabs(M[r * LD + k]);
                        if (v > best) { best = v; bi = r; }
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const T ob = __shfl_xor_sync(0xffffffffu, best, off);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (lane == 0) {
                    if (bi >= m || !(best > (T)0)) {
                        sh_fail = 1;
                        sh_r = 0;
                        sh_piv = (T)1;
                    } else {
                        sh_r = bi;
                        used[bi] = 1;
                        perm[k] = bi;
                        sh_piv = M[bi * LD + k];
                    }
                }
            }
            __syncthreads();
            if (sh_fail) break;
            const int r = sh_r;
            const T inv = (T)1 / sh_piv;
            for (int t = tid; t < m; t += FACT_THREADS) colk[t] = M[t * LD + k];
            __syncthreads();
            for (int t = tid; t < m; t += FACT_THREADS) M[r * LD + t] = (t == k ? (T)1 : M[r * LD + t]) * inv;
            __syncthreads();
            for (int rr = warp; rr < m; rr += FW) {
                if (rr == r) continue;
                const T fct = colk[rr];
                for (int t = lane; t < m; t += 32) {
                    const T old = (t == k) ? (T)0 : M[rr * LD + t];
                    M[rr * LD + t] = old - fct * M[r * LD + t];
                }
            }
            __syncthreads();
        }
        if (sh_fail) break;
        for (int t = tid; t < m; t += FACT_THREADS) rinv[perm[t]] = t;
        __syncthreads();
        T* Gj = G + (long long)j * m * m;
        for (int r = warp; r < m; r += FW) {
            const int pr = perm[r];
            for (int cidx = lane; cidx < m; cidx += 32) Gj[r * m + cidx] = M[pr * LD + rinv[cidx]];
        }
        __syncthreads();
    }
    if (sh_fail && tid == 0) {
        ls[i].status = ST_ESINGULAR;
        ls[i].active = 0;
    }
}

// ------------------------------------------------------------------ solve
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// out[k] = sum_c G[k*m + c] vec[c], one warp per row, lanes across columns.
template <typename T>
__device__ __forceinline__ void block_matvec(const T* __restrict__ G, int m, const T* vec, T* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = warp; k < m; k += NW) {
        const T* row = G + (long long)k * m;
        T acc = (T)0;
#pragma unroll 5
        for (int cidx = lane; cidx < m; cidx += 32) acc += __ldg(row + cidx) * vec[cidx];
        acc = warp_sum(acc);
        if (lane == 0) out[k] = acc;
    }
}

// z = J_i^-1 b with the stored G_j. rhs(j, t) gives b (row j, unknown t);
// out(j, t, z) consumes z. w: global scratch of m*W T. vec, tmp: shared, m T.
template <typename T, class Rhs, class Out>
__device__ void block_solve(const T* __restrict__ G, int m, int W, T beta, T* w, T* vec, T* tmp,
                            Rhs rhs, Out out) {
    const int tid = threadIdx.x;
    for (int j = 0; j < W; ++j) {
        for (int t = tid; t < m; t += NT) {
            T v = rhs(j, t);
            if (j > 0) v += beta * tmp[t];
            vec[t] = v;
            w[j * m + t] = v;
        }
        __syncthreads();
        if (j < W - 1) {
            block_matvec(G + (long long)j * m * m, m, vec, tmp);
            __syncthreads();
        }
    }
    for (int j = W - 1; j >= 0; --j) {
        for (int t = tid; t < m; t += NT) {
            T v = w[j * m + t];
            if (j < W - 1) v += beta * tmp[t];
            vec[t] = v;
        }
        __syncthreads();
        block_matvec(G + (long long)j * m * m, m, vec, tmp);
        __syncthreads();
        for (int t = tid; t < m; t += NT) out(j, t, tmp[t]);
    }
    __syncthreads();
}

// r = bsign * B - J_i z in FP64 with the Jacobian coefficients stored by the
// factor kernel (5-point coupling inside Omega_i only); returns ||r||^2.
__device__ double local_linear_residual(const SubDev& s, double beta, const double* coef, double bsign,
                                        const double* B, const double* z, double* r, double* red) {
    const int wx = s.wx, wy = s.wy, nn = wx * wy;
    const double* ca = coef + 3 * s.noff;
    const double* cb = ca + nn;
    const double* cc = cb + nn;
    double r2 = 0.0, dummy = 0.0;
    for (int q = threadIdx.x; q < nn; q += NT) {
        const int lx = q % wx, ly = q / wx;
        const double zyc = z[2 * q], zpc = z[2 * q + 1];
        double sy = 0.0, sp = 0.0;
        if (lx > 0) { sy += z[2 * (q - 1)]; sp += z[2 * (q - 1) + 1]; }
        if (lx < wx - 1) { sy += z[2 * (q + 1)]; sp += z[2 * (q + 1) + 1]; }
        if (ly > 0) { sy += z[2 * (q - wx)]; sp += z[2 * (q - wx) + 1]; }
        if (ly < wy - 1) { sy += z[2 * (q + wx)]; sp += z[2 * (q + wx) + 1]; }
        const double Jy = beta * (4.0 * zyc - sy) + ca[q] * zyc + cb[q] * zpc;
        const double Jp = beta * (4.0 * zpc - sp) + cc[q] * zyc + ca[q] * zpc;
        const double ry = bsign * B[2 * q] - Jy, rp = bsign * B[2 * q + 1] - Jp;
        r[2 * q] = ry;
        r[2 * q + 1] = rp;
        r2 += ry * ry + rp * rp;
    }
    block_sum2<NT>(r2, dummy, red);
    return r2;
}

// Newton direction d = -J_i^-1 K_i. In mixed precision the FP32 solve is
// followed by FP64 iterative refinement: r = -K - J d with the FP64 Jacobian
// (matrix-free, from the coefficients the factor kernel stored), d += J^-1 r,
// until ||r|| <= ir_rtol ||K|| or ir_max corrections.
template <typename T>
__global__ void __launch_bounds__(NT) k_local_direction(int nsub, const SubDev* __restrict__ subs,
                                                        const ProbDev* __restrict__ probs,
                                                        LocalState* ls, NewtonParams np,
                                                        const double* coef, const T* gpool,
                                                        const double* Kpool, double* dpool,
                                                        double* rpool, T* wpool) {
    __shared__ T vec[MAX_M], tmp[MAX_M];
    __shared__ double red[2 * NT];
    const int i = blockIdx.x;
    if (i >= nsub) return;
    if (!ls[i].active) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const int m = 2 * s.wx, W = s.wy, L = m * W, wx = s.wx, wy = s.wy, nn = wx * wy;
    const double beta = P.beta;
    const double* K = Kpool + s.voff;
    double* d = dpool + s.voff;
    double* r = rpool + s.voff;
    T* w = wpool + s.voff;
    const T* G = gpool + s.goff;
    double b2 = 0.0, dummy = 0.0;
    for (int q = threadIdx.x; q < L; q += NT) {
        const double v = -K[q];
        r[q] = v;
        d[q] = 0.0;
        b2 += v * v;
    }
    block_sum2<NT>(b2, dummy, red);
    const double bnorm = sqrt(b2);
    int nsolves = 0;
    for (int it = 0;; ++it) {
        ++nsolves;
        block_solve<T>(
            G, m, W, (T)beta, w, vec, tmp, [=](int j, int t) { return (T)r[j * m + t]; },
            [=](int j, int t, T z) { d[j * m + t] += (double)z; });
        if (it >= np.ir_max) break;
        const double r2 = local_linear_residual(s, beta, coef, -1.0, K, d, r, red);
        if (sqrt(r2) <= np.ir_rtol * bnorm) break;
    }
    if (threadIdx.x == 0) ls[i].solves += nsolves;
}

// Backtracking (relaxed test with sigma), step, eps update and stop test of
// Alg. 1 for every active subdomain.
__global__ void __launch_bounds__(NT) k_local_linesearch(int nsub, const SubDev* __restrict__ subs,
                                                         const ProbDev* __restrict__ probs,
                                                         const double* X, LocalState* ls,
                                                         NewtonParams np, double* cpool,
                                                         const double* dpool, double* Kpool,
                                                         double* Ktpool, int* active_count) {
    __shared__ double red[2 * NT];
    const int i = blockIdx.x;
    if (i >= nsub) return;
    LocalState L = ls[i];
    if (!L.active) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const int len = 2 * s.wx * s.wy;
    double* c = cpool + s.voff;
    const double* d = dpool + s.voff;
    double* K = Kpool + s.voff;
    double* Kt = Ktpool + s.voff;
    double alpha = 1.0, nt = 0.0, ft = 0.0;
    int h = 0;
    for (;;) {
        const LocalView V = make_view(s, P, X, c, d, alpha);
        double n2, f2;
        local_residual(V, P, L.eps, Kt, n2, f2, red);
        nt = sqrt(n2);
        ft = sqrt(f2);
        if (nt <= np.sigma * L.nrm || h == np.max_halvings) break;
        alpha *= 0.5;
        ++h;
    }
    if (!(nt <= np.sigma * L.nrm)) L.exhausted++;
    L.halvings += h;
    for (int q = threadIdx.x; q < len; q += NT) c[q] = fma(alpha, d[q], c[q]);
    __syncthreads();
    const double en = next_eps(L.eps, np.gamma, np.eps_min);
    if (en == L.eps) {
        for (int q = threadIdx.x; q < len; q += NT) K[q] = Kt[q];
        L.nrm = nt;
        L.flr = ft;
    } else {
        const LocalView V = make_view(s, P, X, c, nullptr, 0.0);
        double n2, f2;
        local_residual(V, P, en, K, n2, f2, red);
        L.nrm = sqrt(n2);
        L.flr = sqrt(f2);
    }
    L.eps = en;
    L.k += 1;
    decide(L, np);
    __syncthreads();
    if (threadIdx.x == 0) {
        ls[i] = L;
        if (L.active) atomicAdd(active_count, 1);
    }
}

// Restricted prolongation (Sec. 4.2): F[owned nodes of i] = C_i.
__global__ void __launch_bounds__(NT) k_local_prolong(int nsub, const SubDev* __restrict__ subs,
                                                      const ProbDev* __restrict__ probs,
                                                      const double* cpool, double* F) {
    const int i = blockIdx.x;
    if (i >= nsub) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const long long nn = (long long)P.n * P.n;
    double* Fy = F + P.ofs;
    const double* c = cpool + s.voff;
    const int no = s.owx * s.owy;
    for (int q = threadIdx.x; q < no; q += NT) {
        const int gx = s.ox0 + q % s.owx, gy = s.oy0 + q / s.owx;
        const int lq = (gy - s.y0) * s.wx + (gx - s.x0);
        const long long g = (long long)gy * P.n + gx;
        Fy[g] = c[2 * lq];
        Fy[nn + g] = c[2 * lq + 1];
    }
}

// Jacobian action of the RASPEN function (Alg. 4):
//   O = -D - sum_i tilde P_i J_i(x^(i))^-1 B_i D,  B_i D = R_i A (I - P_i R_i) D,
// i.e. b = -beta * (sum of D over the 5-point neighbours outside Omega_i).
// With nir > 0 (mixed precision) the local solve is refined nir times in FP64:
// z += J^-1 (b - J z), J from the coefficients at x^(i).
template <typename T>
__global__ void __launch_bounds__(NT) k_local_jvp(int nsub, const SubDev* __restrict__ subs,
                                                  const ProbDev* __restrict__ probs, const T* gpool,
                                                  T* wpool, const double* coef, double* zpool,
                                                  double* rpool, double* bpool, int nir, const double* D,
                                                  double* O) {
    __shared__ T vec[MAX_M], tmp[MAX_M];
    __shared__ double red[2 * NT];
    const int i = blockIdx.x;
    if (i >= nsub) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const int n = P.n, m = 2 * s.wx, W = s.wy;
    const long long nn = (long long)n * n;
    const double beta = P.beta;
    const double* Dy = D + P.ofs;
    double* Oy = O + P.ofs;
    const T* G = gpool + s.goff;
    T* w = wpool + s.voff;
    auto bval = [=](int j, int t) -> double {
        const int lx = t >> 1, f = t & 1;
        const int gx = s.x0 + lx, gy = s.y0 + j;
        const double* Df = Dy + f * nn;
        double b = 0.0;
        if (lx == 0 && gx > 0) b += Df[(long long)gy * n + gx - 1];
        if (lx == s.wx - 1 && gx < n - 1) b += Df[(long long)gy * n + gx + 1];
        if (j == 0 && gy > 0) b += Df[(long long)(gy - 1) * n + gx];
        if (j == W - 1 && gy < n - 1) b += Df[(long long)(gy + 1) * n + gx];
        return -beta * b;
    };
    auto owned_out = [=](int j, int t, double z) {
        const int lx = t >> 1, f = t & 1;
        const int gx = s.x0 + lx, gy = s.y0 + j;
        if (gx >= s.ox0 && gx < s.ox0 + s.owx && gy >= s.oy0 && gy < s.oy0 + s.owy) {
            const long long g = f * nn + (long long)gy * n + gx;
            Oy[g] = -Dy[g] - z;
        }
    };
    if (nir == 0) {
        block_solve<T>(G, m, W, (T)beta, w, vec, tmp, [=](int j, int t) { return (T)bval(j, t); },
                       [=](int j, int t, T z) { owned_out(j, t, (double)z); });
        return;
    }
    const int L = m * W;
    double* b = bpool + s.voff;
    double* z = zpool + s.voff;
    double* r = rpool + s.voff;
    for (int q = threadIdx.x; q < L; q += NT) {
        b[q] = bval(q / m, q % m);
        z[q] = 0.0;
    }
    __syncthreads();
    block_solve<T>(G, m, W, (T)beta, w, vec, tmp, [=](int j, int t) { return (T)b[j * m + t]; },
                   [=](int j, int t, T zz) { z[j * m + t] += (double)zz; });
    for (int it = 0; it < nir; ++it) {
        local_linear_residual(s, beta, coef, 1.0, b, z, r, red);
        block_solve<T>(G, m, W, (T)beta, w, vec, tmp, [=](int j, int t) { return (T)r[j * m + t]; },
                       [=](int j, int t, T zz) { z[j * m + t] += (double)zz; });
    }
    for (int q = threadIdx.x; q < L; q += NT) owned_out(q / m, q % m, z[q]);
}

// Linear RAS preconditioner: Z = sum_i tilde P_i J_i^-1 R_i R.
template <typename T>
__global__ void __launch_bounds__(NT) k_local_precond(int nsub, const SubDev* __restrict__ subs,
                                                      const ProbDev* __restrict__ probs,
                                                      const T* gpool, T* wpool, const double* R,
                                                      double* Z) {
    __shared__ T vec[MAX_M], tmp[MAX_M];
    const int i = blockIdx.x;
    if (i >= nsub) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const int n = P.n, m = 2 * s.wx, W = s.wy;
    const long long nn = (long long)n * n;
    const double* Ry = R + P.ofs;
    double* Zy = Z + P.ofs;
    auto rhs = [=](int j, int t) -> T {
        const int lx = t >> 1, f = t & 1;
        return (T)Ry[f * nn + (long long)(s.y0 + j) * n + s.x0 + lx];
    };
    auto out = [=](int j, int t, T z) {
        const int lx = t >> 1, f = t & 1;
        const int gx = s.x0 + lx, gy = s.y0 + j;
        if (gx >= s.ox0 && gx < s.ox0 + s.owx && gy >= s.oy0 && gy < s.oy0 + s.owy)
            Zy[f * nn + (long long)gy * n + gx] = (double)z;
    };
    block_solve<T>(gpool + s.goff, m, W, (T)P.beta, wpool + s.voff, vec, tmp, rhs, out);
}

template <typename T>
size_t factor_smem(int maxm) {
    return (size_t)maxm * (maxm + 1) * sizeof(T) + (size_t)maxm * sizeof(T) + 3 * (size_t)maxm * sizeof(int);
}

}  // namespace

// ------------------------------------------------------------------ launchers
cudaError_t launch_local_init(cudaStream_t st, int nsub, const SubDev* subs, const ProbDev* probs,
                              const double* X, LocalState* ls, double eps_start, NewtonParams np,
                              double* cpool, double* Kpool, int* active_count) {
    count_launch();
    k_local_init<<<nsub, NT, 0, st>>>(nsub, subs, probs, X, ls, eps_start, np, cpool, Kpool, active_count);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_factor(cudaStream_t st, int nsub, int maxm, const SubDev* subs,
                                const ProbDev* probs, const double* X, LocalState* ls,
                                const double* cpool, double* coef, T* gpool, int only_active) {
    const size_t sm = factor_smem<T>(maxm);
    cudaError_t e = cudaFuncSetAttribute(k_local_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_factor<T><<<nsub, FACT_THREADS, sm, st>>>(nsub, maxm, subs, probs, X, ls, cpool, coef, gpool,
                                                      only_active);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_direction(cudaStream_t st, int nsub, int maxm, const SubDev* subs,
                                   const ProbDev* probs, LocalState* ls, NewtonParams np,
                                   const double* coef, const T* gpool, const double* Kpool,
                                   double* dpool, double* rpool, T* wpool) {
    (void)maxm;
    count_launch();
    k_local_direction<T><<<nsub, NT, 0, st>>>(nsub, subs, probs, ls, np, coef, gpool, Kpool, dpool, rpool,
                                              wpool);
    return cudaGetLastError();
}

cudaError_t launch_local_linesearch(cudaStream_t st, int nsub, const SubDev* subs, const ProbDev* probs,
                                    const double* X, LocalState* ls, NewtonParams np, double* cpool,
                                    const double* dpool, double* Kpool, double* Ktpool,
                                    int* active_count) {
    count_launch();
    k_local_linesearch<<<nsub, NT, 0, st>>>(nsub, subs, probs, X, ls, np, cpool, dpool, Kpool, Ktpool,
                                            active_count);
    return cudaGetLastError();
}

cudaError_t launch_local_prolong(cudaStream_t st, int nsub, const SubDev* subs, const ProbDev* probs,
                                 const double* cpool, double* F) {
    count_launch();
    k_local_prolong<<<nsub, NT, 0, st>>>(nsub, subs, probs, cpool, F);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_jvp(cudaStream_t st, int nsub, int maxm, const SubDev* subs,
                             const ProbDev* probs, const T* gpool, T* wpool, const double* coef,
                             double* zpool, double* rpool, double* bpool, int nir, const double* D,
                             double* O) {
    (void)maxm;
    count_launch();
    k_local_jvp<T><<<nsub, NT, 0, st>>>(nsub, subs, probs, gpool, wpool, coef, zpool, rpool, bpool, nir, D, O);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_precond(cudaStream_t st, int nsub, int maxm, const SubDev* subs,
                                 const ProbDev* probs, const T* gpool, T* wpool, const double* R,
                                 double* Z) {
    (void)maxm;
    count_launch();
    k_local_precond<T><<<nsub, NT, 0, st>>>(nsub, subs, probs, gpool, wpool, R, Z);
    return cudaGetLastError();
}

#define RAS_INSTANTIATE(T)                                                                            \
    template cudaError_t launch_local_factor<T>(cudaStream_t, int, int, const SubDev*, const ProbDev*,  \
                                                const double*, LocalState*, const double*, double*, T*, \
                                                int);                                                   \
    template cudaError_t launch_local_direction<T>(cudaStream_t, int, int, const SubDev*,               \
                                                   const ProbDev*, LocalState*, NewtonParams,           \
                                                   const double*, const T*, const double*, double*,     \
                                                   double*, T*);                                        \
    template cudaError_t launch_local_jvp<T>(cudaStream_t, int, int, const SubDev*, const ProbDev*,     \
                                             const T*, T*, const double*, double*, double*, double*,    \
                                             int, const double*, double*);                              \
    template cudaError_t launch_local_precond<T>(cudaStream_t, int, int, const SubDev*,                 \
                                                 const ProbDev*, const T*, T*, const double*, double*);
RAS_INSTANTIATE(float)
RAS_INSTANTIATE(double)
#undef RAS_INSTANTIATE

}  // namespace ras
