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
// and the factor stores G_j = S_j^-1 (in the packed order of packed_index),
// computed by Gauss-Jordan elimination with partial pivoting inside each
// block. The solves with these factors are in solve.cu.
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
        const long long blk = (long long)s.mp * s.mp;
        const T* Gp = G + (long long)(j > 0 ? j - 1 : 0) * blk;
        for (int r = warp; r < m; r += FW) {
            const int ix = r >> 1, f = r & 1;
            const int q = j * s.wx + ix;
            for (int cidx = lane; cidx < m; cidx += 32) {
                const int cx = cidx >> 1, cf = cidx & 1;
                T v = (j > 0) ? -tbeta2 * Gp[packed_index<T>(r, cidx, s.mp)] : (T)0;
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
        T* Gj = G + (long long)j * blk;
        for (int r = warp; r < s.mp; r += FW) {
            const int pr = r < m ? perm[r] : 0;
            for (int cidx = lane; cidx < s.mp; cidx += 32)
                Gj[packed_index<T>(r, cidx, s.mp)] = (r < m && cidx < m) ? M[pr * LD + rinv[cidx]] : (T)0;
        }
        __syncthreads();
    }
    if (sh_fail && tid == 0) {
        ls[i].status = ST_ESINGULAR;
        ls[i].active = 0;
    }
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

// FP32 factorisation with the block held in registers. Thread (ty, tx) of a
// 16 x 16 CTA owns rows ty + 16a and columns tx + 16b (a, b < R) of the
// 16R x 16R block, so every elimination step updates registers only; the
// pivot column and the scaled pivot row are broadcast through shared memory
// (double-buffered, three barriers per step). Partial pivoting as in the
// generic kernel (max |.| among the not yet eliminated rows, ties to the
// lowest row); an off-diagonal pivot row is swapped in physically and the
// column order of the inverse is restored when G_j is written.
template <int R>
__global__ void __launch_bounds__(FACT_THREADS, 2) k_local_factor_reg(int nsub, const SubDev* __restrict__ subs,
                                                                      const ProbDev* __restrict__ probs,
                                                                      const double* X, LocalState* ls,
                                                                      const double* cpool, double* coef,
                                                                      float* gpool, int only_active) {
    constexpr int MM = 16 * R;
    static_assert(FACT_THREADS == 256, "16 x 16 thread tile");
    __shared__ float colk[2][MM];
    __shared__ float rowb[2][MM];
    __shared__ float swp[MM];
    __shared__ int pivr[MM];
    __shared__ int sinv[MM];
    __shared__ int sh_r[2], sh_fail, sh_nswap;
    __shared__ float sh_piv[2];
    const int i = blockIdx.x;
    if (i >= nsub) return;
    if (only_active && !ls[i].active) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const int m = 2 * s.wx, W = s.wy, nn = s.wx * s.wy, mp = s.mp;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15, warp = tid >> 5, lane = tid & 31;

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

    const float tbeta = (float)beta, tbeta2 = (float)(beta * beta), tdiag = (float)(4.0 * beta);
    const long long blk = (long long)mp * mp;
    float* G = gpool + s.goff;
    float Mr[R][R];
    for (int j = 0; j < W; ++j) {
        // S_j = D_j - beta^2 G_{j-1}
        const float* Gp = G + (long long)(j > 0 ? j - 1 : 0) * blk;
#pragma unroll
        for (int a = 0; a < R; ++a) {
            const int r = ty + 16 * a;
#pragma unroll
            for (int b = 0; b < R; ++b) {
                const int c = tx + 16 * b;
                float v = 0.f;
                if (r < m && c < m) {
                    if (j > 0) v = -tbeta2 * Gp[packed_index<float>(r, c, mp)];
                    const int ix = r >> 1, f = r & 1, cx = c >> 1, cf = c & 1;
                    const int q = j * s.wx + ix;
                    if (cx == ix) {
                        if (cf == f) v += tdiag + (float)ca[q];
                        else if (f == 0) v += (float)cb[q];
                        else v += (float)cc[q];
                    } else if (cf == f && (cx == ix - 1 || cx == ix + 1)) {
                        v -= tbeta;
                    }
                }
                Mr[a][b] = v;
            }
        }
        if (tid == 0) sh_nswap = 0;
        __syncthreads();

        int par = 0;
        bool done = false;
#pragma unroll
        for (int kb = 0; kb < R; ++kb) {
            for (int kt = 0; kt < 16 && !done; ++kt) {
                const int k = 16 * kb + kt;
                if (k >= m) {
                    done = true;
                    break;
                }
                if (tx == kt) {
#pragma unroll
                    for (int a = 0; a < R; ++a) colk[par][ty + 16 * a] = Mr[a][kb];
                }
                __syncthreads();
                if (warp == 0) {
                    float best = -1.f;
                    int bi = 0x7fffffff;
                    for (int r = k + lane; r < m; r += 32) {
                        const float v = fabsf(colk[par][r]);
                        if (v > best) { best = v; bi = r; }
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        const float ob = __shfl_xor_sync(0xffffffffu, best, off);
                        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                    }
                    if (lane == 0) {
                        if (bi >= m || !(best > 0.f)) {
                            sh_fail = 1;
                        } else {
                            sh_r[par] = bi;
                            sh_piv[par] = colk[par][bi];
                            pivr[k] = bi;
                        }
                    }
                }
                __syncthreads();
                if (sh_fail) {
                    done = true;
                    break;
                }
                const int r = sh_r[par];
                if (r != k) {
                    const int tr = r & 15, ar = r >> 4;
                    if (ty == kt) {
#pragma unroll
                        for (int b = 0; b < R; ++b) rowb[par][tx + 16 * b] = Mr[kb][b];
                    }
                    if (ty == tr) {
#pragma unroll
                        for (int a = 0; a < R; ++a)
                            if (a == ar) {
#pragma unroll
                                for (int b = 0; b < R; ++b) swp[tx + 16 * b] = Mr[a][b];
                            }
                    }
                    __syncthreads();
                    if (ty == kt) {
#pragma unroll
                        for (int b = 0; b < R; ++b) Mr[kb][b] = swp[tx + 16 * b];
                    }
                    if (ty == tr) {
#pragma unroll
                        for (int a = 0; a < R; ++a)
                            if (a == ar) {
#pragma unroll
                                for (int b = 0; b < R; ++b) Mr[a][b] = rowb[par][tx + 16 * b];
                            }
                    }
                    if (tid == 0) {
                        const float t = colk[par][k];
                        colk[par][k] = colk[par][r];
                        colk[par][r] = t;
                        sh_nswap += 1;
                    }
                    __syncthreads();
                }
                const float inv = 1.f / sh_piv[par];
                if (ty == kt) {
#pragma unroll
                    for (int b = 0; b < R; ++b) {
                        const int c = tx + 16 * b;
                        rowb[par][c] = (c == k) ? inv : Mr[kb][b] * inv;
                    }
                }
                if (tid == 0) colk[par][k] = 0.f;
                __syncthreads();
                if (tx == kt) {
#pragma unroll
                    for (int a = 0; a < R; ++a) Mr[a][kb] = 0.f;
                }
                float ck[R];
#pragma unroll
                for (int a = 0; a < R; ++a) ck[a] = colk[par][ty + 16 * a];
#pragma unroll
                for (int b = 0; b < R; ++b) {
                    const float rb = rowb[par][tx + 16 * b];
#pragma unroll
                    for (int a = 0; a < R; ++a) Mr[a][b] = fmaf(-ck[a], rb, Mr[a][b]);
                }
                if (ty == kt) {
#pragma unroll
                    for (int b = 0; b < R; ++b) Mr[kb][b] = rowb[par][tx + 16 * b];
                }
                par ^= 1;
            }
        }
        if (sh_fail) break;
        // column order of the inverse: undo the row interchanges in reverse
        if (tid == 0) {
            for (int c = 0; c < m; ++c) sinv[c] = c;
            if (sh_nswap > 0) {
                for (int c = 0; c < m; ++c) swp[c] = __int_as_float(c);   // sig, as bits
                for (int k = m - 1; k >= 0; --k) {
                    const int r = pivr[k];
                    if (r != k) {
                        const float t = swp[k];
                        swp[k] = swp[r];
                        swp[r] = t;
                    }
                }
                for (int c = 0; c < m; ++c) sinv[__float_as_int(swp[c])] = c;
            }
        }
        __syncthreads();
        float* Gj = G + (long long)j * blk;
#pragma unroll
        for (int a = 0; a < R; ++a) {
            const int r = ty + 16 * a;
#pragma unroll
            for (int b = 0; b < R; ++b) {
                const int c = tx + 16 * b;
                if (r < mp && c < mp) {
                    if (r < m && c < m) Gj[packed_index<float>(r, sinv[c], mp)] = Mr[a][b];
                    else Gj[packed_index<float>(r, c, mp)] = 0.f;
                }
            }
        }
        __syncthreads();
    }
    if (sh_fail && tid == 0) {
        ls[i].status = ST_ESINGULAR;
        ls[i].active = 0;
    }
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

template <int R>
cudaError_t launch_factor_reg(cudaStream_t st, int nsub, const SubDev* subs, const ProbDev* probs,
                              const double* X, LocalState* ls, const double* cpool, double* coef,
                              float* gpool, int only_active) {
    count_launch();
    k_local_factor_reg<R><<<nsub, FACT_THREADS, 0, st>>>(nsub, subs, probs, X, ls, cpool, coef, gpool,
                                                         only_active);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_factor(cudaStream_t st, int nsub, int maxm, const SubDev* subs,
                                const ProbDev* probs, const double* X, LocalState* ls,
                                const double* cpool, double* coef, T* gpool, int only_active) {
    if (sizeof(T) == sizeof(float)) {
        // register tile covering the largest packed block (mp <= 16 R)
        const int mpmax = ((maxm + 31) / 32) * 32;
        float* g = reinterpret_cast<float*>(gpool);
        switch (mpmax / 16) {
            case 2: return launch_factor_reg<2>(st, nsub, subs, probs, X, ls, cpool, coef, g, only_active);
            case 4: return launch_factor_reg<4>(st, nsub, subs, probs, X, ls, cpool, coef, g, only_active);
            case 6: return launch_factor_reg<6>(st, nsub, subs, probs, X, ls, cpool, coef, g, only_active);
            case 8: return launch_factor_reg<8>(st, nsub, subs, probs, X, ls, cpool, coef, g, only_active);
            case 10: return launch_factor_reg<10>(st, nsub, subs, probs, X, ls, cpool, coef, g, only_active);
            default: return cudaErrorInvalidValue;
        }
    }
    const size_t sm = factor_smem<T>(maxm);
    cudaError_t e = cudaFuncSetAttribute(k_local_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_factor<T><<<nsub, FACT_THREADS, sm, st>>>(nsub, maxm, subs, probs, X, ls, cpool, coef, gpool,
                                                      only_active);
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

#define RAS_INSTANTIATE(T)                                                                            \
    template cudaError_t launch_local_factor<T>(cudaStream_t, int, int, const SubDev*, const ProbDev*,  \
                                                const double*, LocalState*, const double*, double*, T*, \
                                                int);
RAS_INSTANTIATE(float)
RAS_INSTANTIATE(double)
#undef RAS_INSTANTIATE

}  // namespace ras
