// Per-subdomain kernels of the nonlinear RAS sweep (Alg. 3), its Jacobian
// action (Alg. 4) and the linear RAS preconditioner (Newton_RAS).
//
// One CTA owns one subdomain i for the whole launch. The local problem is
//   K_i(c) = R_i F_eps(x + P_i c) = 0                          (Sec. 4.2)
// solved by Alg. 1 from c = 0. Its Jacobian J_i = R_i F'(x + P_i c) P_i in the
// interleaved (y, p) ordering, grouped by grid rows of Omega_i (planes on the
// cube), is block tridiagonal: diagonal blocks D_j (one grid row or plane,
// m = 2 bl unknowns) and off-diagonal blocks -beta I (the stencil's coupling
// between neighbouring rows or planes, beta = 1/h^2, the same for both
// fields). Its block LU therefore only needs
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

// Value of the local state at local node (lx, ly), field f (square), or
// (lx, ly, lz) (cube): x + c + alpha d on Omega_i, x on the ring outside it,
// 0 outside the grid.
struct LocalView {
    const double* X;   // y-plane of this problem; p-plane at X + nn
    long long nn;
    int n, nz, x0, y0, z0, wx, wy, wz;
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

    __device__ __forceinline__ double val3(int lx, int ly, int lz, int f) const {
        const int gi = x0 + lx, gj = y0 + ly, gk = z0 + lz;
        if (gi < 0 || gi >= n || gj < 0 || gj >= n || gk < 0 || gk >= nz) return 0.0;
        double v = X[f * nn + ((long long)gk * n + gj) * n + gi];
        if (lx >= 0 && lx < wx && ly >= 0 && ly < wy && lz >= 0 && lz < wz) {
            const int lq = 2 * ((lz * wy + ly) * wx + lx) + f;
            double cc = c[lq];
            if (d) cc = fma(alpha, d[lq], cc);
            v += cc;
        }
        return v;
    }

    // the state at local node q of Omega_i itself (either geometry)
    __device__ __forceinline__ double at(int q, int f) const {
        const int lx = q % wx, r = q / wx, ly = r % wy, lz = r / wy;
        double cc = c[2 * q + f];
        if (d) cc = fma(alpha, d[2 * q + f], cc);
        return X[f * nn + ((long long)(z0 + lz) * n + (y0 + ly)) * n + (x0 + lx)] + cc;
    }
};

__device__ __forceinline__ LocalView make_view(const SubDev& s, const ProbDev& P, const double* X,
                                               const double* c, const double* d, double alpha) {
    LocalView V;
    V.X = X + P.ofs;
    V.nn = P.nn;
    V.n = P.n;
    V.nz = P.nz;
    V.x0 = s.x0; V.y0 = s.y0; V.z0 = s.z0; V.wx = s.wx; V.wy = s.wy; V.wz = s.wz;
    V.c = c; V.d = d; V.alpha = alpha;
    return V;
}

// K_i at the view's state and eps (residual F of Sec. 3.3 at the nodes of
// Omega_i). Writes the interleaved residual to `out` when non-null and
// returns (block-wide) its squared 2-norm and, with `with_floor`, the squared
// norm of the nodewise |term| sums (rounding-floor estimate; the stop test
// reads it only at eps_min, so callers ask for it only there; else 0).
__device__ void local_residual(const LocalView& V, const ProbDev& P, double eps, double* out,
                               double& nrm2, double& flr2, double* red, bool with_floor) {
    const int wx = V.wx, nn = wx * V.wy * V.wz;
    const double beta = P.beta, inu = 1.0 / P.nu, mu = P.mu, imu = 1.0 / P.mu, munu = P.mu / P.nu;
    double a = 0.0, b = 0.0;
    if (V.nz > 1) {
        // the cube: 7-point stencil, beta (6 z - sum of the six neighbours)
        for (int q = threadIdx.x; q < nn; q += NT) {
            const int lx = q % wx, r = q / wx, ly = r % V.wy, lz = r / V.wy;
            const long long g = ((long long)(V.z0 + lz) * V.n + (V.y0 + ly)) * V.n + (V.x0 + lx);
            const double yc = V.val3(lx, ly, lz, 0), pc = V.val3(lx, ly, lz, 1);
            const double yw = V.val3(lx - 1, ly, lz, 0), ye = V.val3(lx + 1, ly, lz, 0);
            const double ys = V.val3(lx, ly - 1, lz, 0), yn = V.val3(lx, ly + 1, lz, 0);
            const double yb = V.val3(lx, ly, lz - 1, 0), yt = V.val3(lx, ly, lz + 1, 0);
            const double pw = V.val3(lx - 1, ly, lz, 1), pe = V.val3(lx + 1, ly, lz, 1);
            const double ps = V.val3(lx, ly - 1, lz, 1), pn = V.val3(lx, ly + 1, lz, 1);
            const double pb = V.val3(lx, ly, lz - 1, 1), pt = V.val3(lx, ly, lz + 1, 1);
            double ph, d1, d2;
            phi_eval(P.phi, P.kappa, yc, ph, d1, d2);
            const double fv = P.f ? P.f[g] : 0.0;
            const double xq = -pc * imu;
            const double dq = P_eps_minus_id(xq, eps);
            const double Fy = beta * (6.0 * yc - yw - ye - ys - yn - yb - yt) + ph - fv + munu * dq;
            const double Fp = beta * (6.0 * pc - pw - pe - ps - pn - pb - pt) + d1 * pc - yc + P.yd[g];
            if (with_floor) {
                const double My = beta * (6.0 * fabs(yc) + fabs(yw) + fabs(ye) + fabs(ys) + fabs(yn) + fabs(yb) +
                                          fabs(yt)) +
                                  fabs(ph) + fabs(fv) + inu * (fabs(pc) + mu * fabs(xq + dq));
                const double Mp = beta * (6.0 * fabs(pc) + fabs(pw) + fabs(pe) + fabs(ps) + fabs(pn) + fabs(pb) +
                                          fabs(pt)) +
                                  fabs(d1 * pc) + fabs(yc) + fabs(P.yd[g]);
                b += My * My + Mp * Mp;
            }
            if (out) {
                out[2 * q] = Fy;
                out[2 * q + 1] = Fp;
            }
            a += Fy * Fy + Fp * Fp;
        }
        block_sum2<NT>(a, b, red);
        nrm2 = a;
        flr2 = b;
        return;
    }
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
        // -u = (mu/nu)(P_eps(x) - x), x = -p/mu (control of Sec. 3.2)
        const double xq = -pc * imu;
        const double dq = P_eps_minus_id(xq, eps);
        const double Fy = beta * (4.0 * yc - yw - ye - ys - yn) + ph - fv + munu * dq;
        const double Fp = beta * (4.0 * pc - pw - pe - ps - pn) + d1 * pc - yc + P.yd[g];
        if (with_floor) {
            const double My = beta * (4.0 * fabs(yc) + fabs(yw) + fabs(ye) + fabs(ys) + fabs(yn)) + fabs(ph) +
                              fabs(fv) + inu * (fabs(pc) + mu * fabs(xq + dq));
            const double Mp = beta * (4.0 * fabs(pc) + fabs(pw) + fabs(pe) + fabs(ps) + fabs(pn)) +
                              fabs(d1 * pc) + fabs(yc) + fabs(P.yd[g]);
            b += My * My + Mp * Mp;
        }
        if (out) {
            out[2 * q] = Fy;
            out[2 * q + 1] = Fp;
        }
        a += Fy * Fy + Fp * Fp;
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

// pstart[p]: eps at which the local solves of problem p start (eps_0 with
// continuation, eps_min without); <= 0 means problem p does not take part.
__global__ void __launch_bounds__(NT) k_local_init(int nsub, const SubDev* __restrict__ subs,
                                                   const ProbDev* __restrict__ probs, const double* X,
                                                   LocalState* ls, const double* __restrict__ pstart,
                                                   NewtonParams np, double* cpool, double* Kpool,
                                                   int* active_count) {
    __shared__ double red[2 * NT];
    const int i = blockIdx.x;
    if (i >= nsub) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const double eps_start = pstart[s.prob];
    if (!(eps_start > 0.0)) {
        if (threadIdx.x == 0) {
            LocalState st{};
            st.status = ST_SKIP;
            st.active = 0;
            ls[i] = st;
        }
        return;
    }
    const int L = 2 * s.wx * s.wy * s.wz;
    double* c = cpool + s.voff;
    for (int q = threadIdx.x; q < L; q += NT) c[q] = 0.0;
    __syncthreads();
    const LocalView V = make_view(s, P, X, c, nullptr, 0.0);
    double n2, f2;
    local_residual(V, P, eps_start, Kpool + s.voff, n2, f2, red, eps_start == np.eps_min);
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
    if (ls[i].status == ST_SKIP) return;
    const SubDev s = subs[i];
    if (s.mp > MAX_M) return;   // wide block: k_local_factor_big
    const ProbDev P = probs[s.prob];
    const int m = 2 * s.bl, W = s.bw, nn = s.wx * s.wy * s.wz, LD = maxm + 1;
    const bool cube = P.nz > 1;
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
    double* ca = s.cptr;
    double* cb = ca + nn;
    double* cc = cb + nn;
    {
        const double* c = cpool + s.voff;
        const LocalView V = make_view(s, P, X, c, nullptr, 0.0);
        for (int q = tid; q < nn; q += FACT_THREADS) {
            const double y = V.at(q, 0), p = V.at(q, 1);
            double ph, d1, d2;
            phi_eval(P.phi, P.kappa, y, ph, d1, d2);
            ca[q] = d1;
            cb[q] = inu * one_minus_dP_eps(-p / mu, eps);
            cc[q] = d2 * p - 1.0;
        }
    }
    if (tid == 0) sh_fail = 0;
    __syncthreads();

    const T tbeta = (T)beta, tbeta2 = (T)(beta * beta), tdiag = (T)P.diag;
    T* G = static_cast<T*>(s.gptr);
    for (int j = 0; j < W; ++j) {
        // S_j = D_j - beta^2 G_{j-1}
        const long long blk = (long long)s.mp * s.mp;
        const T* Gp = G + (long long)(j > 0 ? j - 1 : 0) * blk;
        for (int r = warp; r < m; r += FW) {
            const int ix = r >> 1, f = r & 1;
            const int q = j * s.bl + ix;
            for (int cidx = lane; cidx < m; cidx += 32) {
                const int cx = cidx >> 1, cf = cidx & 1;
                T v = (j > 0) ? -tbeta2 * Gp[packed_index<T>(r, cidx, s.mp)] : (T)0;
                if (cx == ix) {
                    if (cf == f) v += tdiag + (T)ca[q];
                    else if (f == 0) v += (T)cb[q];
                    else v += (T)cc[q];
                } else if (cf == f && row_neighbour(ix, cx, s.wx, cube)) {
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
    const int len = 2 * s.wx * s.wy * s.wz;
    double* c = cpool + s.voff;
    const double* d = dpool + s.voff;
    double* K = Kpool + s.voff;
    double* Kt = Ktpool + s.voff;
    double alpha = 1.0, nt = 0.0, ft = 0.0;
    int h = 0;
    for (;;) {
        const LocalView V = make_view(s, P, X, c, d, alpha);
        double n2, f2;
        local_residual(V, P, L.eps, Kt, n2, f2, red, L.eps == np.eps_min);
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
        local_residual(V, P, en, K, n2, f2, red, en == np.eps_min);
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
                                                      const ProbDev* __restrict__ probs, const LocalState* ls,
                                                      const double* cpool, double* F) {
    const int i = blockIdx.x;
    if (i >= nsub) return;
    if (ls[i].status == ST_SKIP) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const long long nn = P.nn;
    double* Fy = F + P.ofs;
    const double* c = cpool + s.voff;
    const int no = s.owx * s.owy * s.owz;
    for (int q = threadIdx.x; q < no; q += NT) {
        const int r = q / s.owx;
        const int gx = s.ox0 + q % s.owx, gy = s.oy0 + r % s.owy, gz = s.oz0 + r / s.owy;
        const int lq = ((gz - s.z0) * s.wy + (gy - s.y0)) * s.wx + (gx - s.x0);
        const long long g = grid_index(P, gx, gy, gz);
        Fy[g] = c[2 * lq];
        Fy[nn + g] = c[2 * lq + 1];
    }
}

// R consecutive floats of shared memory (16-byte aligned) <-> registers, in
// 16-, 8- and 4-byte pieces.
template <int R>
__device__ __forceinline__ void load_vec(const float* src, float* v) {
#pragma unroll
    for (int q = 0; q + 4 <= R; q += 4) {
        const float4 t = *reinterpret_cast<const float4*>(src + q);
        v[q] = t.x; v[q + 1] = t.y; v[q + 2] = t.z; v[q + 3] = t.w;
    }
    if (R % 4 >= 2) {
        const float2 t = *reinterpret_cast<const float2*>(src + (R / 4) * 4);
        v[(R / 4) * 4] = t.x;
        v[(R / 4) * 4 + 1] = t.y;
    }
    if (R % 2) v[R - 1] = src[R - 1];
}

template <int R>
__device__ __forceinline__ void store_vec(float* dst, const float* v) {
#pragma unroll
    for (int q = 0; q + 4 <= R; q += 4)
        *reinterpret_cast<float4*>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
    if (R % 4 >= 2) *reinterpret_cast<float2*>(dst + (R / 4) * 4) = make_float2(v[(R / 4) * 4], v[(R / 4) * 4 + 1]);
    if (R % 2) dst[R - 1] = v[R - 1];
}

// Entries of D_j (grid row j of the local Jacobian) inside the tile of
// thread (ty, ty + DT): the 2 x 2 node blocks on the diagonal (4 beta + phi',
// the control coupling (1/nu)(1 - P_eps'(-p/mu)) in the y-row and
// phi'' p - 1 in the p-row) and -beta two places off it (the x-neighbours of
// the same field). R is even, so a row's field is a & 1.
template <int R, int DT>
__device__ __forceinline__ void add_band(float (&Mr)[R][R], int ty, int m, int wx, int j, float tdiag,
                                         float tbeta, const double* ca, const double* cb, const double* cc) {
#pragma unroll
    for (int a = 0; a < R; ++a) {
#pragma unroll
        for (int b = 0; b < R; ++b) {
            const int off = DT * R + b - a;
            if (off < -2 || off > 2) continue;
            const int r = ty * R + a, c = r + off;
            if (r >= m || c < 0 || c >= m) continue;
            const int q = j * wx + (r >> 1);
            if (off == 0) Mr[a][b] += tdiag + (float)ca[q];
            else if (off == 1 && (a & 1) == 0) Mr[a][b] += (float)cb[q];
            else if (off == -1 && (a & 1) == 1) Mr[a][b] += (float)cc[q];
            else if (off == 2 || off == -2) Mr[a][b] -= tbeta;
        }
    }
}

// Entries of D_j on the cube (one plane of bl = wx*wy nodes) inside the tile
// of thread (ty, tx), rows ty*R + a and columns tx*R + b: the 2 x 2 node
// blocks on the diagonal as in add_band (6 beta + phi' on the diagonal) and
// -beta at the in-plane neighbours of the same field, node offsets +-1 within
// a grid line and +-wx, which reach tiles away from the diagonal.
template <int R>
__device__ __forceinline__ void add_plane(float (&Mr)[R][R], int ty, int tx, int m, int bl, int wx, int j,
                                          float tdiag, float tbeta, const double* ca, const double* cb,
                                          const double* cc) {
#pragma unroll
    for (int a = 0; a < R; ++a) {
        const int r = ty * R + a;
        if (r >= m) continue;
        const int ix = r >> 1, f = r & 1;
        const int q = j * bl + ix;
#pragma unroll
        for (int b = 0; b < R; ++b) {
            const int c = tx * R + b;
            if (c >= m) continue;
            const int cx = c >> 1, cf = c & 1;
            if (cx == ix) {
                if (cf == f) Mr[a][b] += tdiag + (float)ca[q];
                else if (f == 0) Mr[a][b] += (float)cb[q];
                else Mr[a][b] += (float)cc[q];
            } else if (cf == f && row_neighbour(ix, cx, wx, true)) {
                Mr[a][b] -= tbeta;
            }
        }
    }
}

// The single-pivot Gauss-Jordan sweeps k = kt*R .. kt*R+R-1 restricted to the
// column panel M[:, K], run by its 16 owners (thread column kt: one half of a
// warp, lanes in the mask hm) on their own tiles, so the panel never leaves
// registers. The pivot rows sit in thread (kt, kt) = lane src. Partial
// pivoting is checked, not applied: every lane notes a row not yet
// eliminated (rows of thread rows > kt, and rows after the pivot in thread
// row kt) whose entry in the pivot column is larger than the diagonal, or a
// diagonal that is 0 or not finite; the owners vote once at the end, and
// false means the caller redoes the block row with pivoting.
template <int R>
__device__ __forceinline__ bool panel_sweep(float (&Mr)[R][R], int ty, int kt, int m, unsigned hm, int src) {
    const int nk = min(R, m - kt * R);
    bool bad = false;
#pragma unroll
    for (int kl = 0; kl < R; ++kl) {
        if (kl >= nk) break;
        float t[R];
#pragma unroll
        for (int c = 0; c < R; ++c) t[c] = __shfl_sync(hm, Mr[kl][c], src);
        const float d = t[kl], ad = fabsf(d);
        bad |= !(ad > 0.f && ad < INFINITY);
        {
            // largest candidate of this lane: all its rows below thread row
            // kt, the rows after the pivot in thread row kt, none above
            float mpart = 0.f;
#pragma unroll
            for (int a = kl + 1; a < R; ++a) mpart = fmaxf(mpart, fabsf(Mr[a][kl]));
            float mall = mpart;
#pragma unroll
            for (int a = 0; a <= kl; ++a) mall = fmaxf(mall, fabsf(Mr[a][kl]));
            const float cand = (ty > kt) ? mall : ((ty == kt) ? mpart : 0.f);
            bad |= cand > ad;
        }
        const float inv = __frcp_rn(d);
#pragma unroll
        for (int c = 0; c < R; ++c) t[c] = (c == kl) ? inv : t[c] * inv;
#pragma unroll
        for (int a = 0; a < R; ++a) {
            const float f = Mr[a][kl];
            Mr[a][kl] = 0.f;
#pragma unroll
            for (int c = 0; c < R; ++c) Mr[a][c] = fmaf(-f, t[c], Mr[a][c]);
        }
        if (ty == kt) {
#pragma unroll
            for (int c = 0; c < R; ++c) Mr[kl][c] = t[c];
        }
    }
    return !__any_sync(hm, bad);
}

// FP32 factorisation, one CTA per subdomain. Thread (ty, tx) of the 16 x 16
// CTA (tid = 16 tx + ty: a thread column is one half of a warp) holds the
// R x R tile (rows ty*R + a, columns tx*R + b) of the block row matrix in
// registers for the whole launch: S_j = D_j - beta^2 G_{j-1} is formed in
// place from G_{j-1} (the same tile), inverted in place and written out
// (staged through shared memory in the packed order).
//
// The inverse is the Gauss-Jordan sweep over the pivots k = 0 .. m-1, taken
// R at a time: panel K = kt*R .. kt*R+R-1 holds the columns of thread column
// kt and the rows of thread row kt. With A = M[K,K], sweeping the pivots of K
// gives M[:,K] <- C' = [A^-1; -M[I,K] A^-1] (the column panel after its R
// single-pivot sweeps) and, for every other column J,
//   M[K,J] <- C'[K,K] M[K,J],   M[I,J] <- M[I,J] + C'[I,K] M[K,J].
// Per panel: the 16 owners of column kt sweep it in their registers
// (panel_sweep) and publish C'; the owners of row kt publish M[K,:] with
// zeros in place of M[K,K] and clear their tiles; after one barrier every
// thread adds the rank-R product of the two, which leaves the column panel
// at C' and turns rows K into C'[K,K] M[K,J]. The panel buffers alternate
// between two copies, so one barrier per panel suffices.
//
// Partial pivoting (max |.| in the column among the rows not yet eliminated,
// ties to the lowest row) is optimistic: a block row whose diagonal pivots
// all pass the check is exactly what partial pivoting computes; one that
// fails is redone from S_j (G_{j-1} read back from the factor pool) by a
// shared-memory Gauss-Jordan elimination with partial pivoting.
template <int R>
__global__ void __launch_bounds__(FACT_THREADS, 2) k_local_factor_panel(int nsub, const SubDev* __restrict__ subs,
                                                                        const ProbDev* __restrict__ probs,
                                                                        const double* X, LocalState* ls,
                                                                        const double* cpool, double* coef,
                                                                        float* gpool, int only_active,
                                                                        const int* __restrict__ list, FactorSel sel) {
    constexpr int MM = 16 * R;
    constexpr int PAD = ((R + 3) / 4) * 4;   // owner stride in the panel buffers
    constexpr int LDC = 16 * PAD;            // one panel column (or row) of 16 owners
    constexpr int LDS = MM + 4;              // staging stride of the full block
    static_assert(FACT_THREADS == 256, "16 x 16 thread tile");
    static_assert(R % 2 == 0, "one field per row parity");
    // panel buffers inside the staging area (dead while the panels run):
    // two copies each of the swept column panel (transposed) and the row panel
    constexpr int OFF_CT = 0;
    constexpr int OFF_RW = OFF_CT + 2 * R * LDC;
    static_assert(OFF_RW + 2 * R * LDC <= MM * LDS, "panel buffers fit in the staging area");
    __shared__ float fcol[MM];
    __shared__ int pivr[MM];
    __shared__ int sinv[MM];
    __shared__ int used[MM];
    __shared__ int sh_viol, sh_r, sh_fail;
    __shared__ float sh_piv;
    extern __shared__ __align__(16) float Ms[];
    if ((int)blockIdx.x >= nsub) return;
    if (sel.nwork && min(*sel.nwork, nsub) <= sel.thr) return;   // the 1024-thread kernel's turn
    const int i = list ? list[blockIdx.x] : (int)blockIdx.x;
    if (only_active && !ls[i].active) return;
    if (ls[i].status == ST_SKIP) return;
    const SubDev s = subs[i];
    if (s.mp > 16 * R) return;   // not this register-tile class (wide blocks: k_local_factor_big)
    const ProbDev P = probs[s.prob];
    const int m = 2 * s.bl, W = s.bw, nn = s.wx * s.wy * s.wz, mp = s.mp;
    const bool cube = P.nz > 1;
    const int tid = threadIdx.x, ty = tid & 15, tx = tid >> 4, warp = tid >> 5, lane = tid & 31;

    const double eps = ls[i].eps;
    const double beta = P.beta, inu = 1.0 / P.nu, mu = P.mu;
    double* ca = s.cptr;
    double* cb = ca + nn;
    double* cc = cb + nn;
    {
        const double* c = cpool + s.voff;
        const LocalView V = make_view(s, P, X, c, nullptr, 0.0);
        for (int q = tid; q < nn; q += FACT_THREADS) {
            const double y = V.at(q, 0), p = V.at(q, 1);
            double ph, d1, d2;
            phi_eval(P.phi, P.kappa, y, ph, d1, d2);
            ca[q] = d1;
            cb[q] = inu * one_minus_dP_eps(-p / mu, eps);
            cc[q] = d2 * p - 1.0;
        }
    }
    if (tid == 0) sh_fail = 0;
    __syncthreads();   // coefficients visible to the whole CTA

    const float tbeta = (float)beta, tbeta2 = (float)(beta * beta), tdiag = (float)P.diag;
    const long long blk = (long long)mp * mp;
    float* G = static_cast<float*>(s.gptr);
    float Mr[R][R];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) Mr[a][b] = 0.f;
    bool failed = false;
    auto dval = [=](int j, int r, int c) -> float {
        const int ix = r >> 1, f = r & 1, cx = c >> 1, cf = c & 1;
        const int q = j * s.bl + ix;
        if (cx == ix) {
            if (cf == f) return tdiag + (float)ca[q];
            return (f == 0) ? (float)cb[q] : (float)cc[q];
        }
        return (cf == f && row_neighbour(ix, cx, s.wx, cube)) ? -tbeta : 0.f;
    };
    for (int j = 0; j < W && !failed; ++j) {
        // S_j = D_j - beta^2 G_{j-1}: the tile holds G_{j-1} (zero for j = 0)
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < R; ++b) Mr[a][b] = -tbeta2 * Mr[a][b];
        if (cube) add_plane<R>(Mr, ty, tx, m, s.bl, s.wx, j, tdiag, tbeta, ca, cb, cc);
        else if (tx == ty) add_band<R, 0>(Mr, ty, m, s.bl, j, tdiag, tbeta, ca, cb, cc);
        else if (tx == ty + 1) add_band<R, 1>(Mr, ty, m, s.bl, j, tdiag, tbeta, ca, cb, cc);
        else if (tx == ty - 1) add_band<R, -1>(Mr, ty, m, s.bl, j, tdiag, tbeta, ca, cb, cc);
        if (tid == 0) sh_viol = 0;

        for (int kt = 0; kt < 16 && kt * R < m; ++kt) {
            float* CsT = Ms + OFF_CT + (kt & 1) * (R * LDC);
            float* Rw = Ms + OFF_RW + (kt & 1) * (R * LDC);
            if (ty == kt) {
                if (tx == kt) {
#pragma unroll
                    for (int c = 0; c < R; ++c) {
                        float z[R];
#pragma unroll
                        for (int b = 0; b < R; ++b) z[b] = 0.f;
                        store_vec<R>(Rw + c * LDC + tx * PAD, z);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < R; ++c) store_vec<R>(Rw + c * LDC + tx * PAD, Mr[c]);
                }
                // rows K restart from 0: the update below leaves C'[K,K] M[K,J]
                // there (forming it as M[K,J] + (C'[K,K] - I) M[K,J] would
                // cancel catastrophically, since C'[K,K] ~ 1/(4 beta))
                if (tx != kt) {
#pragma unroll
                    for (int a = 0; a < R; ++a)
#pragma unroll
                        for (int b = 0; b < R; ++b) Mr[a][b] = 0.f;
                }
            }
            if (tx == kt) {
                const int half = kt & 1;
                const unsigned hm = 0xffffu << (16 * half);
                const bool ok = panel_sweep<R>(Mr, ty, kt, m, hm, 16 * half + kt);
                if (!ok && ty == 0) sh_viol = 1;
#pragma unroll
                for (int c = 0; c < R; ++c) {
                    float col[R];
#pragma unroll
                    for (int a = 0; a < R; ++a) col[a] = Mr[a][c];
                    store_vec<R>(CsT + c * LDC + ty * PAD, col);
                }
            }
            __syncthreads();
            if (sh_viol) break;
            // rank-R update M += C' [M[K,:] with 0 at K]
#pragma unroll
            for (int c = 0; c < R; ++c) {
                float rv[R];
                load_vec<R>(Rw + c * LDC + tx * PAD, rv);
                const float* cp = CsT + c * LDC + ty * PAD;
                // the column operand four rows at a time (fewer live registers)
#pragma unroll
                for (int a0 = 0; a0 < R; a0 += 4) {
                    float cv[4];
                    if (a0 + 4 <= R) {
                        const float4 t4 = *reinterpret_cast<const float4*>(cp + a0);
                        cv[0] = t4.x; cv[1] = t4.y; cv[2] = t4.z; cv[3] = t4.w;
                    } else {
                        const float2 t2 = *reinterpret_cast<const float2*>(cp + a0);
                        cv[0] = t2.x; cv[1] = t2.y; cv[2] = 0.f; cv[3] = 0.f;
                    }
#pragma unroll
                    for (int a = a0; a < a0 + 4 && a < R; ++a)
#pragma unroll
                        for (int b = 0; b < R; ++b) Mr[a][b] = fmaf(cv[a - a0], rv[b], Mr[a][b]);
                }
            }
        }
        __syncthreads();   // the panel buffers are dead before the staging area is reused
        if (sh_viol) {
            // Redo this block row with partial pivoting in shared memory:
            // S_j from G_{j-1} (in the factor pool) and D_j, implicit
            // pivoting (rows never move), then G_j[r][c] = M[perm[r]][rinv[c]].
            const float* Gp = G + (long long)(j > 0 ? j - 1 : 0) * blk;
            for (int r = warp; r < m; r += FACT_THREADS / 32) {
                for (int c = lane; c < m; c += 32) {
                    const float v = (j > 0) ? -tbeta2 * Gp[packed_index<float>(r, c, mp)] : 0.f;
                    Ms[r * LDS + c] = v + dval(j, r, c);
                }
            }
            for (int t = tid; t < m; t += FACT_THREADS) used[t] = 0;
            __syncthreads();
            for (int k = 0; k < m; ++k) {
                if (warp == 0) {
                    unsigned bb = 0u;
                    int bi = 0x7fffffff;
                    for (int r = lane; r < m; r += 32) {
                        if (!used[r]) {
                            const unsigned u = __float_as_uint(fabsf(Ms[r * LDS + k]));
                            if (u > bb) { bb = u; bi = r; }
                        }
                    }
                    const unsigned mx = __reduce_max_sync(0xffffffffu, bb);
                    const int r = (int)__reduce_min_sync(0xffffffffu, (unsigned)(bb == mx ? bi : 0x7fffffff));
                    if (lane == 0) {
                        if (mx == 0u || mx >= 0x7f800000u || r >= m) {
                            sh_fail = 1;
                        } else {
                            sh_r = r;
                            used[r] = 1;
                            pivr[k] = r;
                            sh_piv = Ms[r * LDS + k];
                        }
                    }
                }
                __syncthreads();
                if (sh_fail) break;
                const int r = sh_r;
                const float inv = 1.f / sh_piv;
                for (int t = tid; t < m; t += FACT_THREADS) fcol[t] = Ms[t * LDS + k];
                __syncthreads();
                for (int t = tid; t < m; t += FACT_THREADS) Ms[r * LDS + t] = (t == k ? 1.f : Ms[r * LDS + t]) * inv;
                __syncthreads();
                // rows by warp, columns by lane; the pivot row in registers
                constexpr int NC = (MM + 31) / 32;
                float prow[NC];
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    const int t = lane + 32 * q;
                    prow[q] = (t < m) ? Ms[r * LDS + t] : 0.f;
                }
                for (int rr = warp; rr < m; rr += FACT_THREADS / 32) {
                    if (rr == r) continue;
                    const float fct = fcol[rr];
#pragma unroll
                    for (int q = 0; q < NC; ++q) {
                        const int t = lane + 32 * q;
                        if (t < m) Ms[rr * LDS + t] = (t == k ? 0.f : Ms[rr * LDS + t]) - fct * prow[q];
                    }
                }
                __syncthreads();
            }
            if (sh_fail) {
                failed = true;
                break;
            }
            for (int t = tid; t < m; t += FACT_THREADS) sinv[pivr[t]] = t;   // rinv
            __syncthreads();
#pragma unroll
            for (int a = 0; a < R; ++a) {
                const int r = ty * R + a;
#pragma unroll
                for (int b = 0; b < R; ++b) {
                    const int c = tx * R + b;
                    Mr[a][b] = (r < m && c < m) ? Ms[pivr[r] * LDS + sinv[c]] : 0.f;
                }
            }
            __syncthreads();
        }
        // G_j into shared memory, then packed to HBM
#pragma unroll
        for (int a2 = 0; a2 < R; ++a2) {
            const int r = ty * R + a2;
#pragma unroll
            for (int b = 0; b < R; ++b) {
                const int c = tx * R + b;
                if (r < mp && c < mp) Ms[r * LDS + c] = (r < m && c < m) ? Mr[a2][b] : 0.f;
            }
        }
        __syncthreads();
        {
            // slab sl, vector v of thread t = 8 rho + kappa: row rho + 32 sl,
            // columns kappa*cw + 4v .. +3 (the layout of packed_index)
            const int cw = mp >> 3, nv = cw >> 2, nslab = mp >> 5;
            const int rho = tid >> 3, kappa = tid & 7;
            float4* Gj4 = reinterpret_cast<float4*>(G + (long long)j * blk);
            for (int sl = 0; sl < nslab; ++sl) {
                const float* row = Ms + (rho + 32 * sl) * LDS + kappa * cw;
                for (int v = 0; v < nv; ++v)
                    Gj4[(sl * nv + v) * 256 + tid] = *reinterpret_cast<const float4*>(row + 4 * v);
            }
        }
        __syncthreads();
    }
    if (failed && tid == 0) {
        ls[i].status = ST_ESINGULAR;
        ls[i].active = 0;
    }
}

// Entries of D_j (grid row j of the local Jacobian) inside the tile of
// thread (ty, ty + DT) of a wide CTA (R x R tiles, any R): the 2 x 2 node
// blocks on the diagonal (4 beta + phi', the control coupling
// (1/nu)(1 - P_eps'(-p/mu)) in the y-row and phi'' p - 1 in the p-row) and
// -beta two places off it (the x-neighbours of the same field).
template <int R, int DT>
__device__ __forceinline__ void add_band_any(float (&Mr)[R][R], int ty, int m, int wx, int j, float tdiag,
                                             float tbeta, const double* ca, const double* cb, const double* cc) {
#pragma unroll
    for (int a = 0; a < R; ++a) {
#pragma unroll
        for (int b = 0; b < R; ++b) {
            const int off = DT * R + b - a;
            if (off < -2 || off > 2) continue;
            const int r = ty * R + a, c = r + off;
            if (r >= m || c < 0 || c >= m) continue;
            const int q = j * wx + (r >> 1);
            const bool yrow = (r & 1) == 0;
            if (off == 0) Mr[a][b] += tdiag + (float)ca[q];
            else if (off == 1) { if (yrow) Mr[a][b] += (float)cb[q]; }
            else if (off == -1) { if (!yrow) Mr[a][b] += (float)cc[q]; }
            else Mr[a][b] -= tbeta;
        }
    }
}

// FP32 factorisation with one 1024-thread CTA per subdomain (one CTA per SM):
// thread (ty, tx) of the 32 x 32 CTA (tid = 32 tx + ty: a thread column is a
// warp) holds the R x R tile (R = mp / 32) of the block row matrix in
// registers. The algorithm is that of k_local_factor_panel (panels of R
// pivots swept by the panel's column owners, here a whole warp, then one
// rank-R update), with 32 warps sharing each block row: the dependent pivot
// chain of a panel is R pivots of R x R work per lane, and the update is
// spread over four times as many warps.
template <int R>
__global__ void __launch_bounds__(1024, 1) k_local_factor_wide(int nsub, const SubDev* __restrict__ subs,
                                                               const ProbDev* __restrict__ probs,
                                                               const double* X, LocalState* ls,
                                                               const double* cpool, double* coef,
                                                               float* gpool, int only_active,
                                                               const int* __restrict__ list, FactorSel sel) {
    constexpr int NTH = 1024, NWARP = 32;
    constexpr int MM = 32 * R;
    constexpr int PAD = ((R + 3) / 4) * 4;   // owner stride of the row panel
    constexpr int LDR = 32 * PAD;            // one row of the row panel
    constexpr int LDCT = 32 * R;             // one column of the swept panel: [a][ty]
    constexpr int LDS = MM + 4;              // staging stride of the full block
    constexpr int OFF_CT = 0;
    constexpr int OFF_RW = OFF_CT + 2 * R * LDCT;
    static_assert(OFF_RW + 2 * R * LDR <= MM * LDS, "panel buffers fit in the staging area");
    __shared__ float fcol[MM];
    __shared__ int pivr[MM];
    __shared__ int sinv[MM];
    __shared__ int used[MM];
    __shared__ int sh_viol, sh_r, sh_fail;
    __shared__ float sh_piv;
    extern __shared__ __align__(16) float Ms[];
    if ((int)blockIdx.x >= nsub) return;
    if (sel.nwork && min(*sel.nwork, nsub) > sel.thr) return;    // the 256-thread kernel's turn
    const int i = list ? list[blockIdx.x] : (int)blockIdx.x;
    if (only_active && !ls[i].active) return;
    if (ls[i].status == ST_SKIP) return;
    const SubDev s = subs[i];
    if (s.mp > 32 * R) return;   // not this register-tile class (wide blocks: k_local_factor_big)
    const ProbDev P = probs[s.prob];
    const int m = 2 * s.bl, W = s.bw, nn = s.wx * s.wy * s.wz, mp = s.mp;
    const bool cube = P.nz > 1;
    const int tid = threadIdx.x, ty = tid & 31, tx = tid >> 5, warp = tid >> 5, lane = tid & 31;

    const double eps = ls[i].eps;
    const double beta = P.beta, inu = 1.0 / P.nu, mu = P.mu;
    double* ca = s.cptr;
    double* cb = ca + nn;
    double* cc = cb + nn;
    {
        const double* c = cpool + s.voff;
        const LocalView V = make_view(s, P, X, c, nullptr, 0.0);
        for (int q = tid; q < nn; q += NTH) {
            const double y = V.at(q, 0), p = V.at(q, 1);
            double ph, d1, d2;
            phi_eval(P.phi, P.kappa, y, ph, d1, d2);
            ca[q] = d1;
            cb[q] = inu * one_minus_dP_eps(-p / mu, eps);
            cc[q] = d2 * p - 1.0;
        }
    }
    if (tid == 0) sh_fail = 0;
    __syncthreads();   // coefficients visible to the whole CTA

    const float tbeta = (float)beta, tbeta2 = (float)(beta * beta), tdiag = (float)P.diag;
    const long long blk = (long long)mp * mp;
    float* G = static_cast<float*>(s.gptr);
    float Mr[R][R];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) Mr[a][b] = 0.f;
    bool failed = false;
    auto dval = [=](int j, int r, int c) -> float {
        const int ix = r >> 1, f = r & 1, cx = c >> 1, cf = c & 1;
        const int q = j * s.bl + ix;
        if (cx == ix) {
            if (cf == f) return tdiag + (float)ca[q];
            return (f == 0) ? (float)cb[q] : (float)cc[q];
        }
        return (cf == f && row_neighbour(ix, cx, s.wx, cube)) ? -tbeta : 0.f;
    };
    for (int j = 0; j < W && !failed; ++j) {
        // S_j = D_j - beta^2 G_{j-1}: the tile holds G_{j-1} (zero for j = 0)
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < R; ++b) Mr[a][b] = -tbeta2 * Mr[a][b];
        const int dt = tx - ty;
        if (cube) add_plane<R>(Mr, ty, tx, m, s.bl, s.wx, j, tdiag, tbeta, ca, cb, cc);
        else if (dt == 0) add_band_any<R, 0>(Mr, ty, m, s.bl, j, tdiag, tbeta, ca, cb, cc);
        else if (dt == 1) add_band_any<R, 1>(Mr, ty, m, s.bl, j, tdiag, tbeta, ca, cb, cc);
        else if (dt == -1) add_band_any<R, -1>(Mr, ty, m, s.bl, j, tdiag, tbeta, ca, cb, cc);
        else if (R == 1 && dt == 2) add_band_any<R, 2>(Mr, ty, m, s.bl, j, tdiag, tbeta, ca, cb, cc);
        else if (R == 1 && dt == -2) add_band_any<R, -2>(Mr, ty, m, s.bl, j, tdiag, tbeta, ca, cb, cc);
        if (tid == 0) sh_viol = 0;

        for (int kt = 0; kt < 32 && kt * R < m; ++kt) {
            float* CsT = Ms + OFF_CT + (kt & 1) * (R * LDCT);
            float* Rw = Ms + OFF_RW + (kt & 1) * (R * LDR);
            if (ty == kt) {
                if (tx == kt) {
#pragma unroll
                    for (int c = 0; c < R; ++c) {
                        float z[R];
#pragma unroll
                        for (int b = 0; b < R; ++b) z[b] = 0.f;
                        store_vec<R>(Rw + c * LDR + tx * PAD, z);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < R; ++c) store_vec<R>(Rw + c * LDR + tx * PAD, Mr[c]);
                    // rows K restart from 0: the update below leaves C'[K,K] M[K,J]
                    // there (M[K,J] + (C'[K,K] - I) M[K,J] would cancel, C'[K,K] ~ 1/(4 beta))
#pragma unroll
                    for (int a = 0; a < R; ++a)
#pragma unroll
                        for (int b = 0; b < R; ++b) Mr[a][b] = 0.f;
                }
            }
            if (tx == kt) {
                const bool ok = panel_sweep<R>(Mr, ty, kt, m, 0xffffffffu, kt);
                if (!ok && ty == 0) sh_viol = 1;
#pragma unroll
                for (int c = 0; c < R; ++c)
#pragma unroll
                    for (int a = 0; a < R; ++a) CsT[c * LDCT + a * 32 + ty] = Mr[a][c];
            }
            __syncthreads();
            if (sh_viol) break;
            // rank-R update M += C' [M[K,:] with 0 at K]
#pragma unroll
            for (int c = 0; c < R; ++c) {
                float rv[R];
                load_vec<R>(Rw + c * LDR + tx * PAD, rv);
#pragma unroll
                for (int a = 0; a < R; ++a) {
                    const float cv = CsT[c * LDCT + a * 32 + ty];
#pragma unroll
                    for (int b = 0; b < R; ++b) Mr[a][b] = fmaf(cv, rv[b], Mr[a][b]);
                }
            }
        }
        __syncthreads();   // the panel buffers are dead before the staging area is reused
        if (sh_viol) {
            // Redo this block row with partial pivoting in shared memory:
            // S_j from G_{j-1} (in the factor pool) and D_j, implicit
            // pivoting (rows never move), then G_j[r][c] = M[perm[r]][rinv[c]].
            const float* Gp = G + (long long)(j > 0 ? j - 1 : 0) * blk;
            for (int r = warp; r < m; r += NWARP) {
                for (int c = lane; c < m; c += 32) {
                    const float v = (j > 0) ? -tbeta2 * Gp[packed_index<float>(r, c, mp)] : 0.f;
                    Ms[r * LDS + c] = v + dval(j, r, c);
                }
            }
            for (int t = tid; t < m; t += NTH) used[t] = 0;
            __syncthreads();
            for (int k = 0; k < m; ++k) {
                if (warp == 0) {
                    unsigned bb = 0u;
                    int bi = 0x7fffffff;
                    for (int r = lane; r < m; r += 32) {
                        if (!used[r]) {
                            const unsigned u = __float_as_uint(fabsf(Ms[r * LDS + k]));
                            if (u > bb) { bb = u; bi = r; }
                        }
                    }
                    const unsigned mx = __reduce_max_sync(0xffffffffu, bb);
                    const int r = (int)__reduce_min_sync(0xffffffffu, (unsigned)(bb == mx ? bi : 0x7fffffff));
                    if (lane == 0) {
                        if (mx == 0u || mx >= 0x7f800000u || r >= m) {
                            sh_fail = 1;
                        } else {
                            sh_r = r;
                            used[r] = 1;
                            pivr[k] = r;
                            sh_piv = Ms[r * LDS + k];
                        }
                    }
                }
                __syncthreads();
                if (sh_fail) break;
                const int r = sh_r;
                const float inv = 1.f / sh_piv;
                for (int t = tid; t < m; t += NTH) fcol[t] = Ms[t * LDS + k];
                __syncthreads();
                for (int t = tid; t < m; t += NTH) Ms[r * LDS + t] = (t == k ? 1.f : Ms[r * LDS + t]) * inv;
                __syncthreads();
                constexpr int NC = (MM + 31) / 32;
                float prow[NC];
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    const int t = lane + 32 * q;
                    prow[q] = (t < m) ? Ms[r * LDS + t] : 0.f;
                }
                for (int rr = warp; rr < m; rr += NWARP) {
                    if (rr == r) continue;
                    const float fct = fcol[rr];
#pragma unroll
                    for (int q = 0; q < NC; ++q) {
                        const int t = lane + 32 * q;
                        if (t < m) Ms[rr * LDS + t] = (t == k ? 0.f : Ms[rr * LDS + t]) - fct * prow[q];
                    }
                }
                __syncthreads();
            }
            if (sh_fail) {
                failed = true;
                break;
            }
            for (int t = tid; t < m; t += NTH) sinv[pivr[t]] = t;   // rinv
            __syncthreads();
#pragma unroll
            for (int a = 0; a < R; ++a) {
                const int r = ty * R + a;
#pragma unroll
                for (int b = 0; b < R; ++b) {
                    const int c = tx * R + b;
                    Mr[a][b] = (r < m && c < m) ? Ms[pivr[r] * LDS + sinv[c]] : 0.f;
                }
            }
            __syncthreads();
        }
        // G_j into shared memory, then packed to HBM
#pragma unroll
        for (int a2 = 0; a2 < R; ++a2) {
            const int r = ty * R + a2;
#pragma unroll
            for (int b = 0; b < R; ++b) {
                const int c = tx * R + b;
                if (r < mp && c < mp) Ms[r * LDS + c] = (r < m && c < m) ? Mr[a2][b] : 0.f;
            }
        }
        __syncthreads();
        {
            // entry e * 256 + t of the packed block (e = slab sl, vector v;
            // t = 8 rho + kappa): row rho + 32 sl, columns kappa*cw + 4v .. +3
            const int cw = mp >> 3, nv = cw >> 2, nslab = mp >> 5;
            float4* Gj4 = reinterpret_cast<float4*>(G + (long long)j * blk);
            for (int idx = tid; idx < nslab * nv * 256; idx += NTH) {
                const int e = idx >> 8, t = idx & 255;
                const int sl = e / nv, v = e - sl * nv;
                const float* row = Ms + ((t >> 3) + 32 * sl) * LDS + (t & 7) * cw;
                Gj4[idx] = *reinterpret_cast<const float4*>(row + 4 * v);
            }
        }
        __syncthreads();
    }
    if (failed && tid == 0) {
        ls[i].status = ST_ESINGULAR;
        ls[i].active = 0;
    }
}

// ------------------------------------------------------------- wide blocks
// Cluster primitives (the CTAs of one thread-block cluster).
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Every thread of every CTA of the cluster; memory operations before it are
// visible to the cluster after it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// An int in the shared memory of CTA `rank` of the cluster, at the offset of
// `p` in this CTA's.
__device__ __forceinline__ int ld_cluster_int(const int* p, uint32_t rank) {
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    uint32_t ra;
    int v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
    return v;
}

// 16 consecutive T of a panel row (16-byte aligned) <-> registers.
template <typename T>
__device__ __forceinline__ void ld_row16(const T* src, T (&v)[BIG_PANEL]) {
    static_assert(BIG_PANEL == 16, "16 entries per panel row");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 t = reinterpret_cast<const float4*>(src)[q];
            v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const double2 t = reinterpret_cast<const double2*>(src)[q];
            v[2 * q] = t.x; v[2 * q + 1] = t.y;
        }
    }
}

template <typename T>
__device__ __forceinline__ void st_row16(T* dst, const T (&v)[BIG_PANEL]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) reinterpret_cast<double2*>(dst)[q] = make_double2(v[2 * q], v[2 * q + 1]);
    }
}

// Factorisation of a wide-block subdomain (MAX_M < m = 2 bl <= MAX_MW) by one
// cluster of 1024-thread CTAs (BIG_CLUSTER of them; the kernel reads the
// cluster's size, so one CTA per subdomain works too). Block row j is formed
// and inverted in place in its own factor slot (mp x mp): S_j = D_j -
// beta^2 G_{j-1}, inverted by Gauss-Jordan elimination with partial pivoting
// (max |.| among the rows not yet pivots, ties to the lowest row), BIG_PANEL
// pivots at a time and with implicit interchanges: rows never move, perm[k]
// records the row that pivots column k, and the slot ends up holding
// S_j^-1[k][c] at (perm[k], perm^-1[c]). The columns of the block are split
// among the CTAs in whole panels; CTA b forms and updates its own columns only.
// For the panel K of CTA o: thread r of CTA o holds row r of the column panel
// in registers and sweeps it (per pivot: an argmax over the CTA, the pivot row
// passed on in shared memory), writes C' back into M[:, K] and publishes the
// panel's pivot rows P in its shared memory; after one cluster barrier every
// CTA reads C' and P and applies the rank-BIG_PANEL update to its columns: the
// rows of P become C'[P,K] M[P,J] and every other row M[I,J] + C'[I,K] M[P,J].
// One cluster barrier per panel suffices: M[:, K] changes again only in the
// next panel's update, after the next barrier. Once block row j + 1 has read
// G_j (through the pivoting, by gathers that hit L2), slot j is rewritten in
// plain column-major order through a scratch block (the wide solves read G_j
// column-major). A pivot that is 0 or not finite stops the subdomain with
// ST_ESINGULAR.
template <typename T>
__global__ void __launch_bounds__(BIG_THREADS) k_local_factor_big(int count, const int* __restrict__ list,
                                                                  const SubDev* __restrict__ subs,
                                                                  const ProbDev* __restrict__ probs,
                                                                  const double* X, LocalState* ls,
                                                                  const double* cpool, double* coef, T* gpool,
                                                                  int only_active) {
    constexpr int NTH = BIG_THREADS, NWB = NTH / 32, RB = BIG_PANEL;
    static_assert(MAX_MW <= NTH, "one panel row per thread in the sweep");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Cs = reinterpret_cast<T*>(smem_raw);   // C' of the panel: row r at Cs + r * RB
    T* Rs = Cs + MAX_MW * RB;                 // pivot rows of the panel: kk at Rs + kk * MAX_MW
    T* prow = Rs + RB * MAX_MW;               // the pivot row of the current pivot
    __shared__ int perm[MAX_MW];              // perm[k]: row pivoting column k (this block row)
    __shared__ int pprev[MAX_MW], rprev[MAX_MW];   // perm of block row j - 1 and its inverse
    __shared__ unsigned char used[MAX_MW];    // row already a pivot row in this block row
    __shared__ unsigned char inp[MAX_MW];     // row is a pivot row of the current panel
    __shared__ T red_v[NWB];
    __shared__ int red_i[NWB];
    __shared__ int sh_p;                      // pivot row of the current pivot (-1: singular)
    __shared__ int pk[RB];                    // pivot rows of the current panel (every CTA)
    __shared__ int pub[2][RB];                // pivot rows of the panels this CTA swept
    __shared__ int pubf[2];                   // and whether a pivot was 0 or not finite
    const uint32_t nct = cluster_size(), rank = cluster_rank();
    const int sidx = (int)(blockIdx.x / nct);
    if (sidx >= count) return;
    const int i = list[sidx];
    if (only_active && !ls[i].active) return;
    if (ls[i].status == ST_SKIP) return;
    const SubDev s = subs[i];
    const ProbDev P = probs[s.prob];
    const int m = 2 * s.bl, W = s.bw, nn = s.wx * s.wy * s.wz, mp = s.mp;
    const bool cube = P.nz > 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // columns of this CTA: [cl, ch), whole panels
    const int pw = ((m + (int)nct * RB - 1) / ((int)nct * RB)) * RB;
    const int cl = min(m, (int)rank * pw), ch = min(m, cl + pw), ncol = ch - cl;

    const double eps = ls[i].eps;
    const double beta = P.beta, inu = 1.0 / P.nu, mu = P.mu;
    double* ca = s.cptr;
    double* cb = ca + nn;
    double* cc = cb + nn;
    {
        const double* c = cpool + s.voff;
        const LocalView V = make_view(s, P, X, c, nullptr, 0.0);
        for (int q = (int)rank * NTH + tid; q < nn; q += (int)nct * NTH) {
            const double y = V.at(q, 0), p = V.at(q, 1);
            double ph, d1, d2;
            phi_eval(P.phi, P.kappa, y, ph, d1, d2);
            ca[q] = d1;
            cb[q] = inu * one_minus_dP_eps(-p / mu, eps);
            cc[q] = d2 * p - 1.0;
        }
    }
    __threadfence();
    cluster_sync();   // coefficients of the whole box written

    const T tbeta = (T)beta, tbeta2 = (T)(beta * beta), tdiag = (T)P.diag;
    T* G = static_cast<T*>(s.gptr);
    const long long blk = (long long)mp * mp;
    T* scratch = G + (long long)W * blk;      // one more block after the bw factor blocks
    auto dval = [&](int j, int r, int c) -> T {   // entry (r, c) of D_j
        const int ix = r >> 1, f = r & 1, cx = c >> 1, cf = c & 1;
        const int q = j * s.bl + ix;
        if (cx == ix) {
            if (cf == f) return tdiag + (T)ca[q];
            return (f == 0) ? (T)cb[q] : (T)cc[q];
        }
        return (cf == f && row_neighbour(ix, cx, s.wx, cube)) ? -tbeta : (T)0;
    };
    // own columns of M = S_j; G_{j-1}[r][c] = slot j-1 at (pprev[r], rprev[c])
    auto form = [&](int j, T* M) {
        const T* Gp = G + (long long)(j > 0 ? j - 1 : 0) * blk;
        for (int e = tid; e < m * ncol; e += NTH) {
            const int r = e / ncol, c = cl + (e - r * ncol);
            const T g = (j > 0) ? -tbeta2 * Gp[(long long)pprev[r] * mp + rprev[c]] : (T)0;
            M[(long long)r * mp + c] = g + dval(j, r, c);
        }
    };
    // slot j (pivoting pprev / rprev) to plain column-major order: copy the
    // own columns to the scratch block, then write rows c of the storage
    // (column c of G_j) from it
    auto finalize = [&](int j) {
        T* M = G + (long long)j * blk;
        for (int e = tid; e < m * ncol; e += NTH) {
            const int r = e / ncol, c = cl + (e - r * ncol);
            scratch[(long long)r * mp + c] = M[(long long)r * mp + c];
        }
        __threadfence();
        cluster_sync();   // the whole slot copied
        for (int e = tid; e < ncol * m; e += NTH) {
            const int c = cl + e / m, k = e - (e / m) * m;
            M[(long long)c * mp + k] = scratch[(long long)pprev[k] * mp + rprev[c]];
        }
    };
    const int mc = ((ncol + 31) / 32) * 32;        // update: own columns padded to whole warps,
    const int rows_par = (mc > 0) ? NTH / mc : 1;  // rows_par threads per column
    const int ucol = (mc > 0) ? tid % mc : 0, urow = (mc > 0) ? tid / mc : NTH;
    for (int r = tid; r < MAX_MW; r += NTH) inp[r] = 0;

    bool failed = false;
    for (int j = 0; j < W && !failed; ++j) {
        T* M = G + (long long)j * blk;
        // G_{j-1}[r][c] lies in other CTAs' columns: every update of block row j - 1 is done first
        if (j > 0) cluster_sync();
        form(j, M);
        if (j > 0) {
            cluster_sync();   // every CTA has read G_{j-1}
            finalize(j - 1);
        }
        for (int r = tid; r < m; r += NTH) used[r] = 0;
        __syncthreads();
        for (int k0 = 0; k0 < m; k0 += RB) {
            const int nk = min(RB, m - k0);
            const uint32_t owner = (uint32_t)(k0 / pw);
            // the owner's slot: parity of its panels before this one in the block row
            const int slot = ((k0 - (int)owner * pw) / RB) & 1;
            if (rank == owner) {
                // thread r < m: row r of the column panel in registers
                T v[RB];
                if (tid < m) {
                    ld_row16<T>(M + (long long)tid * mp + k0, v);
#pragma unroll
                    for (int kk = 0; kk < RB; ++kk)
                        if (kk >= nk) v[kk] = (T)0;
                }
                int fail = 0;
#pragma unroll
                for (int kk = 0; kk < RB; ++kk) {
                    if (kk < nk && !fail) {
                        // pivot: max |.| of column kk among the rows not yet pivots
                        T best = (tid < m && !used[tid]) ? fabs(v[kk]) : (T)-1;
                        int bi = (tid < m && !used[tid]) ? tid : 0x7fffffff;
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) {
                            const T ob = __shfl_xor_sync(0xffffffffu, best, off);
                            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                        }
                        if (lane == 0) {
                            red_v[warp] = best;
                            red_i[warp] = bi;
                        }
                        __syncthreads();
                        if (warp == 0) {
                            best = (lane < NWB) ? red_v[lane] : (T)-1;
                            bi = (lane < NWB) ? red_i[lane] : 0x7fffffff;
#pragma unroll
                            for (int off = 16; off > 0; off >>= 1) {
                                const T ob = __shfl_xor_sync(0xffffffffu, best, off);
                                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                            }
                            if (lane == 0) sh_p = (bi < m && best > (T)0 && best < (T)INFINITY) ? bi : -1;
                        }
                        __syncthreads();
                        const int p = sh_p;
                        if (p < 0) {
                            fail = 1;   // the same on every thread
                        } else {
                            if (tid == p) {
#pragma unroll
                                for (int c = 0; c < RB; ++c) prow[c] = v[c];
                                used[p] = 1;
                            }
                            if (tid == 0) pub[slot][kk] = p;
                            __syncthreads();
                            const T inv = (T)1 / prow[kk];
                            if (tid == p) {
#pragma unroll
                                for (int c = 0; c < RB; ++c) v[c] = (c == kk) ? inv : prow[c] * inv;
                            } else if (tid < m) {
                                const T f = v[kk];
#pragma unroll
                                for (int c = 0; c < RB; ++c) {
                                    const T t = (c == kk) ? inv : prow[c] * inv;
                                    v[c] = fma(-f, t, (c == kk) ? (T)0 : v[c]);
                                }
                            }
                        }
                    }
                }
                if (tid == 0) pubf[slot] = fail;
                // C' into M[:, K] (columns past m are padding) and into shared memory
                if (!fail && tid < m) {
                    st_row16<T>(M + (long long)tid * mp + k0, v);
                    st_row16<T>(Cs + tid * RB, v);
                }
                __threadfence();
            }
            cluster_sync();   // C' of panel K and its pivot rows visible to the cluster
            if (ld_cluster_int(&pubf[slot], owner)) {
                failed = true;
                break;
            }
            if (tid < nk) {
                const int p = ld_cluster_int(&pub[slot][tid], owner);
                pk[tid] = p;
                perm[k0 + tid] = p;
                used[p] = 1;
                inp[p] = 1;
            }
            if (rank != owner && tid < m) {
                T v[RB];
                ld_row16<T>(M + (long long)tid * mp + k0, v);
#pragma unroll
                for (int kk = 0; kk < RB; ++kk)
                    if (kk >= nk) v[kk] = (T)0;
                st_row16<T>(Cs + tid * RB, v);
            }
            __syncthreads();
            for (int e = tid; e < RB * ncol; e += NTH) {
                const int kk = e / ncol, c = cl + (e - kk * ncol);
                Rs[kk * MAX_MW + c] =
                    (kk < nk && (c < k0 || c >= k0 + nk)) ? M[(long long)pk[kk] * mp + c] : (T)0;
            }
            __syncthreads();
            if (ucol < ncol && urow < rows_par) {
                const int c = cl + ucol;
                if (c < k0 || c >= k0 + nk) {
                    T rv[RB];
#pragma unroll
                    for (int kk = 0; kk < RB; ++kk) rv[kk] = Rs[kk * MAX_MW + c];
                    // UR rows at a time, their loads issued before any is used
                    constexpr int UR = sizeof(T) == 4 ? 8 : 4;
                    for (int r0 = urow; r0 < m; r0 += UR * rows_par) {
                        T acc[UR];
#pragma unroll
                        for (int u = 0; u < UR; ++u) {
                            const int r = r0 + u * rows_par;
                            acc[u] = (r < m && !inp[r]) ? M[(long long)r * mp + c] : (T)0;
                        }
#pragma unroll
                        for (int u = 0; u < UR; ++u) {
                            const int r = r0 + u * rows_par;
                            if (r < m) {
                                if constexpr (sizeof(T) == 4) {
                                    T cv[RB];
                                    ld_row16<T>(Cs + r * RB, cv);
#pragma unroll
                                    for (int kk = 0; kk < RB; ++kk) acc[u] = fma(cv[kk], rv[kk], acc[u]);
                                } else {
#pragma unroll
                                    for (int kk = 0; kk < RB; ++kk) acc[u] = fma(Cs[r * RB + kk], rv[kk], acc[u]);
                                }
                                M[(long long)r * mp + c] = acc[u];
                            }
                        }
                    }
                }
            }
            __syncthreads();
            if (tid < nk) inp[pk[tid]] = 0;
        }
        if (failed) break;
        // this block row's pivoting becomes the previous one's
        __syncthreads();
        for (int r = tid; r < m; r += NTH) {
            pprev[r] = perm[r];
            rprev[perm[r]] = r;
        }
        __syncthreads();
    }
    if (failed) {
        if (rank == 0 && tid == 0) {
            ls[i].status = ST_ESINGULAR;
            ls[i].active = 0;
        }
    } else {
        cluster_sync();   // every CTA's last update is done
        finalize(W - 1);
    }
    cluster_sync();   // no CTA leaves while another may read its shared memory
}

template <typename T>
size_t factor_smem(int maxm) {
    return (size_t)maxm * (maxm + 1) * sizeof(T) + (size_t)maxm * sizeof(T) + 3 * (size_t)maxm * sizeof(int);
}

// Loop condition of the local Newton sweep (see launch_sweep_cond).
__global__ void k_sweep_cond(cudaGraphConditionalHandle c, const int* active, int* guard, int limit, int reset) {
    const int g = reset ? 0 : *guard;
    *guard = g + 1;
    cudaGraphSetConditional(c, (*active > 0 && g <= limit) ? 1u : 0u);
}

}  // namespace

// ------------------------------------------------------------------ launchers
cudaError_t launch_local_init(cudaStream_t st, int nsub, const SubDev* subs, const ProbDev* probs,
                              const double* X, LocalState* ls, const double* pstart, NewtonParams np,
                              double* cpool, double* Kpool, int* active_count) {
    count_launch();
    k_local_init<<<nsub, NT, 0, st>>>(nsub, subs, probs, X, ls, pstart, np, cpool, Kpool, active_count);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_factor_panel(cudaStream_t st, int count, const SubDev* subs, const ProbDev* probs,
                              const double* X, LocalState* ls, const double* cpool, double* coef,
                              float* gpool, int only_active, const int* list, FactorSel fs) {
    const size_t sm = (size_t)(16 * R) * (16 * R + 4) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_local_factor_panel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_factor_panel<R><<<count, FACT_THREADS, sm, st>>>(count, subs, probs, X, ls, cpool, coef, gpool,
                                                           only_active, list, fs);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_factor_wide(cudaStream_t st, int count, const SubDev* subs, const ProbDev* probs,
                               const double* X, LocalState* ls, const double* cpool, double* coef,
                               float* gpool, int only_active, const int* list, FactorSel fs) {
    const size_t sm = (size_t)(32 * R) * (32 * R + 4) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_local_factor_wide<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_factor_wide<R><<<count, 1024, sm, st>>>(count, subs, probs, X, ls, cpool, coef, gpool, only_active,
                                                    list, fs);
    return cudaGetLastError();
}

cudaError_t launch_local_factor_f32(cudaStream_t st, int tile, int count, const int* list, const SubDev* subs,
                                    const ProbDev* probs, const double* X, LocalState* ls, const double* cpool,
                                    double* coef, float* gpool, int only_active, int wide, FactorSel fs) {
    if (wide) {
        switch (tile) {
            case 2: return launch_factor_wide<1>(st, count, subs, probs, X, ls, cpool, coef, gpool, only_active, list, fs);
            case 4: return launch_factor_wide<2>(st, count, subs, probs, X, ls, cpool, coef, gpool, only_active, list, fs);
            case 6: return launch_factor_wide<3>(st, count, subs, probs, X, ls, cpool, coef, gpool, only_active, list, fs);
            case 8: return launch_factor_wide<4>(st, count, subs, probs, X, ls, cpool, coef, gpool, only_active, list, fs);
            case 10: return launch_factor_wide<5>(st, count, subs, probs, X, ls, cpool, coef, gpool, only_active, list, fs);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (tile) {
        case 2: return launch_factor_panel<2>(st, count, subs, probs, X, ls, cpool, coef, gpool, only_active, list, fs);
        case 4: return launch_factor_panel<4>(st, count, subs, probs, X, ls, cpool, coef, gpool, only_active, list, fs);
        case 6: return launch_factor_panel<6>(st, count, subs, probs, X, ls, cpool, coef, gpool, only_active, list, fs);
        case 8: return launch_factor_panel<8>(st, count, subs, probs, X, ls, cpool, coef, gpool, only_active, list, fs);
        case 10: return launch_factor_panel<10>(st, count, subs, probs, X, ls, cpool, coef, gpool, only_active, list, fs);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_local_factor(cudaStream_t st, int nsub, int maxm, const SubDev* subs,
                                const ProbDev* probs, const double* X, LocalState* ls,
                                const double* cpool, double* coef, T* gpool, int only_active) {
    if (sizeof(T) == sizeof(float)) {
        const int mpmax = ((maxm + 31) / 32) * 32;
        return launch_local_factor_f32(st, mpmax / 16, nsub, nullptr, subs, probs, X, ls, cpool, coef,
                                       reinterpret_cast<float*>(gpool), only_active, 0);
    }
    const size_t sm = factor_smem<T>(maxm);
    cudaError_t e = cudaFuncSetAttribute(k_local_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_factor<T><<<nsub, FACT_THREADS, sm, st>>>(nsub, maxm, subs, probs, X, ls, cpool, coef, gpool,
                                                      only_active);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_factor_big(cudaStream_t st, int count, const int* list, const SubDev* subs,
                                    const ProbDev* probs, const double* X, LocalState* ls, const double* cpool,
                                    double* coef, T* gpool, int only_active) {
    if (count <= 0) return cudaSuccess;
    const size_t sm = (size_t)(2 * MAX_MW * BIG_PANEL + BIG_PANEL) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_local_factor_big<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // one cluster of BIG_CLUSTER CTAs per subdomain, fewer if the device cannot place that many
    static int csize = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(BIG_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    if (csize == 0) {
        for (int c = BIG_CLUSTER; c >= 1; c /= 2) {
            cfg.gridDim = dim3((unsigned)c);
            attr[0].val.clusterDim.x = (unsigned)c;
            int ncl = 0;
            if (cudaOccupancyMaxActiveClusters(&ncl, k_local_factor_big<T>, &cfg) == cudaSuccess && ncl > 0) {
                csize = c;
                break;
            }
            cudaGetLastError();
        }
        if (csize == 0) return cudaErrorLaunchOutOfResources;
    }
    cfg.gridDim = dim3((unsigned)(count * csize));
    attr[0].val.clusterDim.x = (unsigned)csize;
    count_launch();
    return cudaLaunchKernelEx(&cfg, k_local_factor_big<T>, count, list, subs, probs, X, ls, cpool, coef, gpool,
                              only_active);
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

cudaError_t launch_sweep_cond(cudaStream_t st, cudaGraphConditionalHandle c, const int* active, int* guard,
                              int limit, int reset) {
    count_launch();
    k_sweep_cond<<<1, 1, 0, st>>>(c, active, guard, limit, reset);
    return cudaGetLastError();
}

cudaError_t add_sweep_cond_node(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle c,
                                const int* active, int* guard, int limit, int reset, cudaGraphNode_t* out) {
    cudaKernelNodeParams kp{};
    void* args[] = {&c, &active, &guard, &limit, &reset};
    kp.func = reinterpret_cast<void*>(k_sweep_cond);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
}

cudaError_t launch_local_prolong(cudaStream_t st, int nsub, const SubDev* subs, const ProbDev* probs,
                                 const LocalState* ls, const double* cpool, double* F) {
    count_launch();
    k_local_prolong<<<nsub, NT, 0, st>>>(nsub, subs, probs, ls, cpool, F);
    return cudaGetLastError();
}

#define RAS_INSTANTIATE(T)                                                                                 \
    template cudaError_t launch_local_factor<T>(cudaStream_t, int, int, const SubDev*, const ProbDev*,       \
                                                const double*, LocalState*, const double*, double*, T*,      \
                                                int);                                                        \
    template cudaError_t launch_local_factor_big<T>(cudaStream_t, int, const int*, const SubDev*,            \
                                                    const ProbDev*, const double*, LocalState*, const double*, \
                                                    double*, T*, int);
RAS_INSTANTIATE(float)
RAS_INSTANTIATE(double)
#undef RAS_INSTANTIATE

}  // namespace ras
