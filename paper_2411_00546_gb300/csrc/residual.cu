// Grid-wide kernels: the residual F(x, eps) of Sec. 3.3 on the whole grid,
// the Jacobian action F'(x, eps) v (Newton_RAS's Krylov operator), and the
// vector kernels of GMRES (multi-dot, multi-axpy, scaling). All reductions use
// a fixed grid (VEC_BLOCKS) and fixed trees, so results do not depend on
// scheduling.
#include "ras_internal.cuh"

namespace ras {

namespace {

constexpr int NT = VEC_THREADS;
constexpr int NB = VEC_BLOCKS;

__device__ __forceinline__ double gval(const double* Z, int n, int i, int j) {
    return (i < 0 || i >= n || j < 0 || j >= n) ? 0.0 : Z[(long long)j * n + i];
}

// F at x + alpha d (d may be null). Writes Fy/Fp when non-null; per-block
// partial sums of ||F||^2 into partials[blockIdx] and, with FLOOR, of the
// rounding-floor estimate (nodewise sums of |terms|) into
// partials[NB + blockIdx]. Block b takes the grid rows b, b + NB, ...; its
// threads take the nodes of a row, so no node index is divided.
template <bool FLOOR>
__global__ void __launch_bounds__(NT) k_residual_global(ProbDev P, const double* __restrict__ y,
                                                        const double* __restrict__ p,
                                                        const double* __restrict__ dy,
                                                        const double* __restrict__ dp, double alpha,
                                                        double eps, double* Fy, double* Fp,
                                                        double* partials) {
    __shared__ double red[2 * NT];
    const int n = P.n;
    const double beta = P.beta, inu = 1.0 / P.nu, mu = P.mu, imu = 1.0 / P.mu, munu = P.mu / P.nu;
    auto vy = [=](int i, int j) -> double {
        if (i < 0 || i >= n || j < 0 || j >= n) return 0.0;
        const long long g = (long long)j * n + i;
        return dy ? fma(alpha, dy[g], y[g]) : y[g];
    };
    auto vp = [=](int i, int j) -> double {
        if (i < 0 || i >= n || j < 0 || j >= n) return 0.0;
        const long long g = (long long)j * n + i;
        return dp ? fma(alpha, dp[g], p[g]) : p[g];
    };
    double a = 0.0, b = 0.0;
    for (int j = blockIdx.x; j < n; j += NB) {
        for (int i = threadIdx.x; i < n; i += NT) {
            const long long g = (long long)j * n + i;
            const double yc = vy(i, j), yw = vy(i - 1, j), ye = vy(i + 1, j), ys = vy(i, j - 1), yn = vy(i, j + 1);
            const double pc = vp(i, j), pw = vp(i - 1, j), pe = vp(i + 1, j), ps = vp(i, j - 1), pn = vp(i, j + 1);
            double ph, d1, d2;
            phi_eval(P.phi, P.kappa, yc, ph, d1, d2);
            const double fv = P.f ? P.f[g] : 0.0;
            // -u = (mu/nu)(P_eps(x) - x), x = -p/mu (control of Sec. 3.2)
            const double xq = -pc * imu;
            const double dq = P_eps_minus_id(xq, eps);
            const double Fyv = beta * (4.0 * yc - yw - ye - ys - yn) + ph - fv + munu * dq;
            const double Fpv = beta * (4.0 * pc - pw - pe - ps - pn) + d1 * pc - yc + P.yd[g];
            if (Fy) Fy[g] = Fyv;
            if (Fp) Fp[g] = Fpv;
            a += Fyv * Fyv + Fpv * Fpv;
            if (FLOOR) {
                const double My = beta * (4.0 * fabs(yc) + fabs(yw) + fabs(ye) + fabs(ys) + fabs(yn)) + fabs(ph) +
                                  fabs(fv) + inu * (fabs(pc) + mu * fabs(xq + dq));
                const double Mp = beta * (4.0 * fabs(pc) + fabs(pw) + fabs(pe) + fabs(ps) + fabs(pn)) +
                                  fabs(d1 * pc) + fabs(yc) + fabs(P.yd[g]);
                b += My * My + Mp * Mp;
            }
        }
    }
    block_sum2<NT>(a, b, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = a;
        partials[NB + blockIdx.x] = b;
    }
}

// The same on the cube (7-point stencil): block b takes the grid lines
// (j, k) with j + n k = b, b + NB, ...; its threads take the nodes of a line.
template <bool FLOOR>
__global__ void __launch_bounds__(NT) k_residual_global3(ProbDev P, const double* __restrict__ y,
                                                         const double* __restrict__ p,
                                                         const double* __restrict__ dy,
                                                         const double* __restrict__ dp, double alpha,
                                                         double eps, double* Fy, double* Fp,
                                                         double* partials) {
    __shared__ double red[2 * NT];
    const int n = P.n;
    const double beta = P.beta, inu = 1.0 / P.nu, mu = P.mu, imu = 1.0 / P.mu, munu = P.mu / P.nu;
    auto vy = [=](int i, int j, int k) -> double {
        if (i < 0 || i >= n || j < 0 || j >= n || k < 0 || k >= n) return 0.0;
        const long long g = ((long long)k * n + j) * n + i;
        return dy ? fma(alpha, dy[g], y[g]) : y[g];
    };
    auto vp = [=](int i, int j, int k) -> double {
        if (i < 0 || i >= n || j < 0 || j >= n || k < 0 || k >= n) return 0.0;
        const long long g = ((long long)k * n + j) * n + i;
        return dp ? fma(alpha, dp[g], p[g]) : p[g];
    };
    double a = 0.0, b = 0.0;
    for (int jr = blockIdx.x; jr < n * n; jr += NB) {
        const int j = jr % n, k = jr / n;
        for (int i = threadIdx.x; i < n; i += NT) {
            const long long g = ((long long)k * n + j) * n + i;
            const double yc = vy(i, j, k), pc = vp(i, j, k);
            const double yw = vy(i - 1, j, k), ye = vy(i + 1, j, k), ys = vy(i, j - 1, k), yn = vy(i, j + 1, k);
            const double yb = vy(i, j, k - 1), yt = vy(i, j, k + 1);
            const double pw = vp(i - 1, j, k), pe = vp(i + 1, j, k), ps = vp(i, j - 1, k), pn = vp(i, j + 1, k);
            const double pb = vp(i, j, k - 1), pt = vp(i, j, k + 1);
            double ph, d1, d2;
            phi_eval(P.phi, P.kappa, yc, ph, d1, d2);
            const double fv = P.f ? P.f[g] : 0.0;
            const double xq = -pc * imu;
            const double dq = P_eps_minus_id(xq, eps);
            const double Fyv = beta * (6.0 * yc - yw - ye - ys - yn - yb - yt) + ph - fv + munu * dq;
            const double Fpv = beta * (6.0 * pc - pw - pe - ps - pn - pb - pt) + d1 * pc - yc + P.yd[g];
            if (Fy) Fy[g] = Fyv;
            if (Fp) Fp[g] = Fpv;
            a += Fyv * Fyv + Fpv * Fpv;
            if (FLOOR) {
                const double My = beta * (6.0 * fabs(yc) + fabs(yw) + fabs(ye) + fabs(ys) + fabs(yn) + fabs(yb) +
                                          fabs(yt)) +
                                  fabs(ph) + fabs(fv) + inu * (fabs(pc) + mu * fabs(xq + dq));
                const double Mp = beta * (6.0 * fabs(pc) + fabs(pw) + fabs(pe) + fabs(ps) + fabs(pn) + fabs(pb) +
                                          fabs(pt)) +
                                  fabs(d1 * pc) + fabs(yc) + fabs(P.yd[g]);
                b += My * My + Mp * Mp;
            }
        }
    }
    block_sum2<NT>(a, b, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = a;
        partials[NB + blockIdx.x] = b;
    }
}

// out[v] = sum over the nparts partials of row v, in index order (one warp per row).
__global__ void k_reduce_partials(const double* __restrict__ partials, int nparts, int nvals,
                                  double* out) {
    const int v = blockIdx.x;
    if (v >= nvals) return;
    __shared__ double red[NT];
    double a = 0.0;
    for (int k = threadIdx.x; k < nparts; k += NT) a += partials[(long long)v * nparts + k];
    a = block_sum1<NT>(a, red);
    if (threadIdx.x == 0) out[v] = a;
}

// Jacobian coefficients at (x, eps): phi'(y), (1/nu)(1 - P_eps'(-p/mu)), phi''(y) p - 1.
__global__ void __launch_bounds__(NT) k_coef_global(ProbDev P, const double* __restrict__ y,
                                                    const double* __restrict__ p, double eps,
                                                    double* coef) {
    const long long nn = P.nn;
    const double inu = 1.0 / P.nu, mu = P.mu;
    for (long long g = (long long)blockIdx.x * NT + threadIdx.x; g < nn; g += (long long)NB * NT) {
        double ph, d1, d2;
        const double yv = y[g], pv = p[g];
        phi_eval(P.phi, P.kappa, yv, ph, d1, d2);
        coef[g] = d1;
        coef[nn + g] = inu * one_minus_dP_eps(-pv / mu, eps);
        coef[2 * nn + g] = d2 * pv - 1.0;
    }
}

// F'(x, eps) v with stored coefficients (Jacobian of Sec. 3.3).
__global__ void __launch_bounds__(NT) k_jacvec_global(ProbDev P, const double* __restrict__ coef,
                                                      const double* __restrict__ vy,
                                                      const double* __restrict__ vp, double* oy,
                                                      double* op) {
    const int n = P.n;
    const long long nn = P.nn, pl = (long long)n * n;
    const double beta = P.beta;
    const bool cube = P.nz > 1;
    for (long long g = (long long)blockIdx.x * NT + threadIdx.x; g < nn; g += (long long)NB * NT) {
        const long long gp = g % pl;
        const int i = (int)(gp % n), j = (int)(gp / n), k = (int)(g / pl);
        const double yc = vy[g], pc = vp[g];
        const double* wy = vy + (long long)k * pl;
        const double* wp = vp + (long long)k * pl;
        double sy = gval(wy, n, i - 1, j) + gval(wy, n, i + 1, j) + gval(wy, n, i, j - 1) + gval(wy, n, i, j + 1);
        double sp = gval(wp, n, i - 1, j) + gval(wp, n, i + 1, j) + gval(wp, n, i, j - 1) + gval(wp, n, i, j + 1);
        double dg = 4.0;
        if (cube) {
            dg = 6.0;
            if (k > 0) { sy += vy[g - pl]; sp += vp[g - pl]; }
            if (k < n - 1) { sy += vy[g + pl]; sp += vp[g + pl]; }
        }
        const double a = coef[g], b = coef[nn + g], c = coef[2 * nn + g];
        oy[g] = beta * (dg * yc - sy) + a * yc + b * pc;
        op[g] = beta * (dg * pc - sp) + c * yc + a * pc;
    }
}

// partials[v * NB + block] = partial dot of V_v (row v of V, stride ld) with w.
// Per-thread accumulators, then warp shuffles and one pass over the 8 warps'
// partials in warp order (fixed order: deterministic).
constexpr int MAXV = 32;
template <int NVC>
__global__ void __launch_bounds__(NT) k_dot_multi(const double* __restrict__ V, long long ld, int nv,
                                                  const double* __restrict__ w, long long len,
                                                  double* partials) {
    __shared__ double red[NT / 32][NVC];
    double acc[NVC];
#pragma unroll
    for (int v = 0; v < NVC; ++v) acc[v] = 0.0;
    for (long long g = (long long)blockIdx.x * NT + threadIdx.x; g < len; g += (long long)NB * NT) {
        const double wv = w[g];
#pragma unroll
        for (int v = 0; v < NVC; ++v) acc[v] += V[(long long)v * ld + g] * wv;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int v = 0; v < NVC; ++v) {
        double a = acc[v];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) red[warp][v] = a;
    }
    __syncthreads();
    if (threadIdx.x < NVC) {
        double a = 0.0;
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) a += red[k][threadIdx.x];
        partials[(long long)threadIdx.x * NB + blockIdx.x] = a;
    }
}

// w += sign * sum_v h[v] V_v
__global__ void __launch_bounds__(NT) k_axpy_multi(const double* __restrict__ V, long long ld, int nv,
                                                   const double* __restrict__ h, double sign, double* w,
                                                   long long len) {
    __shared__ double hs[MAXV];
    if (threadIdx.x < nv && threadIdx.x < MAXV) hs[threadIdx.x] = sign * h[threadIdx.x];
    __syncthreads();
    for (long long g = (long long)blockIdx.x * NT + threadIdx.x; g < len; g += (long long)NB * NT) {
        double acc = w[g];
        for (int v = 0; v < nv; ++v) acc += hs[v] * V[(long long)v * ld + g];
        w[g] = acc;
    }
}

// dst = sign * src * num / den (num, den: device scalars; null means 1).
__global__ void __launch_bounds__(NT) k_scale_copy(const double* src, const double* num,
                                                   const double* den, double sign, double* dst,
                                                   long long len) {
    double s = sign;
    if (num) s *= *num;
    if (den) s /= *den;
    for (long long g = (long long)blockIdx.x * NT + threadIdx.x; g < len; g += (long long)NB * NT)
        dst[g] = s * src[g];
}

__global__ void __launch_bounds__(NT) k_axpy(double a, const double* __restrict__ x, double* y,
                                             long long len) {
    for (long long g = (long long)blockIdx.x * NT + threadIdx.x; g < len; g += (long long)NB * NT)
        y[g] = fma(a, x[g], y[g]);
}

// out = fma(alpha, d, x): the same rounding as the trial point of the residual kernel.
__global__ void __launch_bounds__(NT) k_add_scaled(const double* x, const double* d,
                                                   double alpha, double* out, long long len) {
    for (long long g = (long long)blockIdx.x * NT + threadIdx.x; g < len; g += (long long)NB * NT)
        out[g] = fma(alpha, d[g], x[g]);
}


// ------------------------------------------------------------------ segmented
// 1-D grid over a SegGrid table: block b works on problem tab[b].x, as its
// tab[b].y-th of nbps blocks, grid-striding over that problem's segment.
// Reductions use fixed trees and a fixed block order (deterministic for a
// given table).
__host__ __device__ constexpr int pow2_ceil(int v) { return v <= 1 ? 1 : 2 * pow2_ceil((v + 1) / 2); }

template <int NVC>
__global__ void __launch_bounds__(NT) k_seg_dot(SegGrid sg_, const Seg* __restrict__ segs,
                                                const double* __restrict__ V, long long ld,
                                                const double* __restrict__ w, double* partials) {
    constexpr int P = pow2_ceil(NVC);   // values per lane, padded with zeros
    __shared__ double red[NT / 32][NVC];
    const int2 e = sg_.tab[blockIdx.x];
    if (e.x < 0) return;
    const int pb = e.x, bi = e.y, nb = sg_.nbps[pb];
    const Seg sg = segs[pb];
    double acc[P];
#pragma unroll
    for (int v = 0; v < P; ++v) acc[v] = 0.0;
    for (long long g = (long long)bi * NT + threadIdx.x; g < sg.len; g += (long long)nb * NT) {
        const long long x = sg.ofs + g;
        const double wv = w[x];
#pragma unroll
        for (int v = 0; v < NVC; ++v) acc[v] += V[(long long)v * ld + x] * wv;
    }
    // Warp sums of the P values by a transposing butterfly: at offset s each
    // lane keeps one half of its remaining values (the upper half when
    // lane & s) and adds the partner's copy of that half, so the FP64 adds
    // per lane are P - 1 (plus one per remaining level) instead of 5 P.
    // Lane l then holds value vi(l) summed over the lanes that share its
    // bits below the last transposing offset.
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int vi = 0;
    int s = 16;
#pragma unroll
    for (int cnt = P; cnt > 1; cnt >>= 1) {
        const int half = cnt >> 1;
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const double send = up ? acc[k] : acc[k + half];
            const double keep = up ? acc[k + half] : acc[k];
            acc[k] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
        if (up) vi += half;
        s >>= 1;
    }
    double a = acc[0];
    for (int off = s; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if ((lane & ((32 / P) - 1)) == 0 && vi < NVC) red[warp][vi] = a;
    __syncthreads();
    if (threadIdx.x < NVC) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) t += red[k][threadIdx.x];
        partials[((long long)pb * SEG_STRIDE + threadIdx.x) * VEC_BLOCKS + bi] = t;
    }
}

// out[p*32 + v] = sum over the nbps[p] partials of (p, v), in block order.
__global__ void k_seg_reduce(const int* __restrict__ nbps, const double* __restrict__ partials, double* out) {
    const int v = blockIdx.x, pb = blockIdx.y;
    const int nb = nbps[pb];
    if (nb == 0) return;
    __shared__ double red[NT];
    double a = 0.0;
    for (int k = threadIdx.x; k < nb; k += NT) a += partials[((long long)pb * SEG_STRIDE + v) * VEC_BLOCKS + k];
    a = block_sum1<NT>(a, red);
    if (threadIdx.x == 0) out[pb * SEG_STRIDE + v] = a;
}

// w += sign * sum_v h[p*32 + v] V_v on each segment.
__global__ void __launch_bounds__(NT) k_seg_axpy(SegGrid sg_, const Seg* __restrict__ segs,
                                                 const double* __restrict__ V, long long ld, int nv,
                                                 const double* __restrict__ h, double sign, double* w) {
    __shared__ double hs[SEG_STRIDE];
    const int2 e = sg_.tab[blockIdx.x];
    if (e.x < 0) return;
    const int pb = e.x, bi = e.y, nb = sg_.nbps[pb];
    if (threadIdx.x < nv) hs[threadIdx.x] = sign * h[pb * SEG_STRIDE + threadIdx.x];
    __syncthreads();
    const Seg sg = segs[pb];
    for (long long g = (long long)bi * NT + threadIdx.x; g < sg.len; g += (long long)nb * NT) {
        const long long x = sg.ofs + g;
        double acc = w[x];
        for (int v = 0; v < nv; ++v) acc += hs[v] * V[(long long)v * ld + x];
        w[x] = acc;
    }
}

// dst = sign * src / sqrt(n2[p*32]) (n2 null: dst = sign * src) on each segment.
__global__ void __launch_bounds__(NT) k_seg_scale(SegGrid sg_, const Seg* __restrict__ segs, const double* src,
                                                  const double* __restrict__ n2, double sign, double* dst) {
    const int2 e = sg_.tab[blockIdx.x];
    if (e.x < 0) return;
    const int pb = e.x, bi = e.y, nb = sg_.nbps[pb];
    const double s = n2 ? sign / sqrt(n2[pb * SEG_STRIDE]) : sign;
    const Seg sg = segs[pb];
    for (long long g = (long long)bi * NT + threadIdx.x; g < sg.len; g += (long long)nb * NT)
        dst[sg.ofs + g] = s * src[sg.ofs + g];
}

// out = fma(alpha, d, x) on each segment.
__global__ void __launch_bounds__(NT) k_seg_add_scaled(SegGrid sg_, const Seg* __restrict__ segs, const double* x,
                                                       const double* d, double alpha, double* out) {
    const int2 e = sg_.tab[blockIdx.x];
    const int pb = e.x, bi = e.y, nb = sg_.nbps[pb];
    const Seg sg = segs[pb];
    for (long long g = (long long)bi * NT + threadIdx.x; g < sg.len; g += (long long)nb * NT)
        out[sg.ofs + g] = fma(alpha, d[sg.ofs + g], x[sg.ofs + g]);
}

// One Arnoldi step's Hessenberg column, Givens rotation and stop test per
// problem (see launch_gmres_givens); the same operations in the same order
// as the textbook GMRES least-squares update.
__global__ void __launch_bounds__(NT) k_gmres_givens(int nprob, int m, int j, int* act, const double* h1,
                                                     const double* h2, const double* n2, double* H, double* cs,
                                                     double* sn, double* g, int* its, int* steps,
                                                     const double* target, int maxit, int* any_out) {
    int any = 0;
    for (int p = threadIdx.x; p < nprob; p += NT) {
        if (!act[p]) continue;
        double* Hp = H + (long long)p * (m + 1) * m;
        double* csp = cs + (long long)p * m;
        double* snp = sn + (long long)p * m;
        double* gp = g + (long long)p * (m + 1);
        for (int i = 0; i <= j; ++i) Hp[i * m + j] = h1[p * SEG_STRIDE + i] + h2[p * SEG_STRIDE + i];
        const double hn = sqrt(n2[p * SEG_STRIDE]);
        Hp[(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
            const double t = csp[i] * Hp[i * m + j] + snp[i] * Hp[(i + 1) * m + j];
            Hp[(i + 1) * m + j] = -snp[i] * Hp[i * m + j] + csp[i] * Hp[(i + 1) * m + j];
            Hp[i * m + j] = t;
        }
        const double den = hypot(Hp[j * m + j], Hp[(j + 1) * m + j]);
        csp[j] = Hp[j * m + j] / den;
        snp[j] = Hp[(j + 1) * m + j] / den;
        Hp[j * m + j] = den;
        Hp[(j + 1) * m + j] = 0.0;
        gp[j + 1] = -snp[j] * gp[j];
        gp[j] = csp[j] * gp[j];
        its[p] += 1;
        steps[p] = j + 1;
        if (hn == 0.0 || fabs(gp[j + 1]) <= target[p] || its[p] >= maxit) act[p] = 0;
        else any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) *any_out = any;
}

__global__ void __launch_bounds__(NT) k_seg_table(int nprob, const int* act, const Seg* segs, int vb, int cap,
                                                  int2* tab, int* nbps, int* offs) {
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int p = 0; p < nprob; ++p)
            if (act[p]) tot += (double)segs[p].len;
        int o = 0;
        for (int p = 0; p < nprob; ++p) {
            int nb = 0;
            if (act[p]) {
                const double len = (double)segs[p].len;
                const int most = (int)fmax(1.0, ceil(len / 512.0));
                nb = (int)floor(vb * len / tot + 0.5);
                nb = max(1, min(nb, min(most, vb)));
            }
            nbps[p] = nb;
            offs[p] = o;
            o += nb;
        }
        offs[nprob] = o;
    }
    __syncthreads();
    const int used = offs[nprob];
    for (int b = threadIdx.x; b < cap; b += NT) {
        if (b >= used) {
            tab[b] = make_int2(-1, 0);
            continue;
        }
        int lo = 0, hi = nprob - 1;   // the problem p with offs[p] <= b < offs[p + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offs[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        tab[b] = make_int2(lo, b - offs[lo]);
    }
}

__global__ void k_set_conditional(cudaGraphConditionalHandle c, const int* any) {
    cudaGraphSetConditional(c, *any ? 1u : 0u);
}

}  // namespace

cudaError_t launch_seg_table(cudaStream_t st, int nprob, const int* act, const Seg* segs, int vec_blocks, int cap,
                             int2* tab, int* nbps, int* offs) {
    count_launch();
    k_seg_table<<<1, NT, 0, st>>>(nprob, act, segs, vec_blocks, cap, tab, nbps, offs);
    return cudaGetLastError();
}

cudaError_t launch_gmres_givens(cudaStream_t st, int nprob, int m, int j, int* act, const double* h1,
                                const double* h2, const double* n2, double* H, double* cs, double* sn, double* g,
                                int* its, int* steps, const double* target, int maxit, int* any) {
    count_launch();
    k_gmres_givens<<<1, NT, 0, st>>>(nprob, m, j, act, h1, h2, n2, H, cs, sn, g, its, steps, target, maxit, any);
    return cudaGetLastError();
}

cudaError_t add_set_conditional_node(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle c,
                                     const int* any, cudaGraphNode_t* out) {
    cudaKernelNodeParams kp{};
    void* args[] = {&c, &any};
    kp.func = reinterpret_cast<void*>(k_set_conditional);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
}

cudaError_t launch_seg_dot(cudaStream_t st, SegGrid g, const Seg* segs, const double* V, long long ld, int nv,
                           const double* w, double* partials) {
    if (g.nblocks == 0) return cudaSuccess;
    count_launch();
    switch (nv) {
#define RAS_SEG_CASE(K) \
    case K: k_seg_dot<K><<<g.nblocks, NT, 0, st>>>(g, segs, V, ld, w, partials); break;
        RAS_SEG_CASE(1) RAS_SEG_CASE(2) RAS_SEG_CASE(3) RAS_SEG_CASE(4) RAS_SEG_CASE(5) RAS_SEG_CASE(6)
        RAS_SEG_CASE(7) RAS_SEG_CASE(8) RAS_SEG_CASE(9) RAS_SEG_CASE(10) RAS_SEG_CASE(11) RAS_SEG_CASE(12)
        RAS_SEG_CASE(13) RAS_SEG_CASE(14) RAS_SEG_CASE(15) RAS_SEG_CASE(16) RAS_SEG_CASE(17) RAS_SEG_CASE(18)
        RAS_SEG_CASE(19) RAS_SEG_CASE(20) RAS_SEG_CASE(21) RAS_SEG_CASE(22) RAS_SEG_CASE(23) RAS_SEG_CASE(24)
        RAS_SEG_CASE(25) RAS_SEG_CASE(26) RAS_SEG_CASE(27) RAS_SEG_CASE(28) RAS_SEG_CASE(29) RAS_SEG_CASE(30)
        RAS_SEG_CASE(31) RAS_SEG_CASE(32)
#undef RAS_SEG_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_seg_reduce(cudaStream_t st, int nprob, const int* nbps, int nv, const double* partials,
                              double* out) {
    if (nv < 1 || nv > SEG_STRIDE) return cudaErrorInvalidValue;
    count_launch();
    k_seg_reduce<<<dim3(nv, nprob), NT, 0, st>>>(nbps, partials, out);
    return cudaGetLastError();
}

cudaError_t launch_seg_axpy(cudaStream_t st, SegGrid g, const Seg* segs, const double* V, long long ld, int nv,
                            const double* h, double sign, double* w) {
    if (nv < 1 || nv > SEG_STRIDE) return cudaErrorInvalidValue;
    if (g.nblocks == 0) return cudaSuccess;
    count_launch();
    k_seg_axpy<<<g.nblocks, NT, 0, st>>>(g, segs, V, ld, nv, h, sign, w);
    return cudaGetLastError();
}

cudaError_t launch_seg_scale(cudaStream_t st, SegGrid g, const Seg* segs, const double* src, const double* n2,
                             double sign, double* dst) {
    if (g.nblocks == 0) return cudaSuccess;
    count_launch();
    k_seg_scale<<<g.nblocks, NT, 0, st>>>(g, segs, src, n2, sign, dst);
    return cudaGetLastError();
}

cudaError_t launch_seg_add_scaled(cudaStream_t st, SegGrid g, const Seg* segs, const double* x, const double* d,
                                  double alpha, double* out) {
    if (g.nblocks == 0) return cudaSuccess;
    count_launch();
    k_seg_add_scaled<<<g.nblocks, NT, 0, st>>>(g, segs, x, d, alpha, out);
    return cudaGetLastError();
}

cudaError_t launch_residual_global(cudaStream_t st, const ProbDev& P, const double* y, const double* p,
                                   const double* dy, const double* dp, double alpha, double eps,
                                   double* Fy, double* Fp, double* partials, int floor) {
    count_launch();
    if (P.nz > 1) {
        if (floor)
            k_residual_global3<true><<<NB, NT, 0, st>>>(P, y, p, dy, dp, alpha, eps, Fy, Fp, partials);
        else
            k_residual_global3<false><<<NB, NT, 0, st>>>(P, y, p, dy, dp, alpha, eps, Fy, Fp, partials);
    } else if (floor) {
        k_residual_global<true><<<NB, NT, 0, st>>>(P, y, p, dy, dp, alpha, eps, Fy, Fp, partials);
    } else {
        k_residual_global<false><<<NB, NT, 0, st>>>(P, y, p, dy, dp, alpha, eps, Fy, Fp, partials);
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(cudaStream_t st, const double* partials, int nparts, int nvals,
                                   double* out) {
    count_launch();
    k_reduce_partials<<<nvals, NT, 0, st>>>(partials, nparts, nvals, out);
    return cudaGetLastError();
}

cudaError_t launch_coef_global(cudaStream_t st, const ProbDev& P, const double* y, const double* p,
                               double eps, double* coef) {
    count_launch();
    k_coef_global<<<NB, NT, 0, st>>>(P, y, p, eps, coef);
    return cudaGetLastError();
}

cudaError_t launch_jacvec_global(cudaStream_t st, const ProbDev& P, const double* coef,
                                 const double* vy, const double* vp, double* oy, double* op) {
    count_launch();
    k_jacvec_global<<<NB, NT, 0, st>>>(P, coef, vy, vp, oy, op);
    return cudaGetLastError();
}

cudaError_t launch_dot_multi(cudaStream_t st, const double* V, long long ld, int nv, const double* w,
                             long long len, double* partials) {
    if (nv > MAXV || nv < 1) return cudaErrorInvalidValue;
    count_launch();
    // one instantiation per count: every issued FP64 FMA is a useful one (the
    // FP64 pipe, not HBM, bounds this kernel on GB300)
    switch (nv) {
#define RAS_DOT_CASE(K) \
    case K: k_dot_multi<K><<<NB, NT, 0, st>>>(V, ld, nv, w, len, partials); break;
        RAS_DOT_CASE(1) RAS_DOT_CASE(2) RAS_DOT_CASE(3) RAS_DOT_CASE(4) RAS_DOT_CASE(5) RAS_DOT_CASE(6)
        RAS_DOT_CASE(7) RAS_DOT_CASE(8) RAS_DOT_CASE(9) RAS_DOT_CASE(10) RAS_DOT_CASE(11) RAS_DOT_CASE(12)
        RAS_DOT_CASE(13) RAS_DOT_CASE(14) RAS_DOT_CASE(15) RAS_DOT_CASE(16) RAS_DOT_CASE(17) RAS_DOT_CASE(18)
        RAS_DOT_CASE(19) RAS_DOT_CASE(20) RAS_DOT_CASE(21) RAS_DOT_CASE(22) RAS_DOT_CASE(23) RAS_DOT_CASE(24)
        RAS_DOT_CASE(25) RAS_DOT_CASE(26) RAS_DOT_CASE(27) RAS_DOT_CASE(28) RAS_DOT_CASE(29) RAS_DOT_CASE(30)
        RAS_DOT_CASE(31) RAS_DOT_CASE(32)
#undef RAS_DOT_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_axpy_multi(cudaStream_t st, const double* V, long long ld, int nv, const double* h,
                              double sign, double* w, long long len) {
    if (nv > MAXV || nv < 1) return cudaErrorInvalidValue;
    count_launch();
    k_axpy_multi<<<NB, NT, 0, st>>>(V, ld, nv, h, sign, w, len);
    return cudaGetLastError();
}

cudaError_t launch_scale_copy(cudaStream_t st, const double* src, const double* num, const double* den,
                              double sign, double* dst, long long len) {
    count_launch();
    k_scale_copy<<<NB, NT, 0, st>>>(src, num, den, sign, dst, len);
    return cudaGetLastError();
}

cudaError_t launch_axpy(cudaStream_t st, double a, const double* x, double* y, long long len) {
    count_launch();
    k_axpy<<<NB, NT, 0, st>>>(a, x, y, len);
    return cudaGetLastError();
}

cudaError_t launch_add_scaled(cudaStream_t st, const double* x, const double* d, double alpha,
                              double* out, long long len) {
    count_launch();
    k_add_scaled<<<NB, NT, 0, st>>>(x, d, alpha, out, len);
    return cudaGetLastError();
}

}  // namespace ras
