// Handle-free residual entry point that allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc or cudaFree, for example
// code that runs while another allocator (a framework's caching allocator or a
// pre-reserved memory pool) owns all of the device memory, or a latency-bound
// loop in which a cudaMalloc/cudaFree (which can synchronise the device) is not
// acceptable. ras_create allocates its buffers, so such callers cannot use the
// handle-based ras_residual; this variant computes the same F(x, eps) and its
// norm with the norm's partial sums kept in a fixed array that is part of the
// loaded library.
//
// The array holds two FP64 partial sums per grid row, for at most
// RAS_STATIC_MAX_N rows (128 KiB). Every GPU that loads the library keeps it
// until the process exits. Host code must not pass the array's name to a
// kernel (on the host it is only a stand-in for the symbol); its device address
// is fetched once per device with cudaGetSymbolAddress, the first time this
// entry point runs on that device with that device current.
#include <mutex>

#include "ras.h"
#include "ras_internal.cuh"

namespace {

constexpr int ROW_THREADS = 256;
constexpr int MAX_DEVICES = 64;

// Two partial sums (||F||^2 and the rounding-floor estimate) per grid row.
static __device__ __align__(256) double g_row_partials[2 * RAS_STATIC_MAX_N];

std::mutex g_setup_mu;
double* g_partials_dev[MAX_DEVICES] = {};

// Device address of g_row_partials on the current device (set up once).
cudaError_t partials_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_partials_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_row_partials);
        if (e != cudaSuccess) return e;
        g_partials_dev[dev] = static_cast<double*>(p);
    }
    *out = g_partials_dev[dev];
    return cudaSuccess;
}

__device__ __forceinline__ double at(const double* Z, int n, int i, int j) {
    return (i < 0 || i >= n || j < 0 || j >= n) ? 0.0 : Z[(long long)j * n + i];
}

// One CTA per grid row j: F at the row's nodes (same expression as the
// handle-based residual kernel) and the row's two partial sums.
__global__ void __launch_bounds__(ROW_THREADS) k_residual_rows(ras::ProbDev P, const double* __restrict__ y,
                                                               const double* __restrict__ p, double eps,
                                                               double* Fy, double* Fp, double* partials) {
    __shared__ double red[2 * ROW_THREADS];
    const int n = P.n, j = blockIdx.x;
    const double beta = P.beta, inu = 1.0 / P.nu, mu = P.mu;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += ROW_THREADS) {
        const long long g = (long long)j * n + i;
        const double yc = y[g], yw = at(y, n, i - 1, j), ye = at(y, n, i + 1, j), ys = at(y, n, i, j - 1),
                     yn = at(y, n, i, j + 1);
        const double pc = p[g], pw = at(p, n, i - 1, j), pe = at(p, n, i + 1, j), ps = at(p, n, i, j - 1),
                     pn = at(p, n, i, j + 1);
        double ph, d1, d2;
        ras::phi_eval(P.phi, P.kappa, yc, ph, d1, d2);
        const double fv = P.f ? P.f[g] : 0.0;
        const double pe_ = ras::P_eps(-pc / mu, eps);
        const double Fyv = beta * (4.0 * yc - yw - ye - ys - yn) + ph - fv + inu * (pc + mu * pe_);
        const double Fpv = beta * (4.0 * pc - pw - pe - ps - pn) + d1 * pc - yc + P.yd[g];
        const double My = beta * (4.0 * fabs(yc) + fabs(yw) + fabs(ye) + fabs(ys) + fabs(yn)) + fabs(ph) +
                          fabs(fv) + inu * (fabs(pc) + mu * fabs(pe_));
        const double Mp = beta * (4.0 * fabs(pc) + fabs(pw) + fabs(pe) + fabs(ps) + fabs(pn)) +
                          fabs(d1 * pc) + fabs(yc) + fabs(P.yd[g]);
        if (Fy) Fy[g] = Fyv;
        if (Fp) Fp[g] = Fpv;
        a += Fyv * Fyv + Fpv * Fpv;
        b += My * My + Mp * Mp;
    }
    ras::block_sum2<ROW_THREADS>(a, b, red);
    if (threadIdx.x == 0) {
        partials[2 * j] = a;
        partials[2 * j + 1] = b;
    }
}

// norm[0] = sqrt(sum of the n row partials of ||F||^2), summed in row order.
__global__ void __launch_bounds__(ROW_THREADS) k_reduce_rows(const double* __restrict__ partials, int n,
                                                             double* norm) {
    __shared__ double red[ROW_THREADS];
    double a = 0.0;
    for (int j = threadIdx.x; j < n; j += ROW_THREADS) a += partials[2 * j];
    a = ras::block_sum1<ROW_THREADS>(a, red);
    if (threadIdx.x == 0) norm[0] = sqrt(a);
}

}  // namespace

extern "C" int ras_residual_static(int n, int phi, double nu, double mu, double kappa, double eps,
                                   const double* y, const double* p, const double* y_d, const double* f,
                                   double* Fy, double* Fp, double* norm_dev, void* stream) {
    if (n < 2 || n > RAS_STATIC_MAX_N || phi < 0 || phi > 2 || !(nu > 0) || !(mu > 0) || !(eps > 0) || !y ||
        !p || !y_d)
        return RAS_EINVAL;
    double* partials = nullptr;
    if (partials_address(&partials) != cudaSuccess) return RAS_ECUDA;
    ras::ProbDev P{};
    P.n = n;
    P.phi = phi;
    P.h = 1.0 / (n + 1);
    P.beta = 1.0 / (P.h * P.h);
    P.nu = nu;
    P.mu = mu;
    P.kappa = kappa;
    P.yd = y_d;
    P.f = f;
    P.ofs = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ras::count_launch();
    k_residual_rows<<<n, ROW_THREADS, 0, st>>>(P, y, p, eps, Fy, Fp, partials);
    if (cudaGetLastError() != cudaSuccess) return RAS_ECUDA;
    if (norm_dev) {
        ras::count_launch();
        k_reduce_rows<<<1, ROW_THREADS, 0, st>>>(partials, n, norm_dev);
        if (cudaGetLastError() != cudaSuccess) return RAS_ECUDA;
    }
    return RAS_OK;
}
