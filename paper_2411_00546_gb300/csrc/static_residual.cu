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
// The array holds one FP64 partial sum of ||F||^2 per grid row, for at most
// RAS_STATIC_MAX_N rows (64 KiB). Every GPU that loads the library keeps it
// until the process exits. Host code must not pass the array's name to a
// kernel (on the host it is only a stand-in for the symbol); its device address
// is looked up with cudaGetSymbolAddress, with the caller's device current, on
// every call. The lookup allocates nothing, and doing it per call keeps the
// address right after a cudaDeviceReset or with another context current, where
// a cached address would dangle. The first call on a device may load the
// library's device code; make it before any stream capture.
#include "ras.h"
#include "ras_internal.cuh"

namespace {

constexpr int ROW_THREADS = 256;

// One partial sum of ||F||^2 per grid row.
static __device__ __align__(256) double g_row_partials[RAS_STATIC_MAX_N];

// Device address of g_row_partials in the current context.
cudaError_t partials_address(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_row_partials);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

__device__ __forceinline__ double at(const double* Z, int n, int i, int j) {
    return (i < 0 || i >= n || j < 0 || j >= n) ? 0.0 : Z[(long long)j * n + i];
}

// One CTA per grid row j: F at the row's nodes (the expression of the
// handle-based residual kernel, operation for operation) and the row's
// partial sum of ||F||^2.
__global__ void __launch_bounds__(ROW_THREADS) k_residual_rows(ras::ProbDev P, const double* __restrict__ y,
                                                               const double* __restrict__ p, double eps,
                                                               double* Fy, double* Fp, double* partials) {
    __shared__ double red[ROW_THREADS];
    const int n = P.n, j = blockIdx.x;
    const double beta = P.beta, imu = 1.0 / P.mu, munu = P.mu / P.nu;
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += ROW_THREADS) {
        const long long g = (long long)j * n + i;
        const double yc = y[g], yw = at(y, n, i - 1, j), ye = at(y, n, i + 1, j), ys = at(y, n, i, j - 1),
                     yn = at(y, n, i, j + 1);
        const double pc = p[g], pw = at(p, n, i - 1, j), pe = at(p, n, i + 1, j), ps = at(p, n, i, j - 1),
                     pn = at(p, n, i, j + 1);
        double ph, d1, d2;
        ras::phi_eval(P.phi, P.kappa, yc, ph, d1, d2);
        const double fv = P.f ? P.f[g] : 0.0;
        // -u = (mu/nu)(P_eps(x) - x), x = -p/mu (control of Sec. 3.2)
        const double dq = ras::P_eps_minus_id(-pc * imu, eps);
        const double Fyv = beta * (4.0 * yc - yw - ye - ys - yn) + ph - fv + munu * dq;
        const double Fpv = beta * (4.0 * pc - pw - pe - ps - pn) + d1 * pc - yc + P.yd[g];
        if (Fy) Fy[g] = Fyv;
        if (Fp) Fp[g] = Fpv;
        a += Fyv * Fyv + Fpv * Fpv;
    }
    a = ras::block_sum1<ROW_THREADS>(a, red);
    if (threadIdx.x == 0) partials[j] = a;
}

// norm[0] = sqrt(sum of the n row partials of ||F||^2), summed in row order.
__global__ void __launch_bounds__(ROW_THREADS) k_reduce_rows(const double* __restrict__ partials, int n,
                                                             double* norm) {
    __shared__ double red[ROW_THREADS];
    double a = 0.0;
    for (int j = threadIdx.x; j < n; j += ROW_THREADS) a += partials[j];
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
    P.nz = 1;
    P.nn = (long long)n * n;
    P.phi = phi;
    P.h = 1.0 / (n + 1);
    P.beta = 1.0 / (P.h * P.h);
    P.diag = 4.0 * P.beta;
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
