// Local block-tridiagonal solves J_i z = b with the stored factors G_j:
//   w_0 = b_0, w_j = b_j + beta G_{j-1} w_{j-1};
//   z_{W-1} = G_{W-1} w_{W-1},  z_j = G_j (w_j + beta z_{j+1}),
// used by the Newton direction of the local solves (Alg. 1 inside Alg. 3),
// the Jacobian action of the RASPEN function (Alg. 4) and the linear RAS
// preconditioner. One CTA (256 threads) per subdomain.
//
// The solve is a chain of 2W-1 dependent matrix-vector products; each reads
// one mp x mp block (100 KB in FP32 at mp = 160) that does not depend on the
// chain. The blocks are therefore streamed ahead of the chain: every block is
// stored as mp/32 contiguous slabs (packed_index), and a ring of D slab
// buffers in shared memory (as many as fit in RING_BYTES) is filled by TMA
// bulk copies (cp.async.bulk, completion on an mbarrier) issued D slabs ahead
// of the slab being used.
// Thread t = 8 rho + kappa multiplies its own contiguous part of a slab (row
// rho + 32 s, column chunk kappa) with the vector and the 8 partial sums of a
// row are added with warp shuffles. Every mbarrier wait is bounded; on timeout
// the CTA waits (bounded) for its copies in flight, records ST_ETIMEOUT in
// *err and returns.
#include <stdint.h>

#include <algorithm>

#include "ras_internal.cuh"

namespace ras {

namespace {

constexpr int NT = LOC_THREADS;
static_assert(NT == 256, "packed layout assumes 256 threads");
static_assert(MAX_M <= NT, "one entry of a block row per thread");
constexpr long long WAIT_LIMIT = 1LL << 22;   // try_wait rounds before giving up

// The slab ring: RING_BYTES of shared memory split into as many slab slots as
// fit for the block size at hand (at most MAXD), so narrow blocks keep more
// slabs in flight. Two CTAs fit on an SM.
template <typename T>
struct Ring {
    static constexpr int RING_BYTES = 80 * 1024;
    static constexpr int MAXD = 16;
    static constexpr int SLAB_MAX = 256 * ((MAX_M / 8) / (16 / (int)sizeof(T))) * 16;  // bytes
    static_assert(RING_BYTES >= 2 * SLAB_MAX, "at least two slabs in flight");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arm `bar` for `bytes` and copy them from global `src` to shared `dst`.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait for phase `parity` of `bar` (at most `limit` polls); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = WAIT_LIMIT) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <typename T>
__device__ __forceinline__ T shfl_x(T v, int m) {
    return __shfl_xor_sync(0xffffffffu, v, m);
}

// Shared state of one CTA's slab stream. Every solve uses slots 0..D-1 round
// robin and consumes every slab it issues, so between solves all slots are
// idle and D may change; `phase` (uniform over the CTA) holds the parity that
// each slot's mbarrier completes next.
template <typename T>
struct Stream {
    unsigned char* ring;   // RING_BYTES of slab slots
    uint64_t* full;        // MAXD mbarriers
    int* fail;             // shared flag
    uint32_t phase;        // bit k: parity of slot k's next completion
};

template <typename T>
__device__ void stream_init(Stream<T>& S, unsigned char* smem) {
    constexpr int MD = Ring<T>::MAXD;
    S.ring = smem;
    S.full = reinterpret_cast<uint64_t*>(smem + Ring<T>::RING_BYTES);
    S.fail = reinterpret_cast<int*>(S.full + MD);
    S.phase = 0u;
    if (threadIdx.x == 0) {
        for (int k = 0; k < MD; ++k) mbar_init(&S.full[k], 1);
        *S.fail = 0;
        fence_barrier_init();
    }
    __syncthreads();
}

// On a timeout: wait (bounded) for the copies still in flight (relative
// slabs first .. last-1, slab `first` in slot k0 of a ring of D), then report.
template <typename T>
__device__ void stream_abort(Stream<T>& S, uint32_t first, uint32_t last, uint32_t k0, uint32_t D, int* err) {
    if (threadIdx.x == 0) {
        uint32_t k = k0;
        for (uint32_t q = first; q < last; ++q, k = (k + 1 == D) ? 0u : k + 1)
            mbar_wait(&S.full[k], (S.phase >> k) & 1u);
        if (err) atomicExch(err, ST_ETIMEOUT);
    }
    __syncthreads();
}

// z = J_i^-1 b (see the file comment). rhs(j, t) -> T gives b; pre(j, t) ->
// double loads what out needs besides z; out(j, t, z, pre) consumes z. rhs,
// pre and the read-back of w are called one block row ahead, so their global
// loads overlap the streamed products instead of stalling every row.
// vec, tmp: shared arrays of mp T. w: global scratch, m*W T. m <= NT: thread
// t handles entry t of every block row. Returns false if a wait timed out
// (the CTA must then return). err[0] is the timeout flag; err[1] != 0 is the
// timeout test of ras_opts.wait_test: the first slab wait of the solve then
// polls zero times, so it runs out with its copy still in flight, and the
// copies issued so far are drained with the normal limit before the return.
template <typename T, class Rhs, class Pre, class Out>
__device__ bool stream_solve(Stream<T>& S, const T* __restrict__ G, int m, int mp, int W, T beta, T* w, T* vec,
                             T* tmp, Rhs rhs, Pre pre, Out out, int* err) {
    constexpr int VE = 16 / (int)sizeof(T);
    const int tid = threadIdx.x, kappa = tid & 7, rho = tid >> 3;
    const int cw = mp >> 3, nv = cw / VE, nslab = mp >> 5;
    const uint32_t slab_elems = 256u * nv * VE;
    const uint32_t slab_bytes = slab_elems * sizeof(T);
    const uint32_t D = min((uint32_t)Ring<T>::MAXD, (uint32_t)Ring<T>::RING_BYTES / slab_bytes);
    const long long blk = (long long)mp * mp;
    const uint32_t total = (uint32_t)((2 * W - 1) * nslab);
    const bool first_zero = err && err[1] != 0;
    // slab q of this solve: forward blocks 0..W-2, then backward W-1..0
    auto src = [&](uint32_t q) -> const T* {
        const int f = (W - 1) * nslab;
        int jb, sl;
        if ((int)q < f) {
            jb = q / nslab;
            sl = q % nslab;
        } else {
            const int r = q - f;
            jb = W - 1 - r / nslab;
            sl = r % nslab;
        }
        return G + jb * blk + (long long)sl * slab_elems;
    };
    if (tid == 0) {
        fence_proxy_async();
        for (uint32_t q = 0; q < total && q < D; ++q)
            tma_load_1d(S.ring + q * slab_bytes, src(q), slab_bytes, &S.full[q]);
    }
    uint32_t q = 0, k = 0;   // slab q of this solve sits in slot k = q mod D
    // one mp x mp product from the stream: tmp = G_(next block) vec
    auto matvec = [&]() -> bool {
        for (int sl = 0; sl < nslab; ++sl, ++q, k = (k + 1 == D) ? 0u : k + 1) {
            const bool ok = mbar_wait(&S.full[k], (S.phase >> k) & 1u, (q == 0 && first_zero) ? 0 : WAIT_LIMIT);
            const T* slot = reinterpret_cast<const T*>(S.ring + k * slab_bytes);
            T acc = (T)0;
            if (ok) {
                const T* vk = vec + kappa * cw;
                for (int v = 0; v < nv; ++v) {
                    const T* gv = slot + ((long long)v * 256 + tid) * VE;
#pragma unroll
                    for (int l = 0; l < VE; ++l) acc += gv[l] * vk[v * VE + l];
                }
            }
            if (__syncthreads_or(!ok)) {
                // copies issued so far: relative slabs < min(total, q + D)
                stream_abort(S, q, min(total, q + D), k, D, err);
                return false;
            }
            S.phase ^= 1u << k;
            if (tid == 0 && q + D < total) {
                fence_proxy_async();
                tma_load_1d(S.ring + k * slab_bytes, src(q + D), slab_bytes, &S.full[k]);
            }
            acc += shfl_x(acc, 1);
            acc += shfl_x(acc, 2);
            acc += shfl_x(acc, 4);
            if (kappa == 0) tmp[rho + 32 * sl] = acc;
        }
        __syncthreads();
        return true;
    };
    for (int t = m + tid; t < mp; t += NT) vec[t] = (T)0;
    const bool mine = tid < m;
    T nb = mine ? rhs(0, tid) : (T)0;   // b of the next block row
    for (int j = 0; j < W; ++j) {
        if (mine) {
            T v = nb;
            if (j > 0) v += beta * tmp[tid];
            vec[tid] = v;
            w[j * m + tid] = v;
            if (j + 1 < W) nb = rhs(j + 1, tid);
        }
        __syncthreads();
        if (j < W - 1 && !matvec()) return false;
    }
    T nw = mine ? w[(W - 1) * m + tid] : (T)0;   // w and pre of the next block row (backward)
    double np_ = mine ? pre(W - 1, tid) : 0.0;
    for (int j = W - 1; j >= 0; --j) {
        double cur = 0.0;
        if (mine) {
            T v = nw;
            if (j < W - 1) v += beta * tmp[tid];
            vec[tid] = v;
            cur = np_;
            if (j > 0) {
                nw = w[(j - 1) * m + tid];
                np_ = pre(j - 1, tid);
            }
        }
        __syncthreads();
        if (!matvec()) return false;
        if (mine) out(j, tid, tmp[tid], cur);
    }
    __syncthreads();
    return true;
}

template <typename T>
size_t solve_smem() {
    return (size_t)Ring<T>::RING_BYTES + Ring<T>::MAXD * sizeof(uint64_t) + 16;
}

// Persistent work distribution of the solve kernels: every CTA takes the next
// position of `order` (subdomain indices, largest factors first) from a
// ticket counter that the launcher zeroes, until the list is exhausted.
__device__ __forceinline__ int next_position(int* ticket, int* slot) {
    __syncthreads();   // every thread is done with the previous subdomain
    if (threadIdx.x == 0) *slot = atomicAdd(ticket, 1);
    __syncthreads();
    return *slot;
}

// The same solve for a wide block (MAX_M < m <= MAX_MW = 2 NT) with the
// factor blocks stored column-major (element (r, c) of G_j at c*mp + r).
// Every product reads its block as chunks of whole columns (CB columns, at
// most WSLOT bytes), copied by TMA bulk copies (cp.async.bulk) into a ring of
// WNS shared-memory slots; thread 0 keeps WNS chunks in flight across block
// boundaries (the products run through blocks 0 .. W-2, then W-1 .. 0), and
// thread t adds the chunk's columns times vec into rows t and t + NT. Every
// wait is bounded; on a timeout the copies in flight are waited for (bounded)
// and the solve returns false with ST_ETIMEOUT in *err. err[1] != 0 makes the
// first wait poll zero times (the timeout test of ras_opts.wait_test). rhs,
// pre and out as in stream_solve.
constexpr int WNS = 6;                       // ring slots of the wide solves
constexpr uint32_t WSLOT = 32 * 1024;        // bytes per slot
template <typename T>
size_t wide_solve_smem() {
    return (size_t)WNS * WSLOT + WNS * sizeof(uint64_t) + 16;
}

template <typename T>
__device__ void wide_stream_init(Stream<T>& S, unsigned char* smem) {
    S.ring = smem;
    S.full = reinterpret_cast<uint64_t*>(smem + (size_t)WNS * WSLOT);
    S.fail = reinterpret_cast<int*>(S.full + WNS);
    S.phase = 0u;
    if (threadIdx.x == 0) {
        for (int k = 0; k < WNS; ++k) mbar_init(&S.full[k], 1);
        *S.fail = 0;
        fence_barrier_init();
    }
    __syncthreads();
}

template <typename T, class Rhs, class Pre, class Out>
__device__ bool wide_solve(Stream<T>& S, const T* __restrict__ G, int m, int mp, int W, T beta, T* w, T* vec,
                           T* tmp, Rhs rhs, Pre pre, Out out, int* err) {
    const int r0 = threadIdx.x, r1 = threadIdx.x + NT;
    const bool h0 = r0 < m, h1 = r1 < m;
    const long long blk = (long long)mp * mp;
    const uint32_t colb = (uint32_t)mp * (uint32_t)sizeof(T);   // a multiple of 128 bytes
    const int CB = (int)(WSLOT / colb);                          // >= 1: mp <= MAX_MW
    const int nch = (m + CB - 1) / CB;
    const uint32_t total = (uint32_t)((2 * W - 1) * nch);
    const bool first_zero = err && err[1] != 0;
    auto issue = [&](uint32_t x) {   // chunk x of the sequence into slot x % WNS (thread 0)
        const int v = (int)(x / (uint32_t)nch), ch = (int)(x % (uint32_t)nch);
        const int jb = (v < W - 1) ? v : 2 * W - 2 - v;
        const int c0 = ch * CB, nc = min(CB, m - c0);
        const uint32_t k = x % WNS;
        fence_proxy_async();
        tma_load_1d(S.ring + (size_t)k * WSLOT, G + (long long)jb * blk + (long long)c0 * mp, (uint32_t)nc * colb,
                    &S.full[k]);
    };
    if (threadIdx.x == 0)
        for (uint32_t x = 0; x < (uint32_t)WNS && x < total; ++x) issue(x);
    uint32_t q = 0;   // next chunk to consume
    auto matvec = [&]() -> bool {   // tmp = G_(next block) vec
        T a0 = (T)0, a1 = (T)0;
        for (int ch = 0; ch < nch; ++ch, ++q) {
            const uint32_t k = q % WNS;
            const bool ok = mbar_wait(&S.full[k], (S.phase >> k) & 1u, (q == 0 && first_zero) ? 0 : WAIT_LIMIT);
            if (__syncthreads_or(!ok)) {
                // drain the copies issued and not consumed (chunks q .. q + WNS - 1), then report
                if (threadIdx.x == 0) {
                    for (uint32_t x = q; x < total && x < q + WNS; ++x) {
                        const uint32_t kx = x % WNS;
                        mbar_wait(&S.full[kx], (S.phase >> kx) & 1u);
                    }
                    if (err) atomicExch(err, ST_ETIMEOUT);
                }
                __syncthreads();
                return false;
            }
            S.phase ^= 1u << k;
            const T* cols = reinterpret_cast<const T*>(S.ring + (size_t)k * WSLOT);
            const int c0 = ch * CB, nc = min(CB, m - c0);
            for (int cc = 0; cc < nc; ++cc) {
                const T v = vec[c0 + cc];
                const T* col = cols + cc * mp;
                if (h0) a0 = fma(col[r0], v, a0);
                if (h1) a1 = fma(col[r1], v, a1);
            }
            __syncthreads();   // slot k read by every thread
            if (threadIdx.x == 0 && q + WNS < total) issue(q + WNS);
        }
        if (h0) tmp[r0] = a0;
        if (h1) tmp[r1] = a1;
        __syncthreads();
        return true;
    };
    for (int j = 0; j < W; ++j) {
        if (h0) {
            T v = rhs(j, r0);
            if (j > 0) v += beta * tmp[r0];
            vec[r0] = v;
            w[j * m + r0] = v;
        }
        if (h1) {
            T v = rhs(j, r1);
            if (j > 0) v += beta * tmp[r1];
            vec[r1] = v;
            w[j * m + r1] = v;
        }
        __syncthreads();
        if (j < W - 1 && !matvec()) return false;
    }
    for (int j = W - 1; j >= 0; --j) {
        if (h0) vec[r0] = w[j * m + r0] + ((j < W - 1) ? beta * tmp[r0] : (T)0);
        if (h1) vec[r1] = w[j * m + r1] + ((j < W - 1) ? beta * tmp[r1] : (T)0);
        __syncthreads();
        if (!matvec()) return false;
        if (h0) out(j, r0, tmp[r0], pre(j, r0));
        if (h1) out(j, r1, tmp[r1], pre(j, r1));
    }
    __syncthreads();
    return true;
}

// One local solve: the slab stream (narrow blocks) or the column-chunk stream (wide blocks).
template <typename T, bool WIDE, class Rhs, class Pre, class Out>
__device__ __forceinline__ bool local_solve(Stream<T>& S, const T* G, int m, int mp, int W, T beta, T* w, T* vec,
                                            T* tmp, Rhs rhs, Pre pre, Out out, int* err) {
    if constexpr (WIDE) {
        return wide_solve<T>(S, G, m, mp, W, beta, w, vec, tmp, rhs, pre, out, err);
    } else {
        return stream_solve<T>(S, G, m, mp, W, beta, w, vec, tmp, rhs, pre, out, err);
    }
}

// Subdomain position of a solve kernel: the persistent kernels take the next
// ticket; the wide-block ones run one CTA per listed subdomain.
template <bool WIDE>
__device__ __forceinline__ int solve_position(int it, int* ticket, int* slot) {
    if constexpr (WIDE) {
        return it == 0 ? (int)blockIdx.x : 0x7fffffff;
    } else {
        return next_position(ticket, slot);
    }
}

// r = bsign * B - J_i z in FP64 with the Jacobian coefficients stored by the
// factor kernel (the stencil's coupling inside Omega_i only; diag = 4 beta on
// the square, 6 beta on the cube); returns ||r||^2.
__device__ double local_linear_residual(const SubDev& s, double beta, double diag, const double* coef,
                                        double bsign, const double* B, const double* z, double* r,
                                        double* red) {
    const int wx = s.wx, wy = s.wy, wz = s.wz, nn = wx * wy * wz, pl = wx * wy;
    const double* ca = s.cptr;
    const double* cb = ca + nn;
    const double* cc = cb + nn;
    double r2 = 0.0, dummy = 0.0;
    for (int q = threadIdx.x; q < nn; q += NT) {
        const int lx = q % wx, rq = q / wx, ly = rq % wy, lz = rq / wy;
        const double zyc = z[2 * q], zpc = z[2 * q + 1];
        double sy = 0.0, sp = 0.0;
        if (lx > 0) { sy += z[2 * (q - 1)]; sp += z[2 * (q - 1) + 1]; }
        if (lx < wx - 1) { sy += z[2 * (q + 1)]; sp += z[2 * (q + 1) + 1]; }
        if (ly > 0) { sy += z[2 * (q - wx)]; sp += z[2 * (q - wx) + 1]; }
        if (ly < wy - 1) { sy += z[2 * (q + wx)]; sp += z[2 * (q + wx) + 1]; }
        if (lz > 0) { sy += z[2 * (q - pl)]; sp += z[2 * (q - pl) + 1]; }
        if (lz < wz - 1) { sy += z[2 * (q + pl)]; sp += z[2 * (q + pl) + 1]; }
        const double Jy = beta * (diag * zyc - sy) + ca[q] * zyc + cb[q] * zpc;
        const double Jp = beta * (diag * zpc - sp) + cc[q] * zyc + ca[q] * zpc;
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
template <typename T, bool WIDE>
__global__ void __launch_bounds__(NT) k_local_direction(int nsub, const SubDev* __restrict__ subs,
                                                        const ProbDev* __restrict__ probs, LocalState* ls,
                                                        NewtonParams np, const double* coef, const T* gpool,
                                                        const double* Kpool, double* dpool, double* rpool,
                                                        T* wpool, int* err, const int* order, int* ticket) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) T vec[WIDE ? MAX_MW : MAX_M];
    __shared__ __align__(16) T tmp[WIDE ? MAX_MW : MAX_M];
    __shared__ double red[2 * NT];
    __shared__ int sh_next;
    Stream<T> S;
    if constexpr (WIDE) wide_stream_init(S, smem);
    else stream_init(S, smem);
    for (int it = 0;; ++it) {
    const int pos = solve_position<WIDE>(it, ticket, &sh_next);
    if (pos >= nsub) break;
    const int i = order[pos];
    if (!ls[i].active) continue;
    const SubDev s = subs[i];
    if (!WIDE && s.mp > MAX_M) continue;
    const ProbDev P = probs[s.prob];
    const int m = 2 * s.bl, W = s.bw, L = m * W;
    const double beta = P.beta, sdiag = P.nz > 1 ? 6.0 : 4.0;
    const double* K = Kpool + s.voff;
    double* d = dpool + s.voff;
    double* r = rpool + s.voff;
    T* w = wpool + s.voff;
    const T* G = static_cast<const T*>(s.gptr);
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
        if (!local_solve<T, WIDE>(
                S, G, m, s.mp, W, (T)beta, w, vec, tmp, [=](int j, int t) { return (T)r[j * m + t]; },
                [=](int j, int t) { return d[j * m + t]; },
                [=](int j, int t, T z, double old) { d[j * m + t] = old + (double)z; }, err)) {
            if (threadIdx.x == 0) {
                ls[i].status = ST_ETIMEOUT;
                ls[i].active = 0;
            }
            return;
        }
        if (it >= np.ir_max) break;
        const double r2 = local_linear_residual(s, beta, sdiag, coef, -1.0, K, d, r, red);
        if (sqrt(r2) <= np.ir_rtol * bnorm) break;
    }
    if (threadIdx.x == 0) ls[i].solves += nsolves;
    }
}

// Jacobian action of the RASPEN function (Alg. 4):
//   O = -D - sum_i tilde P_i J_i(x^(i))^-1 B_i D,  B_i D = R_i A (I - P_i R_i) D,
// i.e. b = -beta * (sum of D over the stencil neighbours outside Omega_i).
// With nir > 0 (mixed precision) the local solve is refined nir times in FP64:
// z += J^-1 (b - J z), J from the coefficients at x^(i).
template <typename T, bool WIDE>
__global__ void __launch_bounds__(NT) k_local_jvp(int nsub, const SubDev* __restrict__ subs,
                                                  const ProbDev* __restrict__ probs, const T* gpool, T* wpool,
                                                  const double* coef, double* zpool, double* rpool,
                                                  double* bpool, int nir, const double* D, double* O,
                                                  const int* pmask, int* err, const int* order, int* ticket) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) T vec[WIDE ? MAX_MW : MAX_M];
    __shared__ __align__(16) T tmp[WIDE ? MAX_MW : MAX_M];
    __shared__ double red[2 * NT];
    __shared__ int sh_next;
    Stream<T> S;
    if constexpr (WIDE) wide_stream_init(S, smem);
    else stream_init(S, smem);
    for (int it = 0;; ++it) {
    const int pos = solve_position<WIDE>(it, ticket, &sh_next);
    if (pos >= nsub) break;
    const int i = order[pos];
    const SubDev s = subs[i];
    if (pmask && !pmask[s.prob]) continue;
    if (!WIDE && s.mp > MAX_M) continue;
    const ProbDev P = probs[s.prob];
    const int n = P.n, nz = P.nz, m = 2 * s.bl, W = s.bw;
    const long long nn = P.nn;
    const double beta = P.beta, sdiag = P.nz > 1 ? 6.0 : 4.0;
    const double* Dy = D + P.ofs;
    double* Oy = O + P.ofs;
    const T* G = static_cast<const T*>(s.gptr);
    T* w = wpool + s.voff;
    // local entry (j, t) is node q = j*bl + t/2 of the box, field t & 1
    auto bval = [=](int j, int t) -> double {
        const int f = t & 1;
        int lx, ly, lz;
        local_coords(s, j * s.bl + (t >> 1), lx, ly, lz);
        const int gx = s.x0 + lx, gy = s.y0 + ly, gz = s.z0 + lz;
        const double* Df = Dy + f * nn;
        double b = 0.0;
        if (lx == 0 && gx > 0) b += Df[grid_index(P, gx - 1, gy, gz)];
        if (lx == s.wx - 1 && gx < n - 1) b += Df[grid_index(P, gx + 1, gy, gz)];
        if (ly == 0 && gy > 0) b += Df[grid_index(P, gx, gy - 1, gz)];
        if (ly == s.wy - 1 && gy < n - 1) b += Df[grid_index(P, gx, gy + 1, gz)];
        if (lz == 0 && gz > 0) b += Df[grid_index(P, gx, gy, gz - 1)];
        if (lz == s.wz - 1 && gz < nz - 1) b += Df[grid_index(P, gx, gy, gz + 1)];
        return -beta * b;
    };
    // owned node of local entry (j, t): its global index, else -1
    auto owned = [=](int j, int t) -> long long {
        const int f = t & 1;
        int lx, ly, lz;
        local_coords(s, j * s.bl + (t >> 1), lx, ly, lz);
        const int gx = s.x0 + lx, gy = s.y0 + ly, gz = s.z0 + lz;
        if (gx >= s.ox0 && gx < s.ox0 + s.owx && gy >= s.oy0 && gy < s.oy0 + s.owy && gz >= s.oz0 &&
            gz < s.oz0 + s.owz)
            return f * nn + grid_index(P, gx, gy, gz);
        return -1;
    };
    auto owned_out = [=](int j, int t, double z) {
        const long long g = owned(j, t);
        if (g >= 0) Oy[g] = -Dy[g] - z;
    };
    if (nir == 0) {
        if (!local_solve<T, WIDE>(
                S, G, m, s.mp, W, (T)beta, w, vec, tmp, [=](int j, int t) { return (T)bval(j, t); },
                [=](int j, int t) {
                    const long long g = owned(j, t);
                    return g >= 0 ? -Dy[g] : 0.0;
                },
                [=](int j, int t, T z, double mdy) {
                    const long long g = owned(j, t);
                    if (g >= 0) Oy[g] = mdy - (double)z;
                },
                err))
            return;
        continue;
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
    if (!local_solve<T, WIDE>(
            S, G, m, s.mp, W, (T)beta, w, vec, tmp, [=](int j, int t) { return (T)b[j * m + t]; },
            [=](int, int) { return 0.0; }, [=](int j, int t, T zz, double) { z[j * m + t] = (double)zz; }, err))
        return;
    for (int it = 0; it < nir; ++it) {
        local_linear_residual(s, beta, sdiag, coef, 1.0, b, z, r, red);
        if (!local_solve<T, WIDE>(
                S, G, m, s.mp, W, (T)beta, w, vec, tmp, [=](int j, int t) { return (T)r[j * m + t]; },
                [=](int j, int t) { return z[j * m + t]; },
                [=](int j, int t, T zz, double old) { z[j * m + t] = old + (double)zz; }, err))
            return;
    }
    for (int q = threadIdx.x; q < L; q += NT) owned_out(q / m, q % m, z[q]);
    }
}

// Linear RAS preconditioner: Z = sum_i tilde P_i J_i^-1 R_i R.
template <typename T, bool WIDE>
__global__ void __launch_bounds__(NT) k_local_precond(int nsub, const SubDev* __restrict__ subs,
                                                      const ProbDev* __restrict__ probs, const T* gpool,
                                                      T* wpool, const double* R, double* Z, int* err,
                                                      const int* order, int* ticket) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) T vec[WIDE ? MAX_MW : MAX_M];
    __shared__ __align__(16) T tmp[WIDE ? MAX_MW : MAX_M];
    __shared__ int sh_next;
    Stream<T> S;
    if constexpr (WIDE) wide_stream_init(S, smem);
    else stream_init(S, smem);
    for (int it = 0;; ++it) {
    const int pos = solve_position<WIDE>(it, ticket, &sh_next);
    if (pos >= nsub) break;
    const int i = order[pos];
    const SubDev s = subs[i];
    if (!WIDE && s.mp > MAX_M) continue;
    const ProbDev P = probs[s.prob];
    const int m = 2 * s.bl, W = s.bw;
    const long long nn = P.nn;
    const double* Ry = R + P.ofs;
    double* Zy = Z + P.ofs;
    auto rhs = [=](int j, int t) -> T {
        const int f = t & 1;
        int lx, ly, lz;
        local_coords(s, j * s.bl + (t >> 1), lx, ly, lz);
        return (T)Ry[f * nn + grid_index(P, s.x0 + lx, s.y0 + ly, s.z0 + lz)];
    };
    auto out = [=](int j, int t, T z, double) {
        const int f = t & 1;
        int lx, ly, lz;
        local_coords(s, j * s.bl + (t >> 1), lx, ly, lz);
        const int gx = s.x0 + lx, gy = s.y0 + ly, gz = s.z0 + lz;
        if (gx >= s.ox0 && gx < s.ox0 + s.owx && gy >= s.oy0 && gy < s.oy0 + s.owy && gz >= s.oz0 &&
            gz < s.oz0 + s.owz)
            Zy[f * nn + grid_index(P, gx, gy, gz)] = (double)z;
    };
    if (!local_solve<T, WIDE>(S, static_cast<const T*>(s.gptr), m, s.mp, W, (T)P.beta, wpool + s.voff, vec, tmp, rhs,
                         [=](int, int) { return 0.0; }, out, err))
        return;
    }
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Grid of a persistent solve kernel: as many CTAs as fit on the device at
// once, at most one per subdomain; the ticket is zeroed on the stream first.
template <class K>
cudaError_t persistent_grid(K kernel, size_t smem, int nsub, int ctas_per_sm, cudaStream_t st, int* ticket,
                            int& grid) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, per_sm);
    if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
    grid = std::max(1, std::min(nsub, per_sm * sms));
    return cudaSuccess;
}

}  // namespace

template <typename T>
cudaError_t launch_local_direction(cudaStream_t st, int nsub, int ctas_per_sm, const SubDev* subs,
                                   const ProbDev* probs, LocalState* ls, NewtonParams np,
                                   const double* coef, const T* gpool, const double* Kpool,
                                   double* dpool, double* rpool, T* wpool, int* err, const int* order,
                                   int* ticket) {
    const size_t sm = solve_smem<T>();
    cudaError_t e = set_smem(k_local_direction<T, false>, sm);
    int grid = 0;
    if (e == cudaSuccess) e = persistent_grid(k_local_direction<T, false>, sm, nsub, ctas_per_sm, st, ticket, grid);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_direction<T, false><<<grid, NT, sm, st>>>(nsub, subs, probs, ls, np, coef, gpool, Kpool, dpool, rpool,
                                               wpool, err, order, ticket);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_jvp(cudaStream_t st, int nsub, int ctas_per_sm, const SubDev* subs,
                             const ProbDev* probs, const T* gpool, T* wpool, const double* coef,
                             double* zpool, double* rpool, double* bpool, int nir, const double* D,
                             double* O, const int* pmask, int* err, const int* order, int* ticket) {
    const size_t sm = solve_smem<T>();
    cudaError_t e = set_smem(k_local_jvp<T, false>, sm);
    int grid = 0;
    if (e == cudaSuccess) e = persistent_grid(k_local_jvp<T, false>, sm, nsub, ctas_per_sm, st, ticket, grid);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_jvp<T, false><<<grid, NT, sm, st>>>(nsub, subs, probs, gpool, wpool, coef, zpool, rpool, bpool, nir, D, O,
                                         pmask, err, order, ticket);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_precond(cudaStream_t st, int nsub, int ctas_per_sm, const SubDev* subs,
                                 const ProbDev* probs, const T* gpool, T* wpool, const double* R,
                                 double* Z, int* err, const int* order, int* ticket) {
    const size_t sm = solve_smem<T>();
    cudaError_t e = set_smem(k_local_precond<T, false>, sm);
    int grid = 0;
    if (e == cudaSuccess) e = persistent_grid(k_local_precond<T, false>, sm, nsub, ctas_per_sm, st, ticket, grid);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_precond<T, false><<<grid, NT, sm, st>>>(nsub, subs, probs, gpool, wpool, R, Z, err, order, ticket);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_direction_wide(cudaStream_t st, int count, const int* list, const SubDev* subs,
                                        const ProbDev* probs, LocalState* ls, NewtonParams np,
                                        const double* coef, const T* gpool, const double* Kpool, double* dpool,
                                        double* rpool, T* wpool, int* err) {
    if (count <= 0) return cudaSuccess;
    const size_t sm = wide_solve_smem<T>();
    cudaError_t e = set_smem(k_local_direction<T, true>, sm);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_direction<T, true><<<count, NT, sm, st>>>(count, subs, probs, ls, np, coef, gpool, Kpool, dpool, rpool,
                                                     wpool, err, list, nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_jvp_wide(cudaStream_t st, int count, const int* list, const SubDev* subs,
                                  const ProbDev* probs, const T* gpool, T* wpool, const double* coef,
                                  double* zpool, double* rpool, double* bpool, int nir, const double* D, double* O,
                                  const int* pmask, int* err) {
    if (count <= 0) return cudaSuccess;
    const size_t sm = wide_solve_smem<T>();
    cudaError_t e = set_smem(k_local_jvp<T, true>, sm);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_jvp<T, true><<<count, NT, sm, st>>>(count, subs, probs, gpool, wpool, coef, zpool, rpool, bpool, nir, D,
                                               O, pmask, err, list, nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_local_precond_wide(cudaStream_t st, int count, const int* list, const SubDev* subs,
                                      const ProbDev* probs, const T* gpool, T* wpool, const double* R, double* Z,
                                      int* err) {
    if (count <= 0) return cudaSuccess;
    const size_t sm = wide_solve_smem<T>();
    cudaError_t e = set_smem(k_local_precond<T, true>, sm);
    if (e != cudaSuccess) return e;
    count_launch();
    k_local_precond<T, true><<<count, NT, sm, st>>>(count, subs, probs, gpool, wpool, R, Z, err, list, nullptr);
    return cudaGetLastError();
}

// CTAs of the local-solve kernels that fit on one SM (FP32 or FP64 factors).
cudaError_t solve_ctas_per_sm_max(bool f32, int* per_sm) {
    *per_sm = 0;
    if (f32) {
        cudaError_t e = set_smem(k_local_precond<float, false>, solve_smem<float>());
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_local_precond<float, false>, NT, solve_smem<float>());
    }
    cudaError_t e = set_smem(k_local_precond<double, false>, solve_smem<double>());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_local_precond<double, false>, NT, solve_smem<double>());
}

#define RAS_INSTANTIATE(T)                                                                              \
    template cudaError_t launch_local_direction<T>(cudaStream_t, int, int, const SubDev*, const ProbDev*, \
                                                   LocalState*, NewtonParams, const double*, const T*,    \
                                                   const double*, double*, double*, T*, int*, const int*, \
                                                   int*);                                                 \
    template cudaError_t launch_local_jvp<T>(cudaStream_t, int, int, const SubDev*, const ProbDev*, const T*,  \
                                             T*, const double*, double*, double*, double*, int,                \
                                             const double*, double*, const int*, int*, const int*, int*);      \
    template cudaError_t launch_local_precond<T>(cudaStream_t, int, int, const SubDev*, const ProbDev*,        \
                                                 const T*, T*, const double*, double*, int*, const int*, int*);  \
    template cudaError_t launch_local_direction_wide<T>(cudaStream_t, int, const int*, const SubDev*,         \
                                                        const ProbDev*, LocalState*, NewtonParams,             \
                                                        const double*, const T*, const double*, double*,       \
                                                        double*, T*, int*);                                    \
    template cudaError_t launch_local_jvp_wide<T>(cudaStream_t, int, const int*, const SubDev*, const ProbDev*, \
                                                  const T*, T*, const double*, double*, double*, double*, int, \
                                                  const double*, double*, const int*, int*);                   \
    template cudaError_t launch_local_precond_wide<T>(cudaStream_t, int, const int*, const SubDev*,           \
                                                      const ProbDev*, const T*, T*, const double*, double*,    \
                                                      int*);
RAS_INSTANTIATE(float)
RAS_INSTANTIATE(double)
#undef RAS_INSTANTIATE

}  // namespace ras
