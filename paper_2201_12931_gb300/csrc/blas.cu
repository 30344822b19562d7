// Vector kernels of the CG loop (Algorithm 1: dots, alpha/beta, x/r/p updates;
// all on the device, no host round trip per iteration) and the dense direct
// solve on the coarsest grid (Algorithm 3 "Solve the problem directly"):
// blocked right-looking Cholesky K_c = L L^T, explicit W = L^-1, and per
// application u = W^T (W r) as two triangular matrix-vector products.
// Reductions use a fixed grid of kRedBlocks blocks and a fixed-order second
// pass, so results are bitwise reproducible run to run.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace topo {

namespace {

constexpr int TB = 32;   // dense tile

inline unsigned grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 2147483647LL) b = 2147483647LL;
    return (unsigned)(b < 1 ? 1 : b);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

template <typename A, typename B>
__global__ void __launch_bounds__(256) k_dot(long long n, const A* __restrict__ a, const B* __restrict__ b,
                                             double* __restrict__ partials) {
    __shared__ double sh[32];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += (double)a[i] * (double)b[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__device__ __forceinline__ double sum_partials(const double* __restrict__ p, int n, double* sh) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
    return block_sum(s, sh);
}

__global__ void __launch_bounds__(1024) k_reduce_to(const double* __restrict__ p, int n, double* dst) {
    __shared__ double sh[32];
    const double s = sum_partials(p, n, sh);
    if (threadIdx.x == 0) *dst = s;
}

__global__ void __launch_bounds__(1024) k_cg_alpha(const double* __restrict__ p, int n, Scalars* sc,
                                                   double* __restrict__ hist) {
    __shared__ double sh[32];
    const double pq = sum_partials(p, n, sh);
    if (threadIdx.x == 0) {
        sc->pq = pq;
        if (pq > 0.0 && isfinite(pq) && isfinite(sc->rz)) {
            sc->alpha = sc->rz / pq;
        } else {
            sc->alpha = 0.0;
            sc->aux = 1.0;   // breakdown flag, read by the host
        }
        if (hist) *hist = sc->alpha;
    }
}

__global__ void __launch_bounds__(1024) k_cg_beta(const double* __restrict__ p, int n, Scalars* sc) {
    __shared__ double sh[32];
    const double rz = sum_partials(p, n, sh);
    if (threadIdx.x == 0) {
        const double old = sc->rz;
        sc->rz_old = old;
        sc->rz_new = rz;
        sc->beta = (old != 0.0 && isfinite(rz)) ? rz / old : 0.0;
        if (!isfinite(rz)) sc->aux = 1.0;
        sc->rz = rz;
    }
}

__global__ void __launch_bounds__(1024) k_cg_beta_flexible(const double* __restrict__ p, int n, Scalars* sc) {
    __shared__ double sh[32];
    const double zq = sum_partials(p, n, sh);
    if (threadIdx.x == 0) {
        const double old = sc->rz_old;
        sc->beta = (old != 0.0 && isfinite(zq)) ? -sc->alpha * zq / old : 0.0;
        if (!isfinite(zq)) sc->aux = 1.0;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_update_xr(long long n, const Scalars* __restrict__ sc, const T* __restrict__ p,
                                                   const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r,
                                                   double* __restrict__ partials) {
    __shared__ double sh[32];
    const T a = (T)sc->alpha;
    double s = 0.0;
    long long i0 = 0;
    if constexpr (std::is_same<T, float>::value) {
        // 128-bit accesses; r.r (used only for the stopping test) as FP32
        // sums of 4 squares added in FP64: one FP64 add per 4 entries
        // instead of a conversion and an FP64 FMA per entry
        const long long n4 = n / 4;
        const float4* p4 = reinterpret_cast<const float4*>(p);
        const float4* q4 = reinterpret_cast<const float4*>(q);
        float4* x4 = reinterpret_cast<float4*>(x);
        float4* r4 = reinterpret_cast<float4*>(r);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
             i += (long long)gridDim.x * blockDim.x) {
            const float4 pv = p4[i], qv = q4[i];
            float4 xv = x4[i], rv = r4[i];
            xv.x += a * pv.x;
            xv.y += a * pv.y;
            xv.z += a * pv.z;
            xv.w += a * pv.w;
            rv.x -= a * qv.x;
            rv.y -= a * qv.y;
            rv.z -= a * qv.z;
            rv.w -= a * qv.w;
            x4[i] = xv;
            r4[i] = rv;
            s += (double)(rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
        }
        i0 = 4 * n4;
    }
    for (long long i = i0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        x[i] += a * p[i];
        const T ri = r[i] - a * q[i];
        r[i] = ri;
        s += (double)ri * (double)ri;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// r -= alpha q and per-block partial sums of r.r (as k_update_xr without x)
template <typename T>
__global__ void __launch_bounds__(256) k_update_r(long long n, const Scalars* __restrict__ sc, const T* __restrict__ q,
                                                  T* __restrict__ r, double* __restrict__ partials) {
    __shared__ double sh[32];
    const T a = (T)sc->alpha;
    double s = 0.0;
    long long i0 = 0;
    if constexpr (std::is_same<T, float>::value) {
        const long long n4 = n / 4;
        const float4* q4 = reinterpret_cast<const float4*>(q);
        float4* r4 = reinterpret_cast<float4*>(r);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
             i += (long long)gridDim.x * blockDim.x) {
            const float4 qv = q4[i];
            float4 rv = r4[i];
            rv.x -= a * qv.x;
            rv.y -= a * qv.y;
            rv.z -= a * qv.z;
            rv.w -= a * qv.w;
            r4[i] = rv;
            s += (double)(rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
        }
        i0 = 4 * n4;
    }
    for (long long i = i0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const T ri = r[i] - a * q[i];
        r[i] = ri;
        s += (double)ri * (double)ri;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// x += alpha_j p_j, j = 0 .. count-1 in order: per entry the same fused
// multiply-adds as count successive x += alpha p updates, with x read and
// written once
template <typename T>
struct DirRing {
    const T* p[kDirRing];
};
template <typename T>
__global__ void __launch_bounds__(256) k_flush_x(long long n, DirRing<T> ring, const double* __restrict__ alpha,
                                                 int count, T* __restrict__ x) {
    T a[kDirRing];
#pragma unroll
    for (int j = 0; j < kDirRing; ++j) a[j] = j < count ? (T)alpha[j] : T(0);
    long long i0 = 0;
    if constexpr (std::is_same<T, float>::value) {
        const long long n4 = n / 4;
        float4* x4 = reinterpret_cast<float4*>(x);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
             i += (long long)gridDim.x * blockDim.x) {
            float4 xv = x4[i];
#pragma unroll
            for (int j = 0; j < kDirRing; ++j) {
                if (j < count) {
                    const float4 pv = reinterpret_cast<const float4*>(ring.p[j])[i];
                    xv.x += a[j] * pv.x;
                    xv.y += a[j] * pv.y;
                    xv.z += a[j] * pv.z;
                    xv.w += a[j] * pv.w;
                }
            }
            x4[i] = xv;
        }
        i0 = 4 * n4;
    }
    for (long long i = i0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T xi = x[i];
#pragma unroll
        for (int j = 0; j < kDirRing; ++j)
            if (j < count) xi += a[j] * ring.p[j][i];
        x[i] = xi;
    }
}

template <typename T>
__global__ void k_update_p(long long n, const Scalars* __restrict__ sc, const T* __restrict__ z, T* __restrict__ p) {
    const T b = (T)sc->beta;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = z[i] + b * p[i];
}

template <typename S, typename D>
__global__ void k_convert(long long n, const S* __restrict__ s, D* __restrict__ d) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = (D)s[i];
}

__global__ void k_fill(long long n, double* __restrict__ v, double value) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = value;
}

__global__ void k_axpy_f32(long long n, const float* __restrict__ d, double* __restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

// ---- dense coarse solve --------------------------------------------------

// The dense coarse factorization is a chain of small steps, and FP64
// arithmetic runs on a narrow pipe (1/64 of the FP32 rate on this GPU): the
// kernels below spread each step's FP64 work over as many SMs as it allows,
// in strips of kStrip rows (or columns) of a 32 x 32 tile per CTA of 128
// threads, instead of one tile per CTA.
constexpr int kStrip = 4;

// Cholesky of diagonal block kb by one CTA of 128 threads (right-looking, in
// shared memory; the pivot by one thread: rs = rsqrt(d), L_jj = d rs), then
// L_kk^-1 by forward elimination (row j of X = B_j / L_jj, then
// B_i -= L_ij X_j for the rows below).  L goes back to the block (zeros above
// the diagonal), L_kk^-1 to Dk (block kb: TB x TB row-major at Dk + kb TB^2).
// A non-positive or non-finite pivot sets info to its row + 1 (first one
// wins) and continues with pivot 1.
__global__ void __launch_bounds__(128) k_potrf_diag(double* __restrict__ A, int npad, int kb, int* info,
                                                    double* __restrict__ Dk) {
    __shared__ double sA[TB][TB + 1];
    __shared__ double sX[TB][TB + 1];
    __shared__ double sR[TB];
    const int tid = threadIdx.x;
    const long long base = (long long)kb * TB;
    for (int e = tid; e < TB * TB; e += 128) {
        const int r = e / TB, c = e % TB;
        sA[r][c] = A[(base + r) * npad + base + c];
        sX[r][c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < TB; ++j) {
        if (tid == 0) {
            double d = sA[j][j];
            if (!(d > 0.0) || !isfinite(d)) {
                atomicCAS(info, 0, (int)(base + j) + 1);
                d = 1.0;
            }
            const double rs = rsqrt(d);
            sA[j][j] = d * rs;
            sR[j] = rs;
        }
        __syncthreads();
        if (tid > j && tid < TB) sA[tid][j] *= sR[j];
        __syncthreads();
        for (int e = (j + 1) * TB + tid; e < TB * TB; e += 128) {   // rows below j only
            const int i = e / TB, k = e % TB;
            if (k > j && k <= i) sA[i][k] -= sA[i][j] * sA[k][j];
        }
        __syncthreads();
    }
    for (int j = 0; j < TB; ++j) {
        if (tid <= j) sX[j][tid] *= sR[j];
        __syncthreads();
        for (int e = (j + 1) * TB + tid; e < TB * TB; e += 128) {   // rows below j only
            const int i = e / TB, c = e % TB;
            if (c <= j) sX[i][c] -= sA[i][j] * sX[j][c];
        }
        __syncthreads();
    }
    double* D = Dk + base * TB;
    for (int e = tid; e < TB * TB; e += 128) {
        const int r = e / TB, c = e % TB;
        A[(base + r) * npad + base + c] = (c <= r) ? sA[r][c] : 0.0;
        D[e] = sX[r][c];
    }
}

// L_ib,kb = A_ib,kb L_kk^-T: block row ib = kb+1+blockIdx.y, its rows
// kStrip*blockIdx.x .. +kStrip (threads: 32 columns x kStrip rows)
__global__ void __launch_bounds__(128) k_trsm_panel(double* __restrict__ A, int npad, int kb,
                                                    const double* __restrict__ Dk) {
    __shared__ double sI[TB][TB + 1];
    __shared__ double sA[kStrip][TB + 1];
    const int ib = kb + 1 + blockIdx.y, r0 = kStrip * blockIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TB + tx;
    const long long rb = (long long)ib * TB + r0, cb = (long long)kb * TB;
    for (int e = tid; e < TB * TB; e += 128) sI[e / TB][e % TB] = Dk[cb * TB + e];
    sA[ty][tx] = A[(rb + ty) * npad + cb + tx];
    __syncthreads();
    double s = 0.0;
#pragma unroll 8
    for (int t = 0; t < TB; ++t) s += sA[ty][t] * sI[tx][t];
    A[(rb + ty) * npad + cb + tx] = s;
}

// A_ib,jb -= L_ib,kb L_jb,kb^T for kb < jb <= ib (pair blockIdx.y), rows
// kStrip*blockIdx.x .. +kStrip of the tile
__global__ void __launch_bounds__(128) k_syrk(double* __restrict__ A, int npad, int kb) {
    __shared__ double sI[kStrip][TB + 1];
    __shared__ double sJ[TB][TB + 1];
    const int t = blockIdx.y;
    int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while (ii * (ii + 1) / 2 > t) --ii;
    const int jj = t - ii * (ii + 1) / 2;
    const int ib = kb + 1 + ii, jb = kb + 1 + jj, r0 = kStrip * blockIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TB + tx;
    const long long cb = (long long)kb * TB, rb = (long long)ib * TB + r0, jr = (long long)jb * TB;
    sI[ty][tx] = A[(rb + ty) * npad + cb + tx];
    for (int e = tid; e < TB * TB; e += 128) sJ[e / TB][e % TB] = A[(jr + e / TB) * npad + cb + e % TB];
    __syncthreads();
    double s = 0.0;
#pragma unroll 8
    for (int c = 0; c < TB; ++c) s += sI[ty][c] * sJ[tx][c];
    A[(rb + ty) * npad + jr + tx] -= s;
}

__global__ void k_identity(double* __restrict__ W, int npad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n2 = (long long)npad * npad;
    if (i >= n2) return;
    W[i] = ((i / npad) == (i % npad)) ? 1.0 : 0.0;
}

// W_kb,jb = L_kk^-1 B_kb,jb for jb = blockIdx.y <= kb, its columns
// kStrip*blockIdx.x .. +kStrip (threads: kStrip columns x 32 rows)
__global__ void __launch_bounds__(128) k_trsm_rows(double* __restrict__ W, int npad, int kb,
                                                   const double* __restrict__ Dk) {
    __shared__ double sI[TB][TB + 1];
    __shared__ double sB[TB][kStrip + 1];
    const int jb = blockIdx.y, c0 = kStrip * blockIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kStrip + tx;
    const long long rb = (long long)kb * TB, cb = (long long)jb * TB + c0;
    for (int e = tid; e < TB * TB; e += 128) sI[e / TB][e % TB] = Dk[rb * TB + e];
    sB[ty][tx] = W[(rb + ty) * npad + cb + tx];
    __syncthreads();
    double s = 0.0;
#pragma unroll 8
    for (int t = 0; t < TB; ++t) s += sI[ty][t] * sB[t][tx];
    W[(rb + ty) * npad + cb + tx] = s;
}

// B_ib,jb -= L_ib,kb W_kb,jb for jb = blockIdx.y <= kb, ib = kb+1+blockIdx.z,
// rows kStrip*blockIdx.x .. +kStrip of the tile
__global__ void __launch_bounds__(128) k_gemm_update(const double* __restrict__ L, double* __restrict__ W, int npad,
                                                     int kb) {
    __shared__ double sL[kStrip][TB + 1];
    __shared__ double sW[TB][TB + 1];
    const int jb = blockIdx.y, ib = kb + 1 + blockIdx.z, r0 = kStrip * blockIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TB + tx;
    const long long kbase = (long long)kb * TB, rb = (long long)ib * TB + r0, cb = (long long)jb * TB;
    sL[ty][tx] = L[(rb + ty) * npad + kbase + tx];
    for (int e = tid; e < TB * TB; e += 128) sW[e / TB][e % TB] = W[(kbase + e / TB) * npad + cb + e % TB];
    __syncthreads();
    double s = 0.0;
#pragma unroll 8
    for (int c = 0; c < TB; ++c) s += sL[ty][c] * sW[c][tx];
    W[(rb + ty) * npad + cb + tx] -= s;
}

__global__ void k_transpose(const double* __restrict__ W, double* __restrict__ WT, int npad) {
    __shared__ double s[TB][TB + 1];
    const int bx = blockIdx.x, by = blockIdx.y, tx = threadIdx.x, ty = threadIdx.y;
    s[ty][tx] = W[((long long)by * TB + ty) * npad + (long long)bx * TB + tx];
    __syncthreads();
    WT[((long long)bx * TB + ty) * npad + (long long)by * TB + tx] = s[tx][ty];
}

// y_i = sum_{j<=i} W_ij r_j  (lower) or sum_{j>=i} (upper); warp per row
template <typename T, bool LOWER>
__global__ void k_trigemv(int n, int npad, const T* __restrict__ M, const T* __restrict__ v, T* __restrict__ y) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int j0 = LOWER ? 0 : row, j1 = LOWER ? row + 1 : n;
    double s = 0.0;
    const T* mr = M + (long long)row * npad;
    for (int j = j0 + lane; j < j1; j += 32) s += (double)mr[j] * (double)v[j];
    s = warp_sum(s);
    if (lane == 0) y[row] = (T)s;
}

}  // namespace

template <typename A, typename B>
void dot_partials(const Ctx& c, long long n, const A* a, const B* b, double* partials) {
    k_dot<A, B><<<kRedBlocks, 256, 0, c.s>>>(n, a, b, partials);
    TOPO_LAUNCH_CHECK(c);
}
template void dot_partials<double, double>(const Ctx&, long long, const double*, const double*, double*);
template void dot_partials<float, float>(const Ctx&, long long, const float*, const float*, double*);
template void dot_partials<double, float>(const Ctx&, long long, const double*, const float*, double*);

void reduce_to(const Ctx& c, const double* partials, int n, double* dst) {
    k_reduce_to<<<1, 1024, 0, c.s>>>(partials, n, dst);
    TOPO_LAUNCH_CHECK(c);
}
void cg_alpha(const Ctx& c, const double* partials, int n, Scalars* sc, double* hist) {
    k_cg_alpha<<<1, 1024, 0, c.s>>>(partials, n, sc, hist);
    TOPO_LAUNCH_CHECK(c);
}
void cg_beta(const Ctx& c, const double* partials, int n, Scalars* sc) {
    k_cg_beta<<<1, 1024, 0, c.s>>>(partials, n, sc);
    TOPO_LAUNCH_CHECK(c);
}
void cg_beta_flexible(const Ctx& c, const double* partials, int n, Scalars* sc) {
    k_cg_beta_flexible<<<1, 1024, 0, c.s>>>(partials, n, sc);
    TOPO_LAUNCH_CHECK(c);
}

template <typename T>
void cg_update_xr(const Ctx& c, long long n, const Scalars* sc, const T* p, const T* q, T* x, T* r,
                  double* partials) {
    k_update_xr<T><<<kRedBlocks, 256, 0, c.s>>>(n, sc, p, q, x, r, partials);
    TOPO_LAUNCH_CHECK(c);
}
template void cg_update_xr<double>(const Ctx&, long long, const Scalars*, const double*, const double*, double*,
                                   double*, double*);
template void cg_update_xr<float>(const Ctx&, long long, const Scalars*, const float*, const float*, float*, float*,
                                  double*);

template <typename T>
void cg_update_p(const Ctx& c, long long n, const Scalars* sc, const T* z, T* p) {
    k_update_p<T><<<grid_for(n, 256) > 8192 ? 8192 : grid_for(n, 256), 256, 0, c.s>>>(n, sc, z, p);
    TOPO_LAUNCH_CHECK(c);
}
template void cg_update_p<double>(const Ctx&, long long, const Scalars*, const double*, double*);
template void cg_update_p<float>(const Ctx&, long long, const Scalars*, const float*, float*);

template <typename T>
void cg_update_r(const Ctx& c, long long n, const Scalars* sc, const T* q, T* r, double* partials) {
    k_update_r<T><<<kRedBlocks, 256, 0, c.s>>>(n, sc, q, r, partials);
    TOPO_LAUNCH_CHECK(c);
}
template void cg_update_r<double>(const Ctx&, long long, const Scalars*, const double*, double*, double*);
template void cg_update_r<float>(const Ctx&, long long, const Scalars*, const float*, float*, double*);

template <typename T>
void cg_flush_x(const Ctx& c, long long n, T* const* ring, const double* alpha, int count, T* x) {
    DirRing<T> dr;
    for (int j = 0; j < kDirRing; ++j) dr.p[j] = ring[j];
    k_flush_x<T><<<grid_for(n, 256) > 8192 ? 8192 : grid_for(n, 256), 256, 0, c.s>>>(n, dr, alpha, count, x);
    TOPO_LAUNCH_CHECK(c);
}
template void cg_flush_x<double>(const Ctx&, long long, double* const*, const double*, int, double*);
template void cg_flush_x<float>(const Ctx&, long long, float* const*, const double*, int, float*);

template <typename S, typename D>
void convert(const Ctx& c, long long n, const S* src, D* dst) {
    k_convert<S, D><<<grid_for(n, 256) > 8192 ? 8192 : grid_for(n, 256), 256, 0, c.s>>>(n, src, dst);
    TOPO_LAUNCH_CHECK(c);
}
template void convert<double, float>(const Ctx&, long long, const double*, float*);
template void convert<float, double>(const Ctx&, long long, const float*, double*);
template void convert<bf16, float>(const Ctx&, long long, const bf16*, float*);

void axpy_f32_into_f64(const Ctx& c, long long n, const float* d, double* x) {
    k_axpy_f32<<<grid_for(n, 256) > 8192 ? 8192 : grid_for(n, 256), 256, 0, c.s>>>(n, d, x);
    TOPO_LAUNCH_CHECK(c);
}

template <typename T>
void zero(const Ctx& c, long long n, T* v) {
    cudaMemsetAsync(v, 0, sizeof(T) * (size_t)n, c.s);
}
template void zero<double>(const Ctx&, long long, double*);
template void zero<float>(const Ctx&, long long, float*);

void fill(const Ctx& c, long long n, double* v, double value) {
    k_fill<<<grid_for(n, 256) > 8192 ? 8192 : grid_for(n, 256), 256, 0, c.s>>>(n, v, value);
    TOPO_LAUNCH_CHECK(c);
}

// Blocks of a banded matrix (A_ij = 0 for |i - j| > band) that can be nonzero
// below the diagonal block of block column kb: block rows kb+1 .. kb+bb.
inline int band_blocks(int band) { return (band + TB - 1) / TB; }

void chol_factor(const Ctx& c, double* A, int npad, int band, int* info, double* Dk) {
    // the Cholesky factor of a banded matrix keeps its band, so the panel and
    // the trailing update of step kb touch only the bb block rows below it;
    // the blocks left out are zero in A and L alike
    const int nb = npad / TB, bb = band_blocks(band);
    cudaMemsetAsync(info, 0, sizeof(int), c.s);
    for (int kb = 0; kb < nb; ++kb) {
        k_potrf_diag<<<1, 128, 0, c.s>>>(A, npad, kb, info, Dk);
        TOPO_LAUNCH_CHECK(c);
        const int m = std::min(nb - kb - 1, bb);
        if (m > 0) {
            k_trsm_panel<<<dim3(TB / kStrip, m), dim3(TB, kStrip), 0, c.s>>>(A, npad, kb, Dk);
            TOPO_LAUNCH_CHECK(c);
            k_syrk<<<dim3(TB / kStrip, m * (m + 1) / 2), dim3(TB, kStrip), 0, c.s>>>(A, npad, kb);
            TOPO_LAUNCH_CHECK(c);
        }
    }
}

void tri_inverse(const Ctx& c, const double* L, double* W, int npad, int band, const double* Dk) {
    // W = L^-1 is dense lower triangular; L_ib,kb vanishes beyond the band,
    // so the update after block row kb reaches only the bb block rows below
    const int nb = npad / TB, bb = band_blocks(band);
    const long long n2 = (long long)npad * npad;
    k_identity<<<grid_for(n2, 256), 256, 0, c.s>>>(W, npad);
    TOPO_LAUNCH_CHECK(c);
    for (int kb = 0; kb < nb; ++kb) {
        k_trsm_rows<<<dim3(TB / kStrip, kb + 1), dim3(kStrip, TB), 0, c.s>>>(W, npad, kb, Dk);
        TOPO_LAUNCH_CHECK(c);
        const int m = std::min(nb - kb - 1, bb);
        if (m > 0) {
            k_gemm_update<<<dim3(TB / kStrip, kb + 1, m), dim3(TB, kStrip), 0, c.s>>>(L, W, npad, kb);
            TOPO_LAUNCH_CHECK(c);
        }
    }
}

void transpose_dense(const Ctx& c, const double* W, double* WT, int npad) {
    const int nb = npad / TB;
    k_transpose<<<dim3(nb, nb), dim3(TB, TB), 0, c.s>>>(W, WT, npad);
    TOPO_LAUNCH_CHECK(c);
}

template <typename T>
void coarse_apply(const Ctx& c, int n, int npad, const T* W, const T* WT, const T* rhs, T* y, T* out) {
    const unsigned blocks = (unsigned)((n + 7) / 8);
    k_trigemv<T, true><<<blocks, 256, 0, c.s>>>(n, npad, W, rhs, y);
    TOPO_LAUNCH_CHECK(c);
    k_trigemv<T, false><<<blocks, 256, 0, c.s>>>(n, npad, WT, y, out);
    TOPO_LAUNCH_CHECK(c);
}
template void coarse_apply<double>(const Ctx&, int, int, const double*, const double*, const double*, double*,
                                   double*);
template void coarse_apply<float>(const Ctx&, int, int, const float*, const float*, const float*, float*, float*);

}  // namespace topo
