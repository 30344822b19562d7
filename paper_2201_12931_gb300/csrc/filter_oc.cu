// Density filter (weights of Eqs. Neighbourhood / NB_dist, normalised by the
// in-domain weight sum), its transpose, and the optimality-criteria update with
// bisection on the Lagrange multiplier (Eqs. OCUp1, bisect).
//
// The volume of the filtered new design is evaluated without filtering it:
// mean(H x) = (1/N) sum_e sum_i w_ei x_i / S_e = (1/N) (H^T 1)^T x, so one
// bisection step is a single pass over (x, -dc~, H^T 1) with an FP64 block sum.
#include <math.h>

#include "common.cuh"

namespace topo {

namespace {

inline unsigned grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 2147483647LL) b = 2147483647LL;
    return (unsigned)(b < 1 ? 1 : b);
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    }
    return t;
}

// mode 0: out_e = sum_d w_d in[e+d] / S_e (S_e on the fly)
// mode 1: out_i = sum_d w_d in[i+d]   with in = g / S already divided
// mode 2: out_e = S_e
template <int MODE>
__global__ void __launch_bounds__(256) k_filter(const int4* __restrict__ offs, const double* __restrict__ wts,
                                                int noffs, int nx, int ny, int nz, const double* __restrict__ in,
                                                const double* __restrict__ S, double* __restrict__ out) {
    extern __shared__ int4 soff[];                       // offsets first: 16-byte aligned
    double* sw = reinterpret_cast<double*>(soff + noffs);
    for (int t = threadIdx.x; t < noffs; t += blockDim.x) {
        sw[t] = wts[t];
        soff[t] = offs[t];
    }
    __syncthreads();
    const long long ne = (long long)nx * ny * nz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nx);
        const long long t = e / nx;
        const int j = (int)(t % ny), k = (int)(t / ny);
        double acc = 0.0, ws = 0.0;
        for (int q = 0; q < noffs; ++q) {
            const int4 o = soff[q];
            const int a = i + o.x, b = j + o.y, c = k + o.z;
            if (a < 0 || a >= nx || b < 0 || b >= ny || c < 0 || c >= nz) continue;
            const double w = sw[q];
            const long long nb = a + (long long)nx * (b + (long long)ny * c);
            if (MODE == 0) {
                acc += w * in[nb];
                ws += w;
            } else if (MODE == 1) {
                acc += w * in[nb];   // in = g / S, formed by k_divide
            } else {
                ws += w;
            }
        }
        out[e] = (MODE == 0) ? acc / ws : (MODE == 1 ? acc : ws);
    }
}

// Eq. sensitivity filter: t = rho dc before the normalised filter, and the
// division by max(gamma, rho_e) after it
__global__ void k_mul(long long n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n) return;
    out[e] = a[e] * b[e];
}
__global__ void k_div_max(long long n, double* __restrict__ out, const double* __restrict__ rho, double gamma) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n) return;
    out[e] = out[e] / fmax(gamma, rho[e]);
}

__global__ void k_divide(long long n, const double* __restrict__ a, const double* __restrict__ b,
                         double* __restrict__ out) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n) return;
    out[e] = a[e] / b[e];
}

// q_e = x_e sqrt(max(-dc~_e, 1e-30) / dv~_e): the part of the OC candidate
// x (B)^(1/2), B = -dc~ / (lambda dv~), that does not depend on lambda
// q = x sqrt(max(-dc~, 1e-30) / dv~) (in place over dc~) and the move-limit
// bounds lo = max(0, x - move), hi = min(1, x + move) of Eq. OC
__global__ void k_oc_prepare(long long ne, const double* __restrict__ x, double* dct_q, const double* __restrict__ dv,
                             double move, double* __restrict__ lo, double* __restrict__ hi) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const double xe = x[e];
    dct_q[e] = xe * sqrt(fmax(-dct_q[e], 1e-30) / (dv ? dv[e] : 1.0));
    lo[e] = fmax(0.0, xe - move);
    hi[e] = fmin(1.0, xe + move);
}

// passive elements (0 active, 1 solid, 2 void) take x = 1 / 0 through
// lo = hi and carry no volume (dv = 0); active elements: dv = 1
__global__ void k_oc_prepare_passive(long long ne, const double* __restrict__ x, double* dc_q,
                                     const uint8_t* __restrict__ passive, double move, double* __restrict__ lo,
                                     double* __restrict__ hi, double* __restrict__ dv) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const unsigned p = passive[e];
    if (p != 0) {
        const double v = p == 1 ? 1.0 : 0.0;
        dc_q[e] = 0.0;
        lo[e] = hi[e] = v;
        dv[e] = 0.0;
        return;
    }
    const double xe = x[e];
    dc_q[e] = xe * sqrt(fmax(-dc_q[e], 1e-30));
    lo[e] = fmax(0.0, xe - move);
    hi[e] = fmin(1.0, xe + move);
    dv[e] = 1.0;
}

// Self-weight (design-dependent) load: f_out = f_ext + sum_e rho_e g_e with
// g_e = -(w/8) e_z at the 8 corners of e; one thread per node
__global__ void k_gravity_load(const double* __restrict__ rho, const double* __restrict__ f_ext,
                               double* __restrict__ f_out, double w, int nx, int ny, int nz) {
    const int NX = nx + 1, NY = ny + 1;
    const long long nn = (long long)NX * NY * (nz + 1);
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= nn) return;
    const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / ((long long)NX * NY));
    double s = 0.0;
    for (int dz = -1; dz <= 0; ++dz)
        for (int dy = -1; dy <= 0; ++dy)
            for (int dx = -1; dx <= 0; ++dx) {
                const int ex = i + dx, ey = j + dy, ez = k + dz;
                if (ex < 0 || ex >= nx || ey < 0 || ey >= ny || ez < 0 || ez >= nz) continue;
                s += rho[ex + (long long)nx * (ey + (long long)ny * ez)];
            }
    f_out[3 * n + 0] = f_ext ? f_ext[3 * n + 0] : 0.0;
    f_out[3 * n + 1] = f_ext ? f_ext[3 * n + 1] : 0.0;
    f_out[3 * n + 2] = (f_ext ? f_ext[3 * n + 2] : 0.0) - 0.125 * w * s;
}

// dc_e += 2 u_e^T g_e = -(w/4) sum of u_z over the 8 corners of e
__global__ void k_gravity_sens(const double* __restrict__ u, double* __restrict__ dc, double w, int nx, int ny,
                               int nz) {
    const long long ne = (long long)nx * ny * nz;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int NX = nx + 1, NY = ny + 1;
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long long)nx * ny));
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const long long nd = (i + (a & 1)) + (long long)NX * ((j + ((a >> 1) & 1)) + (long long)NY * (k + (a >> 2)));
        s += u[3 * nd + 2];
    }
    dc[e] += -0.25 * w * s;
}

// lam state: [0] l1, [1] l2, [2] lmid (next to evaluate), [3] done, [4] steps, [5] last lmid
// candidate min(hi, max(lo, q s)) with s = lambda^(-1/2); the three values are
// non-negative, so the clamps compare their IEEE bit patterns as integers
// (same order, exact, and off the FP64 pipe)
__device__ __forceinline__ double oc_candidate(double q, double s, double lo, double hi) {
    long long b = __double_as_longlong(q * s);
    b = max(b, __double_as_longlong(lo));
    b = min(b, __double_as_longlong(hi));
    return __longlong_as_double(b);
}

__global__ void __launch_bounds__(256) k_oc_step(long long ne, const double* __restrict__ lo, const double* __restrict__ hi,
                                                 const double* __restrict__ num, const double* __restrict__ dv,
                                                 double* __restrict__ partials, const double* __restrict__ lam) {
    __shared__ double sh[32];
    if (lam[3] != 0.0) {
        if (threadIdx.x == 0) partials[blockIdx.x] = 0.0;
        return;
    }
    const double sl = rsqrt(lam[2]);
    double s = 0.0;
    if (dv) {
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
             e += (long long)gridDim.x * blockDim.x)
            s += dv[e] * oc_candidate(num[e], sl, lo[e], hi[e]);
    } else {   // no density filter: the volume of the design itself
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
             e += (long long)gridDim.x * blockDim.x)
            s += oc_candidate(num[e], sl, lo[e], hi[e]);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_oc_finalize(const double* __restrict__ partials, double* lam, double volfrac_ne,
                                                      double tol) {
    __shared__ double sh[32];
    if (lam[3] != 0.0) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) s += partials[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        const double lm = lam[2];
        if (s > volfrac_ne) lam[0] = lm;
        else lam[1] = lm;
        lam[5] = lm;
        lam[4] += 1.0;
        const double l1 = lam[0], l2 = lam[1];
        if ((l2 - l1) / (l1 + l2) > tol) lam[2] = 0.5 * (l1 + l2);
        else lam[3] = 1.0;
    }
}

__global__ void __launch_bounds__(256) k_oc_write(long long ne, double* __restrict__ x, const double* __restrict__ lo,
                                                  const double* __restrict__ hi, const double* __restrict__ num,
                                                  const double* __restrict__ lam, double* __restrict__ partials) {
    __shared__ double sh[32];
    const double sl = rsqrt(lam[5]);
    double m = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        const double xo = x[e];
        const double xn = oc_candidate(num[e], sl, lo[e], hi[e]);
        m = fmax(m, fabs(xn - xo));
        x[e] = xn;
    }
    m = block_max(m, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = m;
}

__global__ void __launch_bounds__(1024) k_max_to(const double* __restrict__ partials, double* dst) {
    __shared__ double sh[32];
    double m = 0.0;
    for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) m = fmax(m, partials[i]);
    m = block_max(m, sh);
    if (threadIdx.x == 0) *dst = m;
}

}  // namespace

void filter_launch(const Ctx& c, const Geom& g, const int4* offs, const double* wts, int noffs, const double* in,
                   double* out, int mode, const double* S) {
    unsigned blocks = grid_for(g.ne, 256);
    if (blocks > 16384) blocks = 16384;
    const size_t sm = (sizeof(int4) + sizeof(double)) * (size_t)noffs;
    if (mode == 0) k_filter<0><<<blocks, 256, sm, c.s>>>(offs, wts, noffs, g.nx, g.ny, g.nz, in, S, out);
    else if (mode == 1) k_filter<1><<<blocks, 256, sm, c.s>>>(offs, wts, noffs, g.nx, g.ny, g.nz, in, S, out);
    else k_filter<2><<<blocks, 256, sm, c.s>>>(offs, wts, noffs, g.nx, g.ny, g.nz, in, S, out);
    TOPO_LAUNCH_CHECK(c);
}

void divide(const Ctx& c, long long n, const double* a, const double* b, double* out) {
    k_divide<<<grid_for(n, 256), 256, 0, c.s>>>(n, a, b, out);
    TOPO_LAUNCH_CHECK(c);
}

void sensitivity_filter(const Ctx& c, const Geom& g, const int4* offs, const double* wts, int noffs,
                        const double* rho, const double* dc, double gamma, double* tmp, double* out) {
    k_mul<<<grid_for(g.ne, 256), 256, 0, c.s>>>(g.ne, rho, dc, tmp);
    TOPO_LAUNCH_CHECK(c);
    filter_launch(c, g, offs, wts, noffs, tmp, out, 0, nullptr);
    k_div_max<<<grid_for(g.ne, 256), 256, 0, c.s>>>(g.ne, out, rho, gamma);
    TOPO_LAUNCH_CHECK(c);
}

void oc_prepare(const Ctx& c, long long ne, const double* x, double* dct_q, const double* dv, double move, double* lo,
                double* hi) {
    k_oc_prepare<<<grid_for(ne, 256), 256, 0, c.s>>>(ne, x, dct_q, dv, move, lo, hi);
    TOPO_LAUNCH_CHECK(c);
}

void oc_prepare_passive(const Ctx& c, long long ne, const double* x, double* dct_q, const uint8_t* passive,
                        double move, double* lo, double* hi, double* dv) {
    k_oc_prepare_passive<<<grid_for(ne, 256), 256, 0, c.s>>>(ne, x, dct_q, passive, move, lo, hi, dv);
    TOPO_LAUNCH_CHECK(c);
}

void gravity_load(const Ctx& c, const Geom& g, const double* rho, const double* f_ext, double* f_out, double w) {
    k_gravity_load<<<grid_for(g.nn, 256), 256, 0, c.s>>>(rho, f_ext, f_out, w, g.nx, g.ny, g.nz);
    TOPO_LAUNCH_CHECK(c);
}

void gravity_sensitivity(const Ctx& c, const Geom& g, const double* u, double* dc, double w) {
    k_gravity_sens<<<grid_for(g.ne, 256), 256, 0, c.s>>>(u, dc, w, g.nx, g.ny, g.nz);
    TOPO_LAUNCH_CHECK(c);
}

void oc_bisect_step(const Ctx& c, long long ne, const double* lo, const double* hi, const double* num,
                    const double* dv, double* partials, double* lam_state) {
    k_oc_step<<<kRedBlocks, 256, 0, c.s>>>(ne, lo, hi, num, dv, partials, lam_state);
    TOPO_LAUNCH_CHECK(c);
}

void oc_bisect_finalize(const Ctx& c, const double* partials, double* lam_state, double volfrac_ne, double tol) {
    k_oc_finalize<<<1, 1024, 0, c.s>>>(partials, lam_state, volfrac_ne, tol);
    TOPO_LAUNCH_CHECK(c);
}

void oc_write(const Ctx& c, long long ne, double* x, const double* lo, const double* hi, const double* num,
              const double* lam_state, double* partials, double* change_dst) {
    k_oc_write<<<kRedBlocks, 256, 0, c.s>>>(ne, x, lo, hi, num, lam_state, partials);
    TOPO_LAUNCH_CHECK(c);
    k_max_to<<<1, 1024, 0, c.s>>>(partials, change_dst);
    TOPO_LAUNCH_CHECK(c);
}

}  // namespace topo
