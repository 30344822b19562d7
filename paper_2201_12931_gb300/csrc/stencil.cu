// Matrix-free element-by-element operator (Sec. 4.2.1: "sum of density times
// local stiffness matrices of these 8 elements gives the value equal to global
// stiffness value of that node"), fused with the damped Jacobi sweep
// (Sec. 3.2) and the residual (Eq. residual); coarse-grid assembly; element
// energy and compliance sensitivity (Eq. sensitivity).
//
// Operator with Dirichlet rows: y = P_f K P_f u + (I - P_f) u, P_f zeroing the
// fixed DOFs, K = sum_e E_e A_e^T K0 A_e (E_e already holds 2^l on level l).
#include "common.cuh"
#include "modal.cuh"

namespace topo {

namespace {

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
    return t;   // valid in thread 0
}

// One thread per node; gathers the 8 adjacent elements' rows of E_e K0 u_e.
template <typename T, int MODE, bool DOT>
__global__ void __launch_bounds__(256) k_stencil_gather(
    const T* __restrict__ K0g, const T* __restrict__ E, const uint8_t* __restrict__ mask,
    const T* __restrict__ u, const T* __restrict__ f, T* __restrict__ out, int nx, int ny, int nz,
    T omega, double* __restrict__ partials) {
    __shared__ T sK[576];
    __shared__ double sred[32];
    for (int t = threadIdx.x; t < 576; t += blockDim.x) sK[t] = K0g[t];
    __syncthreads();
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    const long long nn = (long long)NX * NY * NZ;
    double dot = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
         n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % NX);
        const long long t2 = n / NX;
        const int j = (int)(t2 % NY);
        const int k = (int)(t2 / NY);
        const unsigned mk = mask[n];
        T acc[3] = {T(0), T(0), T(0)};
        T dg[3] = {T(0), T(0), T(0)};
#pragma unroll 1
        for (int az = 0; az < 2; ++az) {
            const int ez = k - 1 + az;
            if (ez < 0 || ez >= nz) continue;
#pragma unroll 1
            for (int ay = 0; ay < 2; ++ay) {
                const int ey = j - 1 + ay;
                if (ey < 0 || ey >= ny) continue;
#pragma unroll 1
                for (int ax = 0; ax < 2; ++ax) {
                    const int ex = i - 1 + ax;
                    if (ex < 0 || ex >= nx) continue;
                    const T Ee = E[ex + (long long)nx * (ey + (long long)ny * ez)];
                    const int ln = (1 - ax) + 2 * (1 - ay) + 4 * (1 - az);
#pragma unroll
                    for (int c = 0; c < 3; ++c) dg[c] += Ee * sK[(3 * ln + c) * 24 + 3 * ln + c];
                    if (MODE != ST_JACOBI0) {
                        T s[3] = {T(0), T(0), T(0)};
#pragma unroll
                        for (int m = 0; m < 8; ++m) {
                            const long long nm = (ex + (m & 1)) +
                                                 (long long)NX * ((ey + ((m >> 1) & 1)) + (long long)NY * (ez + (m >> 2)));
                            const unsigned mm = mask[nm];
                            const T v0 = (mm & 1u) ? T(0) : u[3 * nm + 0];
                            const T v1 = (mm & 2u) ? T(0) : u[3 * nm + 1];
                            const T v2 = (mm & 4u) ? T(0) : u[3 * nm + 2];
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const T* row = &sK[(3 * ln + c) * 24 + 3 * m];
                                s[c] += row[0] * v0 + row[1] * v1 + row[2] * v2;
                            }
                        }
#pragma unroll
                        for (int c = 0; c < 3; ++c) acc[c] += Ee * s[c];
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const bool fixed = (mk >> c) & 1u;
            const long long d = 3 * n + c;
            T y;
            if (MODE == ST_APPLY) {
                const T uc = u[d];
                y = fixed ? uc : acc[c];
                if (DOT) dot += (double)uc * (double)y;
            } else if (MODE == ST_RESID) {
                const T Ku = fixed ? u[d] : acc[c];
                y = f[d] - Ku;
                if (DOT) dot += (double)y * (double)y;
            } else if (MODE == ST_JACOBI) {
                const T uc = u[d];
                const T Ku = fixed ? uc : acc[c];
                const T D = fixed ? T(1) : dg[c];
                y = uc + omega * (f[d] - Ku) / D;
                if (DOT) dot += (double)f[d] * (double)y;
            } else {  // ST_JACOBI0
                const T D = fixed ? T(1) : dg[c];
                y = omega * f[d] / D;
                if (DOT) dot += (double)f[d] * (double)y;
            }
            out[d] = y;
        }
    }
    if (DOT) {
        const double t = block_sum(dot, sred);
        if (threadIdx.x == 0) partials[blockIdx.x] = t;
    }
}

template <typename T, int MODE>
void launch_mode(const Ctx& c, const Geom& g, const T* K0, const T* E, const uint8_t* mask, const T* u,
                 const T* f, T* out, T omega, double* dot) {
    const int threads = 256;
    if (dot) {
        k_stencil_gather<T, MODE, true><<<kRedBlocks, threads, 0, c.s>>>(K0, E, mask, u, f, out, g.nx, g.ny,
                                                                       g.nz, omega, dot);
    } else {
        long long blocks = (g.nn + threads - 1) / threads;
        if (blocks > 65535LL * 16) blocks = 65535LL * 16;
        k_stencil_gather<T, MODE, false><<<(unsigned)blocks, threads, 0, c.s>>>(K0, E, mask, u, f, out, g.nx,
                                                                              g.ny, g.nz, omega, nullptr);
    }
    TOPO_LAUNCH_CHECK(c);
}

// Dense assembly of the coarsest operator with identity Dirichlet rows.
__global__ void k_assemble(const double* __restrict__ K0, const double* __restrict__ E,
                           const uint8_t* __restrict__ mask, double* __restrict__ A, int nx, int ny, int nz,
                           int npad) {
    const int e = blockIdx.x;
    const int i = e % nx, j = (e / nx) % ny, k = e / (nx * ny);
    const int NX = nx + 1, NY = ny + 1;
    const double Ee = E[e];
    for (int t = threadIdx.x; t < 576; t += blockDim.x) {
        const int r = t / 24, s = t % 24;
        const int ar = r / 3, cr = r % 3, as = s / 3, cs = s % 3;
        const int nr = (i + (ar & 1)) + NX * ((j + ((ar >> 1) & 1)) + NY * (k + (ar >> 2)));
        const int ns = (i + (as & 1)) + NX * ((j + ((as >> 1) & 1)) + NY * (k + (as >> 2)));
        if (((mask[nr] >> cr) & 1u) || ((mask[ns] >> cs) & 1u)) continue;
        atomicAdd(&A[(long long)(3 * nr + cr) * npad + (3 * ns + cs)], Ee * K0[r * 24 + s]);
    }
}

__global__ void k_assemble_diag(const uint8_t* __restrict__ mask, double* __restrict__ A, int n, int npad) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= npad) return;
    if (d >= n || ((mask[d / 3] >> (d % 3)) & 1u)) A[(long long)d * npad + d] = 1.0;
}

// Element energy u_e^T K0 u_e in the modal (Walsh-Hadamard) basis, compliance
// partial sums sum_e E_e se_e and the sensitivity -p rho^(p-1) (E0-Emin) se_e.
__global__ void __launch_bounds__(256) k_energy_sens(ModalCoef mc, const double* __restrict__ u,
                                                     const double* __restrict__ rho, int nx, int ny, int nz,
                                                     double E0, double Emin, double penal,
                                                     double* __restrict__ dc, double* __restrict__ partials) {
    __shared__ double sred[32];
    const long long ne = (long long)nx * ny * nz;
    const int NX = nx + 1, NY = ny + 1;
    double csum = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nx);
        const long long t = e / nx;
        const int j = (int)(t % ny), k = (int)(t / ny);
        double ue[24];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const long long nd = (i + (a & 1)) + (long long)NX * ((j + ((a >> 1) & 1)) + (long long)NY * (k + (a >> 2)));
#pragma unroll
            for (int c = 0; c < 3; ++c) ue[3 * a + c] = u[3 * nd + c];
        }
        double m[24];
        modal_forward(ue, m);
        const double se = modal_energy(mc, m);
        const double r = rho[e];
        const double Ee = Emin + pow(r, penal) * (E0 - Emin);
        csum += Ee * se;
        if (dc) dc[e] = -penal * pow(r, penal - 1.0) * (E0 - Emin) * se;
    }
    const double tsum = block_sum(csum, sred);
    if (threadIdx.x == 0) partials[blockIdx.x] = tsum;
}

}  // namespace

template <typename T>
void stencil(const Ctx& c, int mode, const Geom& g, const T* K0, const T* E, const uint8_t* mask, const T* u,
             const T* f, T* out, T omega, double* dot) {
    switch (mode) {
        case ST_APPLY: launch_mode<T, ST_APPLY>(c, g, K0, E, mask, u, f, out, omega, dot); break;
        case ST_JACOBI: launch_mode<T, ST_JACOBI>(c, g, K0, E, mask, u, f, out, omega, dot); break;
        case ST_RESID: launch_mode<T, ST_RESID>(c, g, K0, E, mask, u, f, out, omega, dot); break;
        default: launch_mode<T, ST_JACOBI0>(c, g, K0, E, mask, u, f, out, omega, dot); break;
    }
}
template void stencil<double>(const Ctx&, int, const Geom&, const double*, const double*, const uint8_t*,
                              const double*, const double*, double*, double, double*);
template void stencil<float>(const Ctx&, int, const Geom&, const float*, const float*, const uint8_t*,
                             const float*, const float*, float*, float, double*);

void assemble_coarse(const Ctx& c, const Geom& g, const double* K0, const double* E, const uint8_t* mask,
                     double* A, int npad) {
    cudaMemsetAsync(A, 0, sizeof(double) * (size_t)npad * npad, c.s);
    k_assemble<<<(unsigned)g.ne, 128, 0, c.s>>>(K0, E, mask, A, g.nx, g.ny, g.nz, npad);
    TOPO_LAUNCH_CHECK(c);
    k_assemble_diag<<<(npad + 255) / 256, 256, 0, c.s>>>(mask, A, (int)(3 * g.nn), npad);
    TOPO_LAUNCH_CHECK(c);
}

void element_energy_sens(const Ctx& c, const Geom& g, const ModalCoef& mc, const double* u, const double* rho,
                         double E0, double Emin, double penal, double* dc_out, double* partials) {
    k_energy_sens<<<kRedBlocks, 256, 0, c.s>>>(mc, u, rho, g.nx, g.ny, g.nz, E0, Emin, penal, dc_out, partials);
    TOPO_LAUNCH_CHECK(c);
}

}  // namespace topo
