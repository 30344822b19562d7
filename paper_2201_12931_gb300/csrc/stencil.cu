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
#include "operator.cuh"

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

// Element-column z-march operator kernel; see operator.cuh for the scheme.
template <typename T, int MODE, bool DOT>
__global__ void __launch_bounds__(kOpTX * kOpTY) k_op(ModalK<T> mk, const T* __restrict__ E,
                                                      const uint8_t* __restrict__ mask, const T* __restrict__ u,
                                                      const T* __restrict__ f, T* __restrict__ out, int nx, int ny,
                                                      int nz, int cz, T omega, double* __restrict__ partials) {
    constexpr int TX = kOpTX, TY = kOpTY;
    constexpr bool NEEDU = (MODE != ST_JACOBI0);
    constexpr bool NEEDD = (MODE == ST_JACOBI || MODE == ST_JACOBI0);
    constexpr bool NEEDF = (MODE != ST_APPLY);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sU = reinterpret_cast<T*>(smem_raw);        // [2][TY+1][TX+1][3]   masked u of a node plane
    T* sC = sU + 2 * (TY + 1) * (TX + 1) * 3;      // [2][3][TY][TX][3]     corner contributions 10, 01, 11
    T* sE = sC + 2 * 3 * TY * TX * 3;              // [2][TY][TX]           column modulus sums
    __shared__ double sred[32];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int NX = nx + 1, NY = ny + 1;
    const int i0 = blockIdx.x * (TX - 1), j0 = blockIdx.y * (TY - 1);
    const int kz0 = blockIdx.z * cz;
    const int kz1 = min(kz0 + cz, nz + 1);
    const int in = i0 - 1 + tx, jn = j0 - 1 + ty;
    const bool node_ok = in >= 0 && in < NX && jn >= 0 && jn < NY;
    const bool col_ok = in >= 0 && in < nx && jn >= 0 && jn < ny;
    const bool out_ok = tx >= 1 && ty >= 1 && node_ok;
    // one halo node (+x column, +y row, +x+y corner) per thread with tid < TX + TY + 1
    int hsx = TX, hsy = TY;
    if (tid < TY + 1) { hsx = TX; hsy = tid; }
    else if (tid < TY + 1 + TX) { hsx = tid - TY - 1; hsy = TY; }
    const bool has_halo = tid < TY + 1 + TX;
    const int hx = i0 - 1 + hsx, hy = j0 - 1 + hsy;
    const bool halo_ok = has_halo && hx >= 0 && hx < NX && hy >= 0 && hy < NY;
    const long long nplane = (long long)NX * NY;
    const long long own_xy = node_ok ? (long long)in + (long long)NX * jn : 0;
    const long long halo_xy = halo_ok ? (long long)hx + (long long)NX * hy : 0;
    const long long col_xy = col_ok ? (long long)in + (long long)nx * jn : 0;
    const long long eplane = (long long)nx * ny;

    T fB[12], topPrev[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) fB[i] = topPrev[i] = T(0);
    T st00[3] = {T(0), T(0), T(0)}, st10[3] = {T(0), T(0), T(0)}, st01[3] = {T(0), T(0), T(0)},
      st11[3] = {T(0), T(0), T(0)};
    T stE = T(0);
    // own-node history (raw u, mask, f) of planes P-1 (h1) and P-2 (h2)
    T h1u[3] = {T(0), T(0), T(0)}, h2u[3] = {T(0), T(0), T(0)};
    T h1f[3] = {T(0), T(0), T(0)}, h2f[3] = {T(0), T(0), T(0)};
    unsigned h1m = 0, h2m = 0;
    T Elast = T(0);       // E of own column, layer P-2
    double dot = 0.0;

    // prefetched data of plane P
    T nu[3] = {T(0), T(0), T(0)}, nf[3] = {T(0), T(0), T(0)}, hu[3] = {T(0), T(0), T(0)};
    unsigned nm = 0, hm = 0;
    T nE = T(0);          // E of own column, layer P-1
    auto fetch = [&](int P) {
        const bool pin = P >= 0 && P <= nz;
        const long long ob = (long long)P * nplane;
        if (NEEDU || NEEDF) {
            const bool ok = pin && node_ok;
            nm = ok ? mask[ob + own_xy] : 0u;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (NEEDU) nu[c] = ok ? u[3 * (ob + own_xy) + c] : T(0);
                if (NEEDF) nf[c] = ok ? f[3 * (ob + own_xy) + c] : T(0);
            }
        }
        if (NEEDU) {
            const bool okh = pin && halo_ok;
            hm = okh ? mask[ob + halo_xy] : 0u;
#pragma unroll
            for (int c = 0; c < 3; ++c) hu[c] = okh ? u[3 * (ob + halo_xy) + c] : T(0);
        }
        const int L = P - 1;
        nE = (col_ok && L >= 0 && L < nz) ? E[(long long)L * eplane + col_xy] : T(0);
    };

    fetch(kz0 - 1);
    for (int P = kz0 - 1; P <= kz1 + 1; ++P) {
        const int b = P & 1;
        // current plane data
        T cu[3], cf[3];
        const unsigned cm = nm;
        const T cE = nE;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cu[c] = nu[c];
            cf[c] = nf[c];
        }
        T chu[3] = {hu[0], hu[1], hu[2]};
        const unsigned chm = hm;
        if (P + 1 <= kz1) fetch(P + 1);   // prefetch the next plane
        // (2) publish this plane's masked u and the stashed contributions of plane P-2
        if (NEEDU) {
            T* us = &sU[((b * (TY + 1) + ty) * (TX + 1) + tx) * 3];
#pragma unroll
            for (int c = 0; c < 3; ++c) us[c] = ((cm >> c) & 1u) ? T(0) : cu[c];
            if (has_halo) {
                T* hs = &sU[((b * (TY + 1) + hsy) * (TX + 1) + hsx) * 3];
#pragma unroll
                for (int c = 0; c < 3; ++c) hs[c] = ((chm >> c) & 1u) ? T(0) : chu[c];
            }
            T* c0 = &sC[(((b * 3 + 0) * TY + ty) * TX + tx) * 3];
            T* c1 = &sC[(((b * 3 + 1) * TY + ty) * TX + tx) * 3];
            T* c2 = &sC[(((b * 3 + 2) * TY + ty) * TX + tx) * 3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                c0[c] = st10[c];
                c1[c] = st01[c];
                c2[c] = st11[c];
            }
        }
        if (NEEDD) sE[(b * TY + ty) * TX + tx] = stE;
        __syncthreads();
        // (3) output node plane Q = P - 2
        const int Q = P - 2;
        if (out_ok && Q >= kz0 && Q < kz1) {
            T y[3] = {T(0), T(0), T(0)};
            if (NEEDU) {
                const T* a0 = &sC[(((b * 3 + 0) * TY + ty) * TX + tx - 1) * 3];
                const T* a1 = &sC[(((b * 3 + 1) * TY + ty - 1) * TX + tx) * 3];
                const T* a2 = &sC[(((b * 3 + 2) * TY + ty - 1) * TX + tx - 1) * 3];
#pragma unroll
                for (int c = 0; c < 3; ++c) y[c] = st00[c] + a0[c] + a1[c] + a2[c];
            }
            T D = T(1);
            if (NEEDD) {
                const T* e = &sE[b * TY * TX];
                D = mk.kdiag * (e[ty * TX + tx] + e[ty * TX + tx - 1] + e[(ty - 1) * TX + tx] +
                                e[(ty - 1) * TX + tx - 1]);
            }
            const long long n = (long long)Q * nplane + own_xy;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool fixed = (h2m >> c) & 1u;
                T r;
                if (MODE == ST_APPLY) {
                    r = fixed ? h2u[c] : y[c];
                    if (DOT) dot += (double)h2u[c] * (double)r;
                } else if (MODE == ST_RESID) {
                    r = h2f[c] - (fixed ? h2u[c] : y[c]);
                    if (DOT) dot += (double)r * (double)r;
                } else if (MODE == ST_JACOBI) {
                    const T Ku = fixed ? h2u[c] : y[c];
                    r = h2u[c] + omega * (h2f[c] - Ku) / (fixed ? T(1) : D);
                    if (DOT) dot += (double)h2f[c] * (double)r;
                } else {
                    r = omega * h2f[c] / (fixed ? T(1) : D);
                    if (DOT) dot += (double)h2f[c] * (double)r;
                }
                out[3 * n + c] = r;
            }
        }
        // (4) face modes of plane P and the element of layer P-1 (plane P-1 completes)
        if (P >= kz0 && P <= kz1) {
            if (NEEDU) {
                T fT[12];
                const T* s00 = &sU[((b * (TY + 1) + ty) * (TX + 1) + tx) * 3];
                const T* s10 = s00 + 3;
                const T* s01 = s00 + (TX + 1) * 3;
                const T* s11 = s01 + 3;
                face_forward<T>(s00, s10, s01, s11, fT);
                T Bo[12], To[12];
                if (cE != T(0)) {
                    element_modal<T>(mk, cE, fB, fT, Bo, To);
                } else {
#pragma unroll
                    for (int i = 0; i < 12; ++i) Bo[i] = To[i] = T(0);
                }
                T A[12];
#pragma unroll
                for (int i = 0; i < 12; ++i) {
                    A[i] = topPrev[i] + Bo[i];
                    topPrev[i] = To[i];
                    fB[i] = fT[i];
                }
                face_inverse<T>(A, st00, st10, st01, st11);
            }
            if (NEEDD) stE = Elast + cE;
        } else if (NEEDU && P == kz0 - 1) {
            const T* s00 = &sU[((b * (TY + 1) + ty) * (TX + 1) + tx) * 3];
            face_forward<T>(s00, s00 + 3, s00 + (TX + 1) * 3, s00 + (TX + 1) * 3 + 3, fB);
        }
        Elast = cE;
        // shift the own-node history
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            h2u[c] = h1u[c];
            h2f[c] = h1f[c];
            h1u[c] = cu[c];
            h1f[c] = cf[c];
        }
        h2m = h1m;
        h1m = cm;
    }
    if (DOT) {
        double v = dot;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int w = tid >> 5, l = tid & 31;
        if (l == 0) sred[w] = v;
        __syncthreads();
        if (w == 0) {
            double t = (l < (TX * TY) / 32) ? sred[l] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (l == 0) partials[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
        }
    }
}

template <typename T>
constexpr size_t op_smem_bytes() {
    return sizeof(T) * (2 * (kOpTY + 1) * (kOpTX + 1) * 3 + 2 * 3 * kOpTY * kOpTX * 3 + 2 * kOpTY * kOpTX);
}

template <typename T, int MODE, bool DOT>
void launch_op(const Ctx& c, const OpLaunch& L, const ModalK<T>& mk, const T* E, const uint8_t* mask, const T* u,
               const T* f, T* out, T omega, double* dot) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_op<T, MODE, DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)op_smem_bytes<T>());
        attr = true;
    }
    k_op<T, MODE, DOT><<<dim3(L.gx, L.gy, L.gz), dim3(kOpTX, kOpTY), op_smem_bytes<T>(), c.s>>>(
        mk, E, mask, u, f, out, L.g.nx, L.g.ny, L.g.nz, L.cz, omega, dot);
    TOPO_LAUNCH_CHECK(c);
}

template <typename T, int MODE>
void launch_mode(const Ctx& c, const OpLaunch& L, const ModalK<T>& mk, const T* E, const uint8_t* mask, const T* u,
                 const T* f, T* out, T omega, double* dot) {
    if (dot) launch_op<T, MODE, true>(c, L, mk, E, mask, u, f, out, omega, dot);
    else launch_op<T, MODE, false>(c, L, mk, E, mask, u, f, out, omega, nullptr);
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

OpLaunch op_launch(const Geom& g) {
    OpLaunch L;
    L.g = g;
    L.gx = (g.nx + 1 + kOpTX - 2) / (kOpTX - 1);
    L.gy = (g.ny + 1 + kOpTY - 2) / (kOpTY - 1);
    const long long xy = (long long)L.gx * L.gy;
    const int NZ = g.nz + 1;
    const long long gz_target = (4096 + xy - 1) / xy;
    int cz = (int)((NZ + gz_target - 1) / gz_target);
    cz = cz < 8 ? (NZ < 8 ? NZ : 8) : cz;
    L.cz = cz;
    L.gz = (NZ + cz - 1) / cz;
    return L;
}

template <typename T>
int stencil(const Ctx& c, int mode, const OpLaunch& L, const ModalK<T>& mk, const T* E, const uint8_t* mask,
            const T* u, const T* f, T* out, T omega, double* dot) {
    switch (mode) {
        case ST_APPLY: launch_mode<T, ST_APPLY>(c, L, mk, E, mask, u, f, out, omega, dot); break;
        case ST_JACOBI: launch_mode<T, ST_JACOBI>(c, L, mk, E, mask, u, f, out, omega, dot); break;
        case ST_RESID: launch_mode<T, ST_RESID>(c, L, mk, E, mask, u, f, out, omega, dot); break;
        default: launch_mode<T, ST_JACOBI0>(c, L, mk, E, mask, u, f, out, omega, dot); break;
    }
    return L.gx * L.gy * L.gz;
}
template int stencil<double>(const Ctx&, int, const OpLaunch&, const ModalK<double>&, const double*, const uint8_t*,
                             const double*, const double*, double*, double, double*);
template int stencil<float>(const Ctx&, int, const OpLaunch&, const ModalK<float>&, const float*, const uint8_t*,
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
