// Grid transfers and per-level set-up.
//   restriction  r_c = diag(free_c) P^T diag(free_f) r_f  (Algorithm 3,
//                "Restrict to next coarser grid"; trilinear P, 1D weights
//                1 at coincident and 1/2 at midpoint nodes)
//   prolongation u_f += diag(free_f) P diag(free_c) e_c  (Algorithm 3,
//                "Prolongation correction")
//   homogenization: coarse density (or modulus) = mean of the 8 children (Sec. 4.2.2)
//   SIMP moduli E_l = 2^l (Emin + rho^p (E0 - Emin)) (Eq. K_mod)
#include "common.cuh"

namespace topo {

namespace {

inline unsigned grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 2147483647LL) b = 2147483647LL;
    return (unsigned)(b < 1 ? 1 : b);
}

// Restriction r_c = diag(free_c) P^T diag(free_f) r_f.
// Restriction marching along z: one thread per coarse (I, J) node column and
// a chunk of coarse planes.  s_k = the masked in-plane 3 x 3 sum (weights
// 1, 1/2) of fine plane k around (2I, 2J); r_c(K) = s_{2K-1}/2 + s_{2K} +
// s_{2K+1}/2, and s_{2K+1} is reused as the lower plane of K + 1, so every
// fine plane is summed once per coarse column.
template <typename T>
__global__ void __launch_bounds__(256) k_restrict_z(const uint8_t* __restrict__ maskf, const uint8_t* __restrict__ maskc,
                                                    const T* __restrict__ rf, T* __restrict__ rc, int nxf, int nyf,
                                                    int nzf, int czc) {
    const int NXf = nxf + 1, NYf = nyf + 1;
    const int NXc = nxf / 2 + 1, NYc = nyf / 2 + 1, NZc = nzf / 2 + 1;
    const int I = blockIdx.x * 32 + threadIdx.x, J = blockIdx.y * 8 + threadIdx.y;
    if (I >= NXc || J >= NYc) return;
    const int K0 = blockIdx.z * czc, K1 = min(K0 + czc, NZc);
    const long long fplane = (long long)NXf * NYf;
    auto plane_sum = [&](int k, T* s) {
        s[0] = s[1] = s[2] = T(0);
        if (k < 0 || k > nzf) return;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int j = 2 * J + dy;
            if (j < 0 || j >= NYf) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int i = 2 * I + dx;
                if (i < 0 || i >= NXf) continue;
                const T w = (dx ? T(0.5) : T(1)) * (dy ? T(0.5) : T(1));
                const long long n = i + (long long)NXf * j + fplane * k;
                const unsigned mf = maskf[n];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (!((mf >> c) & 1u)) s[c] += w * rf[3 * n + c];
            }
        }
    };
    T lo[3], mid[3], hi[3];
    plane_sum(2 * K0 - 1, lo);
    const long long ccol = I + (long long)NXc * J, cplane = (long long)NXc * NYc;
    for (int K = K0; K < K1; ++K) {
        plane_sum(2 * K, mid);
        plane_sum(2 * K + 1, hi);
        const long long N = ccol + cplane * K;
        const unsigned mc = maskc[N];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rc[3 * N + c] = ((mc >> c) & 1u) ? T(0) : T(0.5) * lo[c] + mid[c] + T(0.5) * hi[c];
            lo[c] = hi[c];
        }
    }
}

constexpr int kRestrictCz = 8;

// Prolongation u_f += diag(free_f) P diag(free_c) e_c, marching along z: one
// thread per fine (i, j) node column and a chunk of fine planes.  The
// in-plane interpolation of a coarse plane (up to four coarse nodes) is
// formed once and serves the two fine planes around it, so a fine node costs
// about two coarse gathers instead of up to eight, and no 64-bit index
// division is needed.  T: arithmetic; TE / TU: storage of the coarse
// correction and of the fine iterate.
template <typename T, typename TE = T, typename TU = T>
__global__ void __launch_bounds__(256) k_prolong_z(const uint8_t* __restrict__ maskf, const uint8_t* __restrict__ maskc,
                                                   const TE* __restrict__ ec, TU* __restrict__ uf, int nxf, int nyf,
                                                   int nzf, int cz) {
    const int NXf = nxf + 1, NYf = nyf + 1, NZf = nzf + 1;
    const int NXc = nxf / 2 + 1, NYc = nyf / 2 + 1;
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    if (i >= NXf || j >= NYf) return;
    const int k0 = blockIdx.z * cz, k1 = min(k0 + cz, NZf);
    const bool two_x = i & 1, two_y = j & 1;
    const int I0 = i >> 1, J0 = j >> 1;
    const T w = (two_x ? T(0.5) : T(1)) * (two_y ? T(0.5) : T(1));
    const long long ncp = (long long)NXc * NYc;
    const long long c00 = I0 + (long long)NXc * J0;
    auto coarse_plane = [&](int K, T* v) {
        v[0] = v[1] = v[2] = T(0);
        const long long b = (long long)K * ncp + c00;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int dx = q & 1, dy = q >> 1;
            if ((dx && !two_x) || (dy && !two_y)) continue;
            const long long N = b + dx + (long long)NXc * dy;
            const unsigned mc = maskc[N];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (!((mc >> c) & 1u)) v[c] += w * (T)ec[3 * N + c];
        }
    };
    T va[3], vb[3];
    int Ka = -1;   // coarse plane whose interpolation is held in va
    const long long col = i + (long long)NXf * j, fplane = (long long)NXf * NYf;
    // the fine node's mask and iterate are loaded one plane ahead (before
    // the stores of the current plane), so that each thread keeps a load in
    // flight while it interpolates and stores
    unsigned mf_n = 0u;
    TU un[3];
    if (k0 < k1) {
        const long long n = col + fplane * k0;
        mf_n = maskf[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) un[c] = uf[3 * n + c];
    }
    for (int k = k0; k < k1; ++k) {
        const unsigned mf = mf_n;
        T uo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) uo[c] = (T)un[c];
        if (k + 1 < k1) {
            const long long n1 = col + fplane * (k + 1);
            mf_n = maskf[n1];
#pragma unroll
            for (int c = 0; c < 3; ++c) un[c] = uf[3 * n1 + c];
        }
        const int K = k >> 1;
        if (Ka != K) {
            coarse_plane(K, va);
            Ka = K;
        }
        T val[3] = {va[0], va[1], va[2]};
        if (k & 1) {   // midway between coarse planes K and K + 1
            coarse_plane(K + 1, vb);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                val[c] = T(0.5) * (va[c] + vb[c]);
                va[c] = vb[c];
            }
            Ka = K + 1;
        }
        const long long n = col + fplane * k;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (!((mf >> c) & 1u)) uf[3 * n + c] = (TU)(uo[c] + val[c]);
    }
}

constexpr int kProlongCz = 16;

// z chunk of a transfer kernel with `columns` (i, j) threads over `planes`
// planes: as long as cz_max (plane sums reused along the march) while the
// grid still fills a GB300 (152 SMs x 2048 threads), shorter on small levels,
// whose launches are bound by the latency of the march, not by memory
inline int transfer_cz(long long columns, int planes, int cz_max) {
    constexpr long long kFull = 152LL * 2048;
    const long long chunks = (kFull + columns - 1) / columns;
    const long long cz = (planes + chunks - 1) / chunks;
    return (int)(cz < 1 ? 1 : (cz > cz_max ? cz_max : cz));
}

inline int prolong_cz(const Geom& gf) {
    return transfer_cz((long long)(gf.nx + 1) * (gf.ny + 1), gf.nz + 1, kProlongCz);
}

inline dim3 prolong_grid(const Geom& gf) {
    const int cz = prolong_cz(gf);
    return dim3((gf.nx + 1 + 31) / 32, (gf.ny + 1 + 7) / 8, (gf.nz + 1 + cz - 1) / cz);
}

__global__ void k_homogenize(const double* __restrict__ rf, double* __restrict__ rc, int nxf, int nyf,
                             int nzf, double scale) {
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const long long nec = (long long)nxc * nyc * nzc;
    const long long E = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (E >= nec) return;
    const int I = (int)(E % nxc);
    const long long t = E / nxc;
    const int J = (int)(t % nyc), K = (int)(t / nyc);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long e = (2 * I + (c & 1)) + (long long)nxf * ((2 * J + ((c >> 1) & 1)) + (long long)nyf * (2 * K + (c >> 2)));
        s += rf[e];
    }
    rc[E] = (0.125 * scale) * s;
}

// rho^p: repeated multiplication for integer p (FP64 pow is slow on this part)
__device__ __forceinline__ double rpow(double r, double p, int ip) {
    if (ip >= 0) {
        double v = 1.0;
        for (int i = 0; i < ip; ++i) v *= r;
        return v;
    }
    return pow(r, p);
}

// D^-1 of the first two pre-smoothing sweeps: node (i, j, k) sums E over the
// in-grid elements (i-1..i, j-1..j, k-1..k) in a fixed order (E carries the
// level scale 2^l); one thread per node of an x-y tile, z from the grid
template <typename T>
__global__ void __launch_bounds__(256) k_diag_inv(const T* __restrict__ E, int nx, int ny, int nz, T kdiag,
                                                  T* __restrict__ D) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i > nx || j > ny) return;
    T s = T(0);
    for (int ez = k - 1; ez <= k; ++ez)
        for (int ey = j - 1; ey <= j; ++ey)
            for (int ex = i - 1; ex <= i; ++ex)
                if (ex >= 0 && ex < nx && ey >= 0 && ey < ny && ez >= 0 && ez < nz)
                    s += E[ex + nx * (ey + ny * ez)];
    D[i + (nx + 1) * (j + (ny + 1) * k)] = s > T(0) ? T(1) / (kdiag * s) : T(0);
}

__global__ void k_simp(long long ne, const double* __restrict__ rho, double scale, double E0, double Emin,
                       double penal, int ipenal, double* __restrict__ E64, float* __restrict__ E32, int* bad) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const double r = rho[e];
    if (!(r >= 0.0 && r <= 1.0)) atomicExch(bad, 1);
    const double rc = fmin(fmax(r, 0.0), 1.0);
    const double E = scale * (Emin + rpow(rc, penal, ipenal) * (E0 - Emin));
    E64[e] = E;
    E32[e] = (float)E;
}

__global__ void k_mask_from_dofs(long long nn, const uint8_t* __restrict__ fixed, uint8_t* __restrict__ mask) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= nn) return;
    mask[n] = (uint8_t)((fixed[3 * n] ? 1 : 0) | (fixed[3 * n + 1] ? 2 : 0) | (fixed[3 * n + 2] ? 4 : 0));
}

__global__ void k_inject_mask(const uint8_t* __restrict__ maskf, uint8_t* __restrict__ maskc, int nxf, int nyf,
                              int nzf) {
    const int NXc = nxf / 2 + 1, NYc = nyf / 2 + 1, NZc = nzf / 2 + 1;
    const long long nnc = (long long)NXc * NYc * NZc;
    const long long N = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (N >= nnc) return;
    const int I = (int)(N % NXc);
    const long long t = N / NXc;
    const int J = (int)(t % NYc), K = (int)(t / NYc);
    maskc[N] = maskf[2 * I + (long long)(nxf + 1) * (2 * J + (long long)(nyf + 1) * 2 * K)];
}

__global__ void k_masked_copy(long long nn, const uint8_t* __restrict__ mask, const double* __restrict__ fin,
                              double* __restrict__ fout) {
    const long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (d >= 3 * nn) return;
    fout[d] = ((mask[d / 3] >> (d % 3)) & 1u) ? 0.0 : fin[d];
}

}  // namespace

template <typename T>
void restrict_residual(const Ctx& c, const Geom& gf, const uint8_t* maskf, const uint8_t* maskc, const T* rf,
                       T* rc) {
    const int czc = transfer_cz((long long)(gf.nx / 2 + 1) * (gf.ny / 2 + 1), gf.nz / 2 + 1, kRestrictCz);
    const dim3 grid((gf.nx / 2 + 1 + 31) / 32, (gf.ny / 2 + 1 + 7) / 8, (gf.nz / 2 + 1 + czc - 1) / czc);
    k_restrict_z<T><<<grid, dim3(32, 8), 0, c.s>>>(maskf, maskc, rf, rc, gf.nx, gf.ny, gf.nz, czc);
    TOPO_LAUNCH_CHECK(c);
}
template void restrict_residual<double>(const Ctx&, const Geom&, const uint8_t*, const uint8_t*, const double*,
                                        double*);
template void restrict_residual<float>(const Ctx&, const Geom&, const uint8_t*, const uint8_t*, const float*,
                                       float*);

template <typename T>
void prolong_add(const Ctx& c, const Geom& gf, const uint8_t* maskf, const uint8_t* maskc, const T* ec, T* uf) {
    k_prolong_z<T><<<prolong_grid(gf), dim3(32, 8), 0, c.s>>>(maskf, maskc, ec, uf, gf.nx, gf.ny, gf.nz, prolong_cz(gf));
    TOPO_LAUNCH_CHECK(c);
}
template void prolong_add<double>(const Ctx&, const Geom&, const uint8_t*, const uint8_t*, const double*,
                                  double*);
template void prolong_add<float>(const Ctx&, const Geom&, const uint8_t*, const uint8_t*, const float*, float*);

template <typename TE>
void prolong_add_bf16(const Ctx& c, const Geom& gf, const uint8_t* maskf, const uint8_t* maskc, const TE* ec,
                      bf16* uf) {
    k_prolong_z<float, TE, bf16><<<prolong_grid(gf), dim3(32, 8), 0, c.s>>>(maskf, maskc, ec, uf, gf.nx, gf.ny, gf.nz,
                                                                        prolong_cz(gf));
    TOPO_LAUNCH_CHECK(c);
}
template void prolong_add_bf16<float>(const Ctx&, const Geom&, const uint8_t*, const uint8_t*, const float*, bf16*);
template void prolong_add_bf16<bf16>(const Ctx&, const Geom&, const uint8_t*, const uint8_t*, const bf16*, bf16*);

void homogenize(const Ctx& c, const Geom& gf, const double* rho_f, double* rho_c, double scale) {
    const long long nec = (long long)(gf.nx / 2) * (gf.ny / 2) * (gf.nz / 2);
    k_homogenize<<<grid_for(nec, 256), 256, 0, c.s>>>(rho_f, rho_c, gf.nx, gf.ny, gf.nz, scale);
    TOPO_LAUNCH_CHECK(c);
}

template <typename T>
void diag_inverse(const Ctx& c, const Geom& g, const T* E, T kdiag, T* Dinv) {
    const dim3 grid((g.nx + 1 + 31) / 32, (g.ny + 1 + 7) / 8, g.nz + 1);
    k_diag_inv<T><<<grid, dim3(32, 8), 0, c.s>>>(E, g.nx, g.ny, g.nz, kdiag, Dinv);
    TOPO_LAUNCH_CHECK(c);
}
template void diag_inverse<double>(const Ctx&, const Geom&, const double*, double, double*);
template void diag_inverse<float>(const Ctx&, const Geom&, const float*, float, float*);

void simp_moduli(const Ctx& c, long long ne, const double* rho, double scale, double E0, double Emin, double penal,
                 double* E64, float* E32, int* bad_flag) {
    const int ip = (penal == (double)(int)penal && penal >= 0.0 && penal <= 16.0) ? (int)penal : -1;
    k_simp<<<grid_for(ne, 256), 256, 0, c.s>>>(ne, rho, scale, E0, Emin, penal, ip, E64, E32, bad_flag);
    TOPO_LAUNCH_CHECK(c);
}

void mask_from_dofs(const Ctx& c, long long nn, const uint8_t* fixed_dofs, uint8_t* mask) {
    k_mask_from_dofs<<<grid_for(nn, 256), 256, 0, c.s>>>(nn, fixed_dofs, mask);
    TOPO_LAUNCH_CHECK(c);
}

void inject_mask(const Ctx& c, const Geom& gf, const uint8_t* maskf, uint8_t* maskc) {
    const long long nnc = (long long)(gf.nx / 2 + 1) * (gf.ny / 2 + 1) * (gf.nz / 2 + 1);
    k_inject_mask<<<grid_for(nnc, 256), 256, 0, c.s>>>(maskf, maskc, gf.nx, gf.ny, gf.nz);
    TOPO_LAUNCH_CHECK(c);
}

void masked_copy_load(const Ctx& c, long long nn, const uint8_t* mask, const double* fin, double* fout) {
    k_masked_copy<<<grid_for(3 * nn, 256), 256, 0, c.s>>>(nn, mask, fin, fout);
    TOPO_LAUNCH_CHECK(c);
}

}  // namespace topo
