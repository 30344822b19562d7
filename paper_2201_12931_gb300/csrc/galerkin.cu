// Galerkin coarse operators with stored coarse element matrices: the
// "standard" scheme the paper compares its homogenization against
// (Sec. 4.2.2, Sec. 6, Table homogenization_comp).
//
// On a structured grid the Galerkin product P^T K P is itself a sum of
// coarse element matrices: with trilinear interpolation each fine element
// lies inside one coarse element, and its nodal values are interpolated
// from that coarse element's 8 nodes only, so
//     Ke_{l+1}(E) = sum over the 8 children o of E of  P_o^T Ke_l(child) P_o,
// P_o = Q_o (x) I_3, Q_o[b][a] = prod_d w(o_d + b_d, a_d), w(p, a) the 1-D
// hat weight of coarse node a at fine position p in {0, 1, 2}.  Level 0 is
// Ke_0(e) = E_e K0.  Fixed DOFs are applied on each level as in the
// matrix-free operator (P_f K P_f + I - P_f, fixed u read as zero); for
// supports on coarse-grid nodes (every fixed fine DOF interpolates from
// fixed coarse DOFs only) this equals the Galerkin product of the
// constrained operators.
//
// Storage: element-major, Ke[E * 576 + 24 r + s], FP64 (and an FP32 copy for
// mixed-precision handles).  The operator on a Galerkin level gathers per
// node the 3 rows of its <= 8 elements (deterministic, no atomics) and forms
// the Jacobi diagonal from the same rows.
#include "common.cuh"

namespace topo {

namespace {

__constant__ double c_Q[8 * 64];   // Q_o[b][a], o-major
// Level 1: Ke_1(E) = sum_o E_child(o) G_o with G_o = P_o^T K0 P_o (o-major,
// 8 x 576), one thread per (coarse element, entry)
__global__ void k_galerkin_build1(const double* __restrict__ G, const double* __restrict__ Ef, double* __restrict__ Kc,
                                  int nxf, int nyf, int nzf) {
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const long long total = (long long)nxc * nyc * nzc * 576;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const long long E = t / 576;
    const int q = (int)(t % 576);
    const int I = (int)(E % nxc), J = (int)((E / nxc) % nyc), K = (int)(E / ((long long)nxc * nyc));
    double v = 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const long long ec = (2 * I + (o & 1)) + (long long)nxf * ((2 * J + ((o >> 1) & 1)) + (long long)nyf * (2 * K + (o >> 2)));
        v += Ef[ec] * G[o * 576 + q];
    }
    Kc[t] = v;
}

// One CTA per coarse element E: Ke_{l+1}(E) = sum_o P_o^T Kc_o P_o by the
// Kronecker form: T = Kc Q_o (per 3x3 component block), then Q_o^T T.
// Children are elements of the finer level; Kc = Ecf[child] * K0 when Kf is
// null (level 0 children), else Kf[child].
__global__ void __launch_bounds__(192) k_galerkin_build(const double* __restrict__ K0, const double* __restrict__ Ecf,
                                                        const double* __restrict__ Kf, double* __restrict__ Kc,
                                                        int nxf, int nyf, int nzf) {
    __shared__ double sK[576], sT[576], sQ[64];
    const int nxc = nxf / 2, nyc = nyf / 2;
    const long long E = blockIdx.x;
    const int I = (int)(E % nxc), J = (int)((E / nxc) % nyc), K = (int)(E / ((long long)nxc * nyc));
    double acc[3] = {0.0, 0.0, 0.0};   // entries t, t + 192, t + 384
    for (int o = 0; o < 8; ++o) {
        const long long ec = (2 * I + (o & 1)) + (long long)nxf * ((2 * J + ((o >> 1) & 1)) + (long long)nyf * (2 * K + (o >> 2)));
        const double s = Kf ? 1.0 : Ecf[ec];
        const double* src = Kf ? Kf + ec * 576 : K0;
        for (int t = threadIdx.x; t < 576; t += blockDim.x) sK[t] = s * src[t];
        for (int t = threadIdx.x; t < 64; t += blockDim.x) sQ[t] = c_Q[o * 64 + t];
        __syncthreads();
        // T[3b + c][3a' + d] = sum_b' Kc[3b + c][3b' + d] Q[b'][a']
        for (int t = threadIdx.x; t < 576; t += blockDim.x) {
            const int r = t / 24, col = t % 24, ap = col / 3, d = col % 3;
            double v = 0.0;
#pragma unroll
            for (int bp = 0; bp < 8; ++bp) v += sK[r * 24 + 3 * bp + d] * sQ[bp * 8 + ap];
            sT[t] = v;
        }
        __syncthreads();
        // Ke[3a + c][col] += sum_b Q[b][a] T[3b + c][col]
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int t = threadIdx.x + 192 * q;
            const int r = t / 24, col = t % 24, a = r / 3, c = r % 3;
            double v = 0.0;
#pragma unroll
            for (int b = 0; b < 8; ++b) v += sQ[b * 8 + a] * sT[(3 * b + c) * 24 + col];
            acc[q] += v;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) Kc[E * 576 + threadIdx.x + 192 * q] = acc[q];
}

// y = op(u) on a Galerkin level, one thread per DOF (node n, component c):
// rows 3a + c of the <= 8 element matrices around n; same modes and
// Dirichlet convention as the matrix-free operator.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_elem_op(const T* __restrict__ Ke, const uint8_t* __restrict__ mask,
                                                 const T* __restrict__ u, const T* __restrict__ f, T* __restrict__ out,
                                                 int nx, int ny, int nz, T omega) {
    const int NX = nx + 1, NY = ny + 1;
    const long long ndof = 3LL * NX * NY * (nz + 1);
    const long long dof = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (dof >= ndof) return;
    const long long n = dof / 3;
    const int c = (int)(dof % 3);
    const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / ((long long)NX * NY));
    const bool fixed = (mask[n] >> c) & 1u;
    T y = T(0), dg = T(0);
    for (int az = 0; az < 2; ++az)
        for (int ay = 0; ay < 2; ++ay)
            for (int ax = 0; ax < 2; ++ax) {
                // element whose corner (ax, ay, az) is node n
                const int ex = i - ax, ey = j - ay, ez = k - az;
                if (ex < 0 || ex >= nx || ey < 0 || ey >= ny || ez < 0 || ez >= nz) continue;
                const long long e = ex + (long long)nx * (ey + (long long)ny * ez);
                const int row = 3 * (ax + 2 * ay + 4 * az) + c;
                const T* kr = Ke + e * 576 + row * 24;
                dg += kr[row];
                if (MODE != ST_JACOBI0) {
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        const long long nb = (ex + (b & 1)) + (long long)NX * ((ey + ((b >> 1) & 1)) + (long long)NY * (ez + (b >> 2)));
                        const unsigned mb = mask[nb];
#pragma unroll
                        for (int d = 0; d < 3; ++d)
                            if (!((mb >> d) & 1u)) y += kr[3 * b + d] * u[3 * nb + d];
                    }
                }
            }
    const T uo = MODE != ST_JACOBI0 ? u[dof] : T(0);
    const T fo = MODE != ST_APPLY ? f[dof] : T(0);
    T r;
    if (MODE == ST_APPLY) r = fixed ? uo : y;
    else if (MODE == ST_RESID) r = fo - (fixed ? uo : y);
    else if (MODE == ST_JACOBI) r = fixed ? uo + omega * (fo - uo) : uo + omega * (fo - y) / dg;
    else r = omega * fo / (fixed ? T(1) : dg);
    out[dof] = r;
}

}  // namespace

static void interpolation_blocks(double* Q) {
    for (int o = 0; o < 8; ++o)
        for (int b = 0; b < 8; ++b)
            for (int a = 0; a < 8; ++a) {
                double w = 1.0;
                for (int d = 0; d < 3; ++d) {
                    const int p = ((o >> d) & 1) + ((b >> d) & 1);   // fine position 0..2
                    const int ad = (a >> d) & 1;                      // coarse node at 0 or 2
                    const int dist = p > 2 * ad ? p - 2 * ad : 2 * ad - p;
                    w *= dist == 0 ? 1.0 : (dist == 1 ? 0.5 : 0.0);
                }
                Q[o * 64 + b * 8 + a] = w;
            }
}

// Q_o in constant memory of each device (call with the device current)
void galerkin_init_constants() {
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && done[dev]) return;
    double Q[8 * 64];
    interpolation_blocks(Q);
    cudaMemcpyToSymbol(c_Q, Q, sizeof(Q));
    if (dev < 64) done[dev] = true;
}

// G_o = P_o^T K0 P_o on the host: G[o*576 + (3a + c)*24 + 3a' + d] =
// sum_{b, b'} Q_o[b][a] K0[3b + c][3b' + d] Q_o[b'][a']
void galerkin_child_matrices(const double* K0, double* G) {
    double Q[8 * 64];
    interpolation_blocks(Q);
    for (int o = 0; o < 8; ++o)
        for (int r = 0; r < 24; ++r)
            for (int col = 0; col < 24; ++col) {
                const int a = r / 3, c = r % 3, ap = col / 3, d = col % 3;
                double v = 0.0;
                for (int b = 0; b < 8; ++b)
                    for (int bp = 0; bp < 8; ++bp)
                        v += Q[o * 64 + b * 8 + a] * K0[(3 * b + c) * 24 + 3 * bp + d] * Q[o * 64 + bp * 8 + ap];
                G[o * 576 + r * 24 + col] = v;
            }
}

void galerkin_build(const Ctx& c, const Geom& gf, const double* K0, const double* G, const double* Ef, const double* Kf,
                    double* Kc) {
    const long long nec = (long long)(gf.nx / 2) * (gf.ny / 2) * (gf.nz / 2);
    if (!Kf) {   // children on level 0: scaled sum of the constant G_o
        const long long total = nec * 576;
        k_galerkin_build1<<<(unsigned)((total + 255) / 256), 256, 0, c.s>>>(G, Ef, Kc, gf.nx, gf.ny, gf.nz);
    } else {
        k_galerkin_build<<<(unsigned)nec, 192, 0, c.s>>>(K0, Ef, Kf, Kc, gf.nx, gf.ny, gf.nz);
    }
    TOPO_LAUNCH_CHECK(c);
}

template <typename T>
void elem_op(const Ctx& c, int mode, const Geom& g, const T* Ke, const uint8_t* mask, const T* u, const T* f, T* out,
             T omega) {
    const long long nd = 3 * g.nn;
    const unsigned blocks = (unsigned)((nd + 255) / 256);
    switch (mode) {
        case ST_APPLY: k_elem_op<T, ST_APPLY><<<blocks, 256, 0, c.s>>>(Ke, mask, u, f, out, g.nx, g.ny, g.nz, omega); break;
        case ST_JACOBI: k_elem_op<T, ST_JACOBI><<<blocks, 256, 0, c.s>>>(Ke, mask, u, f, out, g.nx, g.ny, g.nz, omega); break;
        case ST_RESID: k_elem_op<T, ST_RESID><<<blocks, 256, 0, c.s>>>(Ke, mask, u, f, out, g.nx, g.ny, g.nz, omega); break;
        default: k_elem_op<T, ST_JACOBI0><<<blocks, 256, 0, c.s>>>(Ke, mask, u, f, out, g.nx, g.ny, g.nz, omega); break;
    }
    TOPO_LAUNCH_CHECK(c);
}
template void elem_op<double>(const Ctx&, int, const Geom&, const double*, const uint8_t*, const double*, const double*,
                              double*, double);
template void elem_op<float>(const Ctx&, int, const Geom&, const float*, const uint8_t*, const float*, const float*,
                             float*, float);

}  // namespace topo
