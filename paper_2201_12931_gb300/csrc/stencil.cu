// Matrix-free element-by-element operator (Sec. 4.2.1: a node's row of K is
// the modulus-weighted sum of the reference element matrix over the 8
// elements around it), fused with the damped Jacobi sweep
// (Sec. 3.2) and the residual (Eq. residual); coarse-grid assembly; element
// energy and compliance sensitivity (Eq. sensitivity).
//
// Operator with Dirichlet rows: y = P_f K P_f u + (I - P_f) u, P_f zeroing the
// fixed DOFs, K = sum_e E_e A_e^T K0 A_e (E_e already holds 2^l on level l).
#include <type_traits>

#include "common.cuh"
#include "modal.cuh"
#include "operator.cuh"
#include "opio.cuh"

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
// The per-plane body is a generic lambda called with a compile-time buffer
// parity B = P & 1, so that double buffers and the two-plane register history
// are addressed statically (no register moves, no dynamic indexing).
// T: arithmetic, f, E; TU: storage of u; TO: storage of the output.
template <typename T, typename TU, typename TO, int MODE, bool DOT>
__global__ void __launch_bounds__(kOpTX * op_ty<T>(), sizeof(T) == 4 ? 2 : 1)
    k_op(const ModalK<T> mk, const typename OpStore<T>::type* __restrict__ E, const uint8_t* __restrict__ mask,
         const TU* __restrict__ u, const typename OpStore<T>::type* __restrict__ f, TO* __restrict__ out,
         const int nx, const int ny, const int nz, const int cz, const T omega, double* __restrict__ partials,
         TO* __restrict__ pout, const double* __restrict__ beta, const typename OpStore<T>::type* __restrict__ Dinv) {
    constexpr int TX = kOpTX, TY = op_ty<T>();
    constexpr bool NEEDU = (MODE != ST_JACOBI0);
    constexpr bool NEEDD = (MODE == ST_JACOBI || MODE == ST_JACOBI0 || MODE == ST_JACOBI2);
    constexpr bool J2 = (MODE == ST_JACOBI2);   // u1 = omega D^-1 f formed from f: u is not read
    constexpr bool NEEDF = (MODE != ST_APPLY);   // ST_APPLY_P: p_old in the f slots
    constexpr bool PUPD = (MODE == ST_APPLY_P);
    constexpr int nU = (TY + 1) * (TX + 1) * 4, nC = 3 * TY * TX * 4, nEs = TY * TX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sred[32];
    // double-FP32 arithmetic: the node values of each plane are shifted by
    // that plane's value at the tile's corner node (in FP64, before the
    // split), so that the FP32 pairs carry the displacement relative to the
    // tile rather than its absolute size.  K annihilates a translation, and
    // within a plane the shift is one; between the two planes of an element
    // it leaves only the z-difference of the mean mode, which is added back
    // (4 (ref_P - ref_{P-1}) in element_modal).  Thread 0 keeps the last
    // reference (sref_last) and publishes the split correction of each plane
    // in a ring of four slots (szc).
    constexpr bool kDF = std::is_same<T, dfl>::value;
    __shared__ double sref_last[4];
    __shared__ __align__(16) float szc[4][8];
    if (kDF && threadIdx.x == 0 && threadIdx.y == 0) sref_last[0] = sref_last[1] = sref_last[2] = 0.0;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int NX = nx + 1, NY = ny + 1;
    const int i0 = blockIdx.x * (TX - 1), j0 = blockIdx.y * (TY - 1);
    const int kz0 = blockIdx.z * cz;
    const int kz1 = min(kz0 + cz, nz + 1);
    const int in = i0 - 1 + tx, jn = j0 - 1 + ty;
    const bool node_ok = in >= 0 && in < NX && jn >= 0 && jn < NY;
    const bool col_ok = in >= 0 && in < nx && jn >= 0 && jn < ny;
    const bool out_ok = tx >= 1 && ty >= 1 && node_ok;
    const bool has_halo = tid < TY + 1 + TX;
    [[maybe_unused]] const bool halo_warp = (tid >> 5) <= ((TY + TX) >> 5);   // warp holds halo threads
    const int hsx = tid < TY + 1 ? TX : tid - TY - 1;
    const int hsy = tid < TY + 1 ? tid : TY;
    const int hx = i0 - 1 + hsx, hy = j0 - 1 + hsy;
    const bool halo_ok = has_halo && hx >= 0 && hx < NX && hy >= 0 && hy < NY;
    // 32-bit vector indices (topo_create_grid keeps 3 * nodes below 2^31):
    // fewer address instructions; the fused K.p keeps 64-bit indices, with
    // which it needs fewer registers (measured: 32-bit spilled and was slower)
    using Ix = std::conditional_t<PUPD, long long, int>;
    const Ix nplane = (Ix)NX * NY;
    const int own_xy = node_ok ? in + NX * jn : 0;
    const int halo_xy = halo_ok ? hx + NX * hy : 0;
    const int col_xy = col_ok ? in + nx * jn : 0;
    const int uoff = (ty * (TX + 1) + tx) * 4;      // own slot in a plane buffer
    const int hoff = (hsy * (TX + 1) + hsx) * 4;    // halo slot
    const int coff = (ty * TX + tx) * 4;            // own slot in a contribution buffer

    T fb[2][12], top[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) fb[0][i] = fb[1][i] = top[i] = T(0);
    T st00[3] = {}, st10[3] = {}, st01[3] = {}, st11[3] = {};
    T stE = T(0);
    double dot = 0.0;
    [[maybe_unused]] float dotf = 0.0f;
    // per-plane register slots, slot = plane & 3: own node raw u, f, mask,
    // the column modulus of the layer below the plane, and (two slots) the
    // halo node; planes P-2 .. P+1 are live in step P, so no copies occur.
    // Double-FP32 arithmetic keeps the loaded FP64 words in the slots and
    // splits them where they are used (a load is never consumed in the step
    // that issues it), and fetches f only one step ahead of its use.
    using TSl = std::conditional_t<kDF, double, T>;
    TSl su[4][3], sf[4][3], sE[4];
    unsigned sm[4];
    TSl shv[2][3];
    [[maybe_unused]] T shf[2][3] = {};        // halo p_old (ST_APPLY_P) or halo f (ST_JACOBI2)
    [[maybe_unused]] T sdv[4] = {};           // own node D^-1 per plane slot (ST_JACOBI2)
    [[maybe_unused]] T shd[2] = {};           // halo node D^-1 (ST_JACOBI2)
    [[maybe_unused]] const T bet = (PUPD && beta) ? T(*beta) : T(0);
    unsigned shm[2];
    [[maybe_unused]] double srf[2][3];   // plane references (double-FP32)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        su[q][0] = su[q][1] = su[q][2] = TSl(0);
        sf[q][0] = sf[q][1] = sf[q][2] = TSl(0);
        sE[q] = TSl(0);
        sm[q] = 0u;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        shv[q][0] = shv[q][1] = shv[q][2] = TSl(0);
        shm[q] = 0u;
        srf[q][0] = srf[q][1] = srf[q][2] = 0.0;
    }
    const int own3 = 3 * own_xy, halo3 = 3 * halo_xy;
    [[maybe_unused]] const int ref3 = 3 * (i0 + NX * j0);   // tile corner node (always in the grid)

    // load plane P into slot S (plane-uniform base + per-thread offset)
    auto fetch = [&](auto Sc, int P) {
        constexpr int S = decltype(Sc)::value;
        const bool pin = P >= 0 && P <= nz;
        const Ix pb = (Ix)P * nplane;
        if constexpr (kDF) {
            // raw FP64 words: own and halo node, the plane's reference (tile
            // corner node); f is loaded by the step (one plane behind)
            const bool ok = pin && node_ok;
            sm[S] = ok ? mask[pb + own_xy] : 0u;
            const TU* ub = u + 3 * pb + own3;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                su[S][c] = ok ? (double)ub[c] : 0.0;
                srf[S & 1][c] = pin ? (double)u[3 * pb + ref3 + c] : 0.0;
            }
            const bool okh = pin && halo_ok;
            shm[S & 1] = okh ? mask[pb + halo_xy] : 0u;
            const TU* hb = u + 3 * pb + halo3;
#pragma unroll
            for (int c = 0; c < 3; ++c) shv[S & 1][c] = okh ? (double)hb[c] : 0.0;
        } else if (NEEDU || NEEDF) {
            const bool ok = pin && node_ok;
            sm[S] = ok ? mask[pb + own_xy] : 0u;
            const TU* ub = u + 3 * pb + own3;
            const typename OpStore<T>::type* fb_ = f + 3 * pb + own3;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (NEEDU && !J2) su[S][c] = ok ? (T)ldv(ub + c) : T(0);
                if (NEEDF) sf[S][c] = ok ? (T)fb_[c] : T(0);
            }
            if constexpr (J2) sdv[S] = ok ? (T)Dinv[pb + own_xy] : T(0);
        }
        // residual and K.u: the halo loads behind a warp-uniform branch (two of
        // the eight warps hold halo threads); measured faster there, slower in
        // the Jacobi and fused modes
        [[maybe_unused]] constexpr bool kHaloBranch = (MODE == ST_RESID || MODE == ST_APPLY);
        if constexpr (NEEDU && !kDF) if (!kHaloBranch || halo_warp) {
            const bool okh = pin && halo_ok;
            shm[S & 1] = okh ? mask[pb + halo_xy] : 0u;
            [[maybe_unused]] const TU* hb = u + 3 * pb + halo3;
            if constexpr (!J2) {
#pragma unroll
                for (int c = 0; c < 3; ++c) shv[S & 1][c] = okh ? (T)ldv(hb + c) : T(0);
            }
            if constexpr (PUPD || J2) {
                const typename OpStore<T>::type* hf = f + 3 * pb + halo3;
#pragma unroll
                for (int c = 0; c < 3; ++c) shf[S & 1][c] = okh ? (T)hf[c] : T(0);
                if constexpr (J2) shd[S & 1] = okh ? (T)Dinv[pb + halo_xy] : T(0);
            }
        }
        sE[S] = (col_ok && P >= 1 && P <= nz) ? (TSl)E[(Ix)(P - 1) * nx * ny + col_xy] : TSl(0);
    };

    // step of node plane P, B = P & 3 (static)
    auto step = [&](auto Bc, int P) {
        constexpr int B = decltype(Bc)::value;
        constexpr int B2 = B & 1;                 // shared-memory buffer
        constexpr int SN = (B + 1) & 3;           // slot of plane P + 1
        constexpr int SO = (B + 2) & 3;           // slot of plane P - 2 (output)
        [[maybe_unused]] constexpr int SL = (B + 3) & 3;   // slot of plane P - 1
        T* const U = reinterpret_cast<T*>(smem_raw) + B2 * nU;
        T* const Cb = reinterpret_cast<T*>(smem_raw) + 2 * nU + B2 * nC;
        [[maybe_unused]] T* const Eb = reinterpret_cast<T*>(smem_raw) + 2 * nU + 2 * nC + B2 * nEs;
        // publish plane P (masked) and the stashed contributions of plane P - 2
        if constexpr (kDF) {
            // masked, shifted by the plane reference in FP64, then split
            const unsigned cm = sm[B];
            T mu[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) mu[c] = T((((cm >> c) & 1u) ? 0.0 : su[B][c]) - srf[B & 1][c]);
            if (tid == 0) {   // correction of the element between planes P - 1 and P
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const dfl d = df_from_double(srf[B & 1][c] - sref_last[c]);
                    szc[B][2 * c] = 4.0f * d.h;   // exact: a power of two
                    szc[B][2 * c + 1] = 4.0f * d.l;
                    sref_last[c] = srf[B & 1][c];
                }
            }
            st3(U + uoff, mu);
            if (has_halo) {
                const unsigned chm = shm[B & 1];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    mu[c] = T((((chm >> c) & 1u) ? 0.0 : shv[B & 1][c]) - srf[B & 1][c]);
                st3(U + hoff, mu);
            }
        } else if (NEEDU) {
            if constexpr (J2) {   // first sweep from zero: u1 = omega D^-1 f (no scaling at fixed DOFs)
                const unsigned cm1 = sm[B], chm1 = shm[B & 1];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    su[B][c] = omega * sf[B][c] * (((cm1 >> c) & 1u) ? T(1) : sdv[B]);
                    shv[B & 1][c] = omega * shf[B & 1][c] * (((chm1 >> c) & 1u) ? T(1) : shd[B & 1]);
                }
            }
            if constexpr (PUPD) {   // p = z + beta p_old (own and halo node)
                if (beta) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        su[B][c] = su[B][c] + bet * sf[B][c];
                        shv[B & 1][c] = shv[B & 1][c] + bet * shf[B & 1][c];
                    }
                }
            }
            const unsigned cm = sm[B];
            T mu[3] = {su[B][0], su[B][1], su[B][2]};
            if (cm) {
#pragma unroll
                for (int c = 0; c < 3; ++c) mu[c] = ((cm >> c) & 1u) ? T(0) : su[B][c];
            }
            st3(U + uoff, mu);
            if (has_halo) {
                const unsigned chm = shm[B & 1];
#pragma unroll
                for (int c = 0; c < 3; ++c) mu[c] = ((chm >> c) & 1u) ? T(0) : shv[B & 1][c];
                st3(U + hoff, mu);
            }
            st3(Cb + coff, st10);
            st3(Cb + nC / 3 + coff, st01);
            st3(Cb + 2 * (nC / 3) + coff, st11);
        }
        if constexpr (NEEDD && !J2) Eb[ty * TX + tx] = stE;
        // start loading plane P + 1 (its slot held plane P - 3, no longer needed)
        if (P + 1 <= kz1) fetch(std::integral_constant<int, SN>{}, P + 1);
        if constexpr (kDF && NEEDF) {
            // f of plane P - 1, output by the next step (slot SL is not read here)
            const bool okf = P - 1 >= 0 && P - 1 <= nz && node_ok;
            const double* ff = f + 3 * ((Ix)(P - 1) * nplane) + own3;
#pragma unroll
            for (int c = 0; c < 3; ++c) sf[SL][c] = okf ? ff[c] : 0.0;
        }
        __syncthreads();
        // output node plane Q = P - 2
        const int Q = P - 2;
        if (out_ok && Q >= kz0 && Q < kz1) {
            T y[3] = {T(0), T(0), T(0)};
            if (NEEDU) {
                T a0[3], a1[3], a2[3];
                ld3(Cb + coff - 4, a0);
                ld3(Cb + nC / 3 + coff - TX * 4, a1);
                ld3(Cb + 2 * (nC / 3) + coff - TX * 4 - 4, a2);
                if constexpr (kDF) {   // x and y in paired form (the same operations)
                    st2(y, add2(add2(add2(ld2(st00), ld2(a0)), ld2(a1)), ld2(a2)));
                    y[2] = st00[2] + a0[2] + a1[2] + a2[2];
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) y[c] = st00[c] + a0[c] + a1[c] + a2[c];
                }
            }
            // D^-1 of the output node: stored (first two sweeps) or formed
            // from the column sums of E over the two layers around plane Q
            [[maybe_unused]] T rD = T(1);
            if constexpr (J2) {
                rD = sdv[SO];
            } else if constexpr (NEEDD) {
                const T* e = Eb + ty * TX + tx;
                rD = recip(mk.kdiag * (e[0] + e[-1] + e[-TX] + e[-TX - 1]));
            }
            TO* o = out + 3 * ((Ix)Q * nplane) + own3;
            const unsigned m2 = sm[SO];
            typename DotAcc<T>::type d32 = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool fixed = (m2 >> c) & 1u;
                [[maybe_unused]] T uo;
                [[maybe_unused]] const T fo = T(sf[SO][c]);
                if constexpr (kDF) {   // fixed rows read u itself (the slots are not kept)
                    uo = fixed ? T((double)u[3 * ((Ix)Q * nplane) + own3 + c]) : T(0);
                } else {
                    uo = su[SO][c];
                }
                T r;
                if constexpr (MODE == ST_APPLY || MODE == ST_APPLY_P) {
                    r = fixed ? uo : y[c];
                    if (DOT) d32 += to_acc(uo) * to_acc(r);
                    if constexpr (PUPD) stv(pout + 3 * ((Ix)Q * nplane) + own3 + c, uo);
                } else if constexpr (MODE == ST_RESID) {
                    r = fo - (fixed ? uo : y[c]);
                    if (DOT) d32 += to_acc(r) * to_acc(r);
                } else if constexpr (MODE == ST_JACOBI || MODE == ST_JACOBI2) {
                    r = fixed ? uo + omega * (fo - uo) : uo + omega * (fo - y[c]) * rD;
                    if (DOT) d32 += fo * r;
                } else {
                    r = omega * fo * (fixed ? T(1) : rD);
                    if (DOT) d32 += fo * r;
                }
                stv(o + c, r);
            }
            if constexpr (DOT) {
                // FP32 kernels: FP32 per thread (one column of a z chunk),
                // FP64 across threads and CTAs, fixed order
                if constexpr (kDF || std::is_same<T, float>::value) dotf += d32;
                else dot += (double)d32;
            }
        }
        // face modes of plane P; element of layer P - 1; plane P - 1 completes
        if (P >= kz0 && P <= kz1) {
            if (NEEDU) {
                T c00[3], c10[3], c01[3], c11[3];
                ld3(U + uoff, c00);
                ld3(U + uoff + 4, c10);
                ld3(U + uoff + (TX + 1) * 4, c01);
                ld3(U + uoff + (TX + 1) * 4 + 4, c11);
                face_forward<T>(c00, c10, c01, c11, fb[B2]);
                T Bo[12], To[12];
                if constexpr (kDF) {
                    T zc[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) zc[c] = T(szc[B][2 * c], szc[B][2 * c + 1]);
                    element_modal<T>(mk, T(sE[B]), fb[B2 ^ 1], fb[B2], Bo, To, zc);
                } else {
                    element_modal<T>(mk, sE[B], fb[B2 ^ 1], fb[B2], Bo, To);
                }
                T A[12];
                if constexpr (kDF) {   // x and y of each corner group in paired form
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        st2(A + 3 * g, add2(ld2(top + 3 * g), ld2(Bo + 3 * g)));
                        A[3 * g + 2] = top[3 * g + 2] + Bo[3 * g + 2];
                    }
#pragma unroll
                    for (int i = 0; i < 12; ++i) top[i] = To[i];
                } else {
#pragma unroll
                    for (int i = 0; i < 12; ++i) {
                        A[i] = top[i] + Bo[i];
                        top[i] = To[i];
                    }
                }
                face_inverse<T>(A, st00, st10, st01, st11);
                if constexpr (kDF) {
                    // contributions to the neighbours' corners of plane P - 1 go
                    // straight to the buffer the next step's output reads (every
                    // thread has passed this step's barrier, so nobody reads it)
                    T* const Cn = reinterpret_cast<T*>(smem_raw) + 2 * nU + (B2 ^ 1) * nC;
                    st3(Cn + coff, st10);
                    st3(Cn + nC / 3 + coff, st01);
                    st3(Cn + 2 * (nC / 3) + coff, st11);
                }
            }
            if constexpr (NEEDD && !J2) stE = sE[SL] + sE[B];
        } else if (NEEDU && P == kz0 - 1) {
            T c00[3], c10[3], c01[3], c11[3];
            ld3(U + uoff, c00);
            ld3(U + uoff + 4, c10);
            ld3(U + uoff + (TX + 1) * 4, c01);
            ld3(U + uoff + (TX + 1) * 4 + 4, c11);
            face_forward<T>(c00, c10, c01, c11, fb[B2]);
        }
    };

    using S0 = std::integral_constant<int, 0>;
    using S1 = std::integral_constant<int, 1>;
    using S2 = std::integral_constant<int, 2>;
    using S3 = std::integral_constant<int, 3>;
    // planes kz0-1 .. kz1+1 are processed; the range is widened to whole
    // groups of four (P = 0 mod 4 first) -- the extra steps are guarded no-ops
    const int Pfirst = kz0 - 1;
    int P = Pfirst - (((Pfirst % 4) + 4) % 4);
    switch (Pfirst - P) {   // prefetch plane Pfirst into its slot
        case 0: fetch(S0{}, Pfirst); break;
        case 1: fetch(S1{}, Pfirst); break;
        case 2: fetch(S2{}, Pfirst); break;
        default: fetch(S3{}, Pfirst); break;
    }
    for (; P <= kz1 + 1; P += 4) {
        step(S0{}, P);
        step(S1{}, P + 1);
        step(S2{}, P + 2);
        step(S3{}, P + 3);
    }
    if (DOT) {
        double v = (kDF || std::is_same<T, float>::value) ? (double)dotf : dot;
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
    constexpr int TY = op_ty<T>();
    return sizeof(T) * (2 * (TY + 1) * (kOpTX + 1) * 4 + 2 * 3 * TY * kOpTX * 4 + 2 * TY * kOpTX);
}

template <typename T, int MODE, bool DOT, typename TU = T, typename TO = T>
void launch_op(const Ctx& c, const OpLaunch& L, const ModalK<T>& mk, const typename OpStore<T>::type* E,
               const uint8_t* mask, const TU* u, const typename OpStore<T>::type* f, TO* out, T omega, double* dot,
               TO* pout = nullptr, const double* beta = nullptr,
               const typename OpStore<T>::type* Dinv = nullptr) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_op<T, TU, TO, MODE, DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)op_smem_bytes<T>());
        attr = true;
    }
    k_op<T, TU, TO, MODE, DOT><<<dim3(L.gx, L.gy, L.gz), dim3(kOpTX, op_ty<T>()), op_smem_bytes<T>(), c.s>>>(
        mk, E, mask, u, f, out, L.g.nx, L.g.ny, L.g.nz, L.cz, omega, dot, pout, beta, Dinv);
    TOPO_LAUNCH_CHECK(c);
}

template <typename T, int MODE>
void launch_mode(const Ctx& c, const OpLaunch& L, const ModalK<T>& mk, const T* E, const uint8_t* mask, const T* u,
                 const T* f, T* out, T omega, double* dot, const T* Dinv, T* pout = nullptr,
                 const double* beta = nullptr) {
    if (dot) launch_op<T, MODE, true>(c, L, mk, E, mask, u, f, out, omega, dot, pout, beta, Dinv);
    else launch_op<T, MODE, false>(c, L, mk, E, mask, u, f, out, omega, nullptr, pout, beta, Dinv);
}

// Dense assembly of the coarsest operator with identity Dirichlet rows.
// Dense coarsest operator, deterministic: one thread per (row DOF, neighbour
// node, column component) gathers, in a fixed order, the <= 8 elements that
// contain both nodes -- element matrices E_e K0, or the stored Ke[e] of a
// Galerkin level.  Rows and columns of fixed DOFs stay zero here.
__global__ void k_assemble(const double* __restrict__ K0, const double* __restrict__ E,
                           const double* __restrict__ Ke, const uint8_t* __restrict__ mask, double* __restrict__ A,
                           int nx, int ny, int nz, int npad) {
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    const long long total = 3LL * NX * NY * NZ * 81;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int d = (int)(t % 3);
    const int o = (int)((t / 3) % 27);
    const long long rdof = t / 81;
    const int c = (int)(rdof % 3);
    const long long nr = rdof / 3;
    const int i = (int)(nr % NX), j = (int)((nr / NX) % NY), k = (int)(nr / ((long long)NX * NY));
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int i2 = i + dx, j2 = j + dy, k2 = k + dz;
    if (i2 < 0 || i2 >= NX || j2 < 0 || j2 >= NY || k2 < 0 || k2 >= NZ) return;
    const long long nc = i2 + (long long)NX * (j2 + (long long)NY * k2);
    if (((mask[nr] >> c) & 1u) || ((mask[nc] >> d) & 1u)) return;
    double v = 0.0;
    for (int ez = (k > k2 ? k : k2) - 1; ez <= (k < k2 ? k : k2); ++ez)
        for (int ey = (j > j2 ? j : j2) - 1; ey <= (j < j2 ? j : j2); ++ey)
            for (int ex = (i > i2 ? i : i2) - 1; ex <= (i < i2 ? i : i2); ++ex) {
                if (ex < 0 || ex >= nx || ey < 0 || ey >= ny || ez < 0 || ez >= nz) continue;
                const long long e = ex + (long long)nx * (ey + (long long)ny * ez);
                const int a = (i - ex) + 2 * (j - ey) + 4 * (k - ez);
                const int b = (i2 - ex) + 2 * (j2 - ey) + 4 * (k2 - ez);
                const int r = 3 * a + c, s = 3 * b + d;
                v += Ke ? Ke[e * 576 + r * 24 + s] : E[e] * K0[r * 24 + s];
            }
    A[(3 * nr + c) * (long long)npad + 3 * nc + d] = v;
}

__global__ void k_assemble_diag(const uint8_t* __restrict__ mask, double* __restrict__ A, int n, int npad) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= npad) return;
    if (d >= n || ((mask[d / 3] >> (d % 3)) & 1u)) A[(long long)d * npad + d] = 1.0;
}

// rho^p by repeated multiplication for integer p (FP64 pow is slow on GB300)
__device__ __forceinline__ double ipow(double r, double p, int ip) {
    if (ip >= 0) {
        double v = 1.0;
        for (int i = 0; i < ip; ++i) v *= r;
        return v;
    }
    return pow(r, p);
}

// Element energy u_e^T K0 u_e in the modal (Walsh-Hadamard) basis, compliance
// partial sums sum_e E_e se_e and the sensitivity -p rho^(p-1) (E0-Emin) se_e,
// in FP64 (FP64 handles; mixed-precision handles use k_energy_sens_z).
__global__ void __launch_bounds__(256) k_energy_sens(ModalCoef mc, const double* __restrict__ u,
                                                     const double* __restrict__ rho, int nx, int ny, int nz,
                                                     double E0, double Emin, double penal, int ipenal,
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
        const double rp1 = ipenal >= 1 ? ipow(r, penal - 1.0, ipenal - 1) : pow(r, penal - 1.0);
        const double Ee = Emin + rp1 * r * (E0 - Emin);
        csum += Ee * se;
        if (dc) dc[e] = -penal * rp1 * (E0 - Emin) * se;
    }
    const double tsum = block_sum(csum, sred);
    if (threadIdx.x == 0) partials[blockIdx.x] = tsum;
}

// Mixed-precision handles: the corner-0 displacement is subtracted (K0
// annihilates translations, so the energy is unchanged) and the small
// relative displacements are transformed and contracted in FP32; the
// compliance is still accumulated in FP64.  The subtraction uses the integer
// split of each FP64 value into FP32 words h + l (dfloat.cuh): (h - h0) +
// (l - l0) in FP32 carries the difference to FP32 accuracy without FP64
// instructions, which run on a narrow pipe.  Indices are 32-bit (the grid
// limit of create_grid).
// Marching along z: a work item is an (i, j) element column and a chunk of
// cz layers; the upper face
// of one element (4 nodes, split once into FP32 words) is the lower face of
// the next, so every node is read and split about once per chunk instead of
// once per element around it; the FP64 compliance partials are summed per
// thread in z order.
__global__ void __launch_bounds__(256) k_energy_sens_z(ModalCoef mc, const double* __restrict__ u,
                                                       const double* __restrict__ rho, int nx, int ny, int nz,
                                                       int cz, double E0, double Emin, double penal, int ipenal,
                                                       double* __restrict__ dc, double* __restrict__ partials) {
    __shared__ double sred[32];
    const int NX = nx + 1, NY = ny + 1;
    const int ncol = nx * ny, nplane = NX * NY, nchunk = (nz + cz - 1) / cz;
    const int items = ncol * nchunk;
    double csum = 0.0;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        const int col = it % ncol, q = it / ncol;
        const int i = col % nx, j = col / nx;
        const int k0 = q * cz, k1 = min(nz, k0 + cz);
        const int n00 = i + NX * j;
        dfl lo[12], hi[12];
        auto face = [&](int k, dfl* f) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int nd = n00 + (a & 1) + NX * (a >> 1) + nplane * k;
#pragma unroll
                for (int c = 0; c < 3; ++c) f[3 * a + c] = df_from_double(u[3 * nd + c]);
            }
        };
        face(k0, lo);
        for (int k = k0; k < k1; ++k) {
            face(k + 1, hi);
            float ue[24];
            ue[0] = ue[1] = ue[2] = 0.f;
#pragma unroll
            for (int a = 1; a < 8; ++a) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const dfl v = a < 4 ? lo[3 * a + c] : hi[3 * (a - 4) + c];
                    ue[3 * a + c] = __fadd_rn(__fsub_rn(v.h, lo[c].h), __fsub_rn(v.l, lo[c].l));
                }
            }
            float m[24];
            modal_forward(ue, m);
            const double se = (double)modal_energy<float>(mc, m);
            const int e = col + ncol * k;
            const double r = rho[e];
            const double rp1 = ipenal >= 1 ? ipow(r, penal - 1.0, ipenal - 1) : pow(r, penal - 1.0);
            const double Ee = Emin + rp1 * r * (E0 - Emin);
            csum += Ee * se;
            if (dc) dc[e] = -penal * rp1 * (E0 - Emin) * se;
#pragma unroll
            for (int x = 0; x < 12; ++x) lo[x] = hi[x];
        }
    }
    const double tsum = block_sum(csum, sred);
    if (threadIdx.x == 0) partials[blockIdx.x] = tsum;
}

}  // namespace

// Launch geometry: x-y tiles of (kOpTX - 1) x (ty - 1) output node columns
// and z chunks of at least 16 planes (each chunk recomputes one layer and
// pays about 4.5 extra exchange steps).  At least target_ctas CTAs; beyond
// that the number of chunks minimises (waves of resident CTAs) x (steps per
// CTA), so that a last, nearly empty wave does not cost a whole CTA time.
OpLaunch op_launch(const Geom& g, int ty, int target_ctas, int resident_ctas) {
    OpLaunch L;
    L.g = g;
    L.gx = (g.nx + 1 + kOpTX - 2) / (kOpTX - 1);
    L.gy = (g.ny + 1 + ty - 2) / (ty - 1);
    const long long xy = (long long)L.gx * L.gy;
    const int NZ = g.nz + 1;
    const long long gz_min = (target_ctas + xy - 1) / xy;
    // chunks of at least 4 planes (each chunk re-reads 3 planes): small
    // levels get many short chunks, as their launches are bound by the
    // latency of the march, not by memory
    constexpr int kMinCz = 4;
    auto chunk = [&](long long gz) {
        int cz = (int)((NZ + gz - 1) / gz);
        return cz < kMinCz ? (NZ < kMinCz ? NZ : kMinCz) : cz;
    };
    int best_cz = chunk(gz_min);
    double best_cost = -1.0;
    for (long long gz = gz_min; gz <= 8 * gz_min; ++gz) {
        const int cz = chunk(gz);
        const long long gz_eff = (NZ + cz - 1) / cz;
        const long long waves = (xy * gz_eff + resident_ctas - 1) / resident_ctas;
        const double cost = (double)waves * (cz + 4.5);
        if (best_cost < 0.0 || cost < best_cost) {
            best_cost = cost;
            best_cz = cz;
        }
        if (cz <= kMinCz) break;   // chunks cannot get shorter
    }
    L.cz = best_cz;
    L.gz = (NZ + best_cz - 1) / best_cz;
    return L;
}

// resident CTAs per SM: 2 for the FP32 kernel (launch bounds 256 x 2), 1 for FP64
OpLaunch op_launch32(const Geom& g, int nsm) { return op_launch(g, op_ty<float>(), 1216, 2 * nsm); }
OpLaunch op_launch64(const Geom& g, int nsm) { return op_launch(g, op_ty<double>(), 608, nsm); }

template <typename T>
int stencil(const Ctx& c, int mode, const OpLaunch& L, const ModalK<T>& mk, const T* E, const uint8_t* mask,
            const T* u, const T* f, T* out, T omega, double* dot, const T* Dinv, T* pout, const double* beta) {
    switch (mode) {
        case ST_APPLY_P:
            launch_mode<T, ST_APPLY_P>(c, L, mk, E, mask, u, f, out, omega, dot, Dinv, pout, beta);
            break;
        case ST_APPLY: launch_mode<T, ST_APPLY>(c, L, mk, E, mask, u, f, out, omega, dot, Dinv); break;
        case ST_JACOBI: launch_mode<T, ST_JACOBI>(c, L, mk, E, mask, u, f, out, omega, dot, Dinv); break;
        case ST_RESID: launch_mode<T, ST_RESID>(c, L, mk, E, mask, u, f, out, omega, dot, Dinv); break;
        case ST_JACOBI2:   // pre-smoothing only: no dot
            launch_op<T, ST_JACOBI2, false, T, T>(c, L, mk, E, mask, u, f, out, omega, nullptr, nullptr, nullptr, Dinv);
            return 0;
        default: launch_mode<T, ST_JACOBI0>(c, L, mk, E, mask, u, f, out, omega, dot, Dinv); break;
    }
    return L.gx * L.gy * L.gz;
}
template int stencil<double>(const Ctx&, int, const OpLaunch&, const ModalK<double>&, const double*, const uint8_t*,
                             const double*, const double*, double*, double, double*, const double*, double*,
                             const double*);
template int stencil<float>(const Ctx&, int, const OpLaunch&, const ModalK<float>&, const float*, const uint8_t*,
                            const float*, const float*, float*, float, double*, const float*, float*, const double*);

int stencil_bf16(const Ctx& c, int mode, const OpLaunch& L, const ModalK<float>& mk, const float* E,
                 const uint8_t* mask, const bf16* u, const float* f, bf16* out_h, float* out_f, float omega,
                 double* dot, const float* Dinv) {
    if (mode == ST_JACOBI0 && out_h && !dot) {
        launch_op<float, ST_JACOBI0, false, bf16, bf16>(c, L, mk, E, mask, u, f, out_h, omega, nullptr, nullptr, nullptr, Dinv);
    } else if (mode == ST_JACOBI && out_h && !dot) {
        launch_op<float, ST_JACOBI, false, bf16, bf16>(c, L, mk, E, mask, u, f, out_h, omega, nullptr, nullptr, nullptr, Dinv);
    } else if (mode == ST_JACOBI && out_f) {
        if (dot) launch_op<float, ST_JACOBI, true, bf16, float>(c, L, mk, E, mask, u, f, out_f, omega, dot, nullptr, nullptr, Dinv);
        else launch_op<float, ST_JACOBI, false, bf16, float>(c, L, mk, E, mask, u, f, out_f, omega, nullptr, nullptr, nullptr, Dinv);
    } else if (mode == ST_RESID && out_f && !dot) {
        launch_op<float, ST_RESID, false, bf16, float>(c, L, mk, E, mask, u, f, out_f, omega, nullptr, nullptr, nullptr, Dinv);
    } else {
        return -1;   // combination not instantiated
    }
    return dot ? L.gx * L.gy * L.gz : 0;
}

int stencil_df(const Ctx& c, int mode, const OpLaunch& L, const ModalK<dfl>& mk, const double* E, const uint8_t* mask,
               const double* u, const double* f, double* out64, float* out32, double* dot) {
    const dfl om(0.0f, 0.0f);   // no damping in these modes
    if (mode == ST_APPLY && out64 && !dot) {
        launch_op<dfl, ST_APPLY, false, double, double>(c, L, mk, E, mask, u, nullptr, out64, om, nullptr);
    } else if (mode == ST_RESID && out64 && !dot) {
        launch_op<dfl, ST_RESID, false, double, double>(c, L, mk, E, mask, u, f, out64, om, nullptr);
    } else if (mode == ST_RESID && out32 && dot) {
        launch_op<dfl, ST_RESID, true, double, float>(c, L, mk, E, mask, u, f, out32, om, dot);
    } else {
        return -1;   // combination not instantiated
    }
    return dot ? L.gx * L.gy * L.gz : 0;
}

void assemble_coarse(const Ctx& c, const Geom& g, const double* K0, const double* E, const double* Ke,
                     const uint8_t* mask, double* A, int npad) {
    cudaMemsetAsync(A, 0, sizeof(double) * (size_t)npad * npad, c.s);
    const long long total = 3 * g.nn * 81;
    k_assemble<<<(unsigned)((total + 255) / 256), 256, 0, c.s>>>(K0, E, Ke, mask, A, g.nx, g.ny, g.nz, npad);
    TOPO_LAUNCH_CHECK(c);
    k_assemble_diag<<<(npad + 255) / 256, 256, 0, c.s>>>(mask, A, (int)(3 * g.nn), npad);
    TOPO_LAUNCH_CHECK(c);
}

void element_energy_sens(const Ctx& c, const Geom& g, const ModalCoef& mc, const double* u, const double* rho,
                         double E0, double Emin, double penal, double* dc_out, double* partials, bool low) {
    const int ip = (penal == (double)(int)penal && penal >= 1.0 && penal <= 16.0) ? (int)penal : -1;
    if (low) {
        // chunks of the z columns so that every thread of the fixed grid gets
        // about four work items (a chunk re-reads one face)
        const long long ncol = (long long)g.nx * g.ny, threads = (long long)kRedBlocks * 256;
        long long nch = (4 * threads + ncol - 1) / ncol;
        if (nch > g.nz) nch = g.nz;
        if (nch < 1) nch = 1;
        const int cz = (int)((g.nz + nch - 1) / nch);
        k_energy_sens_z<<<kRedBlocks, 256, 0, c.s>>>(mc, u, rho, g.nx, g.ny, g.nz, cz, E0, Emin, penal, ip, dc_out,
                                                      partials);
    } else
        k_energy_sens<<<kRedBlocks, 256, 0, c.s>>>(mc, u, rho, g.nx, g.ny, g.nz, E0, Emin, penal, ip, dc_out,
                                                            partials);
    TOPO_LAUNCH_CHECK(c);
}

}  // namespace topo
