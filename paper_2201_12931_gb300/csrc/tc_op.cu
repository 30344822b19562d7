// Operator kernel with the element products on the 5th-generation tensor
// cores (Sec. 4.2.1 element-by-element product, GB300 form).
//
// The z-march, tiles, shared-memory exchange and epilogues are those of the
// modal kernel (operator.cuh, stencil.cu); only the element computation
// differs.  Per layer, the 256 element columns of a CTA form the rows of
// A (256 x 72): the element's 24 nodal values minus its corner-0 value (K0
// annihilates the translation, which keeps FP32 cancellation out of the
// product), split into TF32 pairs hi + lo and laid out as [hi | hi | lo].
// (hi is the value rounded to TF32 with integer operations, lo = x - hi.)
// B (32 x 72) holds [K0_hi | K0_lo | K0_hi] (rows 24..31 zero), so one
// tcgen05.mma chain (M = 128 twice, N = 32, K = 72 in nine steps of 8)
// accumulates hi K0_hi + hi K0_lo + lo K0_hi in FP32 in tensor memory: about
// 21 significant bits of each product.  One thread issues the MMAs; every
// thread reads its element's row back with tcgen05.ld and scales it by the
// modulus E_e.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// core matrices of 8 rows x 16 bytes, k-blocks of a row group adjacent
// (leading byte offset 128), row groups 18 k-blocks apart (stride byte
// offset 2304).
//
// Every wait on the MMA completion is bounded; a wait that runs out sets
// *err (read by the host after the launch) and the kernel carries on with
// whatever tensor memory holds, so the launch always ends.
#include <cuda_runtime.h>

#include <type_traits>

#include "common.cuh"
#include "operator.cuh"
#include "opio.cuh"

namespace topo {

constexpr int kTcK = 72;                  // [hi | hi | lo] x 24
constexpr int kTcKB = kTcK / 4;           // 16-byte k-blocks per row
constexpr int kTcN = 32;                  // MMA N (24 outputs + 8 zero rows of B)
constexpr int kTcRows = 256;              // element columns of a CTA (two M = 128 blocks)
constexpr uint32_t kTcABytes = kTcRows * kTcK * 4;
constexpr uint32_t kTcBBytes = kTcN * kTcK * 4;
constexpr int kTcTY = 8;

// B operand in its shared-memory image (kTcBBytes / 4 words of TF32 bit
// patterns): [K0_hi | K0_lo | K0_hi] with K0 rows as MMA N rows
void tc_b_image(const double* K0, uint32_t* img) {
    auto tf32_rna = [](float x) {   // round to the nearest TF32 value, ties away from zero (host)
        uint32_t b;
        memcpy(&b, &x, 4);
        if ((b & 0x7F800000u) != 0x7F800000u) b = (b + 0x1000u) & 0xFFFFE000u;
        return b;
    };
    for (int i = 0; i < kTcN * kTcK; ++i) img[i] = 0u;
    for (int n = 0; n < 24; ++n)
        for (int k = 0; k < kTcK; ++k) {
            const int kk = k % 24, part = k / 24;
            const float v = (float)K0[n * 24 + kk];
            const uint32_t hi = tf32_rna(v);
            float hf;
            memcpy(&hf, &hi, 4);
            const uint32_t w = (part == 1) ? tf32_rna(v - hf) : hi;
            img[((n >> 3) * kTcKB + (k >> 2)) * 32 + (n & 7) * 4 + (k & 3)] = w;
        }
}

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// TF32 high part by integer rounding of the FP32 pattern (finite inputs):
// round half away from zero to 10 stored mantissa bits
__device__ __forceinline__ uint32_t tf32_hi(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

// shared-memory matrix descriptor: K-major, no swizzle (version 1)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: FP32 accumulate, TF32 A and B, both K-major
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < (1 << 20); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 24; ++i) v[i] = __uint_as_float(r[i]);
}

// The z-march of k_op (stencil.cu) in FP32 with tensor-core element products.
// Dynamic shared memory: A | B | two node planes | two contribution buffers |
// two modulus-sum buffers.
template <int MODE, bool DOT>
__global__ void __launch_bounds__(kOpTX * kTcTY, 1)
    k_op_tc(const float kdiag, const float* __restrict__ E, const uint8_t* __restrict__ mask,
            const float* __restrict__ u, const float* __restrict__ f, float* __restrict__ out, const int nx,
            const int ny, const int nz, const int cz, const float omega, const uint32_t* __restrict__ Bimg,
            double* __restrict__ partials, int* __restrict__ err) {
    constexpr int TX = kOpTX, TY = kTcTY;
    constexpr bool NEEDD = (MODE == ST_JACOBI);
    constexpr bool NEEDF = (MODE != ST_APPLY);
    constexpr int nU = (TY + 1) * (TX + 1) * 4, nC = 3 * TY * TX * 4, nEs = TY * TX;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ double sred[32];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar;
    uint32_t* const As = reinterpret_cast<uint32_t*>(smem_raw);
    uint32_t* const Bs = reinterpret_cast<uint32_t*>(smem_raw + kTcABytes);
    float* const planes = reinterpret_cast<float*>(smem_raw + kTcABytes + kTcBBytes);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int warp = tid >> 5;
    const int NX = nx + 1, NY = ny + 1;
    const int i0 = blockIdx.x * (TX - 1), j0 = blockIdx.y * (TY - 1);
    const int kz0 = blockIdx.z * cz;
    const int kz1 = min(kz0 + cz, nz + 1);
    const int in = i0 - 1 + tx, jn = j0 - 1 + ty;
    const bool node_ok = in >= 0 && in < NX && jn >= 0 && jn < NY;
    const bool col_ok = in >= 0 && in < nx && jn >= 0 && jn < ny;
    const bool out_ok = tx >= 1 && ty >= 1 && node_ok;
    const bool has_halo = tid < TY + 1 + TX;
    const int hsx = tid < TY + 1 ? TX : tid - TY - 1;
    const int hsy = tid < TY + 1 ? tid : TY;
    const int hx = i0 - 1 + hsx, hy = j0 - 1 + hsy;
    const bool halo_ok = has_halo && hx >= 0 && hx < NX && hy >= 0 && hy < NY;
    const long long nplane = (long long)NX * NY;
    const int own_xy = node_ok ? in + NX * jn : 0;
    const int halo_xy = halo_ok ? hx + NX * hy : 0;
    const int col_xy = col_ok ? in + nx * jn : 0;
    const int uoff = (ty * (TX + 1) + tx) * 4;
    const int hoff = (hsy * (TX + 1) + hsx) * 4;
    const int coff = (ty * TX + tx) * 4;
    const int own3 = 3 * own_xy, halo3 = 3 * halo_xy;

    // operand B, tensor memory (64 columns: two 32-column accumulators), mbarrier
    for (int i = tid; i < (int)(kTcBBytes / 16); i += TX * TY)
        reinterpret_cast<uint4*>(Bs)[i] = reinterpret_cast<const uint4*>(Bimg)[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t my_tmem = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
    uint32_t phase = 0;

    float cprev[12], top[12];   // corners of the plane below (c00, c10, c01, c11); contributions to them
#pragma unroll
    for (int i = 0; i < 12; ++i) cprev[i] = top[i] = 0.f;
    float st00[3] = {}, st10[3] = {}, st01[3] = {}, st11[3] = {};
    float stE = 0.f;
    double dot = 0.0;
    float su[4][3], sf[4][3], sE[4];
    unsigned sm[4];
    float shv[2][3];
    unsigned shm[2];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        su[q][0] = su[q][1] = su[q][2] = 0.f;
        sf[q][0] = sf[q][1] = sf[q][2] = 0.f;
        sE[q] = 0.f;
        sm[q] = 0u;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        shv[q][0] = shv[q][1] = shv[q][2] = 0.f;
        shm[q] = 0u;
    }

    auto fetch = [&](auto Sc, int P) {
        constexpr int S = decltype(Sc)::value;
        const bool pin = P >= 0 && P <= nz;
        const long long pb = (long long)P * nplane;
        const bool ok = pin && node_ok;
        sm[S] = ok ? mask[pb + own_xy] : 0u;
        const float* ub = u + 3 * pb + own3;
        const float* fb_ = NEEDF ? f + 3 * pb + own3 : nullptr;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            su[S][c] = ok ? ub[c] : 0.f;
            if (NEEDF) sf[S][c] = ok ? fb_[c] : 0.f;
        }
        const bool okh = pin && halo_ok;
        shm[S & 1] = okh ? mask[pb + halo_xy] : 0u;
        const float* hb = u + 3 * pb + halo3;
#pragma unroll
        for (int c = 0; c < 3; ++c) shv[S & 1][c] = okh ? hb[c] : 0.f;
        sE[S] = (col_ok && P >= 1 && P <= nz) ? E[(long long)(P - 1) * nx * ny + col_xy] : 0.f;
    };

    auto step = [&](auto Bc, int P) {
        constexpr int B = decltype(Bc)::value;
        constexpr int B2 = B & 1;
        constexpr int SN = (B + 1) & 3;   // slot of plane P + 1
        constexpr int SO = (B + 2) & 3;   // slot of plane P - 2 (output)
        [[maybe_unused]] constexpr int SL = (B + 3) & 3;   // slot of plane P - 1
        float* const U = planes + B2 * nU;
        float* const Cb = planes + 2 * nU + B2 * nC;
        [[maybe_unused]] float* const Eb = planes + 2 * nU + 2 * nC + B2 * nEs;
        {   // publish plane P (masked) and the stashed contributions of plane P - 2
            const unsigned cm = sm[B];
            float mu[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) mu[c] = ((cm >> c) & 1u) ? 0.f : su[B][c];
            st3(U + uoff, mu);
            if (has_halo) {
                const unsigned chm = shm[B & 1];
#pragma unroll
                for (int c = 0; c < 3; ++c) mu[c] = ((chm >> c) & 1u) ? 0.f : shv[B & 1][c];
                st3(U + hoff, mu);
            }
            st3(Cb + coff, st10);
            st3(Cb + nC / 3 + coff, st01);
            st3(Cb + 2 * (nC / 3) + coff, st11);
        }
        if constexpr (NEEDD) Eb[tid] = stE;
        if (P + 1 <= kz1) fetch(std::integral_constant<int, SN>{}, P + 1);
        __syncthreads();
        // output node plane Q = P - 2
        const int Q = P - 2;
        if (out_ok && Q >= kz0 && Q < kz1) {
            float a0[3], a1[3], a2[3], y[3];
            ld3(Cb + coff - 4, a0);
            ld3(Cb + nC / 3 + coff - TX * 4, a1);
            ld3(Cb + 2 * (nC / 3) + coff - TX * 4 - 4, a2);
#pragma unroll
            for (int c = 0; c < 3; ++c) y[c] = st00[c] + a0[c] + a1[c] + a2[c];
            [[maybe_unused]] float rD = 1.f;
            if constexpr (NEEDD) {
                const float* e = Eb + tid;
                rD = recip(kdiag * (e[0] + e[-1] + e[-TX] + e[-TX - 1]));
            }
            float* o = out + 3 * ((long long)Q * nplane) + own3;
            const unsigned m2 = sm[SO];
            float d32 = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool fixed = (m2 >> c) & 1u;
                const float uo = su[SO][c];
                [[maybe_unused]] const float fo = sf[SO][c];
                float r;
                if constexpr (MODE == ST_APPLY) {
                    r = fixed ? uo : y[c];
                    if (DOT) d32 += uo * r;
                } else if constexpr (MODE == ST_RESID) {
                    r = fo - (fixed ? uo : y[c]);
                    if (DOT) d32 += r * r;
                } else {
                    r = fixed ? uo + omega * (fo - uo) : uo + omega * (fo - y[c]) * rD;
                    if (DOT) d32 += fo * r;
                }
                o[c] = r;
            }
            if (DOT) dot += (double)d32;
        }
        if (P == kz0 - 1) {   // corners of the first plane of the chunk
            ld3(U + uoff, cprev);
            ld3(U + uoff + 4, cprev + 3);
            ld3(U + uoff + (TX + 1) * 4, cprev + 6);
            ld3(U + uoff + (TX + 1) * 4 + 4, cprev + 9);
        } else if (P >= kz0 && P <= kz1) {
            // element of layer P - 1 | P: corners a = ax + 2 ay + 4 az
            float ue[24];
#pragma unroll
            for (int i = 0; i < 12; ++i) ue[i] = cprev[i];
            ld3(U + uoff, ue + 12);
            ld3(U + uoff + 4, ue + 15);
            ld3(U + uoff + (TX + 1) * 4, ue + 18);
            ld3(U + uoff + (TX + 1) * 4 + 4, ue + 21);
#pragma unroll
            for (int i = 0; i < 12; ++i) cprev[i] = ue[12 + i];
            {   // A row: corner-0 translation removed, TF32 hi / lo split
                const float r0 = ue[0], r1 = ue[1], r2 = ue[2];
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    ue[3 * a] -= r0;
                    ue[3 * a + 1] -= r1;
                    ue[3 * a + 2] -= r2;
                }
                uint32_t* const Arow = As + (tid >> 3) * kTcKB * 32 + (tid & 7) * 4;
#pragma unroll
                for (int kb = 0; kb < 6; ++kb) {
                    // hi rounded to TF32; lo = x - hi is exact in FP32 and the
                    // tensor core reads its top 11 bits (|lo| <= 2^-11 |x|)
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        h[j] = tf32_hi(ue[4 * kb + j]);
                        l[j] = __float_as_uint(ue[4 * kb + j] - __uint_as_float(h[j]));
                    }
                    const uint4 hv = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4*>(Arow + kb * 32) = hv;
                    *reinterpret_cast<uint4*>(Arow + (6 + kb) * 32) = hv;
                    *reinterpret_cast<uint4*>(Arow + (12 + kb) * 32) = make_uint4(l[0], l[1], l[2], l[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
                for (int blk = 0; blk < 2; ++blk) {
#pragma unroll
                    for (int s = 0; s < kTcK / 8; ++s) {
                        const uint64_t ad = smem_desc(a0 + blk * (16 * kTcKB * 128) + s * 256, 128, kTcKB * 128);
                        const uint64_t bd = smem_desc(b0 + s * 256, 128, kTcKB * 128);
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + 32 * blk),
                            "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(s));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&mbar))
                             : "memory");
            }
            if (!mbar_wait(smem_u32(&mbar), phase)) atomicExch(err, 1);
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float v[24];
            tmem_ld32(my_tmem, v);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            const float Ee = sE[B];
            float A[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                A[i] = top[i] + Ee * v[i];
                top[i] = Ee * v[12 + i];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                st00[c] = A[c];
                st10[c] = A[3 + c];
                st01[c] = A[6 + c];
                st11[c] = A[9 + c];
            }
            if constexpr (NEEDD) stE = sE[SL] + sE[B];
        }
    };

    using S0 = std::integral_constant<int, 0>;
    using S1 = std::integral_constant<int, 1>;
    using S2 = std::integral_constant<int, 2>;
    using S3 = std::integral_constant<int, 3>;
    const int Pfirst = kz0 - 1;
    int P = Pfirst - (((Pfirst % 4) + 4) % 4);
    switch (Pfirst - P) {
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
        double v = dot;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int l = tid & 31;
        if (l == 0) sred[warp] = v;
        __syncthreads();
        if (warp == 0) {
            double t = (l < (TX * TY) / 32) ? sred[l] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (l == 0) partials[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
    }
}

constexpr size_t tc_smem_bytes() {
    return kTcABytes + kTcBBytes +
           sizeof(float) * (2 * (kTcTY + 1) * (kOpTX + 1) * 4 + 2 * 3 * kTcTY * kOpTX * 4 + 2 * kTcTY * kOpTX);
}

template <int MODE, bool DOT>
void launch_tc(const Ctx& c, const OpLaunch& L, float kdiag, const float* E, const uint8_t* mask, const float* u,
               const float* f, float* out, float omega, const uint32_t* Bimg, double* dot, int* err) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_op_tc<MODE, DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes());
        attr = true;
    }
    k_op_tc<MODE, DOT><<<dim3(L.gx, L.gy, L.gz), dim3(kOpTX, kTcTY), tc_smem_bytes(), c.s>>>(
        kdiag, E, mask, u, f, out, L.g.nx, L.g.ny, L.g.nz, L.cz, omega, Bimg, dot, err);
    TOPO_LAUNCH_CHECK(c);
}

}  // namespace

OpLaunch op_launch_tc(const Geom& g, int nsm) { return op_launch(g, kTcTY, 2 * nsm, nsm); }

int stencil_tc(const Ctx& c, int mode, const OpLaunch& L, float kdiag, const float* E, const uint8_t* mask,
               const float* u, const float* f, float* out, float omega, const uint32_t* Bimg, double* dot,
               int* err) {
    switch (mode) {
        case ST_APPLY:
            if (dot) launch_tc<ST_APPLY, true>(c, L, kdiag, E, mask, u, f, out, omega, Bimg, dot, err);
            else launch_tc<ST_APPLY, false>(c, L, kdiag, E, mask, u, f, out, omega, Bimg, nullptr, err);
            break;
        case ST_JACOBI:
            if (dot) launch_tc<ST_JACOBI, true>(c, L, kdiag, E, mask, u, f, out, omega, Bimg, dot, err);
            else launch_tc<ST_JACOBI, false>(c, L, kdiag, E, mask, u, f, out, omega, Bimg, nullptr, err);
            break;
        case ST_RESID:
            if (dot) launch_tc<ST_RESID, true>(c, L, kdiag, E, mask, u, f, out, omega, Bimg, dot, err);
            else launch_tc<ST_RESID, false>(c, L, kdiag, E, mask, u, f, out, omega, Bimg, nullptr, err);
            break;
        default:
            return -1;   // the first sweep from zero needs no K.u: modal kernel
    }
    return dot ? L.gx * L.gy * L.gz : 0;
}

}  // namespace topo
