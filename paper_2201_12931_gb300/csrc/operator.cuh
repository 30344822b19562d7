// Element-by-element operator kernel (Sec. 4.2.1), GB300 form.
//
// Work decomposition.  A CTA of TX x TY threads owns an x-y tile of element
// columns and marches along z through a chunk of node planes.  Thread (tx, ty)
// owns the element column (i0-1+tx, j0-1+ty) and the node at its lower corner;
// per layer it computes that column's element once, in the Walsh-Hadamard
// (modal) basis of the brick (see modal.cuh):
//     in-plane 2x2 transform of the new node plane (reused by the next layer)
//     -> z butterfly -> 9-coefficient block stiffness scaled by E_e
//     -> inverse z butterfly -> face accumulation with the layer below
//     -> inverse in-plane transform = contributions to the 4 column corners.
// Nodal values and corner contributions move between threads through
// double-buffered shared memory with one __syncthreads per layer; each node
// is read from HBM once per chunk (plus a one-node halo on the +x/+y sides
// and one extra plane per chunk), and each output node is written once.
// Outputs per CTA: (TX-1) x (TY-1) node columns.
//
// Operator with Dirichlet rows: y = P_f K P_f u + (I - P_f) u.  Epilogues:
// K.u, damped Jacobi (Sec. 3.2) with the diagonal kdiag * sum_e E_e formed on
// the fly, residual (Eq. residual), first Jacobi sweep from zero; each can
// also emit per-CTA FP64 partial sums of a dot product.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "dfloat.cuh"

namespace topo {

// storage type of the modulus and right-hand side read by the operator
// kernel for arithmetic type T (double-FP32 arithmetic reads FP64 arrays)
template <typename T>
struct OpStore {
    using type = T;
};
template <>
struct OpStore<dfl> {
    using type = double;
};

template <typename T>
struct ModalK {           // structure verified on the host (build_modal_k)
    T nd, no;             // normal-strain block: diagonal - off, off
    T sc;                 // shear pairs: all four entries
    T bp, bq;             // bilinear pairs: diagonal, off
    T td, to;             // bilinear triple: diagonal - off, off
    T cg;                 // trilinear diagonal
    T kdiag;              // diagonal of K0 (the same for every DOF)
};

constexpr int kOpTX = 32;
// CTA height (32 x 8 threads; measured faster than 32 x 16 for FP32, and
// the FP64 body needs ~220 registers)
template <typename T>
__host__ __device__ constexpr int op_ty() { return 8; }

// FP32 helpers: components x and y of a node travel as one float2 and are
// combined with the paired FP32 instructions of sm_100+ (z stays scalar)
__device__ __forceinline__ float2 ld2(const float* p) { return make_float2(p[0], p[1]); }
__device__ __forceinline__ void st2(float* p, float2 v) {
    p[0] = v.x;
    p[1] = v.y;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Double-FP32 counterpart: the x and y components of a node as dfl2 (high
// words in one float2, low words in another), so that each step of the
// TwoSum-based add of dfloat.cuh runs as one paired instruction for both
// components -- lane by lane the same IEEE operations as df_add / df_sub.
struct dfl2 {
    float2 h, l;
};
__device__ __forceinline__ dfl2 ld2(const dfl* p) {
    return dfl2{make_float2(p[0].h, p[1].h), make_float2(p[0].l, p[1].l)};
}
__device__ __forceinline__ void st2(dfl* p, dfl2 v) {
    p[0] = dfl{v.h.x, v.l.x};
    p[1] = dfl{v.h.y, v.l.y};
}
__device__ __forceinline__ dfl2 add2(dfl2 a, dfl2 b) {
    const float2 s = add2(a.h, b.h), t = add2(a.l, b.l);
    const float2 v = sub2(s, a.h);
    const float2 p = sub2(s, v), q = sub2(b.h, v);
    const float2 e = add2(sub2(a.h, p), q);
    return dfl2{s, add2(e, t)};
}
__device__ __forceinline__ dfl2 sub2(dfl2 a, dfl2 b) {
    return add2(a, dfl2{make_float2(-b.h.x, -b.h.y), make_float2(-b.l.x, -b.l.y)});
}

template <typename T>
__device__ __forceinline__ void face_forward(const T* c00, const T* c10, const T* c01, const T* c11, T* F) {
    // F[3*g + c], g = bx + 2 by
    if constexpr (std::is_same<T, float>::value || std::is_same<T, dfl>::value) {
        using V2 = std::conditional_t<std::is_same<T, float>::value, float2, dfl2>;
        const V2 s0 = add2(ld2(c10), ld2(c00)), d0 = sub2(ld2(c10), ld2(c00));
        const V2 s1 = add2(ld2(c11), ld2(c01)), d1 = sub2(ld2(c11), ld2(c01));
        st2(F + 0, add2(s1, s0));
        st2(F + 3, add2(d1, d0));
        st2(F + 6, sub2(s1, s0));
        st2(F + 9, sub2(d1, d0));
        const T z0 = c10[2] + c00[2], e0 = c10[2] - c00[2];
        const T z1 = c11[2] + c01[2], e1 = c11[2] - c01[2];
        F[2] = z1 + z0;
        F[5] = e1 + e0;
        F[8] = z1 - z0;
        F[11] = e1 - e0;
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T s0 = c10[c] + c00[c], d0 = c10[c] - c00[c];
            const T s1 = c11[c] + c01[c], d1 = c11[c] - c01[c];
            F[0 + c] = s1 + s0;
            F[3 + c] = d1 + d0;
            F[6 + c] = s1 - s0;
            F[9 + c] = d1 - d0;
        }
    }
}

template <typename T>
__device__ __forceinline__ void face_inverse(const T* A, T* c00, T* c10, T* c01, T* c11) {
    if constexpr (std::is_same<T, float>::value || std::is_same<T, dfl>::value) {
        using V2 = std::conditional_t<std::is_same<T, float>::value, float2, dfl2>;
        const V2 lo0 = sub2(ld2(A + 0), ld2(A + 6)), hi0 = add2(ld2(A + 0), ld2(A + 6));
        const V2 lo1 = sub2(ld2(A + 3), ld2(A + 9)), hi1 = add2(ld2(A + 3), ld2(A + 9));
        st2(c00, sub2(lo0, lo1));
        st2(c10, add2(lo0, lo1));
        st2(c01, sub2(hi0, hi1));
        st2(c11, add2(hi0, hi1));
        const T l0 = A[2] - A[8], h0 = A[2] + A[8];
        const T l1 = A[5] - A[11], h1 = A[5] + A[11];
        c00[2] = l0 - l1;
        c10[2] = l0 + l1;
        c01[2] = h0 - h1;
        c11[2] = h0 + h1;
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T lo0 = A[0 + c] - A[6 + c], hi0 = A[0 + c] + A[6 + c];   // bx = 0 : ay = 0 / 1
            const T lo1 = A[3 + c] - A[9 + c], hi1 = A[3 + c] + A[9 + c];   // bx = 1
            c00[c] = lo0 - lo1;
            c10[c] = lo0 + lo1;
            c01[c] = hi0 - hi1;
            c11[c] = hi0 + hi1;
        }
    }
}

// element: bottom face modes FB, top face modes FT (12 each), modulus E ->
// modal outputs folded back to face space: Bo (bottom), To (top).  zc (3,
// optional): added to the z-difference of the mean mode (modes 12..14) when
// the two faces were shifted by different translations.
template <typename T>
__device__ __forceinline__ void element_modal(const ModalK<T>& k, T E, const T* FB, const T* FT, T* Bo, T* To,
                                              const T* zc = nullptr) {
    T m[24];
    if constexpr (std::is_same<T, float>::value || std::is_same<T, dfl>::value) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            st2(m + 3 * g, add2(ld2(FT + 3 * g), ld2(FB + 3 * g)));
            st2(m + 3 * (g + 4), sub2(ld2(FT + 3 * g), ld2(FB + 3 * g)));
            m[3 * g + 2] = FT[3 * g + 2] + FB[3 * g + 2];
            m[3 * (g + 4) + 2] = FT[3 * g + 2] - FB[3 * g + 2];
        }
    } else {
#pragma unroll
        for (int g = 0; g < 4; ++g)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                m[3 * g + c] = FT[3 * g + c] + FB[3 * g + c];
                m[3 * (g + 4) + c] = FT[3 * g + c] - FB[3 * g + c];
            }
    }
    if (zc) {
#pragma unroll
        for (int c = 0; c < 3; ++c) m[12 + c] = m[12 + c] + zc[c];
    }
    const T nd = E * k.nd, no = E * k.no, sc = E * k.sc, bp = E * k.bp, bq = E * k.bq;
    const T td = E * k.td, to = E * k.to, cg = E * k.cg;
    T w[24];
    {   // normal strains {3, 7, 14}
        const T s = no * (m[3] + m[7] + m[14]);
        w[3] = nd * m[3] + s;
        w[7] = nd * m[7] + s;
        w[14] = nd * m[14] + s;
    }
    {   // shear pairs
        w[4] = w[6] = sc * (m[4] + m[6]);
        w[5] = w[12] = sc * (m[5] + m[12]);
        w[8] = w[13] = sc * (m[8] + m[13]);
    }
    {   // bilinear pairs
        w[9] = bp * m[9] + bq * m[20];
        w[20] = bq * m[9] + bp * m[20];
        w[10] = bp * m[10] + bq * m[17];
        w[17] = bq * m[10] + bp * m[17];
        w[15] = bp * m[15] + bq * m[19];
        w[19] = bq * m[15] + bp * m[19];
    }
    {   // bilinear triple {11, 16, 18}
        const T s = to * (m[11] + m[16] + m[18]);
        w[11] = td * m[11] + s;
        w[16] = td * m[16] + s;
        w[18] = td * m[18] + s;
    }
    w[21] = cg * m[21];
    w[22] = cg * m[22];
    w[23] = cg * m[23];
    // inverse z butterfly: bottom corner (az = 0) gets w_g - w_{g+4}; w_0..2 = 0
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Bo[c] = -w[12 + c];
        To[c] = w[12 + c];
    }
    if constexpr (std::is_same<T, float>::value || std::is_same<T, dfl>::value) {
#pragma unroll
        for (int g = 1; g < 4; ++g) {
            st2(Bo + 3 * g, sub2(ld2(w + 3 * g), ld2(w + 3 * (g + 4))));
            st2(To + 3 * g, add2(ld2(w + 3 * g), ld2(w + 3 * (g + 4))));
            Bo[3 * g + 2] = w[3 * g + 2] - w[3 * (g + 4) + 2];
            To[3 * g + 2] = w[3 * g + 2] + w[3 * (g + 4) + 2];
        }
    } else {
#pragma unroll
        for (int g = 1; g < 4; ++g)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Bo[3 * g + c] = w[3 * g + c] - w[3 * (g + 4) + c];
                To[3 * g + c] = w[3 * g + c] + w[3 * (g + 4) + c];
            }
    }
}

}  // namespace topo
