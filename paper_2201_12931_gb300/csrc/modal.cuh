// Walsh-Hadamard ("modal") basis of the hex8 element.
//
// For corner a = (a_x, a_y, a_z) and mode b = (b_x, b_y, b_z) in {0,1}^3 let
// s(a, b) = prod_d (2 a_d - 1)^(b_d).  The modal coefficients of a nodal field
// v are m_b = sum_a s(a, b) v_a (three butterflies of 4 pairs each), and the
// nodal field of a modal vector w is v_a = sum_b s(a, b) w_b.  With T the
// 24x24 transform (per displacement component, index 3 b + c),
// K0 = T^T X T where X = T K0 T^T / 64.  For the cube the modes 1, x, y, z,
// xy, yz, xz, xyz are orthogonal, so X has only 45 non-zeros in fixed small
// symmetric blocks (index 3 b + c, b = b_x + 2 b_y + 4 b_z):
//   normal strains  {3, 7, 14}          3x3
//   shear pairs     {4, 6} {5, 12} {8, 13}      2x2 each
//   bilinear pairs  {9, 20} {10, 17} {15, 19}   2x2 each
//   bilinear triple {11, 16, 18}        3x3
//   trilinear       21, 22, 23          diagonal
// and the rigid translations (b = 0) carry no energy.  Applying K0 in this
// form costs about 190 operations instead of 576 multiply-adds.  The block
// values depend on nu only; build_modal() computes them from K0 and checks
// that K0 has this structure.
#pragma once

#include <string>

namespace topo {

struct ModalCoef {
    double N[3][3];
    double S[3][2][2];
    double B[3][2][2];
    double T3[3][3];
    double C[3];
};

// index sets of the blocks (see above)
__host__ __device__ constexpr int kN(int r) { return r == 0 ? 3 : (r == 1 ? 7 : 14); }
__host__ __device__ constexpr int kS(int g, int r) { return g == 0 ? (r ? 6 : 4) : (g == 1 ? (r ? 12 : 5) : (r ? 13 : 8)); }
__host__ __device__ constexpr int kB(int g, int r) { return g == 0 ? (r ? 20 : 9) : (g == 1 ? (r ? 17 : 10) : (r ? 19 : 15)); }
__host__ __device__ constexpr int kT(int r) { return r == 0 ? 11 : (r == 1 ? 16 : 18); }
__host__ __device__ constexpr int kC(int r) { return 21 + r; }

// nodal (3a + c) -> modal (3b + c); butterflies along x, y, z
template <typename T>
__host__ __device__ __forceinline__ void modal_forward(const T* v, T* m) {
#pragma unroll
    for (int i = 0; i < 24; ++i) m[i] = v[i];
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) {
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            if (a & bit) continue;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T lo = m[3 * a + c], hi = m[3 * (a | bit) + c];
                m[3 * a + c] = hi + lo;
                m[3 * (a | bit) + c] = hi - lo;
            }
        }
    }
}

// modal (3b + c) -> nodal (3a + c):  v_a = sum_b s(a, b) w_b
template <typename T>
__host__ __device__ __forceinline__ void modal_inverse(const T* w, T* v) {
#pragma unroll
    for (int i = 0; i < 24; ++i) v[i] = w[i];
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) {
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            if (a & bit) continue;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T b0 = v[3 * a + c], b1 = v[3 * (a | bit) + c];
                v[3 * a + c] = b0 - b1;        // corner coordinate 0 along this axis
                v[3 * (a | bit) + c] = b0 + b1;  // corner coordinate 1
            }
        }
    }
}

// w = X m  (only the 45 structural non-zeros); w[0..2] = 0
template <typename T, typename C>
__host__ __device__ __forceinline__ void modal_apply(const C& mc, const T* m, T* w) {
#pragma unroll
    for (int i = 0; i < 24; ++i) w[i] = T(0);
#pragma unroll
    for (int r = 0; r < 3; ++r)
        w[kN(r)] = T(mc.N[r][0]) * m[kN(0)] + T(mc.N[r][1]) * m[kN(1)] + T(mc.N[r][2]) * m[kN(2)];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            w[kS(g, r)] = T(mc.S[g][r][0]) * m[kS(g, 0)] + T(mc.S[g][r][1]) * m[kS(g, 1)];
            w[kB(g, r)] = T(mc.B[g][r][0]) * m[kB(g, 0)] + T(mc.B[g][r][1]) * m[kB(g, 1)];
        }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
        w[kT(r)] = T(mc.T3[r][0]) * m[kT(0)] + T(mc.T3[r][1]) * m[kT(1)] + T(mc.T3[r][2]) * m[kT(2)];
#pragma unroll
    for (int r = 0; r < 3; ++r) w[kC(r)] = T(mc.C[r]) * m[kC(r)];
}

// m^T X m
template <typename T, typename C>
__host__ __device__ __forceinline__ T modal_energy(const C& mc, const T* m) {
    T w[24];
    modal_apply<T, C>(mc, m, w);
    T e = T(0);
#pragma unroll
    for (int i = 3; i < 24; ++i) e += m[i] * w[i];
    return e;
}

// Host: X = T K0 T^T / 64, structure check, block extraction.  Returns false
// (with a message) if K0 has entries outside the structural pattern.
bool build_modal(const double K0[576], ModalCoef* mc, std::string* err);

}  // namespace topo
