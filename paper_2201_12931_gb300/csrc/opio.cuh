// Shared-memory and vector element helpers of the operator kernels
// (modal z-march kernel and tensor-core variant).
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace topo {

// Shared-memory slots hold one node's three components padded to four, so a
// slot moves with one 128-bit access (FP32) or a 128 + 64-bit pair (FP64).
__device__ __forceinline__ void st3(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], 0.f);
}
__device__ __forceinline__ void ld3(const float* p, float* v) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
}
__device__ __forceinline__ void st3(double* p, const double* v) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    p[2] = v[2];
}
__device__ __forceinline__ void ld3(const double* p, double* v) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = p[2];
}
__device__ __forceinline__ void st3(dfl* p, const dfl* v) {
    float* q = reinterpret_cast<float*>(p);
    *reinterpret_cast<float4*>(q) = make_float4(v[0].h, v[0].l, v[1].h, v[1].l);
    *reinterpret_cast<float2*>(q + 4) = make_float2(v[2].h, v[2].l);
}
__device__ __forceinline__ void ld3(const dfl* p, dfl* v) {
    const float* q = reinterpret_cast<const float*>(p);
    const float4 a = *reinterpret_cast<const float4*>(q);
    const float2 b = *reinterpret_cast<const float2*>(q + 4);
    v[0] = dfl(a.x, a.y);
    v[1] = dfl(a.z, a.w);
    v[2] = dfl(b.x, b.y);
}
// vector element loads / stores with widening from and rounding to the
// storage type (BF16 iterates of the V-cycle; arithmetic stays in T)
__device__ __forceinline__ float ldv(const float* p) { return *p; }
__device__ __forceinline__ double ldv(const double* p) { return *p; }
__device__ __forceinline__ float ldv(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stv(float* p, float v) { *p = v; }
__device__ __forceinline__ void stv(double* p, double v) { *p = v; }
__device__ __forceinline__ void stv(bf16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void stv(double* p, dfl v) { *p = df_to_double(v); }
__device__ __forceinline__ void stv(float* p, dfl v) { *p = df_to_float(v); }
// per-thread accumulator of the fused dot products
template <typename T>
struct DotAcc {
    using type = T;
};
template <>
struct DotAcc<dfl> {
    using type = float;
};
__device__ __forceinline__ float to_acc(dfl v) { return df_to_float(v); }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
// Jacobi diagonal inverse: the hardware approximate reciprocal (rcp.approx,
// about 1 ulp); any fixed diagonal keeps the smoother symmetric
__device__ __forceinline__ float recip(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

}  // namespace topo
