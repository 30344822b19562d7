// Host-side solver entry points shared by capi.cu and solver.cu.
#pragma once
#include <functional>

#include "common.cuh"

namespace topo {
// returns the number of dot partials written (0 without dot)
template <typename T>
int op_apply(topo_grid* h, int mode, int l, const T* u, const T* f, T* out, double* dot, T* pout = nullptr,
             const double* beta = nullptr);
template <typename T>
int vcycle(topo_grid* h, int l, const T* f, T* out, T* tmp, double* dot);
// V-cycle with BF16 iterates on levels 0 .. L-2 (FP32 arithmetic, FP32
// right-hand sides and residuals, FP32 coarsest solve); the level-0 result
// is written in FP32 to out.  f and out are level-0 FP32 vectors distinct
// from the level's v32.a (used for the residual).
int vcycle_bf16(topo_grid* h, int l, const float* f, float* out, double* dot);
int solve_fp64(topo_grid* h, double tol, int max_it, int* iters, double* relres);
// FP64 D^-1 of every level (read by the FP64 V-cycle), formed once per density
void ensure_dinv64(topo_grid* h);
int solve_mixed(topo_grid* h, double tol, int max_it, int* iters, double* relres);
// ||f - K x|| / ||f|| of the current iterate in FP64 (1 when x is known to be 0)
double current_relres(topo_grid* h);
// Captures the launches of body() (which enqueues on h->stream) into gr on a
// private stream; gr.failed when capture is not possible (then launch directly)
void capture_launches(topo_grid* h, PcgGraph& gr, const std::function<void()>& body);
}  // namespace topo
