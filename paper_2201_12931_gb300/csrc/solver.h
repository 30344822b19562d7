// Host-side solver entry points shared by capi.cu and solver.cu.
#pragma once
#include "common.cuh"

namespace topo {
// returns the number of dot partials written (0 without dot)
template <typename T>
int op_apply(topo_grid* h, int mode, int l, const T* u, const T* f, T* out, double* dot);
template <typename T>
int vcycle(topo_grid* h, int l, const T* f, T* out, T* tmp, double* dot);
int solve_fp64(topo_grid* h, double tol, int max_it, int* iters, double* relres);
int solve_mixed(topo_grid* h, double tol, int max_it, int* iters, double* relres);
}  // namespace topo
