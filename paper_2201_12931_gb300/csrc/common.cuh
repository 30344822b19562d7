// Internal declarations of the GB300 topology-optimisation library.
// Layout in HBM (all device arrays, natural x-fastest indexing):
//   nodal vectors  : interleaved 3*nn scalars, dof = 3*n + c
//   element arrays : ne scalars, e = i + nx*(j + ny*k)
//   Dirichlet mask : one byte per node, bit c set = DOF c fixed
//   per level      : modulus E_l (FP64 and FP32 copies) with the element
//                    scale 2^l folded in, homogenized density, mask, and the
//                    V-cycle work vectors of each precision.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dfloat.cuh"
#include "modal.cuh"
#include "topo.h"

namespace topo {

using bf16 = __nv_bfloat16;

struct Ctx {
    cudaStream_t s;
    long long* launches;
};

struct Geom {
    int nx, ny, nz;       // elements per axis
    long long nn, ne;     // nodes, elements
    int NX() const { return nx + 1; }
    int NY() const { return ny + 1; }
    int NZ() const { return nz + 1; }
};

struct OpLaunch {          // launch geometry of the operator kernel on one level
    Geom g;
    int gx = 1, gy = 1, gz = 1, cz = 1;
    long long ctas() const { return (long long)gx * gy * gz; }
};

template <typename T>
struct ModalK;

template <typename T>
struct VBuf {             // V-cycle work vectors of one level in one precision
    T* a = nullptr;
    T* b = nullptr;
    T* f = nullptr;       // right-hand side (levels > 0)
};

struct Level {
    Geom g;
    bf16* ha = nullptr;       // BF16 V-cycle iterates (TOPO_MIXED_BF16, levels < L-1)
    bf16* hb = nullptr;
    double* Ke64 = nullptr;   // stored Galerkin element matrices (homogenize = 2, levels >= 1)
    float* Ke32 = nullptr;
    OpLaunch op32, op64;      // operator launch geometry per precision
    OpLaunch optc;            // tensor-core FP32 operator (tc_op.cu)
    double scale = 1.0;       // 2^l
    double* rho = nullptr;    // homogenized density
    double* E64 = nullptr;    // 2^l * (Emin + rho^p (E0 - Emin))
    float* E32 = nullptr;
    double* Dinv64 = nullptr; // per node 1 / (kdiag * sum of E over the <= 8 elements around it)
    float* Dinv32 = nullptr;
    uint8_t* mask = nullptr;
    VBuf<double> v64;
    VBuf<float> v32;
};

struct Coarse {           // dense coarsest-grid solve: K_c^-1 = W^T W, W = L^-1
    int n = 0, npad = 0;
    double* A = nullptr;      // npad^2 work matrix (assembly, Cholesky factor)
    double* W64 = nullptr;    // L^-1 (lower, row-major npad^2)
    double* WT64 = nullptr;   // (L^-1)^T (upper, row-major)
    float* W32 = nullptr;
    float* WT32 = nullptr;
    double* y64 = nullptr;    // temporaries of length npad
    float* y32 = nullptr;
    int* info = nullptr;      // device: first non-positive pivot + 1 (0 = ok)
    double* Dk = nullptr;     // inverses of the 32 x 32 diagonal blocks of L (npad x 32)
};

constexpr int kDirRing = 8;   // CG direction buffers of the fused iterations

struct PcgGraph {             // a captured launch sequence (a PCG iteration, or the coarsest factorization)
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;   // kernel launches per replay
    bool failed = false;      // capture not possible: direct launches
};

struct Scalars {              // device-resident CG scalars
    double rz, rz_new, pq, rr, alpha, beta, ff, aux;
    double rz_old;            // z.r of the previous iteration (flexible beta)
};

}  // namespace topo

struct topo_grid {
    topo_params prm{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int L = 1;
    std::vector<topo::Level> lev;
    topo::Coarse cs;
    // fine-level vectors (interleaved, 3*nn)
    double *x = nullptr, *f = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
    double* K0d = nullptr;          // reference element matrix (E = 1, h = 1), 24x24
    float* K0f = nullptr;
    topo::ModalCoef modal{};
    topo::ModalK<double>* mk64 = nullptr;   // host copies of the operator coefficients
    topo::ModalK<float>* mk32 = nullptr;
    topo::ModalK<topo::dfl>* mkdf = nullptr;  // double-FP32 split of mk64
    uint32_t* tcB = nullptr;        // B operand image of the tensor-core operator (tc_b_image)
    int* tc_err = nullptr;          // device: a tensor-core MMA wait ran out (0 = ok)
    long long npartials = 0;                // size of the partials buffer
    double* dc_work = nullptr;      // element work arrays (filter / OC)
    double* xnew_work = nullptr;
    double* oc_hi = nullptr;        // OC upper move-limit bounds
    double* G64 = nullptr;          // Galerkin child matrices P_o^T K0 P_o (homogenize = 2)
    double* oc_dv = nullptr;        // active-element indicator of a passive OC step (lazy)
    double* S_cache = nullptr;      // filter weight sums S_e for S_radius
    double* dv_cache = nullptr;     // H^T 1 for S_radius
    int4* offs = nullptr;           // filter offsets for S_radius
    double* wts = nullptr;          // filter weights for S_radius
    int noffs = 0;
    double S_radius = -1.0;
    double* lam = nullptr;          // OC bisection state (device)
    double* dtmp = nullptr;         // device scratch scalars
    int* dflag = nullptr;           // device: density out of [0,1] seen
    bool coarse_dirty = true;
    bool dinv64_dirty = true;       // FP64 D^-1 of the levels: formed when an FP64 V-cycle first needs it
    bool x_zero = true;             // warm start is u = 0 (initial residual is f)
    // launch timing of fine-level operator kernels (topo_profile_enable)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;     // 2 per record
    std::vector<int> prof_kind;           // mode * 2 + (float ? 1 : 0)
    int prof_n = 0;
    double* partials = nullptr;     // reduction partials
    topo::Scalars* sc = nullptr;    // device scalars
    double* host_sc = nullptr;      // pinned host mirror
    bool have_density = false, have_bc = false, fp64_ready = false, fp32_ready = false, bf16_ready = false;
    long long launches = 0;
    // CG directions of the fused iterations: a ring of kDirRing buffers (p,
    // level 0's v.b, and these), so that x += alpha p runs once per ring
    // (cg_flush_x) instead of once per iteration
    double* dring64[topo::kDirRing - 2] = {};
    float* dring32[topo::kDirRing - 2] = {};
    double* alpha_hist = nullptr;   // device: alpha of each ring slot
    topo::PcgGraph graph64[topo::kDirRing], graph32[topo::kDirRing];   // captured PCG iterations per ring slot
    topo::PcgGraph coarse_graph;            // captured coarsest-grid assembly, factorization and inverse
    cudaStream_t cap_stream = nullptr;  // private stream the graphs are captured on
    topo_solve_stats stats{};
    std::string err;
    topo::Ctx ctx() { return topo::Ctx{stream, &launches}; }
};

namespace topo {

constexpr int kRedBlocks = 1024;   // fixed grid of reduction kernels (deterministic order)
constexpr int kProfMax = 65536;    // launch records of topo_profile_enable

// ---- stencil.cu ----------------------------------------------------------
// ST_APPLY_P: K.p of CG with the direction update fused in: p = u + beta p_old
// (u = z, f = p_old, beta from the device scalars or 0 when null), q = K p
// written to out and p to pout
// ST_JACOBI2: the first two damped-Jacobi sweeps from u = 0 in one pass:
// u1 = omega D^-1 f formed per node from f and D^-1, then u2 = u1 + omega
// D^-1 (f - K u1) (u unused)
enum StencilMode { ST_APPLY = 0, ST_JACOBI = 1, ST_RESID = 2, ST_JACOBI0 = 3, ST_APPLY_P = 4, ST_JACOBI2 = 5 };
// out = op(u, f); with dot != nullptr also writes per-CTA partial sums of
//   APPLY: u.out   JACOBI/JACOBI0: f.out   RESID: out.out
// and returns the number of partials written.
// nsm: multiprocessors of the device (wave-aware z chunking)
OpLaunch op_launch32(const Geom& g, int nsm);
OpLaunch op_launch64(const Geom& g, int nsm);
template <typename T>
int stencil(const Ctx& c, int mode, const OpLaunch& L, const ModalK<T>& mk, const T* E, const uint8_t* mask,
            const T* u, const T* f, T* out, T omega, double* dot_partials, const T* Dinv, T* pout = nullptr,
            const double* beta = nullptr);
// V-cycle operators with BF16 iterates and FP32 arithmetic: u BF16, f FP32,
// output BF16 (out_h) or FP32 (out_f).  Instantiated: JACOBI0 -> BF16,
// JACOBI -> BF16, JACOBI -> FP32 (with or without dot), RESID -> FP32;
// returns -1 for any other combination, else as stencil().
int stencil_bf16(const Ctx& c, int mode, const OpLaunch& L, const ModalK<float>& mk, const float* E,
                 const uint8_t* mask, const bf16* u, const float* f, bf16* out_h, float* out_f, float omega,
                 double* dot_partials, const float* Dinv);
// Operator in double-FP32 arithmetic (dfloat.cuh) on FP64 storage: u, f and
// the modulus E are FP64, split into FP32 pairs on load; launch geometry of
// the FP64 kernel.  Instantiated: APPLY -> FP64 out; RESID -> FP64 out; RESID
// -> FP32 out with r.r partials (the outer residual of the mixed solve).
// Returns -1 for any other combination, else as stencil().
int stencil_df(const Ctx& c, int mode, const OpLaunch& L, const ModalK<dfl>& mk, const double* E, const uint8_t* mask,
               const double* u, const double* f, double* out64, float* out32, double* dot_partials);
// ---- tc_op.cu: FP32 operators with the element products on tcgen05 tensor cores
OpLaunch op_launch(const Geom& g, int ty, int target_ctas, int resident_ctas);
OpLaunch op_launch_tc(const Geom& g, int nsm);
constexpr int kTcBWords = 2304;
// host: shared-memory image of B = [K0_hi | K0_lo | K0_hi] (TF32), kTcBWords words
void tc_b_image(const double* K0, uint32_t* img);
// APPLY / JACOBI / RESID (with or without dot partials) as stencil(); -1 for
// JACOBI0.  *err is set if a bounded wait on the tensor cores ran out.
int stencil_tc(const Ctx& c, int mode, const OpLaunch& L, float kdiag, const float* E, const uint8_t* mask,
               const float* u, const float* f, float* out, float omega, const uint32_t* Bimg, double* dot_partials,
               int* err);
// dense coarsest operator from E_e K0, or from stored element matrices Ke (non-null)
void assemble_coarse(const Ctx& c, const Geom& g, const double* K0, const double* E, const double* Ke,
                     const uint8_t* mask, double* A, int npad);
// ---- galerkin.cu: stored Galerkin coarse element matrices ------------------
void galerkin_init_constants();
// host: the 8 child matrices G_o = P_o^T K0 P_o (8 x 576, o-major)
void galerkin_child_matrices(const double* K0, double* G);
// Kc (coarse elements of the level below gf) = sum_o P_o^T Kchild P_o; the
// children are Ef[e] K0 (Kf null: scaled sum of G) or Kf[e] (576 per
// element, element-major)
void galerkin_build(const Ctx& c, const Geom& gf, const double* K0, const double* G, const double* Ef, const double* Kf,
                    double* Kc);
// the operator modes of stencil() on a level given by element matrices (no dot)
template <typename T>
void elem_op(const Ctx& c, int mode, const Geom& g, const T* Ke, const uint8_t* mask, const T* u, const T* f, T* out,
             T omega);
// low = true: FP32 modal contraction of FP64-relative displacements (mixed modes)
void element_energy_sens(const Ctx& c, const Geom& g, const ModalCoef& mc, const double* u, const double* rho,
                         double E0, double Emin, double penal, double* dc_out, double* partials, bool low);

// ---- transfer.cu ---------------------------------------------------------
template <typename T>
void restrict_residual(const Ctx& c, const Geom& gf, const uint8_t* maskf, const uint8_t* maskc,
                       const T* rf, T* rc);
template <typename T>
void prolong_add(const Ctx& c, const Geom& gf, const uint8_t* maskf, const uint8_t* maskc,
                 const T* ec, T* uf);
// uf (BF16) += P~ ec with FP32 arithmetic; ec FP32 (coarsest solve) or BF16
template <typename TE>
void prolong_add_bf16(const Ctx& c, const Geom& gf, const uint8_t* maskf, const uint8_t* maskc, const TE* ec,
                      bf16* uf);
// coarse = scale * mean of the 8 children (densities: scale 1; moduli: scale 2)
void homogenize(const Ctx& c, const Geom& gf, const double* rho_f, double* rho_c, double scale);
// per node D^-1 = 1 / (kdiag * sum of E over the <= 8 elements around it),
// in the precision of E (indices in 32 bits: the grid limit of create_grid)
template <typename T>
void diag_inverse(const Ctx& c, const Geom& g, const T* E, T kdiag, T* Dinv);
void simp_moduli(const Ctx& c, long long ne, const double* rho, double scale, double E0,
                 double Emin, double penal, double* E64, float* E32, int* bad_flag);
void mask_from_dofs(const Ctx& c, long long nn, const uint8_t* fixed_dofs, uint8_t* mask);
void inject_mask(const Ctx& c, const Geom& gf, const uint8_t* maskf, uint8_t* maskc);
void masked_copy_load(const Ctx& c, long long nn, const uint8_t* mask, const double* fin, double* fout);

// ---- blas.cu -------------------------------------------------------------
template <typename A, typename B>
void dot_partials(const Ctx& c, long long n, const A* a, const B* b, double* partials);
// reduces n partials into *dst (device double), fixed order
void reduce_to(const Ctx& c, const double* partials, int n, double* dst);
// CG scalar steps, all on device: alpha = rz/pq ; beta = rz_new/rz, rz = rz_new
// hist != nullptr: alpha is also stored there (the direction ring's slot)
void cg_alpha(const Ctx& c, const double* partials, int n, Scalars* sc, double* hist = nullptr);
void cg_beta(const Ctx& c, const double* partials, int n, Scalars* sc);
// flexible (Polak-Ribiere) beta for a preconditioner that varies between
// applications: beta = z_new.(r_new - r_old) / z_old.r_old = -alpha z_new.q / rz_old,
// from the partial sums of z_new.q; run after cg_beta
void cg_beta_flexible(const Ctx& c, const double* partials_zq, int n, Scalars* sc);
template <typename T>
void cg_update_xr(const Ctx& c, long long n, const Scalars* sc, const T* p, const T* q, T* x, T* r,
                  double* partials);
template <typename T>
void cg_update_p(const Ctx& c, long long n, const Scalars* sc, const T* z, T* p);
// r -= alpha q with partial sums of r.r (x updated later by cg_flush_x)
template <typename T>
void cg_update_r(const Ctx& c, long long n, const Scalars* sc, const T* q, T* r, double* partials);
// x += alpha_j p_j for j = 0 .. count-1 in that order (the same operations as
// count successive x += alpha p steps); p_j = ring[j], alpha_j = alpha[j]
template <typename T>
void cg_flush_x(const Ctx& c, long long n, T* const* ring, const double* alpha, int count, T* x);
template <typename S, typename D>
void convert(const Ctx& c, long long n, const S* src, D* dst);
void axpy_f32_into_f64(const Ctx& c, long long n, const float* d, double* x);
template <typename T>
void zero(const Ctx& c, long long n, T* v);
void fill(const Ctx& c, long long n, double* v, double value);
// dense coarse solve
// band: half-bandwidth of A in entries (npad for a dense matrix); Dk
// (npad x 32 doubles) receives the inverses of the 32 x 32 diagonal blocks of
// L, which tri_inverse reads
void chol_factor(const Ctx& c, double* A, int npad, int band, int* info, double* Dk);
void tri_inverse(const Ctx& c, const double* L, double* W, int npad, int band, const double* Dk);
void transpose_dense(const Ctx& c, const double* W, double* WT, int npad);
template <typename T>
void coarse_apply(const Ctx& c, int n, int npad, const T* W, const T* WT, const T* rhs, T* y, T* out);

// ---- filter_oc.cu --------------------------------------------------------
// message returned by topo_last_error(NULL)
void set_global_error(const std::string& msg);
// mode 0: filter, 1: transpose of an input already divided by S, 2: weight sums S
void filter_launch(const Ctx& c, const Geom& g, const int4* offs, const double* wts, int noffs, const double* in,
                   double* out, int mode, const double* S);
void divide(const Ctx& c, long long n, const double* a, const double* b, double* out);
// q = x sqrt(max(-dc~, 1e-30) / dv~)
// Eq. sensitivity filter: out = H(rho dc) / max(gamma, rho), tmp: work array
void sensitivity_filter(const Ctx& c, const Geom& g, const int4* offs, const double* wts, int noffs,
                        const double* rho, const double* dc, double gamma, double* tmp, double* out);
// q = x sqrt(max(-dc~,1e-30)/dv~) in place over dc~ (dv~ null: 1); lo / hi:
// move-limit bounds.  The bisection steps take dv~ null for the volume of x
// itself (no density filter).
void oc_prepare(const Ctx& c, long long ne, const double* x, double* dct_q, const double* dv, double move, double* lo,
                double* hi);
// passive elements (0 active, 1 solid, 2 void): lo = hi = 1 / 0, q = 0,
// dv = 0; active: q = x sqrt(max(-dc, 1e-30)), move-limit bounds, dv = 1
void oc_prepare_passive(const Ctx& c, long long ne, const double* x, double* dct_q, const uint8_t* passive,
                        double move, double* lo, double* hi, double* dv);
// self-weight load f_out = f_ext (null: 0) - (w/8) sum of rho over the elements at each node, in z
void gravity_load(const Ctx& c, const Geom& g, const double* rho, const double* f_ext, double* f_out, double w);
// dc_e += -(w/4) sum of u_z over the corners of e
void gravity_sensitivity(const Ctx& c, const Geom& g, const double* u, double* dc, double w);
void oc_bisect_step(const Ctx& c, long long ne, const double* lo, const double* hi, const double* num,
                    const double* dv, double* partials, double* lam_state);
void oc_bisect_finalize(const Ctx& c, const double* partials, double* lam_state, double volfrac_ne,
                        double tol);
void oc_write(const Ctx& c, long long ne, double* x, const double* lo, const double* hi, const double* num,
              const double* lam_state, double* partials, double* change_dst);

}  // namespace topo

#define TOPO_LAUNCH_CHECK(ctx)                 \
    do {                                       \
        ++*(ctx).launches;                     \
    } while (0)
