// extern "C" entry points of include/topo.h: argument checks, device
// workspace, per-level set-up (Sec. 4.2.2 homogenization), and dispatch to the
// solver and the element / filter / OC kernels.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "operator.cuh"
#include "solver.h"

using namespace topo;

namespace {

std::string g_create_err;
constexpr int kMaxCoarseDofs = 12000;

topo_status fail(topo_grid* h, topo_status st, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_err = msg;
    return st;
}

#define CK(h, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), TOPO_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
topo_status dalloc(topo_grid* h, T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(h, e == cudaErrorMemoryAllocation ? TOPO_OOM : TOPO_CUDA,
                    std::string("cudaMalloc(") + std::to_string(sizeof(T) * n) + " bytes): " + cudaGetErrorString(e));
    }
    return TOPO_OK;
}

#define ALLOC(h, p, n)                               \
    do {                                             \
        topo_status s_ = dalloc((h), &(p), (n));     \
        if (s_ != TOPO_OK) return s_;                \
    } while (0)

// K0 of the unit cube by 2x2x2 Gauss quadrature of B^T D B (isotropic, E = 1).
// Local corner a = ax + 2 ay + 4 az, DOF 3 a + c.
void element_matrix(double nu, double K[576]) {
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
    double D[6][6] = {};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[i][j] = lam + (i == j ? 2.0 * mu : 0.0);
    D[3][3] = D[4][4] = D[5][5] = mu;
    const double gp[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
    std::memset(K, 0, sizeof(double) * 576);
    for (int q = 0; q < 8; ++q) {
        const double x = gp[q & 1], y = gp[(q >> 1) & 1], z = gp[q >> 2];
        double B[6][24] = {};
        for (int a = 0; a < 8; ++a) {
            const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
            const double lx = ax ? x : 1.0 - x, ly = ay ? y : 1.0 - y, lz = az ? z : 1.0 - z;
            const double sx = ax ? 1.0 : -1.0, sy = ay ? 1.0 : -1.0, sz = az ? 1.0 : -1.0;
            const double dx = sx * ly * lz, dy = lx * sy * lz, dz = lx * ly * sz;
            B[0][3 * a] = dx;
            B[1][3 * a + 1] = dy;
            B[2][3 * a + 2] = dz;
            B[3][3 * a] = dy;
            B[3][3 * a + 1] = dx;
            B[4][3 * a + 1] = dz;
            B[4][3 * a + 2] = dy;
            B[5][3 * a] = dz;
            B[5][3 * a + 2] = dx;
        }
        double DB[6][24];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 24; ++j) {
                double s = 0.0;
                for (int k = 0; k < 6; ++k) s += D[i][k] * B[k][j];
                DB[i][j] = s;
            }
        for (int i = 0; i < 24; ++i)
            for (int j = 0; j < 24; ++j) {
                double s = 0.0;
                for (int k = 0; k < 6; ++k) s += B[k][i] * DB[k][j];
                K[i * 24 + j] += 0.125 * s;
            }
    }
}

Geom make_geom(int nx, int ny, int nz) {
    Geom g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    g.ne = (long long)nx * ny * nz;
    return g;
}

topo_status alloc_precision(topo_grid* h, bool fp64) {
    if (fp64 && h->fp64_ready) return TOPO_OK;
    if (!fp64 && h->fp32_ready) return TOPO_OK;
    const long long n0 = 3 * h->lev[0].g.nn;
    for (int l = 0; l < h->L; ++l) {
        const long long n = 3 * h->lev[l].g.nn;
        if (fp64) {
            ALLOC(h, h->lev[l].v64.a, n);
            ALLOC(h, h->lev[l].v64.b, n);
            ALLOC(h, h->lev[l].v64.f, n);
        } else {
            ALLOC(h, h->lev[l].v32.a, n);
            ALLOC(h, h->lev[l].v32.b, n);
            ALLOC(h, h->lev[l].v32.f, n);
        }
    }
    if (fp64) {
        ALLOC(h, h->z, n0);
        ALLOC(h, h->p, n0);
        ALLOC(h, h->q, n0);
        for (auto& d : h->dring64) ALLOC(h, d, n0);
        h->fp64_ready = true;
    } else {
        ALLOC(h, h->r32, n0);
        ALLOC(h, h->z32, n0);
        ALLOC(h, h->p32, n0);
        ALLOC(h, h->q32, n0);
        ALLOC(h, h->d32, n0);
        for (auto& d : h->dring32) ALLOC(h, d, n0);
        h->fp32_ready = true;
    }
    return TOPO_OK;
}

// BF16 V-cycle iterates on levels 0 .. L-2 (TOPO_MIXED_BF16)
topo_status alloc_bf16(topo_grid* h) {
    if (h->bf16_ready) return TOPO_OK;
    for (int l = 0; l + 1 < h->L; ++l) {
        const long long n = 3 * h->lev[l].g.nn;
        ALLOC(h, h->lev[l].ha, n);
        ALLOC(h, h->lev[l].hb, n);
    }
    h->bf16_ready = true;
    return TOPO_OK;
}

void free_all(topo_grid* h) {
    auto F = [](void* p) {
        if (p) cudaFree(p);
    };
    for (auto& l : h->lev) {
        F(l.rho); F(l.E64); F(l.E32); F(l.mask);
        F(l.Dinv64); F(l.Dinv32);
        F(l.v64.a); F(l.v64.b); F(l.v64.f);
        F(l.v32.a); F(l.v32.b); F(l.v32.f);
        F(l.ha); F(l.hb); F(l.Ke64); F(l.Ke32);
    }
    F(h->cs.A); F(h->cs.W64); F(h->cs.WT64); F(h->cs.W32); F(h->cs.WT32); F(h->cs.y64); F(h->cs.y32);
    F(h->cs.info); F(h->cs.Dk);
    F(h->x); F(h->f); F(h->r); F(h->z); F(h->p); F(h->q);
    F(h->r32); F(h->z32); F(h->p32); F(h->q32); F(h->d32); F(h->alpha_hist);
    for (auto& d : h->dring64) F(d);
    for (auto& d : h->dring32) F(d);
    F(h->K0d); F(h->K0f);
    F(h->dc_work); F(h->xnew_work); F(h->oc_hi); F(h->G64); F(h->oc_dv); F(h->S_cache); F(h->dv_cache); F(h->offs); F(h->wts);
    F(h->lam); F(h->dtmp); F(h->dflag); F(h->tc_err); F(h->tcB); F(h->partials); F(h->sc);
    if (h->host_sc) cudaFreeHost(h->host_sc);
    delete h->mk64;
    delete h->mk32;
    delete h->mkdf;
    h->mk64 = nullptr;
    h->mk32 = nullptr;
    h->mkdf = nullptr;
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    for (int q = 0; q < kDirRing; ++q) {
        if (h->graph64[q].exec) cudaGraphExecDestroy(h->graph64[q].exec);
        if (h->graph32[q].exec) cudaGraphExecDestroy(h->graph32[q].exec);
        h->graph64[q].exec = h->graph32[q].exec = nullptr;
    }
    if (h->coarse_graph.exec) cudaGraphExecDestroy(h->coarse_graph.exec);
    h->coarse_graph.exec = nullptr;
    for (auto e : h->prof_ev) cudaEventDestroy(e);
    h->prof_ev.clear();
}

// The dense coarsest-grid workspace is allocated on first use, so that handles
// used only for filtering or single-level operators need no coarse factor.
topo_status ensure_coarse(topo_grid* h) {
    if (!h->coarse_dirty) return TOPO_OK;
    if (!h->have_density || !h->have_bc) return fail(h, TOPO_BADARG, "density and boundary conditions must be set");
    Level& lc = h->lev[h->L - 1];
    Coarse& cs = h->cs;
    if (cs.n > kMaxCoarseDofs)
        return fail(h, TOPO_BADARG, "coarsest grid has " + std::to_string(cs.n) + " DOFs (> " +
                                        std::to_string(kMaxCoarseDofs) + "): use more levels");
    if (!cs.A) {
        const size_t n2 = (size_t)cs.npad * cs.npad;
        ALLOC(h, cs.A, n2);
        ALLOC(h, cs.W64, n2);
        ALLOC(h, cs.WT64, n2);
        ALLOC(h, cs.W32, n2);
        ALLOC(h, cs.WT32, n2);
        ALLOC(h, cs.y64, cs.npad);
        ALLOC(h, cs.y32, cs.npad);
        ALLOC(h, cs.info, 1);
        ALLOC(h, cs.Dk, (size_t)cs.npad * 32);
    }
    // half-bandwidth of the coarsest matrix: DOFs of nodes up to one step
    // apart in each direction (node order x fastest, 3 DOFs per node)
    const int NXc = lc.g.nx + 1, NYc = lc.g.ny + 1;
    const int band = 3 * (1 + NXc + NXc * NYc) + 2;
    // assembly, Cholesky, L^-1, its transpose and FP32 copies: a fixed
    // sequence of a few hundred small launches, captured once per handle into
    // a CUDA graph and replayed for each new density (the pointers do not
    // change); the pivot check reads info after the whole sequence
    auto body = [&]() {
        const Ctx cc = h->ctx();
        assemble_coarse(cc, lc.g, h->K0d, lc.E64, h->prm.homogenize == 2 && h->L > 1 ? lc.Ke64 : nullptr, lc.mask,
                        cs.A, cs.npad);
        chol_factor(cc, cs.A, cs.npad, band, cs.info, cs.Dk);
        tri_inverse(cc, cs.A, cs.W64, cs.npad, band, cs.Dk);
        transpose_dense(cc, cs.W64, cs.WT64, cs.npad);
        const long long n2 = (long long)cs.npad * cs.npad;
        convert<double, float>(cc, n2, cs.W64, cs.W32);
        convert<double, float>(cc, n2, cs.WT64, cs.WT32);
    };
    PcgGraph& gr = h->coarse_graph;
    if (h->prm.graphs != 0 && !gr.exec && !gr.failed) capture_launches(h, gr, body);
    if (gr.exec) {
        CK(h, cudaGraphLaunch(gr.exec, h->stream));
        h->launches += gr.launches;
    } else {
        body();
    }
    int info = 0;
    CK(h, cudaMemcpyAsync(&info, cs.info, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (info != 0)
        return fail(h, TOPO_BREAKDOWN, "coarsest-grid matrix not positive definite at row " + std::to_string(info - 1));
    h->coarse_dirty = false;
    return TOPO_OK;
}

topo_status prepare_filter(topo_grid* h, double r) {
    if (!(r > 0.0) || r > 6.0) return fail(h, TOPO_BADARG, "filter radius must be in (0, 6]");
    if (r == h->S_radius) return TOPO_OK;
    const int R = (int)std::ceil(r);
    std::vector<int4> offs;
    std::vector<double> wts;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                const double w = r - std::sqrt((double)(dx * dx + dy * dy + dz * dz));
                if (w > 0.0) {
                    offs.push_back(make_int4(dx, dy, dz, 0));
                    wts.push_back(w);
                }
            }
    if (h->offs) cudaFree(h->offs);
    if (h->wts) cudaFree(h->wts);
    h->offs = nullptr;
    h->wts = nullptr;
    ALLOC(h, h->offs, offs.size());
    ALLOC(h, h->wts, wts.size());
    CK(h, cudaMemcpyAsync(h->offs, offs.data(), sizeof(int4) * offs.size(), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->wts, wts.data(), sizeof(double) * wts.size(), cudaMemcpyHostToDevice, h->stream));
    h->noffs = (int)offs.size();
    const Ctx c = h->ctx();
    const Geom& g = h->lev[0].g;
    filter_launch(c, g, h->offs, h->wts, h->noffs, nullptr, h->S_cache, 2, nullptr);
    fill(c, g.ne, h->xnew_work, 1.0);
    divide(c, g.ne, h->xnew_work, h->S_cache, h->xnew_work);
    filter_launch(c, g, h->offs, h->wts, h->noffs, h->xnew_work, h->dv_cache, 1, nullptr);
    CK(h, cudaStreamSynchronize(h->stream));   // host vectors above go out of scope
    h->S_radius = r;
    return TOPO_OK;
}

// Operator coefficients of operator.cuh from the modal blocks; checks the
// uniform block structure of the isotropic cube that the kernel relies on.
bool build_modal_k(const ModalCoef& m, const double K0[576], ModalK<double>* k, std::string* err) {
    double mx = 0.0;
    for (int i = 0; i < 576; ++i) mx = std::fmax(mx, std::fabs(K0[i]));
    const double tol = 1e-12 * mx;
    bool ok = true;
    auto same = [&](double a, double b) { ok = ok && std::fabs(a - b) <= tol; };
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            same(m.N[i][j], i == j ? m.N[0][0] : m.N[0][1]);
            same(m.T3[i][j], i == j ? m.T3[0][0] : m.T3[0][1]);
        }
    for (int g = 0; g < 3; ++g)
        for (int r = 0; r < 2; ++r)
            for (int q = 0; q < 2; ++q) {
                same(m.S[g][r][q], m.S[0][0][0]);
                same(m.B[g][r][q], r == q ? m.B[0][0][0] : m.B[0][0][1]);
            }
    for (int r = 0; r < 3; ++r) same(m.C[r], m.C[0]);
    for (int i = 0; i < 24; ++i) same(K0[i * 24 + i], K0[0]);
    if (!ok) {
        if (err) *err = "element matrix lacks the uniform modal block structure of the isotropic cube";
        return false;
    }
    k->nd = m.N[0][0] - m.N[0][1];
    k->no = m.N[0][1];
    k->sc = m.S[0][0][0];
    k->bp = m.B[0][0][0];
    k->bq = m.B[0][0][1];
    k->td = m.T3[0][0] - m.T3[0][1];
    k->to = m.T3[0][1];
    k->cg = m.C[0];
    k->kdiag = K0[0];
    return true;
}

topo_status check_handle(topo_grid* h) {
    if (!h) return TOPO_BADARG;
    h->err.clear();
    CK(h, cudaSetDevice(h->device));
    return TOPO_OK;
}

}  // namespace

void topo::ensure_dinv64(topo_grid* h) {
    if (!h->dinv64_dirty) return;
    const Ctx c = h->ctx();
    for (int l = 0; l < h->L; ++l) {
        Level& lv = h->lev[l];
        diag_inverse<double>(c, lv.g, lv.E64, h->mk64->kdiag, lv.Dinv64);
    }
    h->dinv64_dirty = false;
}

void topo::set_global_error(const std::string& msg) { g_create_err = msg; }

extern "C" {

topo_status topo_default_params(topo_params* p) {
    if (!p) return TOPO_BADARG;
    p->E0 = 1.0;
    p->Emin = 1e-9;
    p->nu = 0.3;
    p->penal = 3.0;
    p->levels = 3;
    p->pre = 2;
    p->post = 2;
    p->omega = 0.35;
    p->precision = TOPO_FP64;
    p->inner_tol = 1e-4;
    p->inner_max_it = 500;
    p->max_refine = 12;
    p->homogenize = 0;
    p->graphs = 1;
    p->outer_residual = 0;
    p->tensor_cores = 0;
    p->cg_check = 0;
    return TOPO_OK;
}

topo_status topo_create_grid(int nx, int ny, int nz, const topo_params* prm, void* stream, topo_handle* out) {
    if (!out) return fail(nullptr, TOPO_BADARG, "out is NULL");
    *out = nullptr;
    if (!prm) return fail(nullptr, TOPO_BADARG, "params is NULL");
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(nullptr, TOPO_BADARG, "grid dimensions must be positive");
    const topo_params& p = *prm;
    if (p.levels < 1 || p.levels > 16) return fail(nullptr, TOPO_BADARG, "levels must be in [1, 16]");
    const int div = 1 << (p.levels - 1);
    if (nx % div || ny % div || nz % div)
        return fail(nullptr, TOPO_BADARG, "grid dimensions must be divisible by 2^(levels-1) = " + std::to_string(div));
    if (!(p.nu >= 0.0 && p.nu < 0.5)) return fail(nullptr, TOPO_BADARG, "nu must be in [0, 0.5)");
    if (!(p.E0 > 0.0) || !(p.Emin >= 0.0) || !(p.Emin < p.E0)) return fail(nullptr, TOPO_BADARG, "need 0 <= Emin < E0");
    if (!(p.penal >= 1.0 && p.penal <= 10.0)) return fail(nullptr, TOPO_BADARG, "penal must be in [1, 10]");
    if (!(p.omega > 0.0 && p.omega <= 1.0)) return fail(nullptr, TOPO_BADARG, "omega must be in (0, 1]");
    if (p.pre < 0 || p.post < 0 || p.pre > 32 || p.post > 32) return fail(nullptr, TOPO_BADARG, "bad sweep counts");
    if (p.precision < TOPO_FP64 || p.precision > TOPO_MIXED_BF16) return fail(nullptr, TOPO_BADARG, "bad precision");
    if (!(p.inner_tol > 0.0 && p.inner_tol < 1.0) || p.inner_max_it < 1 || p.max_refine < 1)
        return fail(nullptr, TOPO_BADARG, "bad inner solver parameters");
    if (p.homogenize < 0 || p.homogenize > 2) return fail(nullptr, TOPO_BADARG, "homogenize must be 0, 1 or 2");
    if (p.outer_residual < 0 || p.outer_residual > 1) return fail(nullptr, TOPO_BADARG, "outer_residual must be 0 or 1");
    if (p.tensor_cores < 0 || p.tensor_cores > 1) return fail(nullptr, TOPO_BADARG, "tensor_cores must be 0 or 1");
    if (p.cg_check < 0 || p.cg_check > 1) return fail(nullptr, TOPO_BADARG, "cg_check must be 0 or 1");
    if (p.homogenize == 2 && p.precision == TOPO_MIXED_BF16)
        return fail(nullptr, TOPO_BADARG, "homogenize = 2 (stored Galerkin operators) is not combined with BF16 iterates");
    // the operator kernels index the nodal vectors with 32-bit integers
    if ((long long)(nx + 1) * (ny + 1) * (nz + 1) * 3 >= (1LL << 31))
        return fail(nullptr, TOPO_BADARG, "grid too large: 3 * nodes must be below 2^31");

    topo_grid* h = new (std::nothrow) topo_grid();
    if (!h) return fail(nullptr, TOPO_OOM, "host allocation failed");
    h->prm = p;
    h->stream = (cudaStream_t)stream;
    h->L = p.levels;
    auto bail = [&](topo_status st) {
        g_create_err = h->err;
        free_all(h);
        delete h;
        return st;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        h->err = "no CUDA device";
        return bail(TOPO_CUDA);
    }
    double K0[576];
    element_matrix(p.nu, K0);
    if (!build_modal(K0, &h->modal, &h->err)) return bail(TOPO_BADARG);
    h->mk64 = new ModalK<double>();
    h->mk32 = new ModalK<float>();
    if (!build_modal_k(h->modal, K0, h->mk64, &h->err)) return bail(TOPO_BADARG);
    {
        const ModalK<double>& a = *h->mk64;
        ModalK<float>& b = *h->mk32;
        b.nd = (float)a.nd; b.no = (float)a.no; b.sc = (float)a.sc; b.bp = (float)a.bp; b.bq = (float)a.bq;
        b.td = (float)a.td; b.to = (float)a.to; b.cg = (float)a.cg; b.kdiag = (float)a.kdiag;
        // double-FP32 pairs: nearest FP32 value and the FP32-rounded remainder
        auto split = [](double v) { const float hi = (float)v; return dfl(hi, (float)(v - (double)hi)); };
        h->mkdf = new ModalK<dfl>();
        ModalK<dfl>& d = *h->mkdf;
        d.nd = split(a.nd); d.no = split(a.no); d.sc = split(a.sc); d.bp = split(a.bp); d.bq = split(a.bq);
        d.td = split(a.td); d.to = split(a.to); d.cg = split(a.cg); d.kdiag = split(a.kdiag);
    }
    h->lev.resize(h->L);
    h->npartials = kRedBlocks;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || nsm <= 0) {
        cudaGetLastError();
        nsm = 152;
    }
    for (int l = 0; l < h->L; ++l) {
        Level& lv = h->lev[l];
        lv.g = make_geom(nx >> l, ny >> l, nz >> l);
        lv.scale = (double)(1 << l);
        lv.op32 = op_launch32(lv.g, nsm);
        lv.op64 = op_launch64(lv.g, nsm);
        lv.optc = op_launch_tc(lv.g, nsm);
        h->npartials = std::max(h->npartials, std::max(lv.op32.ctas(), std::max(lv.op64.ctas(), lv.optc.ctas())));
    }
    topo_status st;
#define TRY(expr)                          \
    do {                                   \
        st = (expr);                       \
        if (st != TOPO_OK) return bail(st); \
    } while (0)
    for (auto& lv : h->lev) {
        TRY(dalloc(h, &lv.rho, lv.g.ne));
        TRY(dalloc(h, &lv.E64, lv.g.ne));
        TRY(dalloc(h, &lv.E32, lv.g.ne));
        TRY(dalloc(h, &lv.mask, lv.g.nn));
        TRY(dalloc(h, &lv.Dinv64, lv.g.nn));
        TRY(dalloc(h, &lv.Dinv32, lv.g.nn));
    }
    const Geom& g0 = h->lev[0].g;
    const long long n0 = 3 * g0.nn;
    TRY(dalloc(h, &h->x, n0));
    TRY(dalloc(h, &h->f, n0));
    TRY(dalloc(h, &h->r, n0));
    TRY(dalloc(h, &h->K0d, 576));
    TRY(dalloc(h, &h->K0f, 576));
    TRY(dalloc(h, &h->dc_work, g0.ne));
    TRY(dalloc(h, &h->xnew_work, g0.ne));
    TRY(dalloc(h, &h->oc_hi, g0.ne));
    TRY(dalloc(h, &h->S_cache, g0.ne));
    TRY(dalloc(h, &h->dv_cache, g0.ne));
    TRY(dalloc(h, &h->lam, 8));
    TRY(dalloc(h, &h->dtmp, 8));
    TRY(dalloc(h, &h->dflag, 4));
    TRY(dalloc(h, &h->tc_err, 1));
    TRY(dalloc(h, &h->tcB, kTcBWords));
    TRY(dalloc(h, &h->partials, (size_t)h->npartials));
    TRY(dalloc(h, &h->sc, 1));
    TRY(dalloc(h, &h->alpha_hist, kDirRing));
    h->cs.n = (int)std::min<long long>(3 * h->lev[h->L - 1].g.nn, 1LL << 30);
    h->cs.npad = (h->cs.n + 31) / 32 * 32;
    TRY(alloc_precision(h, p.precision == TOPO_FP64));
    if (p.precision == TOPO_MIXED_BF16) TRY(alloc_bf16(h));
    if (cudaMallocHost((void**)&h->host_sc, sizeof(Scalars)) != cudaSuccess) {
        h->host_sc = nullptr;
        h->err = "cudaMallocHost failed";
        return bail(TOPO_OOM);
    }
    std::memset(h->host_sc, 0, sizeof(Scalars));
    float K0f[576];
    for (int i = 0; i < 576; ++i) K0f[i] = (float)K0[i];
    std::vector<uint32_t> tcimg(kTcBWords);
    tc_b_image(K0, tcimg.data());
    bool ok = cudaMemcpyAsync(h->K0d, K0, sizeof(K0), cudaMemcpyHostToDevice, h->stream) == cudaSuccess &&
              cudaMemcpyAsync(h->K0f, K0f, sizeof(K0f), cudaMemcpyHostToDevice, h->stream) == cudaSuccess &&
              cudaMemsetAsync(h->x, 0, sizeof(double) * n0, h->stream) == cudaSuccess &&
              cudaMemsetAsync(h->f, 0, sizeof(double) * n0, h->stream) == cudaSuccess &&
              cudaMemsetAsync(h->sc, 0, sizeof(Scalars), h->stream) == cudaSuccess &&
              cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream) == cudaSuccess &&
              cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream) == cudaSuccess &&
              cudaMemcpyAsync(h->tcB, tcimg.data(), sizeof(uint32_t) * kTcBWords, cudaMemcpyHostToDevice,
                              h->stream) == cudaSuccess;
    for (auto& lv : h->lev) ok = ok && cudaMemsetAsync(lv.mask, 0, lv.g.nn, h->stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(h->stream) == cudaSuccess;   // K0 host arrays go out of scope
    if (!ok) {
        h->err = std::string("initialisation failed: ") + cudaGetErrorString(cudaGetLastError());
        return bail(TOPO_CUDA);
    }
#undef TRY
    *out = h;
    return TOPO_OK;
}

topo_status topo_destroy_grid(topo_handle h) {
    if (!h) return TOPO_BADARG;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return TOPO_OK;
}

const char* topo_last_error(topo_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

// the density from device (kind = DeviceToDevice) or host memory
// (HostToDevice) into the level-0 copy, then moduli and coarse levels
static topo_status set_density_from(topo_handle h, const double* rho, cudaMemcpyKind kind) {
    const Ctx c = h->ctx();
    CK(h, cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream));
    CK(h, cudaMemcpyAsync(h->lev[0].rho, rho, sizeof(double) * h->lev[0].g.ne, kind, h->stream));
    if (h->prm.homogenize == 2 && h->L > 1) {   // stored Galerkin element matrices of levels 1 .. L-1
        galerkin_init_constants();
        if (!h->G64) {
            double K0[576];
            element_matrix(h->prm.nu, K0);
            std::vector<double> G(8 * 576);
            galerkin_child_matrices(K0, G.data());
            ALLOC(h, h->G64, 8 * 576);
            CK(h, cudaMemcpyAsync(h->G64, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));   // G goes out of scope
        }
        for (int l = 1; l < h->L; ++l) {
            Level& lv = h->lev[l];
            // both copies: FP32 level operators can be requested on any handle
            if (!lv.Ke64) ALLOC(h, lv.Ke64, 576 * lv.g.ne);
            if (!lv.Ke32) ALLOC(h, lv.Ke32, 576 * lv.g.ne);
        }
    }
    for (int l = 0; l < h->L; ++l) {
        Level& lv = h->lev[l];
        if (l == 0 || h->prm.homogenize != 1)
            simp_moduli(c, lv.g.ne, lv.rho, lv.scale, h->prm.E0, h->prm.Emin, h->prm.penal, lv.E64, lv.E32,
                        h->dflag);
        if (l + 1 < h->L) {
            Level& lc = h->lev[l + 1];
            homogenize(c, lv.g, lv.rho, lc.rho, 1.0);
            if (h->prm.homogenize == 1) {   // E_{l+1} = 2 * mean of the children's E_l
                homogenize(c, lv.g, lv.E64, lc.E64, 2.0);
                convert<double, float>(c, lc.g.ne, lc.E64, lc.E32);
            }
        }
    }
    for (int l = 0; l < h->L; ++l) {   // FP32 Jacobi diagonals from the final moduli of every level
        Level& lv = h->lev[l];
        diag_inverse<float>(c, lv.g, lv.E32, h->mk32->kdiag, lv.Dinv32);
    }
    h->dinv64_dirty = true;   // FP64 ones on demand (ensure_dinv64): FP64 division runs on the slow FP64 pipe
    if (h->prm.homogenize == 2) {
        for (int l = 1; l < h->L; ++l) {
            Level& lv = h->lev[l];
            Level& lf = h->lev[l - 1];
            galerkin_build(c, lf.g, h->K0d, h->G64, lf.E64, l == 1 ? nullptr : lf.Ke64, lv.Ke64);
            convert<double, float>(c, 576 * lv.g.ne, lv.Ke64, lv.Ke32);
        }
    }
    CK(h, cudaGetLastError());
    h->have_density = true;
    h->coarse_dirty = true;
    return TOPO_OK;
}

topo_status topo_set_density(topo_handle h, const double* rho_dev) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!rho_dev) return fail(h, TOPO_BADARG, "rho is NULL");
    return set_density_from(h, rho_dev, cudaMemcpyDeviceToDevice);
}

topo_status topo_set_bc_loads(topo_handle h, const uint8_t* fixed_dev, const double* f_dev) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!fixed_dev || !f_dev) return fail(h, TOPO_BADARG, "NULL pointer");
    const Ctx c = h->ctx();
    mask_from_dofs(c, h->lev[0].g.nn, fixed_dev, h->lev[0].mask);
    for (int l = 0; l + 1 < h->L; ++l) inject_mask(c, h->lev[l].g, h->lev[l].mask, h->lev[l + 1].mask);
    const long long n0 = 3 * h->lev[0].g.nn;
    masked_copy_load(c, h->lev[0].g.nn, h->lev[0].mask, f_dev, h->f);
    CK(h, cudaMemsetAsync(h->x, 0, sizeof(double) * n0, h->stream));
    h->x_zero = true;
    dot_partials<double, double>(c, n0, h->f, h->f, h->partials);
    reduce_to(c, h->partials, kRedBlocks, &h->sc->ff);
    CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->have_bc = true;
    h->coarse_dirty = true;
    return TOPO_OK;
}

topo_status topo_solve_state(topo_handle h, double rel_tol, int max_it, double* u_dev_out, int* iters_out,
                             double* relres_out) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!(rel_tol > 0.0) || max_it < 1) return fail(h, TOPO_BADARG, "rel_tol must be > 0 and max_it >= 1");
    if (!h->have_density || !h->have_bc) return fail(h, TOPO_BADARG, "set density and boundary conditions first");
    const auto t0 = std::chrono::steady_clock::now();
    int bad = 0;
    CK(h, cudaMemcpyAsync(&bad, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (bad) return fail(h, TOPO_BADARG, "density outside [0, 1] or NaN");
    const bool fp64 = h->prm.precision == TOPO_FP64;
    s = alloc_precision(h, fp64);
    if (s != TOPO_OK) return s;
    s = ensure_coarse(h);
    if (s == TOPO_BREAKDOWN) {
        // the coarsest operator is singular (no or too few Dirichlet
        // conditions): no iteration ran; the best iterate is the warm start
        const std::string msg = h->err;
        const double rel = current_relres(h);
        if (u_dev_out)
            CK(h, cudaMemcpyAsync(u_dev_out, h->x, sizeof(double) * 3 * h->lev[0].g.nn, cudaMemcpyDeviceToDevice,
                                  h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        h->stats.inner_iters = 0;
        h->stats.outer_steps = 0;
        h->stats.relres = rel;
        h->stats.status = TOPO_BREAKDOWN;
        if (iters_out) *iters_out = 0;
        if (relres_out) *relres_out = rel;
        h->err = msg;
        return TOPO_BREAKDOWN;
    }
    if (s != TOPO_OK) return s;
    int iters = 0;
    double relres = 0.0;
    int st = TOPO_OK;
    h->stats.graph_replays = 0;
    const double ff = h->host_sc[6];
    if (ff == 0.0) {
        CK(h, cudaMemsetAsync(h->x, 0, sizeof(double) * 3 * h->lev[0].g.nn, h->stream));
        h->stats.outer_steps = 0;
        h->x_zero = true;
    } else if (fp64) {
        st = solve_fp64(h, rel_tol, max_it, &iters, &relres);
        h->x_zero = false;
    } else {
        st = solve_mixed(h, rel_tol, max_it, &iters, &relres);
        h->x_zero = false;
    }
    if (u_dev_out)
        CK(h, cudaMemcpyAsync(u_dev_out, h->x, sizeof(double) * 3 * h->lev[0].g.nn, cudaMemcpyDeviceToDevice,
                              h->stream));
    int tc_bad = 0;
    if (h->prm.tensor_cores) CK(h, cudaMemcpyAsync(&tc_bad, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaGetLastError());
    if (tc_bad) {
        cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream);
        return fail(h, TOPO_CUDA, "tensor-core operator: a bounded wait for the MMA ran out");
    }
    const auto t1 = std::chrono::steady_clock::now();
    h->stats.inner_iters = iters;
    h->stats.relres = relres;
    h->stats.solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    h->stats.status = st;
    if (iters_out) *iters_out = iters;
    if (relres_out) *relres_out = relres;
    if (st == TOPO_MAXITER) h->err = "solver did not reach the tolerance";
    if (st == TOPO_BREAKDOWN) h->err = "CG breakdown (non-positive curvature or non-finite value)";
    return (topo_status)st;
}

topo_status topo_compliance_and_sensitivity(topo_handle h, double* C_out, double* dc_dev_out) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!h->have_density || !h->have_bc) return fail(h, TOPO_BADARG, "set density and boundary conditions first");
    const Ctx c = h->ctx();
    const Geom& g = h->lev[0].g;
    element_energy_sens(c, g, h->modal, h->x, h->lev[0].rho, h->prm.E0, h->prm.Emin, h->prm.penal,
                        dc_dev_out ? dc_dev_out : h->dc_work, h->partials, h->prm.precision != TOPO_FP64);
    reduce_to(c, h->partials, kRedBlocks, h->dtmp);
    if (C_out) {
        CK(h, cudaMemcpyAsync(C_out, h->dtmp, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    CK(h, cudaGetLastError());
    return TOPO_OK;
}

topo_status topo_state_step_host(topo_handle h, const double* rho_host, double rel_tol, int max_it, double* C_out,
                                 double* dc_host_out, int* iters_out, double* relres_out) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!rho_host) return fail(h, TOPO_BADARG, "rho is NULL");
    s = set_density_from(h, rho_host, cudaMemcpyHostToDevice);
    if (s != TOPO_OK) return s;
    const topo_status st = topo_solve_state(h, rel_tol, max_it, nullptr, iters_out, relres_out);
    if (st != TOPO_OK && st != TOPO_MAXITER && st != TOPO_BREAKDOWN) return st;
    const std::string msg = h->err;   // the solve's message survives the steps below
    s = topo_compliance_and_sensitivity(h, C_out, dc_host_out ? h->dc_work : nullptr);
    if (s != TOPO_OK) return s;
    if (dc_host_out) {
        CK(h, cudaMemcpyAsync(dc_host_out, h->dc_work, sizeof(double) * h->lev[0].g.ne, cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    h->err = msg;
    return st;
}

topo_status topo_filter(topo_handle h, double r, const double* in_dev, double* out_dev, int transpose) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!in_dev || !out_dev || in_dev == out_dev) return fail(h, TOPO_BADARG, "bad pointers");
    s = prepare_filter(h, r);
    if (s != TOPO_OK) return s;
    const Ctx c = h->ctx();
    const Geom& g = h->lev[0].g;
    if (transpose) {
        divide(c, g.ne, in_dev, h->S_cache, h->xnew_work);
        filter_launch(c, g, h->offs, h->wts, h->noffs, h->xnew_work, out_dev, 1, nullptr);
    } else {
        filter_launch(c, g, h->offs, h->wts, h->noffs, in_dev, out_dev, 0, nullptr);
    }
    CK(h, cudaGetLastError());
    return TOPO_OK;
}

// bisection of Eq. OC on lambda (reading of the paper: l1 = 0, l2 = 1e9,
// relative tolerance 1e-9) over q = x sqrt(-dc / dv) in dc_work and the
// bounds in xnew_work / oc_hi; dv null: volume of x itself; writes x and change
static topo_status oc_bisection(topo_grid* h, double volfrac, double* rho_dev_inout, const double* dv,
                                double* change_out, double n_volume) {
    const Ctx c = h->ctx();
    const Geom& g = h->lev[0].g;
    const double l1 = 0.0, l2 = 1e9, tol = 1e-9;
    const double init[8] = {l1, l2, 0.5 * (l1 + l2), (l2 - l1) / (l1 + l2) > tol ? 0.0 : 1.0, 0.0, 0.5 * (l1 + l2),
                            0.0, 0.0};
    CK(h, cudaMemcpyAsync(h->lam, init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
    double state[8];
    for (int batch = 0; batch < 25; ++batch) {
        for (int k = 0; k < 16; ++k) {
            oc_bisect_step(c, g.ne, h->xnew_work, h->oc_hi, h->dc_work, dv, h->partials, h->lam);
            oc_bisect_finalize(c, h->partials, h->lam, volfrac * n_volume, tol);
        }
        CK(h, cudaMemcpyAsync(state, h->lam, sizeof(state), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        if (state[3] != 0.0) break;
    }
    if (state[3] == 0.0) return fail(h, TOPO_MAXITER, "bisection did not converge");
    oc_write(c, g.ne, rho_dev_inout, h->xnew_work, h->oc_hi, h->dc_work, h->lam, h->partials, h->dtmp);
    if (change_out) {
        CK(h, cudaMemcpyAsync(change_out, h->dtmp, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    CK(h, cudaGetLastError());
    return TOPO_OK;
}

topo_status topo_oc_update(topo_handle h, double r, double move, double volfrac, double* rho_dev_inout,
                           const double* dc_dev, double* change_out) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!rho_dev_inout || !dc_dev) return fail(h, TOPO_BADARG, "NULL pointer");
    if (!(move > 0.0 && move <= 1.0) || !(volfrac > 0.0 && volfrac < 1.0))
        return fail(h, TOPO_BADARG, "move must be in (0,1], volfrac in (0,1)");
    s = prepare_filter(h, r);
    if (s != TOPO_OK) return s;
    const Ctx c = h->ctx();
    const Geom& g = h->lev[0].g;
    divide(c, g.ne, dc_dev, h->S_cache, h->xnew_work);
    filter_launch(c, g, h->offs, h->wts, h->noffs, h->xnew_work, h->dc_work, 1, nullptr);
    // q over dc_work, lower bounds in xnew_work, upper bounds in oc_hi
    oc_prepare(c, g.ne, rho_dev_inout, h->dc_work, h->dv_cache, move, h->xnew_work, h->oc_hi);
    return oc_bisection(h, volfrac, rho_dev_inout, h->dv_cache, change_out, (double)g.ne);
}

topo_status topo_oc_update_unfiltered(topo_handle h, double move, double volfrac, const uint8_t* passive_dev,
                                      double* rho_dev_inout, const double* dc_dev, double* change_out) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!rho_dev_inout || !dc_dev) return fail(h, TOPO_BADARG, "NULL pointer");
    if (!(move > 0.0 && move <= 1.0) || !(volfrac > 0.0 && volfrac < 1.0))
        return fail(h, TOPO_BADARG, "move must be in (0,1], volfrac in (0,1)");
    const Ctx c = h->ctx();
    const Geom& g = h->lev[0].g;
    CK(h, cudaMemcpyAsync(h->dc_work, dc_dev, sizeof(double) * g.ne, cudaMemcpyDeviceToDevice, h->stream));
    if (!passive_dev) {
        oc_prepare(c, g.ne, rho_dev_inout, h->dc_work, nullptr, move, h->xnew_work, h->oc_hi);
        return oc_bisection(h, volfrac, rho_dev_inout, nullptr, change_out, (double)g.ne);
    }
    if (!h->oc_dv) ALLOC(h, h->oc_dv, g.ne);
    oc_prepare_passive(c, g.ne, rho_dev_inout, h->dc_work, passive_dev, move, h->xnew_work, h->oc_hi, h->oc_dv);
    dot_partials<double, double>(c, g.ne, h->oc_dv, h->oc_dv, h->partials);   // number of active elements
    reduce_to(c, h->partials, kRedBlocks, h->dtmp);
    double n_active = 0.0;
    CK(h, cudaMemcpyAsync(&n_active, h->dtmp, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (!(n_active > 0.0)) return fail(h, TOPO_BADARG, "no active elements");
    return oc_bisection(h, volfrac, rho_dev_inout, h->oc_dv, change_out, n_active);
}

topo_status topo_gravity_load(topo_handle h, double w, const double* rho_dev, const double* f_ext_dev,
                              double* f_out_dev) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!rho_dev || !f_out_dev || f_out_dev == f_ext_dev) return fail(h, TOPO_BADARG, "bad pointers");
    gravity_load(h->ctx(), h->lev[0].g, rho_dev, f_ext_dev, f_out_dev, w);
    CK(h, cudaGetLastError());
    return TOPO_OK;
}

topo_status topo_gravity_sensitivity(topo_handle h, double w, double* dc_dev_inout) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!dc_dev_inout) return fail(h, TOPO_BADARG, "NULL pointer");
    gravity_sensitivity(h->ctx(), h->lev[0].g, h->x, dc_dev_inout, w);
    CK(h, cudaGetLastError());
    return TOPO_OK;
}

topo_status topo_sensitivity_filter(topo_handle h, double r, double gamma, const double* rho_dev,
                                    const double* dc_dev, double* out_dev) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (!rho_dev || !dc_dev || !out_dev || out_dev == rho_dev || out_dev == dc_dev)
        return fail(h, TOPO_BADARG, "bad pointers");
    if (!(gamma > 0.0)) return fail(h, TOPO_BADARG, "gamma must be positive");
    s = prepare_filter(h, r);
    if (s != TOPO_OK) return s;
    sensitivity_filter(h->ctx(), h->lev[0].g, h->offs, h->wts, h->noffs, rho_dev, dc_dev, gamma, h->xnew_work,
                       out_dev);
    CK(h, cudaGetLastError());
    return TOPO_OK;
}

topo_status topo_level_dims(topo_handle h, int level, int* nx, int* ny, int* nz) {
    if (!h || level < 0 || level >= h->L || !nx || !ny || !nz) return TOPO_BADARG;
    *nx = h->lev[level].g.nx;
    *ny = h->lev[level].g.ny;
    *nz = h->lev[level].g.nz;
    return TOPO_OK;
}

static topo_status step_check(topo_grid* h, int level, int precision, bool allow_bf16 = false,
                              bool allow_df = false) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (level < 0 || level >= h->L) return fail(h, TOPO_BADARG, "level out of range");
    if (precision == TOPO_DF32 && allow_df) {
        if (!h->have_density) return fail(h, TOPO_BADARG, "set density first");
        return alloc_precision(h, true);
    }
    if (precision == TOPO_FP32_TC && allow_df) {
        if (!h->have_density) return fail(h, TOPO_BADARG, "set density first");
        return alloc_precision(h, false);
    }
    if (precision == TOPO_MIXED_BF16 && allow_bf16) {
        if (!h->have_density) return fail(h, TOPO_BADARG, "set density first");
        s = alloc_precision(h, false);
        return s != TOPO_OK ? s : alloc_bf16(h);
    }
    if (precision != TOPO_FP64 && precision != TOPO_MIXED)
        return fail(h, TOPO_BADARG, allow_bf16 ? "precision must be 0, 1 or 2" : "precision must be 0 or 1");
    if (!h->have_density) return fail(h, TOPO_BADARG, "set density first");
    return alloc_precision(h, precision == TOPO_FP64);
}

// runs a level operator in FP32: inputs rounded into level buffers, result widened
enum { OP_APPLY, OP_JACOBI, OP_RESID };
static topo_status level_op(topo_grid* h, int level, int precision, int op, const double* u, const double* f,
                            double* out) {
    topo_status s = step_check(h, level, precision, false, op != OP_JACOBI || precision == TOPO_FP32_TC);
    if (s != TOPO_OK) return s;
    if (!u || !out || (op != OP_APPLY && !f)) return fail(h, TOPO_BADARG, "NULL pointer");
    const int mode = op == OP_APPLY ? ST_APPLY : (op == OP_JACOBI ? ST_JACOBI : ST_RESID);
    const Ctx c = h->ctx();
    Level& lv = h->lev[level];
    const long long n = 3 * lv.g.nn;
    if (precision == TOPO_FP32_TC) {
        if (h->prm.homogenize == 2 && level > 0)
            return fail(h, TOPO_BADARG, "tensor-core kernel: not for stored Galerkin levels");
        convert<double, float>(c, n, u, lv.v32.a);
        if (f) convert<double, float>(c, n, f, lv.v32.f);
        stencil_tc(c, mode, lv.optc, h->mk32->kdiag, lv.E32, lv.mask, lv.v32.a, f ? lv.v32.f : nullptr, lv.v32.b,
                   (float)h->prm.omega, h->tcB, nullptr, h->tc_err);
        convert<float, double>(c, n, lv.v32.b, out);
        int bad = 0;
        CK(h, cudaMemcpyAsync(&bad, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        if (bad) {
            cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream);
            return fail(h, TOPO_CUDA, "tensor-core operator: a bounded wait for the MMA ran out");
        }
    } else if (precision == TOPO_DF32) {
        if (h->prm.homogenize == 2 && level > 0)
            return fail(h, TOPO_BADARG, "double-FP32 kernel: not for stored Galerkin levels");
        if (stencil_df(c, mode, lv.op64, *h->mkdf, lv.E64, lv.mask, u, f, out, nullptr, nullptr) < 0)
            return fail(h, TOPO_BADARG, "double-FP32 kernel: mode not available");
    } else if (precision == TOPO_FP64) {
        op_apply<double>(h, mode, level, u, f, out, nullptr);
    } else {
        convert<double, float>(c, n, u, lv.v32.a);
        if (f) convert<double, float>(c, n, f, lv.v32.f);
        op_apply<float>(h, mode, level, lv.v32.a, f ? lv.v32.f : nullptr, lv.v32.b, nullptr);
        convert<float, double>(c, n, lv.v32.b, out);
    }
    CK(h, cudaGetLastError());
    return TOPO_OK;
}

topo_status topo_apply_operator(topo_handle h, int level, int precision, const double* u_dev, double* y_dev) {
    return level_op(h, level, precision, OP_APPLY, u_dev, nullptr, y_dev);
}
topo_status topo_jacobi_sweep(topo_handle h, int level, int precision, const double* u_dev, const double* f_dev,
                              double* u_out_dev) {
    return level_op(h, level, precision, OP_JACOBI, u_dev, f_dev, u_out_dev);
}
topo_status topo_residual(topo_handle h, int level, int precision, const double* u_dev, const double* f_dev,
                          double* r_dev) {
    return level_op(h, level, precision, OP_RESID, u_dev, f_dev, r_dev);
}

topo_status topo_restrict(topo_handle h, int level, const double* fine_dev, double* coarse_dev) {
    topo_status s = step_check(h, level, TOPO_FP64);
    if (s != TOPO_OK) return s;
    if (level + 1 >= h->L || !fine_dev || !coarse_dev) return fail(h, TOPO_BADARG, "bad level or pointer");
    restrict_residual<double>(h->ctx(), h->lev[level].g, h->lev[level].mask, h->lev[level + 1].mask, fine_dev,
                              coarse_dev);
    CK(h, cudaGetLastError());
    return TOPO_OK;
}

topo_status topo_prolong_add(topo_handle h, int level, const double* coarse_dev, double* fine_dev) {
    topo_status s = step_check(h, level, TOPO_FP64);
    if (s != TOPO_OK) return s;
    if (level + 1 >= h->L || !fine_dev || !coarse_dev) return fail(h, TOPO_BADARG, "bad level or pointer");
    prolong_add<double>(h->ctx(), h->lev[level].g, h->lev[level].mask, h->lev[level + 1].mask, coarse_dev, fine_dev);
    CK(h, cudaGetLastError());
    return TOPO_OK;
}

topo_status topo_level_density(topo_handle h, int level, double* rho_dev_out) {
    topo_status s = step_check(h, level, TOPO_FP64);
    if (s != TOPO_OK) return s;
    if (!rho_dev_out) return fail(h, TOPO_BADARG, "NULL pointer");
    CK(h, cudaMemcpyAsync(rho_dev_out, h->lev[level].rho, sizeof(double) * h->lev[level].g.ne,
                          cudaMemcpyDeviceToDevice, h->stream));
    return TOPO_OK;
}

topo_status topo_vcycle(topo_handle h, int precision, const double* r_dev, double* z_dev) {
    topo_status s = step_check(h, 0, precision, true);
    if (s != TOPO_OK) return s;
    if (!r_dev || !z_dev || r_dev == z_dev) return fail(h, TOPO_BADARG, "bad pointers");
    s = ensure_coarse(h);
    if (s != TOPO_OK) return s;
    Level& l0 = h->lev[0];
    const long long n = 3 * l0.g.nn;
    if (precision == TOPO_FP64) {
        ensure_dinv64(h);
        vcycle<double>(h, 0, r_dev, z_dev, l0.v64.a, nullptr);
    } else if (precision == TOPO_MIXED_BF16) {
        const Ctx c = h->ctx();
        convert<double, float>(c, n, r_dev, l0.v32.f);
        vcycle_bf16(h, 0, l0.v32.f, l0.v32.b, nullptr);
        convert<float, double>(c, n, l0.v32.b, z_dev);
    } else {
        const Ctx c = h->ctx();
        convert<double, float>(c, n, r_dev, l0.v32.f);
        vcycle<float>(h, 0, l0.v32.f, l0.v32.b, l0.v32.a, nullptr);
        convert<float, double>(c, n, l0.v32.b, z_dev);
    }
    CK(h, cudaGetLastError());
    return TOPO_OK;
}

topo_status topo_get_stats(topo_handle h, topo_solve_stats* out) {
    if (!h || !out) return TOPO_BADARG;
    *out = h->stats;
    return TOPO_OK;
}

topo_status topo_launch_count(topo_handle h, long long* out) {
    if (!h || !out) return TOPO_BADARG;
    *out = h->launches;
    return TOPO_OK;
}

topo_status topo_reset_solution(topo_handle h) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    CK(h, cudaMemsetAsync(h->x, 0, sizeof(double) * 3 * h->lev[0].g.nn, h->stream));
    h->x_zero = true;
    return TOPO_OK;
}

topo_status topo_profile_enable(topo_handle h, int on) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    CK(h, cudaStreamSynchronize(h->stream));
    h->prof_on = on != 0;
    if (on) {
        h->prof_n = 0;
        h->prof_kind.clear();
    }
    return TOPO_OK;
}

topo_status topo_profile_read(topo_handle h, int mode, long long* launches, double* total_ms) {
    topo_status s = check_handle(h);
    if (s != TOPO_OK) return s;
    if (mode < 0 || mode > 5 || !launches || !total_ms) return fail(h, TOPO_BADARG, "bad arguments");
    CK(h, cudaStreamSynchronize(h->stream));
    for (int q = 0; q < 5; ++q) {
        launches[q] = 0;
        total_ms[q] = 0.0;
    }
    for (int i = 0; i < h->prof_n; ++i) {
        const int k = h->prof_kind[i];   // mode * 8 + precision slot
        if (k / 8 != mode) continue;
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
        launches[k & 7] += 1;
        total_ms[k & 7] += ms;
    }
    return TOPO_OK;
}

}  // extern "C"
