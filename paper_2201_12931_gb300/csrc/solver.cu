// Host orchestration of the state solve, all work enqueued on the handle's
// stream:
//   * V-cycle (Algorithm 3) with damped-Jacobi smoothing, residual
//     restriction, recursion from a zero iterate, prolongation correction and
//     the direct solve on the coarsest grid;
//   * preconditioned CG (Algorithm 1, standard initialisation r0 = f - K x0,
//     z0 = M^-1 r0, p0 = z0), scalars kept on the device; the direction
//     update fused into K.p, directions kept in a ring of 8 buffers with
//     x += alpha p applied once per ring; iterations after the first
//     replayed from captured CUDA graphs (one per ring slot); flexible beta
//     for the BF16-iterate V-cycle;
//   * FP64 iterative refinement around an FP32 inner MGPCG (mixed modes):
//     r = f - K x in FP64, solve K d ~= r in FP32, x += d, repeat.
#include <chrono>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "operator.cuh"
#include "solver.h"

namespace topo {

template <typename T>
struct P;
template <>
struct P<double> {
    static const ModalK<double>& mk(topo_grid* h) { return *h->mk64; }
    static const OpLaunch& op(Level& l) { return l.op64; }
    static const double* E(Level& l) { return l.E64; }
    static const double* Dinv(Level& l) { return l.Dinv64; }
    static VBuf<double>& vb(Level& l) { return l.v64; }
    static const double* W(topo_grid* h) { return h->cs.W64; }
    static const double* WT(topo_grid* h) { return h->cs.WT64; }
    static double* y(topo_grid* h) { return h->cs.y64; }
    static const double* Ke(Level& l) { return l.Ke64; }
    static PcgGraph* graph(topo_grid* h) { return h->graph64; }
    static double* const* dring(topo_grid* h) { return h->dring64; }
};
template <>
struct P<float> {
    static const ModalK<float>& mk(topo_grid* h) { return *h->mk32; }
    static const OpLaunch& op(Level& l) { return l.op32; }
    static const float* E(Level& l) { return l.E32; }
    static const float* Dinv(Level& l) { return l.Dinv32; }
    static VBuf<float>& vb(Level& l) { return l.v32; }
    static const float* W(topo_grid* h) { return h->cs.W32; }
    static const float* WT(topo_grid* h) { return h->cs.WT32; }
    static float* y(topo_grid* h) { return h->cs.y32; }
    static const float* Ke(Level& l) { return l.Ke32; }
    static PcgGraph* graph(topo_grid* h) { return h->graph32; }
    static float* const* dring(topo_grid* h) { return h->dring32; }
};

template <typename T>
int op_apply(topo_grid* h, int mode, int l, const T* u, const T* f, T* out, double* dot, T* pout,
             const double* beta) {
    Level& lv = h->lev[l];
    // FP32 operators with K.u on the tensor cores (the first sweep needs none)
    const bool tc = std::is_same<T, float>::value && h->prm.tensor_cores != 0 &&
                    (mode == ST_APPLY || mode == ST_JACOBI || mode == ST_RESID);
    const bool rec = h->prof_on && l == 0 && h->prof_n < kProfMax;
    if (rec) {
        if ((int)h->prof_ev.size() < 2 * (h->prof_n + 1)) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            h->prof_ev.push_back(a);
            h->prof_ev.push_back(b);
        }
        cudaEventRecord(h->prof_ev[2 * h->prof_n], h->stream);
    }
    int np = 0;
    if (h->prm.homogenize == 2 && l > 0) {   // stored Galerkin element matrices (no fused dot on coarse levels)
        if (!P<T>::Ke(lv)) {   // not built: set_density forms them; never launch on a null matrix
            set_global_error("Galerkin element matrices missing (set the density first)");
            return 0;
        }
        elem_op<T>(h->ctx(), mode, lv.g, P<T>::Ke(lv), lv.mask, u, f, out, (T)h->prm.omega);
        if (dot) {
            dot_partials<T, T>(h->ctx(), 3 * lv.g.nn, mode == ST_APPLY ? u : (mode == ST_RESID ? out : f), out, dot);
            np = kRedBlocks;
        }
    } else if (tc) {
        if constexpr (std::is_same<T, float>::value)
            np = stencil_tc(h->ctx(), mode, lv.optc, h->mk32->kdiag, lv.E32, lv.mask, u, f, out, (float)h->prm.omega,
                            h->tcB, dot, h->tc_err);
    } else {
        np = stencil<T>(h->ctx(), mode, P<T>::op(lv), P<T>::mk(h), P<T>::E(lv), lv.mask, u, f, out,
                        (T)h->prm.omega, dot, P<T>::Dinv(lv), pout, beta);
    }
    if (rec) {
        cudaEventRecord(h->prof_ev[2 * h->prof_n + 1], h->stream);
        h->prof_kind.resize(h->prof_n + 1);
        h->prof_kind[h->prof_n] = mode * 8 + (sizeof(T) == 4 ? (tc ? 4 : 1) : 0);
        ++h->prof_n;
    }
    return dot ? np : 0;
}
template int op_apply<double>(topo_grid*, int, int, const double*, const double*, double*, double*, double*,
                              const double*);
template int op_apply<float>(topo_grid*, int, int, const float*, const float*, float*, double*, float*,
                             const double*);

template <typename T>
int vcycle(topo_grid* h, int l, const T* f, T* out, T* tmp, double* dot) {
    const Ctx c = h->ctx();
    Level& lv = h->lev[l];
    if (l == h->L - 1) {
        coarse_apply<T>(c, h->cs.n, h->cs.npad, P<T>::W(h), P<T>::WT(h), f, P<T>::y(h), out);
        if (dot) dot_partials<T, T>(c, 3 * lv.g.nn, f, out, dot);
        return dot ? kRedBlocks : 0;
    }
    const int pre = h->prm.pre, post = h->prm.post;
    const int nflip = (pre > 0 ? pre - 1 : 0) + post;
    T* cur = (nflip & 1) ? tmp : out;
    T* oth = (cur == out) ? tmp : out;
    const long long n = 3 * lv.g.nn;
    if (pre > 0) {
        // the first two sweeps from zero as one kernel on matrix-free levels
        const bool two = pre >= 2 && !(h->prm.homogenize == 2 && l > 0);
        if (two) {
            op_apply<T>(h, ST_JACOBI2, l, nullptr, f, oth, nullptr);
            T* t = cur; cur = oth; oth = t;
        } else {
            op_apply<T>(h, ST_JACOBI0, l, nullptr, f, cur, nullptr);
        }
        for (int s = two ? 2 : 1; s < pre; ++s) {
            op_apply<T>(h, ST_JACOBI, l, cur, f, oth, nullptr);
            T* t = cur; cur = oth; oth = t;
        }
        op_apply<T>(h, ST_RESID, l, cur, f, oth, nullptr);
    } else {
        zero<T>(c, n, cur);
        cudaMemcpyAsync(oth, f, sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream);
    }
    Level& lc = h->lev[l + 1];
    VBuf<T>& vc = P<T>::vb(lc);
    restrict_residual<T>(c, lv.g, lv.mask, lc.mask, oth, vc.f);
    vcycle<T>(h, l + 1, vc.f, vc.a, vc.b, nullptr);
    prolong_add<T>(c, lv.g, lv.mask, lc.mask, vc.a, cur);
    int np = 0;
    for (int s = 0; s < post; ++s) {
        np = op_apply<T>(h, ST_JACOBI, l, cur, f, oth, (s == post - 1) ? dot : nullptr);
        T* t = cur; cur = oth; oth = t;
    }
    if (post == 0 && dot) {
        dot_partials<T, T>(c, n, f, cur, dot);
        np = kRedBlocks;
    }
    return dot ? np : 0;
}
template int vcycle<double>(topo_grid*, int, const double*, double*, double*, double*);
template int vcycle<float>(topo_grid*, int, const float*, float*, float*, double*);

// operator launch with BF16 iterates; level-0 launches are recorded for
// topo_profile_read (precision slot 2)
static int op_apply_bf16(topo_grid* h, int mode, int l, const bf16* u, const float* f, bf16* out_h, float* out_f,
                         double* dot) {
    Level& lv = h->lev[l];
    const bool rec = h->prof_on && l == 0 && h->prof_n < kProfMax;
    if (rec) {
        if ((int)h->prof_ev.size() < 2 * (h->prof_n + 1)) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            h->prof_ev.push_back(a);
            h->prof_ev.push_back(b);
        }
        cudaEventRecord(h->prof_ev[2 * h->prof_n], h->stream);
    }
    const int np = stencil_bf16(h->ctx(), mode, lv.op32, *h->mk32, lv.E32, lv.mask, u, f, out_h, out_f,
                                (float)h->prm.omega, dot, lv.Dinv32);
    if (rec) {
        cudaEventRecord(h->prof_ev[2 * h->prof_n + 1], h->stream);
        h->prof_kind.resize(h->prof_n + 1);
        h->prof_kind[h->prof_n] = mode * 8 + 2;
        ++h->prof_n;
    }
    return np;
}

// One level of the BF16 V-cycle (l < L-1).  The iterate lives in the level's
// two BF16 buffers; the residual f - K u is formed in FP32 in v32.a and
// restricted into the next level's FP32 right-hand side.  Returns the BF16
// buffer holding the result, or, with out_f (level 0), writes the last
// post-sweep to out_f in FP32 (and its dot f.out into *dot) and returns null.
static bf16* vcycle_lp(topo_grid* h, int l, const float* f, float* out_f, double* dot, int* np) {
    const Ctx c = h->ctx();
    Level& lv = h->lev[l];
    Level& lc = h->lev[l + 1];
    const int pre = h->prm.pre, post = h->prm.post;
    const long long n = 3 * lv.g.nn;
    bf16* cur = lv.ha;
    bf16* oth = lv.hb;
    float* res = lv.v32.a;
    if (pre > 0) {
        op_apply_bf16(h, ST_JACOBI0, l, nullptr, f, cur, nullptr, nullptr);
        for (int s = 1; s < pre; ++s) {
            op_apply_bf16(h, ST_JACOBI, l, cur, f, oth, nullptr, nullptr);
            bf16* t = cur; cur = oth; oth = t;
        }
        op_apply_bf16(h, ST_RESID, l, cur, f, nullptr, res, nullptr);
    } else {
        cudaMemsetAsync(cur, 0, sizeof(bf16) * n, h->stream);
        cudaMemcpyAsync(res, f, sizeof(float) * n, cudaMemcpyDeviceToDevice, h->stream);
    }
    restrict_residual<float>(c, lv.g, lv.mask, lc.mask, res, lc.v32.f);
    if (l + 1 == h->L - 1) {
        coarse_apply<float>(c, h->cs.n, h->cs.npad, h->cs.W32, h->cs.WT32, lc.v32.f, h->cs.y32, lc.v32.a);
        prolong_add_bf16<float>(c, lv.g, lv.mask, lc.mask, lc.v32.a, cur);
    } else {
        int npc = 0;
        const bf16* e = vcycle_lp(h, l + 1, lc.v32.f, nullptr, nullptr, &npc);
        prolong_add_bf16<bf16>(c, lv.g, lv.mask, lc.mask, e, cur);
    }
    *np = 0;
    for (int s = 0; s < post; ++s) {
        if (out_f && s == post - 1) {
            *np = op_apply_bf16(h, ST_JACOBI, l, cur, f, nullptr, out_f, dot);
            return nullptr;
        }
        op_apply_bf16(h, ST_JACOBI, l, cur, f, oth, nullptr, nullptr);
        bf16* t = cur; cur = oth; oth = t;
    }
    if (out_f) {   // no post-smoothing: widen the iterate
        convert<bf16, float>(c, n, cur, out_f);
        if (dot) {
            dot_partials<float, float>(c, n, f, out_f, dot);
            *np = kRedBlocks;
        }
        return nullptr;
    }
    return cur;
}

int vcycle_bf16(topo_grid* h, int l, const float* f, float* out, double* dot) {
    const Ctx c = h->ctx();
    Level& lv = h->lev[l];
    if (l == h->L - 1) {   // single level: the direct solve
        coarse_apply<float>(c, h->cs.n, h->cs.npad, h->cs.W32, h->cs.WT32, f, h->cs.y32, out);
        if (dot) dot_partials<float, float>(c, 3 * lv.g.nn, f, out, dot);
        return dot ? kRedBlocks : 0;
    }
    int np = 0;
    vcycle_lp(h, l, f, out, dot, &np);
    return dot ? np : 0;
}

// Captures the launches of body() on the handle's stream into gr (the
// launch counter is charged per replay, not for the capture); on any
// failure the handle falls back to direct launches.
// The capture runs on a private non-blocking stream (the handle's stream
// may be the legacy default stream, which cannot be captured); the graph is
// then launched on the handle's stream.
template <typename F>
static void capture_graph(topo_grid* h, PcgGraph& gr, F&& body) {
    cudaGraph_t graph = nullptr;
    const long long l0 = h->launches;
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        h->cap_stream = nullptr;
        gr.failed = true;
        return;
    }
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        gr.failed = true;
        return;
    }
    cudaStream_t own = h->stream;
    h->stream = h->cap_stream;   // every launch of body() goes to the capture
    body();
    h->stream = own;
    const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    gr.launches = h->launches - l0;
    h->launches = l0;
    if (e != cudaSuccess || !graph || cudaGraphInstantiate(&gr.exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        gr.exec = nullptr;
        gr.failed = true;
    }
    if (graph) cudaGraphDestroy(graph);
}

void capture_launches(topo_grid* h, PcgGraph& gr, const std::function<void()>& body) { capture_graph(h, gr, body); }

// copies the scalars to the pinned mirror and waits for them
static void fetch_scalars(topo_grid* h) {
    cudaMemcpyAsync(h->host_sc, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream);
    cudaStreamSynchronize(h->stream);
}

// PCG on level 0 in precision T.  r holds the right-hand side residual on
// entry (r = b - K x already formed, ||r||^2 in *rr0) and is updated in place.
// Returns the number of iterations; *status gets OK / MAXITER / BREAKDOWN.
template <typename T>
static int pcg_core(topo_grid* h, T* x, T* r, T* z, T* p, T* q, double rr0, double target_rr, int max_it,
                    int* status, double* rr_out) {
    const Ctx c = h->ctx();
    Level& l0 = h->lev[0];
    const long long n = 3 * l0.g.nn;
    VBuf<T>& vb = P<T>::vb(l0);
    double rr = rr0;
    *status = TOPO_OK;
    if (rr <= target_rr || max_it <= 0) {
        if (rr > target_rr) *status = TOPO_MAXITER;
        *rr_out = rr;
        return 0;
    }
    cudaMemsetAsync(&h->sc->aux, 0, sizeof(double), h->stream);
    // preconditioner: V-cycle in T, or with BF16 iterates (FP32 solves of
    // TOPO_MIXED_BF16 handles)
    auto precond = [&]() -> int {
        if constexpr (std::is_same<T, float>::value) {
            if (h->prm.precision == TOPO_MIXED_BF16)
                return vcycle_bf16(h, 0, reinterpret_cast<const float*>(r), reinterpret_cast<float*>(z),
                                   h->partials);
        }
        return vcycle<T>(h, 0, r, z, vb.a, h->partials);
    };
    const bool flexible = std::is_same<T, float>::value && h->prm.precision == TOPO_MIXED_BF16;
    // The direction update p = z + beta p is fused into the K.p kernel
    // (ST_APPLY_P), which reads the old direction from one buffer and writes
    // the new one to the other; the tensor-core operator has no fused form.
    const bool fused = !(std::is_same<T, float>::value && h->prm.tensor_cores != 0);
    // With the fused K.p, iteration k writes its direction to ring slot
    // k % R and reads the previous one from the slot before; x += alpha p
    // waits until the ring is full (or the solve ends) and is then applied
    // for all its slots in one pass (cg_flush_x), in the order of the steps.
    constexpr int R = kDirRing;
    T* ring[R];
    ring[0] = p;
    ring[1] = vb.b;   // vb.b of level 0 is free during the solve
    for (int j = 2; j < R; ++j) ring[j] = P<T>::dring(h)[j - 2];
    int np = precond();
    cg_beta(c, h->partials, np, h->sc);   // sets rz (beta unused on the first step)
    if (!fused) cudaMemcpyAsync(p, z, sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream);
    // step k: K p, alpha, r -= alpha q, r.r, and x += alpha p (per step, or
    // per full ring when fused) on the stream current in h; first step (k = 0):
    // p = z, else p = z + beta p_old
    auto step_a = [&](int k) {
        const Ctx cc = h->ctx();
        if (fused) {
            const int s = k % R;
            // (the first step reads z in place of p_old: beta is absent, nothing is added)
            const int npa = op_apply<T>(h, ST_APPLY_P, 0, z, k == 0 ? z : ring[(s + R - 1) % R], q, h->partials,
                                        ring[s], k == 0 ? nullptr : &h->sc->beta);
            cg_alpha(cc, h->partials, npa, h->sc, h->alpha_hist + s);
            cg_update_r<T>(cc, n, h->sc, q, r, h->partials);
            if (s == R - 1) cg_flush_x<T>(cc, n, ring, h->alpha_hist, R, x);
        } else {
            const int npa = op_apply<T>(h, ST_APPLY, 0, p, nullptr, q, h->partials);
            cg_alpha(cc, h->partials, npa, h->sc);
            cg_update_xr<T>(cc, n, h->sc, p, q, x, r, h->partials);
        }
        reduce_to(cc, h->partials, kRedBlocks, &h->sc->rr);
    };
    // z = M^-1 r, beta, p = z + beta p, then K p ... (step k)
    auto step_ba = [&](int k) {
        const Ctx cc = h->ctx();
        const int npb = precond();
        cg_beta(cc, h->partials, npb, h->sc);
        if (flexible) {   // BF16 rounding makes M^-1 vary slightly between applications
            dot_partials<T, T>(cc, n, z, q, h->partials);
            cg_beta_flexible(cc, h->partials, kRedBlocks, h->sc);
        }
        if (!fused) cg_update_p<T>(cc, n, h->sc, z, p);
        step_a(k);
    };
    // Every iteration after the first is one of R fixed sequences of
    // launches (one per ring slot; all scalars live on the device), each
    // captured once into a CUDA graph and replayed; the host only reads r.r
    // between replays.  Not while launches are timed one by one.
    PcgGraph* grs = P<T>::graph(h);
    bool use_graph = h->prm.graphs != 0 && !h->prof_on;
    for (int j = 0; j < R; ++j) use_graph = use_graph && !grs[j].failed;
    step_a(0);
    int it = 1;   // steps taken
    // The host reads r.r (one stream synchronisation) after a batch of
    // iterations: one at a time for the first two, then as many as the
    // observed contraction rate predicts are still needed (at most 8, and
    // rounded down so that the batch does not step past the target while
    // the rate holds).  topo_params.cg_check = 1 reads after every iteration.
    // Iterations beyond convergence or after a breakdown are harmless: CG
    // with a fixed preconditioner keeps reducing the residual, and a step
    // with non-positive curvature is not taken (alpha = 0).
    double rr_prev = rr0;
    int last_batch = 1;
    for (;;) {
        fetch_scalars(h);
        rr = h->host_sc[3];
        if (h->host_sc[7] != 0.0 || !std::isfinite(rr)) {
            *status = TOPO_BREAKDOWN;
            break;
        }
        if (rr <= target_rr || it >= max_it) break;
        int batch = 1;
        if (h->prm.cg_check == 0 && it >= 2 && rr < rr_prev) {
            const double rate = std::pow(rr / rr_prev, 1.0 / last_batch);
            if (rate < 1.0 && rate > 0.0) {
                const double need = std::log(target_rr / rr) / std::log(rate);
                batch = (int)std::fmin(8.0, std::fmax(1.0, std::floor(need)));
            }
        }
        batch = std::min(batch, max_it - it);
        rr_prev = rr;
        last_batch = batch;
        for (int b = 0; b < batch; ++b) {
            const int k = it;
            PcgGraph& gr = grs[fused ? k % R : 0];
            if (use_graph && !gr.exec && k >= 2) capture_graph(h, gr, [&]() { step_ba(k); });
            if (use_graph && gr.exec) {
                cudaGraphLaunch(gr.exec, h->stream);
                h->launches += gr.launches;
                ++h->stats.graph_replays;
            } else {
                step_ba(k);
            }
            ++it;
        }
    }
    // the x updates of the steps since the last full ring (the last step is it - 1)
    if (fused && (it - 1) % R != R - 1) cg_flush_x<T>(c, n, ring, h->alpha_hist, (it - 1) % R + 1, x);
    if (*status == TOPO_OK && rr > target_rr) *status = TOPO_MAXITER;
    *rr_out = rr;
    return it;
}

// r32 = fl32(f - K x) with the double-FP32 operator kernel (FP64 x, f and
// modulus split into FP32 pairs) and ||r||^2 from the same kernel; with x
// known to be zero, r32 = fl32(f) and ||f||^2.  Level-0 launches are recorded
// for topo_profile_read (precision slot 3).
static double residual_df(topo_grid* h) {
    const Ctx c = h->ctx();
    Level& l0 = h->lev[0];
    const long long n = 3 * l0.g.nn;
    if (h->x_zero) {
        convert<double, float>(c, n, h->f, h->r32);
        return h->host_sc[6];
    }
    const bool rec = h->prof_on && h->prof_n < kProfMax;
    if (rec) {
        if ((int)h->prof_ev.size() < 2 * (h->prof_n + 1)) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            h->prof_ev.push_back(a);
            h->prof_ev.push_back(b);
        }
        cudaEventRecord(h->prof_ev[2 * h->prof_n], h->stream);
    }
    const int np = stencil_df(c, ST_RESID, l0.op64, *h->mkdf, l0.E64, l0.mask, h->x, h->f, nullptr, h->r32,
                              h->partials);
    if (rec) {
        cudaEventRecord(h->prof_ev[2 * h->prof_n + 1], h->stream);
        h->prof_kind.resize(h->prof_n + 1);
        h->prof_kind[h->prof_n] = ST_RESID * 8 + 3;
        ++h->prof_n;
    }
    reduce_to(c, h->partials, np, &h->sc->rr);
    fetch_scalars(h);
    return h->host_sc[3];
}

// r = f - K x in FP64 and ||r||^2; with x known to be zero, r = f.
static double residual64(topo_grid* h) {
    if (h->x_zero) {
        cudaMemcpyAsync(h->r, h->f, sizeof(double) * 3 * h->lev[0].g.nn, cudaMemcpyDeviceToDevice, h->stream);
        return h->host_sc[6];
    }
    const int np = op_apply<double>(h, ST_RESID, 0, h->x, h->f, h->r, h->partials);
    reduce_to(h->ctx(), h->partials, np, &h->sc->rr);
    fetch_scalars(h);
    return h->host_sc[3];
}

double current_relres(topo_grid* h) {
    const double ff = h->host_sc[6];
    if (!(ff > 0.0)) return 0.0;
    return h->x_zero ? 1.0 : std::sqrt(residual64(h) / ff);
}

int solve_fp64(topo_grid* h, double tol, int max_it, int* iters, double* relres) {
    ensure_dinv64(h);
    const double ff = h->host_sc[6];
    double rr_true = residual64(h);
    int status = TOPO_OK, it = 0, restarts = 0;
    // CG on the recursively updated residual; when it reports convergence the
    // true residual f - K x is recomputed and, if the two have drifted apart,
    // CG restarts from the true residual (at most 4 restarts)
    for (;;) {
        double rr;
        it += pcg_core<double>(h, h->x, h->r, h->z, h->p, h->q, rr_true, tol * tol * ff, max_it - it, &status, &rr);
        h->x_zero = false;
        rr_true = residual64(h);
        if (status != TOPO_OK || rr_true <= tol * tol * ff || restarts >= 4 || it >= max_it) break;
        ++restarts;
    }
    *iters = it;
    *relres = std::sqrt(rr_true / ff);
    h->stats.outer_steps = restarts;
    if (status == TOPO_OK && rr_true > tol * tol * ff) status = TOPO_MAXITER;
    return status;
}

int solve_mixed(topo_grid* h, double tol, int max_it, int* iters, double* relres) {
    const Ctx c = h->ctx();
    const long long n = 3 * h->lev[0].g.nn;
    const double ff = h->host_sc[6];
    // outer residual: double-FP32 kernel straight into the FP32 inner
    // right-hand side (default), or the FP64 kernel into r then rounded
    bool df = h->prm.outer_residual == 0;
    auto outer_residual = [&]() { return df ? residual_df(h) : residual64(h); };
    double rr = outer_residual();
    int total = 0, outer = 0, status = TOPO_OK;
    double best = rr;
    for (;;) {
    while (std::sqrt(rr / ff) > tol) {
        if (outer >= h->prm.max_refine || total >= max_it) {
            status = TOPO_MAXITER;
            break;
        }
        double rr32 = rr;
        if (!df) {
            convert<double, float>(c, n, h->r, h->r32);
            dot_partials<float, float>(c, n, h->r32, h->r32, h->partials);
            reduce_to(c, h->partials, kRedBlocks, &h->sc->rr);
            fetch_scalars(h);
            rr32 = h->host_sc[3];
        }
        zero<float>(c, n, h->d32);
        int st;
        double rr_in;
        // inner reduction: inner_tol, loosened on the last step to what is
        // still missing (with a factor 2 margin) so that it does not overshoot
        const double missing = tol / std::sqrt(rr / ff);
        const double red = std::fmin(0.5, std::fmax(h->prm.inner_tol, 0.5 * missing));
        const double target = red * red * rr32;
        const int it = pcg_core<float>(h, h->d32, h->r32, h->z32, h->p32, h->q32, rr32, target,
                                       max_it - total, &st, &rr_in);
        total += it;
        axpy_f32_into_f64(c, n, h->d32, h->x);
        h->x_zero = false;
        ++outer;
        const double rr_new = outer_residual();
        if (st == TOPO_BREAKDOWN || !std::isfinite(rr_new)) {
            status = TOPO_BREAKDOWN;
            rr = rr_new;
            break;
        }
        if (rr_new > 0.25 * best && std::sqrt(rr_new / ff) > tol) {   // refinement stagnates
            if (df) {
                // below the double-FP32 residual's accuracy: continue with
                // the FP64 residual (FP64 r, rounded into the inner solve)
                df = false;
                rr = residual64(h);
                best = rr;
                continue;
            }
            rr = rr_new;
            status = TOPO_MAXITER;
            break;
        }
        best = std::fmin(best, rr_new);
        rr = rr_new;
    }
    // tolerances within two decades of the double-FP32 residual's accuracy
    // (~1e-12 of the load) are confirmed with the FP64 residual
    if (df && status == TOPO_OK && tol < 1e-9 && !h->x_zero) {
        df = false;
        rr = residual64(h);
        best = rr;
        if (std::sqrt(rr / ff) > tol) continue;
    }
    break;
    }
    *iters = total;
    *relres = std::sqrt(rr / ff);
    h->stats.outer_steps = outer;
    return status;
}

}  // namespace topo
