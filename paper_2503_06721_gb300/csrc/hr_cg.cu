// hr_cg.cu -- conjugate gradient on the normal equations (Sec. 4.1.2) with
// even/odd preconditioning (Sec. 4.3.3), plain FP64 or as FP64 defect
// correction around an inner CG in FP32 / FP16 / BF16.
//
// Per iteration (even/odd system, A = Dhat^dag Dhat):
//   t  = D_oe p                                   hop, store
//   q  = (4+m)^2 p - D_eo t          |q|^2 -> alpha = rr / |q|^2
//   t  = (D^dag)_oe q                             hop, store
//   Ap = (4+m)^2 q - (D^dag)_eo t    fused: x += alpha p, r -= alpha Ap,
//                                    |r|^2 -> beta, convergence flag
//   p  = r + beta p
// Scalars never leave the device; the host reads the per-rhs state every few
// iterations to decide when to stop.  Compensated (double-double) grid sums
// carry the reductions (Sec. 4.1.1).
#include <cmath>
#include <cstring>

#include "hr_api.cuh"

namespace hr {

namespace {

struct Ctx {
    const hr_gauge *g;
    hr_parity sys;
    int nrhs;
    cudaStream_t s;
    long vh, ns;   // sites per parity, sites of a system vector
    int D;
    double m4;
    Scratch sc;    // with solver state
    Scratch sc_ns; // same buffers, no state (launches that must not skip)
};

struct Vecs {
    FieldView x, r, p, q, t;   // t is an odd half field (even/odd system only)
    int P;                     // operator precision of p, q, t
    int PW;                    // precision of r and x
};

hr_status apply_A(const Ctx &c, int P, const FieldView &v, const FieldView &out, const FieldView &q,
                  const FieldView &t)
{
    hr_status st;
    const int D = c.D;
    if (c.sys == HR_EO_PRECOND) {
        st = hop(c.g, P, 1, 0, v, t, nullptr, -0.5, 0.0, c.nrhs, c.s, EPI_STORE, &c.sc_ns);
        if (st == HR_OK) st = hop(c.g, P, 0, 0, t, q, &v, 0.5, c.m4 * c.m4, c.nrhs, c.s, EPI_STORE, &c.sc_ns);
        if (st == HR_OK) st = hop(c.g, P, 1, 1, q, t, nullptr, -0.5, 0.0, c.nrhs, c.s, EPI_STORE, &c.sc_ns);
        if (st == HR_OK) st = hop(c.g, P, 0, 1, t, out, &q, 0.5, c.m4 * c.m4, c.nrhs, c.s, EPI_STORE, &c.sc_ns);
        return st;
    }
    for (int dag = 0; dag < 2; dag++) {
        const FieldView &src = dag ? q : v;
        const FieldView &dst = dag ? out : q;
        for (int par = 0; par < 2; par++) {
            FieldView in = half_view(src, 1 - par, c.vh, D, P), dg = half_view(src, par, c.vh, D, P);
            FieldView o = half_view(dst, par, c.vh, D, P);
            st = hop(c.g, P, par, dag, in, o, &dg, -0.5, c.m4, c.nrhs, c.s, EPI_STORE, &c.sc_ns);
            if (st != HR_OK) return st;
        }
    }
    return HR_OK;
}

hr_status cg_iteration(const Ctx &c, const Vecs &v)
{
    hr_status st;
    const int D = c.D, P = v.P;
    if (c.sys == HR_EO_PRECOND) {
        st = hop(c.g, P, 1, 0, v.p, v.t, nullptr, -0.5, 0.0, c.nrhs, c.s, EPI_STORE, &c.sc);
        if (st == HR_OK)
            st = hop(c.g, P, 0, 0, v.t, v.q, &v.p, 0.5, c.m4 * c.m4, c.nrhs, c.s, EPI_STORE_NORM, &c.sc, FIN_CG_ALPHA);
        if (st == HR_OK) st = hop(c.g, P, 1, 1, v.q, v.t, nullptr, -0.5, 0.0, c.nrhs, c.s, EPI_STORE, &c.sc);
        if (st == HR_OK)
            st = hop(c.g, P, 0, 1, v.t, v.q, &v.q, 0.5, c.m4 * c.m4, c.nrhs, c.s, EPI_CG_UPDATE, &c.sc, FIN_CG_BETA,
                     nullptr, nullptr, &v.r, &v.x, &v.p);
        if (st != HR_OK) return st;
    } else {
        // q = D p  (two halves; the |q|^2 of the even half is carried into the odd one)
        for (int par = 0; par < 2; par++) {
            FieldView in = half_view(v.p, 1 - par, c.vh, D, P), dg = half_view(v.p, par, c.vh, D, P);
            FieldView o = half_view(v.q, par, c.vh, D, P);
            st = hop(c.g, P, par, 0, in, o, &dg, -0.5, c.m4, c.nrhs, c.s, EPI_STORE_NORM, &c.sc,
                     par == 0 ? FIN_WRITE : FIN_CG_ALPHA, par == 0 ? nullptr : c.sc.red, par == 0 ? c.sc.red : nullptr);
            if (st != HR_OK) return st;
        }
        // A p = D^dag q, fused into the update of each half
        for (int par = 0; par < 2; par++) {
            FieldView in = half_view(v.q, 1 - par, c.vh, D, P), dg = half_view(v.q, par, c.vh, D, P);
            FieldView rh = half_view(v.r, par, c.vh, D, v.PW), xh = half_view(v.x, par, c.vh, D, v.PW);
            FieldView ph = half_view(v.p, par, c.vh, D, P);
            st = hop(c.g, P, par, 1, in, in, &dg, -0.5, c.m4, c.nrhs, c.s, EPI_CG_UPDATE, &c.sc,
                     par == 0 ? FIN_WRITE : FIN_CG_BETA, par == 0 ? nullptr : c.sc.carry,
                     par == 0 ? c.sc.carry : nullptr, &rh, &xh, &ph);
            if (st != HR_OK) return st;
        }
    }
    BlasParams bp;
    memset(&bp, 0, sizeof bp);
    bp.nsites = c.ns;
    bp.nrhs = c.nrhs;
    bp.a = v.r;
    bp.c = v.p;
    bp.state = c.sc.state;
    return blas_xpay_beta(D, P, bp, c.s);
}

hr_status read_states(const Ctx &c, std::vector<CgState> &out)
{
    hr_gauge *g = const_cast<hr_gauge *>(c.g);
    const size_t need = sizeof(CgState) * c.nrhs + sizeof(double) * 4 * c.nrhs;
    if (g->pinned_bytes < need) {
        if (g->pinned) cudaFreeHost(g->pinned);
        g->pinned = nullptr;
        g->pinned_bytes = 0;
        HR_CUDA_CHECK(cudaMallocHost(&g->pinned, need));
        g->pinned_bytes = need;
    }
    HR_CUDA_CHECK(cudaMemcpyAsync(g->pinned, c.sc.state, sizeof(CgState) * c.nrhs, cudaMemcpyDeviceToHost, c.s));
    HR_CUDA_CHECK(cudaStreamSynchronize(c.s));
    out.resize(c.nrhs);
    memcpy(out.data(), g->pinned, sizeof(CgState) * c.nrhs);
    return HR_OK;
}

hr_status read_red(const Ctx &c, std::vector<double> &out, int n)
{
    out.resize(n);
    HR_CUDA_CHECK(cudaMemcpyAsync(out.data(), c.sc.red, sizeof(double) * n, cudaMemcpyDeviceToHost, c.s));
    HR_CUDA_CHECK(cudaStreamSynchronize(c.s));
    return HR_OK;
}

// r = b - A x (FP64) with |r|^2, |b|^2 into red[2 rhs], state initialised with tol
hr_status true_residual(const Ctx &c, const FieldView &b, const FieldView &x, const FieldView &r,
                        const FieldView &q, const FieldView &q2, const FieldView &t, double tol)
{
    hr_status st = apply_A(c, HR_F64, x, q2, q, t);
    if (st != HR_OK) return st;
    BlasParams bp;
    memset(&bp, 0, sizeof bp);
    bp.nsites = c.ns;
    bp.nrhs = c.nrhs;
    bp.a = r;
    bp.b = b;
    bp.c = q2;
    bp.partials = c.sc.partials;
    bp.counters = c.sc.counters;
    bp.red_out = c.sc.red;
    bp.state = c.sc.state;
    bp.tol2 = tol * tol;
    return blas_residual_init(c.D, bp, c.s);
}

constexpr int CHECK_EVERY = 8;

// |r| / |b| from the squared norms; NaN whenever either is not finite, and
// 0 for b = 0 (then x = 0 is exact)
double rel_residual(double rr, double b2)
{
    if (!std::isfinite(rr) || !std::isfinite(b2)) return NAN;
    return b2 > 0 ? std::sqrt(rr / b2) : 0.0;
}

// run CG iterations until every rhs converged or the budget is used up
hr_status run_iterations(const Ctx &c, const Vecs &v, int budget, std::vector<CgState> &stt, int *done_iters)
{
    int it = 0;
    hr_status st = read_states(c, stt);
    if (st != HR_OK) return st;
    auto all_done = [&]() {
        for (auto &s : stt)
            if (!s.converged) return false;
        return true;
    };
    while (!all_done() && it < budget) {
        int k = std::min(CHECK_EVERY, budget - it);
        for (int j = 0; j < k; j++) {
            st = cg_iteration(c, v);
            if (st != HR_OK) return st;
        }
        it += k;
        st = read_states(c, stt);
        if (st != HR_OK) return st;
    }
    *done_iters = it;
    return HR_OK;
}

}  // namespace

hr_status cg_solve_impl(const hr_gauge *g, hr_parity sys, const void *b, void *x, int nrhs, const hr_cg_params *prm,
                        hr_cg_result *res, cudaStream_t s)
{
    Ctx c;
    c.g = g;
    c.sys = sys;
    c.nrhs = nrhs;
    c.s = s;
    c.vh = g->geom.vh;
    c.ns = sys == HR_FULL ? 2 * c.vh : c.vh;
    c.D = g->D;
    c.m4 = 4.0 + g->lat.m0;
    const int D = c.D;
    const bool mixed = prm->inner != HR_F64;
    const int Pin = prm->inner;

    // field workspace: r64 | q64 | q2_64 | t64 | [p64] | [r32 | x32 | pP | qP | tP];
    // reductions and solver state live in the separate scratch buffer
    const size_t f64 = field_rhs_bytes(c.ns, D, HR_F64) * nrhs;
    const size_t t64 = field_rhs_bytes(c.vh, D, HR_F64) * nrhs;
    size_t need = 3 * f64 + t64 + 4096;
    size_t f32 = 0, fP = 0, tP = 0;
    if (mixed) {
        f32 = field_rhs_bytes(c.ns, D, HR_F32) * nrhs;
        fP = field_rhs_bytes(c.ns, D, Pin) * nrhs;
        tP = field_rhs_bytes(c.vh, D, Pin) * nrhs;
        need += 2 * f32 + 2 * fP + tP + 4096;
    } else {
        need += f64;   // p
    }
    hr_status st = ws_reserve(g, need, s);
    if (st != HR_OK) return st;
    st = scratch_reserve(g, nrhs, s, &c.sc);
    if (st != HR_OK) return st;
    char *p = g->ws;
    c.sc_ns = c.sc;
    c.sc_ns.state = nullptr;
    auto take = [&](size_t bytes) { char *q = p; p += align_up(bytes, 256); return q; };
    FieldView vb = make_view(const_cast<void *>(b), c.ns, D, HR_F64);
    FieldView vx = make_view(x, c.ns, D, HR_F64);
    FieldView r64 = make_view(take(f64), c.ns, D, HR_F64);
    FieldView q64 = make_view(take(f64), c.ns, D, HR_F64);
    FieldView q2 = make_view(take(f64), c.ns, D, HR_F64);
    FieldView t64v = make_view(take(t64), c.vh, D, HR_F64);

    for (int k = 0; k < nrhs; k++) {
        res[k].iters = 0;
        res[k].outer_iters = 0;
        res[k].true_rel_residual = NAN;
        res[k].status = HR_ERR_NOT_CONVERGED;
    }
    const double tol = prm->tol_rel;
    std::vector<CgState> stt;
    std::vector<double> red;
    int total = 0;

    if (!prm->use_initial_guess) HR_CUDA_CHECK(cudaMemsetAsync(x, 0, f64, s));

    if (!mixed) {
        FieldView p64 = make_view(take(f64), c.ns, D, HR_F64);
        Vecs v{vx, r64, p64, q64, t64v, HR_F64, HR_F64};
        std::vector<int> iters(nrhs, 0);
        for (int restart = 0; restart < 100; restart++) {
            st = true_residual(c, vb, vx, r64, q64, q2, t64v, tol);
            if (st != HR_OK) return st;
            // p = r
            BlasParams bp;
            memset(&bp, 0, sizeof bp);
            bp.nsites = c.ns;
            bp.nrhs = nrhs;
            bp.a = p64;
            bp.b = r64;
            bp.s = 1.0;
            st = blas_convert(D, HR_F64, HR_F64, bp, s);
            if (st != HR_OK) return st;
            int done = 0;
            st = run_iterations(c, v, prm->max_iter - total, stt, &done);
            if (st != HR_OK) return st;
            for (int k = 0; k < nrhs; k++) iters[k] += stt[k].iter;
            total += done;
            // verify with the true residual
            st = true_residual(c, vb, vx, r64, q64, q2, t64v, tol);
            if (st != HR_OK) return st;
            st = read_red(c, red, 2 * nrhs);
            if (st != HR_OK) return st;
            bool all_ok = true, any_bad = false;
            for (int k = 0; k < nrhs; k++) {
                double rel = rel_residual(red[2 * k], red[2 * k + 1]);
                res[k].true_rel_residual = rel;
                res[k].iters = iters[k];
                if (!std::isfinite(rel)) any_bad = true;
                if (!(rel <= tol)) all_ok = false;
            }
            if (all_ok || any_bad || total >= prm->max_iter) break;
        }
    } else {
        FieldView r32 = make_view(take(f32), c.ns, D, HR_F32);
        FieldView x32 = make_view(take(f32), c.ns, D, HR_F32);
        FieldView pP = make_view(take(fP), c.ns, D, Pin);
        FieldView qP = make_view(take(fP), c.ns, D, Pin);
        FieldView tPv = make_view(take(tP), c.vh, D, Pin);
        Vecs v{x32, r32, pP, qP, tPv, Pin, HR_F32};
        std::vector<double> sv(2 * nrhs);
        std::vector<int> iters(nrhs, 0);
        int outer = 0;
        for (; outer < 1000; outer++) {
            st = true_residual(c, vb, vx, r64, q64, q2, t64v, tol);
            if (st != HR_OK) return st;
            st = read_red(c, red, 2 * nrhs);
            if (st != HR_OK) return st;
            bool all_ok = true, any_bad = false;
            double worst = 0;
            for (int k = 0; k < nrhs; k++) {
                const double rr = red[2 * k], b2 = red[2 * k + 1];
                const double rel = rel_residual(rr, b2);
                res[k].true_rel_residual = rel;
                res[k].outer_iters = outer;
                if (!std::isfinite(rel)) any_bad = true;
                const bool ok = rel <= tol;
                if (!ok) all_ok = false;
                sv[k] = (ok || !std::isfinite(rel) || rr <= 0) ? 0.0 : 1.0 / std::sqrt(rr);
                sv[nrhs + k] = sv[k] == 0.0 ? 0.0 : std::sqrt(rr);
                if (!ok && std::isfinite(rel)) worst = std::max(worst, tol / rel);
            }
            if (all_ok || any_bad || total >= prm->max_iter) break;
            HR_CUDA_CHECK(cudaMemcpyAsync(c.sc.sv, sv.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, s));
            const double itol = std::max(prm->inner_tol, 0.5 * worst);
            BlasParams bp;
            memset(&bp, 0, sizeof bp);
            bp.nsites = c.ns;
            bp.nrhs = nrhs;
            bp.a = r32;
            bp.b = r64;
            bp.c = x32;
            bp.d = pP;
            bp.sv = c.sc.sv;
            bp.partials = c.sc.partials;
            bp.counters = c.sc.counters;
            bp.state = c.sc.state;
            bp.tol2 = itol * itol;
            st = blas_inner_init(D, Pin, bp, s);
            if (st != HR_OK) return st;
            int done = 0;
            st = run_iterations(c, v, prm->max_iter - total, stt, &done);
            if (st != HR_OK) return st;
            for (int k = 0; k < nrhs; k++) iters[k] += stt[k].iter;
            total += done;
            memset(&bp, 0, sizeof bp);
            bp.nsites = c.ns;
            bp.nrhs = nrhs;
            bp.a = vx;
            bp.b = x32;
            bp.sv = c.sc.sv + nrhs;
            st = blas_outer_update(D, bp, s);
            if (st != HR_OK) return st;
            HR_CUDA_CHECK(cudaStreamSynchronize(s));   // sv is rewritten next round
        }
        for (int k = 0; k < nrhs; k++) {
            res[k].iters = iters[k];
            res[k].outer_iters = outer;
        }
    }
    hr_status overall = HR_OK;
    for (int k = 0; k < nrhs; k++) {
        const double rel = res[k].true_rel_residual;
        res[k].status = !std::isfinite(rel) ? HR_ERR_NONFINITE : (rel <= tol ? HR_OK : HR_ERR_NOT_CONVERGED);
        if (res[k].status != HR_OK && overall == HR_OK) overall = res[k].status;
    }
    if (overall == HR_ERR_NOT_CONVERGED) set_error("CG stopped above tolerance after %d iterations", total);
    if (overall == HR_ERR_NONFINITE) set_error("CG met a non-finite reduction");
    return overall;
}

}  // namespace hr

using namespace hr;

extern "C" hr_status hr_cg_solve(const hr_gauge *g, hr_parity sys, const void *b, void *x, int nrhs,
                                 const hr_cg_params *params, hr_cg_result *res, void *stream)
{
    if (!g || !b || !x || !params || !res || nrhs < 1) {
        set_error("hr_cg_solve: NULL argument or nrhs < 1");
        return HR_ERR_INVALID;
    }
    if (sys != HR_FULL && sys != HR_EO_PRECOND) {
        set_error("hr_cg_solve: sys must be HR_FULL or HR_EO_PRECOND");
        return HR_ERR_INVALID;
    }
    if (b == x) { set_error("hr_cg_solve: b and x must not overlap"); return HR_ERR_INVALID; }
    if (!(params->tol_rel > 0) || params->max_iter < 1) {
        set_error("hr_cg_solve: tol_rel must be > 0 and max_iter >= 1");
        return HR_ERR_INVALID;
    }
    if (!(g->prec_mask & (1u << HR_F64))) {
        set_error("hr_cg_solve: the gauge handle must hold FP64 links");
        return HR_ERR_INVALID;
    }
    if (params->inner < HR_F64 || params->inner > HR_BF16 || !(g->prec_mask & (1u << params->inner))) {
        set_error("hr_cg_solve: inner precision %d not stored in the handle", (int)params->inner);
        return HR_ERR_INVALID;
    }
    if (params->inner != HR_F64 && !(params->inner_tol > 0 && params->inner_tol < 1)) {
        set_error("hr_cg_solve: inner_tol must be in (0, 1)");
        return HR_ERR_INVALID;
    }
    return cg_solve_impl(g, sys, b, x, nrhs, params, res, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" hr_status hr_cg_solve_batched(int n_inst, const hr_gauge *const *g, hr_parity sys, const void *const *b,
                                         void *const *x, const int *nrhs, const hr_cg_params *params,
                                         hr_cg_result *res, void *stream)
{
    set_error("hr_cg_solve_batched: not built yet");
    return HR_ERR_UNSUPPORTED;
}
