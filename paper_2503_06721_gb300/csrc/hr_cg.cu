// hr_cg.cu -- conjugate gradient on the normal equations (Sec. 4.1.2) with
// even/odd preconditioning (Sec. 4.3.3), plain FP64 or as FP64 defect
// correction around an inner CG in FP32 / FP16 / BF16, for one system or for
// a batch of independent systems (different lattices, masses, rhs counts).
//
// Per iteration (even/odd system, A = Dhat^dag Dhat):
//   t  = D_oe p                                   hop, store
//   q  = (4+m)^2 p - D_eo t          |q|^2 -> alpha = rr / |q|^2
//   t  = (D^dag)_oe q                             hop, store
//   Ap = (4+m)^2 q - (D^dag)_eo t    fused: x += alpha p, r -= alpha Ap,
//                                    |r|^2 -> beta, convergence flag
//   p  = r + beta p
// Scalars never leave the device.  The inner iterations of every instance
// are one CUDA graph: a WHILE conditional node whose body runs K iterations
// of all instances on parallel branches and then a one-thread check kernel
// that keeps the loop going while any right-hand side is neither converged
// nor at its iteration cap (cudaGraphSetConditional).  The host only steps
// in for the FP64 true residual between inner solves.  Compensated
// (double-double) grid sums carry the reductions (Sec. 4.1.1).
#include <cmath>
#include <cstring>

#include "hr_api.cuh"

namespace hr {

namespace {

constexpr int MAX_INST = 16;
constexpr int BODY_ITERS = 4;

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
    bool keep_t1;  // even/odd A: write D_oe v to t1 and keep it (fused force)
    FieldView t1;
};

struct Vecs {
    FieldView x, r, p, q, t;   // t is an odd half field (even/odd system only)
    int P;                     // operator precision of p, q, t
    int PW;                    // precision of r and x
};

struct Inst {
    Ctx c;
    FieldView vb, vx, r64, q64, q2, t64;
    FieldView r32, x32;        // mixed only
    Vecs v;                    // the vectors the (inner) iterations run on
    hr_cg_result *res;
    std::vector<int> iters;
    bool done;
    bool df_ok;                // float-float true residuals requested (and DF64 links held)
    bool df;                   // the current true residual is formed in float-float
    double pred_rel;           // expected true residual after the running inner solve
    // fused force: the last FP64 true residual of the final x leaves D x (q64)
    // and, for the even/odd system, D_oe x (c.t1) and (D^dag)_oe D x (t64)
    bool fused_ok;
    FieldView fx, fy;          // full fields (x, D_oe x) and (D x, (D^dag)_oe D x)
    // host-mapped pinned mailbox for the small host round trips, moved by
    // kernels (never by the copy engines, which the caller may keep busy):
    // mb is the host address, mbd the device address of the same bytes
    char *mb, *mbd;
};

// mailbox layout (bytes) for up to MAX_MB_RHS right-hand sides
constexpr int MAX_MB_RHS = 1024;
constexpr size_t MB_RED = 0;                                                  // [nrhs][2] double
constexpr size_t MB_SV = MB_RED + 16 * MAX_MB_RHS;                            // [2 nrhs] double
constexpr size_t MB_STATE = MB_SV + 16 * MAX_MB_RHS;                          // [nrhs] CgState
constexpr size_t MB_BODIES = MB_STATE + sizeof(CgState) * MAX_MB_RHS;         // unsigned
constexpr size_t MB_BYTES = MB_BODIES + 64;
// the inner graph's loop-body counter sits in the first instance's reduction
// tickets ([8 nrhs] of them), past the ones the kernels use ([0, nrhs))
constexpr int BODIES_SLOT = 4;

hr_status apply_A(const Ctx &c, int P, const FieldView &v, const FieldView &out, const FieldView &q,
                  const FieldView &t)
{
    hr_status st;
    const int D = c.D;
    if (c.sys == HR_EO_PRECOND) {
        const FieldView &t1 = c.keep_t1 && P == HR_F64 ? c.t1 : t;
        st = hop(c.g, P, 1, 0, v, t1, nullptr, -0.5, 0.0, c.nrhs, c.s, EPI_STORE, &c.sc_ns);
        if (st == HR_OK) st = hop(c.g, P, 0, 0, t1, q, &v, 0.5, c.m4 * c.m4, c.nrhs, c.s, EPI_STORE, &c.sc_ns);
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

// r = b - A x (FP64) with |r|^2, |b|^2 into red[2 rhs], state initialised with tol.
// With in.df, A x is computed in float-float: x is split into (hi, lo) pairs in
// r64 (a float-float complex takes 16 bytes, like an FP64 one, so the FP64
// buffers serve), A is applied with the DF64 links, and the product is
// rounded back to FP64 in place before the residual is formed in FP64.
hr_status true_residual(const Inst &in, double tol, int cap, bool x_zero)
{
    const Ctx &c = in.c;
    hr_status st = HR_OK;
    if (x_zero) {
        // A 0 = 0: the residual is b itself
    } else if (in.df) {
        BlasParams cv;
        memset(&cv, 0, sizeof cv);
        cv.nsites = c.ns;
        cv.nrhs = c.nrhs;
        cv.s = 1.0;
        cv.a = in.r64;
        cv.b = in.vx;
        st = blas_convert(c.D, HR_DF64, HR_F64, cv, c.s);
        if (st == HR_OK) st = apply_A(c, HR_DF64, in.r64, in.q2, in.q64, in.t64);
        cv.a = in.q2;
        cv.b = in.q2;
        if (st == HR_OK) st = blas_convert(c.D, HR_F64, HR_DF64, cv, c.s);
    } else {
        st = apply_A(c, HR_F64, in.vx, in.q2, in.q64, in.t64);
    }
    if (st != HR_OK) return st;
    BlasParams bp;
    memset(&bp, 0, sizeof bp);
    bp.nsites = c.ns;
    bp.nrhs = c.nrhs;
    bp.a = in.r64;
    bp.b = in.vb;
    if (!x_zero) bp.c = in.q2;
    bp.partials = c.sc.partials;
    bp.counters = c.sc.counters;
    bp.red_out = c.sc.red;
    bp.state = c.sc.state;
    bp.tol2 = tol * tol;
    bp.cap = cap;
    return blas_residual_init(c.D, bp, c.s);
}

// |r| / |b| from the squared norms; NaN whenever either is not finite, and
// 0 for b = 0 (then x = 0 is exact)
double rel_residual(double rr, double b2)
{
    if (!std::isfinite(rr) || !std::isfinite(b2)) return NAN;
    return b2 > 0 ? std::sqrt(rr / b2) : 0.0;
}

// ------------------------------ the inner graph -----------------------------

struct CheckArgs {
    const CgState *st[MAX_INST];
    int nrhs[MAX_INST];
    int n;
    unsigned *bodies;   // number of loop bodies run (statistics)
};

__global__ void k_loop_check(cudaGraphConditionalHandle h, const CheckArgs a)
{
    if (threadIdx.x != 0) return;
    bool any = false;
    for (int i = 0; i < a.n; i++)
        for (int k = 0; k < a.nrhs[i]; k++) any |= !cg_idle(a.st[i][k]);
    *a.bodies += 1;
    cudaGraphSetConditional(h, any ? 1u : 0u);
}

cudaStream_t branch_stream(int i)
{
    static std::vector<cudaStream_t> pool;
    while ((int)pool.size() <= i) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        pool.push_back(s);
    }
    return pool[i];
}

struct InnerGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned *bodies = nullptr;   // device counter (in the first instance's scratch)
    unsigned *bodies_host = nullptr, *bodies_dev = nullptr;
    long long per_body = 0;       // kernels in one loop body
    ~InnerGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }

    hr_status build(std::vector<Inst> &ins)
    {
        // nothing here allocates or frees device memory: either would
        // synchronise the whole device, including the caller's other streams
        bodies = ins[0].c.sc.counters + BODIES_SLOT * ins[0].c.nrhs;
        bodies_host = reinterpret_cast<unsigned *>(ins[0].mb + MB_BODIES);
        bodies_dev = reinterpret_cast<unsigned *>(ins[0].mbd + MB_BODIES);
        HR_CUDA_CHECK(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle h;
        HR_CUDA_CHECK(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        HR_CUDA_CHECK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        const int n = (int)ins.size();
        cudaStream_t cap = branch_stream(0);
        if (!cap) { set_error("cudaStreamCreate failed"); return HR_ERR_CUDA; }
        std::vector<cudaStream_t> br(n);
        for (int i = 0; i < n; i++) {
            br[i] = branch_stream(i + 1);
            if (!br[i]) { set_error("cudaStreamCreate failed"); return HR_ERR_CUDA; }
        }
        std::vector<cudaEvent_t> ev(n + 1);
        for (auto &e : ev) HR_CUDA_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        HR_CUDA_CHECK(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        const long long before = launch_counter();
        hr_status st = HR_OK;
        cudaError_t e = cudaEventRecord(ev[n], cap);
        for (int i = 0; i < n && e == cudaSuccess; i++) e = cudaStreamWaitEvent(br[i], ev[n], 0);
        if (e != cudaSuccess) st = cuda_fail(e, "graph fork");
        for (int k = 0; k < BODY_ITERS && st == HR_OK; k++)
            for (int i = 0; i < n && st == HR_OK; i++) {
                Ctx c = ins[i].c;
                c.s = br[i];
                st = cg_iteration(c, ins[i].v);
            }
        for (int i = 0; i < n && st == HR_OK; i++) {
            e = cudaEventRecord(ev[i], br[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev[i], 0);
            if (e != cudaSuccess) st = cuda_fail(e, "graph join");
        }
        if (st == HR_OK) {
            CheckArgs a;
            memset(&a, 0, sizeof a);
            a.n = n;
            for (int i = 0; i < n; i++) {
                a.st[i] = ins[i].c.sc.state;
                a.nrhs[i] = ins[i].c.nrhs;
            }
            a.bodies = bodies;
            k_loop_check<<<1, 32, 0, cap>>>(h, a);
            count_launch();
            e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_fail(e, "k_loop_check");
        }
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(cap, &out);
        // captured launches are counted when the graph runs, not here
        per_body = launch_counter() - before;
        count_launch(-per_body);
        for (auto &x : ev) cudaEventDestroy(x);
        if (st != HR_OK) return st;
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        HR_CUDA_CHECK(cudaGraphInstantiate(&exec, graph, 0));
        return HR_OK;
    }

    hr_status run(cudaStream_t s)
    {
        hr_status st = kernel_zero(bodies, sizeof(unsigned), s);
        if (st != HR_OK) return st;
        HR_CUDA_CHECK(cudaGraphLaunch(exec, s));
        // the loop-body count travels to the host with the states; the slot
        // is a reduction ticket of other launches, so it goes back to zero
        st = kernel_copy(bodies_dev, bodies, sizeof(unsigned), s);
        return st == HR_OK ? kernel_zero(bodies, sizeof(unsigned), s) : st;
    }
    // after the stream has synchronised: count the kernels the loop ran
    hr_status account()
    {
        count_launch((long long)*bodies_host * per_body);
        return HR_OK;
    }
};

// solver states -> the instance's mailbox (read on the host after a sync)
hr_status read_states(const Inst &in)
{
    return kernel_copy(in.mbd + MB_STATE, in.c.sc.state, sizeof(CgState) * in.c.nrhs, in.c.s);
}
void take_states(const Inst &in, std::vector<CgState> &out)
{
    out.resize(in.c.nrhs);
    memcpy(out.data(), in.mb + MB_STATE, sizeof(CgState) * in.c.nrhs);
}

// carve the instance's vectors out of its handle's workspace
hr_status prepare(Inst &in, const hr_gauge *g, hr_parity sys, const void *b, void *x, int nrhs, int Pin,
                  int Pres, hr_cg_result *res, cudaStream_t s, bool force_out = false)
{
    Ctx &c = in.c;
    c.g = g;
    c.sys = sys;
    c.nrhs = nrhs;
    c.s = s;
    c.vh = g->geom.vh;
    c.ns = sys == HR_FULL ? 2 * c.vh : c.vh;
    c.D = g->D;
    c.m4 = 4.0 + g->lat.m0;
    const int D = c.D;
    const bool mixed = Pin != HR_F64;
    const size_t f64 = field_rhs_bytes(c.ns, D, HR_F64) * nrhs;
    const size_t t64 = field_rhs_bytes(c.vh, D, HR_F64) * nrhs;
    const size_t full64 = field_rhs_bytes(2 * c.vh, D, HR_F64) * nrhs;
    size_t need = 4 * f64 + t64 + 8192;
    if (force_out && sys == HR_EO_PRECOND) need += 2 * full64 + 512;
    size_t f32 = 0, fP = 0, tP = 0;
    if (mixed) {
        f32 = field_rhs_bytes(c.ns, D, HR_F32) * nrhs;
        fP = field_rhs_bytes(c.ns, D, Pin) * nrhs;
        tP = field_rhs_bytes(c.vh, D, Pin) * nrhs;
        need += 2 * f32 + 2 * fP + tP + 4096;
    }
    hr_status st = ws_reserve(g, need, s);
    if (st != HR_OK) return st;
    st = scratch_reserve(g, nrhs, s, &c.sc);
    if (st != HR_OK) return st;
    if (nrhs > MAX_MB_RHS) {
        set_error("CG: at most %d right-hand sides per instance", MAX_MB_RHS);
        return HR_ERR_INVALID;
    }
    st = pinned_reserve(g, MB_BYTES, s, &in.mb, &in.mbd);
    if (st != HR_OK) return st;
    c.sc_ns = c.sc;
    c.sc_ns.state = nullptr;
    char *p = g->ws;
    auto take = [&](size_t bytes) { char *q = p; p += align_up(bytes, 256); return q; };
    in.vb = make_view(const_cast<void *>(b), c.ns, D, HR_F64);
    in.vx = make_view(x, c.ns, D, HR_F64);
    c.keep_t1 = false;
    in.fused_ok = false;
    in.r64 = make_view(take(f64), c.ns, D, HR_F64);
    if (force_out && sys == HR_EO_PRECOND) {
        // q64 | t64 form the full field (D x, (D^dag)_oe D x); D_oe x goes
        // to the odd half of a full field whose even half receives x
        in.fx = make_view(take(full64), 2 * c.vh, D, HR_F64);
        in.fy = make_view(take(full64), 2 * c.vh, D, HR_F64);
        in.q64 = half_view(in.fy, 0, c.vh, D, HR_F64);
        in.t64 = half_view(in.fy, 1, c.vh, D, HR_F64);
        c.keep_t1 = true;
        c.t1 = half_view(in.fx, 1, c.vh, D, HR_F64);
    } else {
        in.q64 = make_view(take(f64), c.ns, D, HR_F64);
        in.t64 = make_view(take(t64), c.vh, D, HR_F64);
    }
    in.q2 = make_view(take(f64), c.ns, D, HR_F64);
    FieldView p64 = make_view(take(f64), c.ns, D, HR_F64);
    if (mixed) {
        in.r32 = make_view(take(f32), c.ns, D, HR_F32);
        in.x32 = make_view(take(f32), c.ns, D, HR_F32);
        FieldView pP = make_view(take(fP), c.ns, D, Pin);
        FieldView qP = make_view(take(fP), c.ns, D, Pin);
        FieldView tPv = make_view(take(tP), c.vh, D, Pin);
        in.v = Vecs{in.x32, in.r32, pP, qP, tPv, Pin, HR_F32};
    } else {
        in.v = Vecs{in.vx, in.r64, p64, in.q64, in.t64, HR_F64, HR_F64};
    }
    in.res = res;
    in.iters.assign(nrhs, 0);
    in.done = false;
    in.df_ok = mixed && Pres == HR_DF64;
    in.df = false;
    in.pred_rel = 1.0;
    for (int k = 0; k < nrhs; k++) {
        res[k].iters = 0;
        res[k].outer_iters = 0;
        res[k].true_rel_residual = NAN;
        res[k].status = HR_ERR_NOT_CONVERGED;
    }
    return HR_OK;
}

}  // namespace

// the outer loop shared by plain and mixed CG, single and batched
hr_status solve_all(std::vector<Inst> &ins, const hr_cg_params *prm, cudaStream_t s)
{
    const bool mixed = prm->inner != HR_F64;
    const double tol = prm->tol_rel;
    for (auto &in : ins)
        if (!prm->use_initial_guess)
            if (hr_status zs = kernel_zero(in.vx.data, in.vx.rhs_stride * in.c.nrhs, s); zs != HR_OK) return zs;
    // pick the hopping-kernel variants of the inner precision before the
    // iterations are captured into a graph
    for (auto &in : ins) {
        hr_gauge *g = const_cast<hr_gauge *>(in.c.g);
        const int P = in.v.P;
        const int rb = rebuild_for(g, P) ? 1 : 0;
        const bool untuned = (g->mode == HR_LINKS_AUTO && g->auto_mode[P] < 0) ||
                             (hop_variants_of(g, P) != 0x1u && g->tuned[P][rb][EPI_CG_UPDATE][in.c.nrhs > 1 ? 1 : 0] < 0);
        if (g->autotune && g->force_variant < 0 && untuned) {
            hr_status ts = tune_hops(g, P, in.c.nrhs, s);
            if (ts != HR_OK) return ts;
        }
    }
    InnerGraph ig;
    hr_status st = ig.build(ins);
    if (st != HR_OK) return st;
    int total = 0;
    std::vector<std::vector<double>> red(ins.size());
    std::vector<std::vector<CgState>> stt(ins.size());
    for (int outer = 0; outer < 10000; outer++) {
        const int cap = std::max(1, prm->max_iter - total);
        for (auto &in : ins) {
            if (in.done) continue;
            const bool x_zero = outer == 0 && !prm->use_initial_guess;
            // float-float for the intermediate residuals; FP64 for the one the
            // last inner solve is expected to bring to the tolerance
            in.df = in.df_ok && !(in.pred_rel <= 4.0 * tol);
            st = true_residual(in, tol, cap, x_zero);
            if (st != HR_OK) return st;
            in.fused_ok = !x_zero && !in.df;
        }
        for (size_t i = 0; i < ins.size(); i++) {
            if (ins[i].done) continue;
            st = kernel_copy(ins[i].mbd + MB_RED, ins[i].c.sc.red, sizeof(double) * 2 * ins[i].c.nrhs, s);
            if (st != HR_OK) return st;
        }
        HR_CUDA_CHECK(cudaStreamSynchronize(s));
        for (size_t i = 0; i < ins.size(); i++) {
            if (ins[i].done) continue;
            red[i].resize(2 * ins[i].c.nrhs);
            memcpy(red[i].data(), ins[i].mb + MB_RED, sizeof(double) * 2 * ins[i].c.nrhs);
        }
        // a float-float residual that meets the tolerance is confirmed in FP64
        bool rerun = false;
        for (size_t i = 0; i < ins.size(); i++) {
            Inst &in = ins[i];
            if (in.done || !in.df) continue;
            bool all_ok = true;
            for (int k = 0; k < in.c.nrhs; k++) all_ok &= rel_residual(red[i][2 * k], red[i][2 * k + 1]) <= tol;
            if (!all_ok) continue;
            in.df = false;
            st = true_residual(in, tol, cap, false);
            in.fused_ok = true;
            if (st == HR_OK) st = kernel_copy(in.mbd + MB_RED, in.c.sc.red, sizeof(double) * 2 * in.c.nrhs, s);
            if (st != HR_OK) return st;
            rerun = true;
        }
        if (rerun) {
            HR_CUDA_CHECK(cudaStreamSynchronize(s));
            for (size_t i = 0; i < ins.size(); i++)
                if (!ins[i].done) memcpy(red[i].data(), ins[i].mb + MB_RED, sizeof(double) * 2 * ins[i].c.nrhs);
        }
        bool any_active = false;
        double worst = 0;
        for (size_t i = 0; i < ins.size(); i++) {
            Inst &in = ins[i];
            if (in.done) continue;
            bool all_ok = true, bad = false;
            for (int k = 0; k < in.c.nrhs; k++) {
                const double rel = rel_residual(red[i][2 * k], red[i][2 * k + 1]);
                in.res[k].true_rel_residual = rel;
                in.res[k].outer_iters = mixed ? outer : 0;
                if (!std::isfinite(rel)) bad = true;
                if (!(rel <= tol)) {
                    all_ok = false;
                    if (std::isfinite(rel)) worst = std::max(worst, tol / rel);
                }
            }
            in.done = all_ok || bad || total >= prm->max_iter;
            any_active |= !in.done;
        }
        if (!any_active) break;
        // start the inner (or plain) iterations of every active instance
        const double itol = std::max(prm->inner_tol, 0.5 * worst);
        for (size_t i = 0; i < ins.size(); i++) {
            Inst &in = ins[i];
            if (in.done) continue;
            const Ctx &c = in.c;
            BlasParams bp;
            memset(&bp, 0, sizeof bp);
            bp.nsites = c.ns;
            bp.nrhs = c.nrhs;
            if (!mixed) {
                // p = r; the state already holds |r|^2, |b|^2 and stop2 = tol^2 |b|^2
                bp.a = in.v.p;
                bp.b = in.r64;
                bp.s = 1.0;
                st = blas_convert(c.D, HR_F64, HR_F64, bp, s);
            } else {
                std::vector<double> sv(2 * c.nrhs);
                in.pred_rel = 0.0;
                for (int k = 0; k < c.nrhs; k++) {
                    const double rel_k = in.res[k].true_rel_residual;
                    if (!(rel_k <= tol)) in.pred_rel = std::max(in.pred_rel, rel_k * itol);
                }
                for (int k = 0; k < c.nrhs; k++) {
                    const double rr = red[i][2 * k];
                    const bool ok = in.res[k].true_rel_residual <= tol;
                    sv[k] = (ok || !(rr > 0) || !std::isfinite(rr)) ? 0.0 : 1.0 / std::sqrt(rr);
                    sv[c.nrhs + k] = sv[k] == 0.0 ? 0.0 : std::sqrt(rr);
                }
                // the previous outer step's copy of the mailbox has completed
                // (the stream was synchronised since)
                memcpy(in.mb + MB_SV, sv.data(), sizeof(double) * 2 * c.nrhs);
                st = kernel_copy(c.sc.sv, in.mbd + MB_SV, sizeof(double) * 2 * c.nrhs, s);
                if (st != HR_OK) return st;
                bp.a = in.r32;
                bp.b = in.r64;
                bp.c = in.x32;
                bp.d = in.v.p;
                bp.sv = c.sc.sv;
                bp.partials = c.sc.partials;
                bp.counters = c.sc.counters;
                bp.state = c.sc.state;
                bp.tol2 = itol * itol;
                bp.cap = cap;
                st = blas_inner_init(c.D, in.v.P, bp, s);
            }
            if (st != HR_OK) return st;
        }
        st = ig.run(s);
        if (st != HR_OK) return st;
        int ran = 0;
        for (size_t i = 0; i < ins.size(); i++) {
            st = read_states(ins[i]);
            if (st != HR_OK) return st;
        }
        HR_CUDA_CHECK(cudaStreamSynchronize(s));
        for (size_t i = 0; i < ins.size(); i++) take_states(ins[i], stt[i]);
        st = ig.account();
        if (st != HR_OK) return st;
        for (size_t i = 0; i < ins.size(); i++) {
            Inst &in = ins[i];
            if (in.done) continue;
            for (int k = 0; k < in.c.nrhs; k++) {
                in.iters[k] += stt[i][k].iter;
                ran = std::max(ran, stt[i][k].iter);
            }
            if (mixed) {
                BlasParams bp;
                memset(&bp, 0, sizeof bp);
                bp.nsites = in.c.ns;
                bp.nrhs = in.c.nrhs;
                bp.a = in.vx;
                bp.b = in.x32;
                bp.sv = in.c.sc.sv + in.c.nrhs;
                st = blas_outer_update(in.c.D, bp, s);
                if (st != HR_OK) return st;
            }
        }
        total += ran;
        if (mixed) HR_CUDA_CHECK(cudaStreamSynchronize(s));   // sv is rewritten next round
    }
    hr_status overall = HR_OK;
    for (auto &in : ins)
        for (int k = 0; k < in.c.nrhs; k++) {
            const double rel = in.res[k].true_rel_residual;
            in.res[k].iters = in.iters[k];
            in.res[k].status = !std::isfinite(rel) ? HR_ERR_NONFINITE : (rel <= tol ? HR_OK : HR_ERR_NOT_CONVERGED);
            if (in.res[k].status != HR_OK && overall == HR_OK) overall = in.res[k].status;
        }
    if (overall == HR_ERR_NOT_CONVERGED) set_error("CG stopped above tolerance after %d iterations", total);
    if (overall == HR_ERR_NONFINITE) set_error("CG met a non-finite reduction");
    return overall;
}

static hr_status check_params(const hr_gauge *g, hr_parity sys, const hr_cg_params *params)
{
    if (sys != HR_FULL && sys != HR_EO_PRECOND) {
        set_error("CG: sys must be HR_FULL or HR_EO_PRECOND");
        return HR_ERR_INVALID;
    }
    if (!(params->tol_rel > 0) || params->max_iter < 1) {
        set_error("CG: tol_rel must be > 0 and max_iter >= 1");
        return HR_ERR_INVALID;
    }
    if (!(g->prec_mask & (1u << HR_F64))) {
        set_error("CG: the gauge handle must hold FP64 links");
        return HR_ERR_INVALID;
    }
    if (params->inner < HR_F64 || params->inner > HR_BF16 || !(g->prec_mask & (1u << params->inner))) {
        set_error("CG: inner precision %d not stored in the handle", (int)params->inner);
        return HR_ERR_INVALID;
    }
    if (params->inner != HR_F64 && !(params->inner_tol > 0 && params->inner_tol < 1)) {
        set_error("CG: inner_tol must be in (0, 1)");
        return HR_ERR_INVALID;
    }
    if (params->residual != HR_F64 && params->residual != HR_DF64) {
        set_error("CG: residual must be HR_F64 or HR_DF64");
        return HR_ERR_INVALID;
    }
    if (params->residual == HR_DF64 && params->inner != HR_F64 &&
        (!g->rep[HR_DF64][0] || rebuild_for(g, HR_DF64))) {
        set_error("CG: float-float residuals need stored DF64 links in the handle");
        return HR_ERR_INVALID;
    }
    return HR_OK;
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
    if (b == x) { set_error("hr_cg_solve: b and x must not overlap"); return HR_ERR_INVALID; }
    if (g->clover_mode || large_n(g)) {
        // the fused CG kernels carry the constant diagonal (4+m) and exist for
        // the site-parallel hops; with the site-dependent clover diagonal, or
        // for the large-N pairs (colour-parallel hops), the solve runs on the
        // multi-shift engine with the single shift 0 (the same CG iterates)
        if (params->use_initial_guess || params->residual != HR_F64) {
            set_error("hr_cg_solve with a clover term: start from x = 0 with FP64 residuals");
            return HR_ERR_UNSUPPORTED;
        }
        const double zero = 0.0;
        return hr_cg_solve_multishift(g, sys, b, x, nrhs, &zero, 1, params, res, stream);
    }
    hr_status st = check_params(g, sys, params);
    if (st != HR_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<Inst> ins(1);
    st = prepare(ins[0], g, sys, b, x, nrhs, params->inner, params->residual, res, s);
    if (st != HR_OK) return st;
    return solve_all(ins, params, s);
}

extern "C" hr_status hr_cg_solve_force(const hr_gauge *g, hr_parity sys, const void *b, void *x,
                                       const hr_cg_params *params, hr_cg_result *res, void *Y, double coeff,
                                       void *F, void *stream)
{
    if (!g || !b || !x || !params || !res || !F) {
        set_error("hr_cg_solve_force: NULL argument");
        return HR_ERR_INVALID;
    }
    if (b == x) { set_error("hr_cg_solve_force: b and x must not overlap"); return HR_ERR_INVALID; }
    if (g->clover_mode || large_n(g)) {
        set_error("hr_cg_solve_force: not provided with a clover term or for the colour-parallel pairs (use hr_cg_solve + "
                  "hr_dirac_force for the latter)");
        return HR_ERR_UNSUPPORTED;
    }
    hr_status st = check_params(g, sys, params);
    if (st != HR_OK) return st;
    if (!g->rep[HR_F64][0]) {
        set_error("hr_cg_solve_force needs FP64 stored represented links in the handle");
        return HR_ERR_INVALID;
    }
    if (params->residual == HR_DF64 && !g->rep[HR_DF64][0]) {
        set_error("hr_cg_solve_force: the float-float force needs DF64 stored represented links in the handle");
        return HR_ERR_INVALID;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<Inst> ins(1);
    st = prepare(ins[0], g, sys, b, x, 1, params->inner, params->residual, res, s, true);
    if (st != HR_OK) return st;
    st = solve_all(ins, params, s);
    if (st != HR_OK) return st;
    Inst &in = ins[0];
    const Ctx &c = in.c;
    if (!in.fused_ok) {
        // the last true residual was not an FP64 application to the final x
        st = apply_A(c, HR_F64, in.vx, in.q2, in.q64, in.t64);
        if (st != HR_OK) return st;
    }
    const size_t fb = field_rhs_bytes(c.ns, c.D, HR_F64);
    if (Y && (st = kernel_copy(Y, in.q64.data, fb, s)) != HR_OK) return st;
    // the force in the residual's arithmetic: float-float when the caller
    // chose float-float residuals (the handle then holds DF64 links)
    const int arith = params->residual == HR_DF64 ? HR_DF64 : HR_F64;
    if (sys == HR_FULL) return force_full(g, in.vx, in.q64, coeff, reinterpret_cast<double *>(F), arith, s);
    // even/odd: minus the full-operator force on X' = (x, D_oe x), Y' = (Dhat x, (D^dag)_oe Dhat x)
    if ((st = kernel_copy(in.fx.data, x, fb, s)) != HR_OK) return st;
    return force_full(g, in.fx, in.fy, -coeff, reinterpret_cast<double *>(F), arith, s);
}

extern "C" hr_status hr_cg_solve_batched(int n_inst, const hr_gauge *const *g, hr_parity sys, const void *const *b,
                                         void *const *x, const int *nrhs, const hr_cg_params *params,
                                         hr_cg_result *res, void *stream)
{
    if (n_inst < 1 || n_inst > MAX_INST || !g || !b || !x || !nrhs || !params || !res) {
        set_error("hr_cg_solve_batched: bad arguments (1 <= n_inst <= %d)", MAX_INST);
        return HR_ERR_INVALID;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<Inst> ins(n_inst);
    size_t off = 0;
    for (int i = 0; i < n_inst; i++) {
        if (!g[i] || !b[i] || !x[i] || nrhs[i] < 1 || b[i] == x[i]) {
            set_error("hr_cg_solve_batched: instance %d has a NULL pointer, nrhs < 1 or b == x", i);
            return HR_ERR_INVALID;
        }
        if (g[i]->clover_mode || large_n(g[i])) {
            set_error("hr_cg_solve_batched: instance %d has a clover term or is a colour-parallel pair (use hr_cg_solve)", i);
            return HR_ERR_UNSUPPORTED;
        }
        for (int j = 0; j < i; j++)
            if (g[j] == g[i]) {
                set_error("hr_cg_solve_batched: instances %d and %d share a gauge handle", j, i);
                return HR_ERR_INVALID;
            }
        if (g[i]->lat.N != g[0]->lat.N || g[i]->lat.rep != g[0]->lat.rep) {
            set_error("hr_cg_solve_batched: all instances must share N and the representation");
            return HR_ERR_INVALID;
        }
        hr_status st = check_params(g[i], sys, params);
        if (st != HR_OK) return st;
        st = prepare(ins[i], g[i], sys, b[i], x[i], nrhs[i], params->inner, params->residual, res + off, s);
        if (st != HR_OK) return st;
        off += nrhs[i];
    }
    return solve_all(ins, params, s);
}
