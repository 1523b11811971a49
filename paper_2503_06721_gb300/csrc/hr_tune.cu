// hr_tune.cu -- the hopping-kernel variant autotuner and its C ABI.
//
// The hopping kernel exists as a direct variant (each lane loads its own
// neighbour records) and as shared-memory-staged variants (the warp moves
// its 32 records cooperatively) at two register budgets, with the link
// records staged as well, and for blocks of right-hand sides sharing each
// loaded link.  All compute the same bits.  Which is fastest
// depends on the representation (record sizes, registers), the precision,
// the link mode, the epilogue and the lattice, so the choice is measured: every variant of every epilogue is
// launched on zero-filled scratch fields of the handle's lattice, timed with
// CUDA events on the caller's stream, and the fastest is recorded in the
// handle per (precision, link mode, epilogue, nrhs == 1 / > 1).
#include <climits>
#include <cstring>

#include "hr_api.cuh"

namespace hr {

namespace {

struct DeviceBuffer {
    void *p = nullptr;
    ~DeviceBuffer()
    {
        if (p) cudaFree(p);
    }
};

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

constexpr int TUNE_REPS = 3;

}  // namespace

// time the variants of every epilogue in the current link mode of P; record
// the fastest and return one CG iteration's worth of their times
static hr_status tune_mode(hr_gauge *g, int P, int nrhs, cudaStream_t s, float *iteration_ms);

hr_status tune_hops(hr_gauge *g, int P, int nrhs, cudaStream_t s)
{
    // the 16-bit precisions keep their stored links: rebuilt from 16-bit
    // fundamental entries, U_R carries about twice their rounding error, and
    // the inner solves then took more iterations and an extra FP64 correction
    // although each launch was as fast (SU(3) sextet 32^3x64, F16 inner, to
    // 1e-10: 62 iterations, 4 outer steps, 184 ms against 58, 3, 156 ms)
    const bool half = P == HR_F16 || P == HR_BF16;
    const bool both = g->mode == HR_LINKS_AUTO && g->rep[P][0] && g->fund[P][0] && !half;
    if (!both) {
        if (g->mode == HR_LINKS_AUTO) g->auto_mode[P] = g->rep[P][0] ? HR_LINKS_STORED : HR_LINKS_REBUILD;
        if (hop_variants_of(g, P) == 0x1u) return HR_OK;
        float t;
        return tune_mode(g, P, nrhs, s, &t);
    }
    // AUTO: measure both ways of obtaining U_R and keep the faster for P
    float t_mode[2];
    for (int m = HR_LINKS_STORED; m <= HR_LINKS_REBUILD; m++) {
        g->auto_mode[P] = (signed char)m;
        hr_status st = tune_mode(g, P, nrhs, s, &t_mode[m]);
        if (st != HR_OK) {
            g->auto_mode[P] = -1;
            return st;
        }
    }
    g->auto_mode[P] = (signed char)(t_mode[HR_LINKS_REBUILD] < t_mode[HR_LINKS_STORED] ? HR_LINKS_REBUILD : HR_LINKS_STORED);
    return HR_OK;
}

static hr_status tune_mode(hr_gauge *g, int P, int nrhs, cudaStream_t s, float *iteration_ms)
{
    const unsigned mask = hop_variants_of(g, P);
    const bool rb = rebuild_for(g, P);
    const int D = g->D;
    const long vh = g->geom.vh;
    const int PC = P == HR_F64 ? HR_F64 : HR_F32;   // r and x of a fused CG update
    const size_t fP = align_up(field_rhs_bytes(vh, D, P) * nrhs, 256);
    const size_t fC = align_up(field_rhs_bytes(vh, D, PC) * nrhs, 256);
    // per right-hand side: one partial per block of 128 sites, or per 32-site
    // tile for the multi-RHS variant
    const long ntiles = (vh + HR_TILE - 1) / HR_TILE;
    const size_t bpart = align_up(sizeof(double) * (size_t)nrhs * (ntiles + 1), 256);
    const size_t bcnt = align_up(sizeof(unsigned) * nrhs, 256);
    const size_t bstate = align_up(sizeof(CgState) * nrhs, 256);
    const size_t bred = align_up(sizeof(double) * nrhs, 256);
    const size_t total = 3 * fP + 2 * fC + bpart + bcnt + bstate + bred;

    DeviceBuffer mem;
    cudaError_t e = cudaMalloc(&mem.p, total);
    if (e != cudaSuccess) {
        mem.p = nullptr;
        cudaGetLastError();
        set_error("hr_tune: cannot allocate %zu bytes of scratch", total);
        return HR_ERR_NOMEM;
    }
    HR_CUDA_CHECK(cudaMemsetAsync(mem.p, 0, total, s));
    char *q = static_cast<char *>(mem.p);
    auto take = [&](size_t b) { char *r = q; q += b; return r; };
    FieldView vin = make_view(take(fP), vh, D, P);
    FieldView vout = make_view(take(fP), vh, D, P);
    FieldView vaux = make_view(take(fP), vh, D, P);
    FieldView vr = make_view(take(fC), vh, D, PC);
    FieldView vx = make_view(take(fC), vh, D, PC);
    Scratch sc;
    memset(&sc, 0, sizeof sc);
    sc.partials = reinterpret_cast<double *>(take(bpart));
    sc.counters = reinterpret_cast<unsigned *>(take(bcnt));
    sc.state = reinterpret_cast<CgState *>(take(bstate));
    double *red = reinterpret_cast<double *>(take(bred));
    Scratch sc_ns = sc;
    sc_ns.state = nullptr;
    // a solver state that never converges and never reaches its cap, so that
    // every timed CG-update launch does its full work
    std::vector<CgState> st0(nrhs);
    for (auto &c : st0) {
        memset(&c, 0, sizeof c);
        c.rr = 1.0;
        c.stop2 = -1.0;
        c.cap = INT_MAX;
    }
    HR_CUDA_CHECK(cudaMemcpyAsync(sc.state, st0.data(), sizeof(CgState) * nrhs, cudaMemcpyHostToDevice, s));

    // the launch shapes of a CG iteration on the even/odd system
    auto launch = [&](int epi, int v) -> hr_status {
        switch (epi) {
        case EPI_STORE:
            return hop(g, P, 0, 0, vin, vout, nullptr, -0.5, 0.0, nrhs, s, EPI_STORE, nullptr, FIN_WRITE, nullptr,
                       nullptr, nullptr, nullptr, nullptr, v);
        case EPI_STORE_NORM:
            return hop(g, P, 0, 0, vin, vout, &vaux, 0.5, 1.0, nrhs, s, EPI_STORE_NORM, &sc_ns, FIN_WRITE, nullptr,
                       red, nullptr, nullptr, nullptr, v);
        default:
            return hop(g, P, 0, 1, vin, vin, &vaux, 0.5, 1.0, nrhs, s, EPI_CG_UPDATE, &sc, FIN_CG_BETA, nullptr,
                       nullptr, &vr, &vx, &vaux, v);
        }
    };
    EventPair ev;
    HR_CUDA_CHECK(cudaEventCreate(&ev.a));
    HR_CUDA_CHECK(cudaEventCreate(&ev.b));
    *iteration_ms = 0;
    for (int epi = EPI_STORE; epi <= EPI_CG_UPDATE; epi++) {
        float best = 0;
        int best_v = -1;
        for (int v = 0; v < HOP_NVARIANTS; v++) {
            if (!((mask >> v) & 1u) || !hop_variant_fits(v, nrhs)) continue;
            hr_status st = launch(epi, v);   // warm-up (and first-use setup)
            if (st != HR_OK) return st;
            HR_CUDA_CHECK(cudaEventRecord(ev.a, s));
            for (int k = 0; k < TUNE_REPS; k++) {
                st = launch(epi, v);
                if (st != HR_OK) return st;
            }
            HR_CUDA_CHECK(cudaEventRecord(ev.b, s));
            HR_CUDA_CHECK(cudaEventSynchronize(ev.b));
            float ms = 0;
            HR_CUDA_CHECK(cudaEventElapsedTime(&ms, ev.a, ev.b));
            if (best_v < 0 || ms < best) {
                best = ms;
                best_v = v;
            }
        }
        g->tuned[P][rb ? 1 : 0][epi][nrhs > 1 ? 1 : 0] = (signed char)best_v;
        *iteration_ms += (epi == EPI_STORE ? 2.0f : 1.0f) * best / TUNE_REPS;
    }
    HR_CUDA_CHECK(cudaStreamSynchronize(s));
    return HR_OK;
}

}  // namespace hr

using namespace hr;

extern "C" {

hr_status hr_tune(hr_gauge *g, hr_prec prec, int nrhs, void *stream)
{
    if (!g || nrhs < 1 || prec < HR_F64 || prec > HR_DF64 || !(g->prec_mask & (1u << prec))) {
        set_error("hr_tune: NULL handle, nrhs < 1 or precision not stored in the handle");
        return HR_ERR_INVALID;
    }
    return tune_hops(g, prec, nrhs, reinterpret_cast<cudaStream_t>(stream));
}

hr_status hr_gauge_set_tuning(hr_gauge *g, int autotune, int variant)
{
    if (!g || (autotune != 0 && autotune != 1) || variant < -1 || variant > HR_HOP_MRHS) {
        set_error("hr_gauge_set_tuning: bad arguments");
        return HR_ERR_INVALID;
    }
    g->autotune = autotune;
    g->force_variant = variant;
    return HR_OK;
}

int hr_gauge_hop_variant(const hr_gauge *g, hr_prec prec, int epilogue, int nrhs)
{
    if (!g || prec < HR_F64 || prec > HR_DF64 || epilogue < HR_EPI_STORE || epilogue > HR_EPI_CG_UPDATE || nrhs < 1)
        return -1;
    return hop_variant(g, prec, rebuild_for(g, prec), epilogue, nrhs);
}

}  // extern "C"
