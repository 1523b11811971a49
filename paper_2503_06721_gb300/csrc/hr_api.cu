// hr_api.cu -- the C ABI of include/hr.h: argument checking, the gauge
// handle, precision/representation dispatch, operator application and the
// force entry point.  The solver lives in hr_cg.cu.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "hr_api.cuh"

namespace hr {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

hr_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HR_ERR_NOMEM : HR_ERR_CUDA;
}

void count_launch(long long n) { g_launches += n; }
long long launch_counter() { return g_launches.load(); }

// --------------------------- dispatch --------------------------------------
#define HR_PAIRS(X) X(2, HR_FUND) X(2, HR_ADJ) X(2, HR_SYM) X(3, HR_FUND) X(3, HR_ADJ) X(3, HR_SYM) \
    X(3, HR_ASYM) X(4, HR_FUND) X(4, HR_ASYM) X(4, HR_ASYM_REAL)

#define HR_DECL(N_, R_)                                                                                    \
    extern template hr_status launch_hop<N_, R_, HR_F64>(const HopParams &, bool, int, int, cudaStream_t);     \
    extern template hr_status launch_hop<N_, R_, HR_F32>(const HopParams &, bool, int, int, cudaStream_t);     \
    extern template hr_status launch_hop<N_, R_, HR_F16>(const HopParams &, bool, int, int, cudaStream_t);     \
    extern template hr_status launch_hop<N_, R_, HR_BF16>(const HopParams &, bool, int, int, cudaStream_t);    \
    extern template hr_status launch_hop<N_, R_, HR_DF64>(const HopParams &, bool, int, int, cudaStream_t);    \
    extern template hr_status represent_launch<N_, R_>(const hr_gauge &, const double2 *, cudaStream_t); \
    extern template hr_status force_launch<N_, R_>(const ForceParams &, cudaStream_t);
HR_PAIRS(HR_DECL)

// large pairs (the fundamental of large N, and the SU(4) adjoint and
// symmetric representations with D_R = 15 and 10): represent and force as
// above, the hop by the colour-parallel kernel (FP64 and FP32, stored links)
#define HR_LARGE_PAIRS(X) X(5, HR_FUND) X(6, HR_FUND) X(8, HR_FUND) X(4, HR_ADJ) X(4, HR_SYM)
#define HR_DECL_LARGE(N_, R_)                                                                          \
    extern template hr_status launch_colour<N_, R_, HR_F64>(const HopParams &, int, cudaStream_t);     \
    extern template hr_status launch_colour<N_, R_, HR_F32>(const HopParams &, int, cudaStream_t);     \
    extern template hr_status represent_launch<N_, R_>(const hr_gauge &, const double2 *, cudaStream_t); \
    extern template hr_status force_launch<N_, R_>(const ForceParams &, cudaStream_t);
HR_LARGE_PAIRS(HR_DECL_LARGE)

bool pair_supported(int N, int rep)
{
#define HR_SUP(N_, R_) if (N == N_ && rep == R_) return true;
    HR_PAIRS(HR_SUP)
    HR_LARGE_PAIRS(HR_SUP)
#undef HR_SUP
    return false;
}

hr_status hop_dispatch(int N, int rep, int P, const HopParams &prm, bool rebuild, int epi, int variant,
                       cudaStream_t stream)
{
#define HR_HOP(N_, R_)                                                                             \
    if (N == N_ && rep == R_) {                                                                    \
        switch (P) {                                                                               \
        case HR_F64: return launch_hop<N_, R_, HR_F64>(prm, rebuild, epi, variant, stream);        \
        case HR_F32: return launch_hop<N_, R_, HR_F32>(prm, rebuild, epi, variant, stream);        \
        case HR_F16: return launch_hop<N_, R_, HR_F16>(prm, rebuild, epi, variant, stream);        \
        case HR_BF16: return launch_hop<N_, R_, HR_BF16>(prm, rebuild, epi, variant, stream);      \
        case HR_DF64: return launch_hop<N_, R_, HR_DF64>(prm, rebuild, epi, variant, stream);      \
        }                                                                                          \
    }
    HR_PAIRS(HR_HOP)
#undef HR_HOP
#define HR_HOP_LARGE(N_, R_)                                                                          \
    if (N == N_ && rep == R_) {                                                                       \
        if (rebuild || (P != HR_F64 && P != HR_F32)) {                                                \
            set_error("SU(%d) rep %d: the colour-parallel kernel takes stored FP64 or FP32 links", N, rep); \
            return HR_ERR_UNSUPPORTED;                                                                \
        }                                                                                             \
        (void)variant;                                                                                \
        return P == HR_F64 ? launch_colour<N_, R_, HR_F64>(prm, epi, stream)                          \
                           : launch_colour<N_, R_, HR_F32>(prm, epi, stream);                         \
    }
    HR_LARGE_PAIRS(HR_HOP_LARGE)
#undef HR_HOP_LARGE
    set_error("SU(%d) representation %d not compiled", N, rep);
    return HR_ERR_UNSUPPORTED;
}

hr_status represent_dispatch(const hr_gauge &g, const double2 *UF, cudaStream_t stream)
{
#define HR_REPR(N_, R_) \
    if (g.lat.N == N_ && g.lat.rep == R_) return represent_launch<N_, R_>(g, UF, stream);
    HR_PAIRS(HR_REPR)
    HR_LARGE_PAIRS(HR_REPR)
#undef HR_REPR
    set_error("SU(%d) representation %d not compiled", g.lat.N, (int)g.lat.rep);
    return HR_ERR_UNSUPPORTED;
}

hr_status force_dispatch(const hr_gauge &g, const ForceParams &fp, cudaStream_t stream)
{
#define HR_FRC(N_, R_) \
    if (g.lat.N == N_ && g.lat.rep == R_) return force_launch<N_, R_>(fp, stream);
    HR_PAIRS(HR_FRC)
    HR_LARGE_PAIRS(HR_FRC)
#undef HR_FRC
    set_error("SU(%d) representation %d not compiled", g.lat.N, (int)g.lat.rep);
    return HR_ERR_UNSUPPORTED;
}

// --------------------------- helpers ---------------------------------------
long lat_volume(const hr_lattice_desc &l) { return (long)l.dims[0] * l.dims[1] * l.dims[2] * l.dims[3]; }

hr_status check_lattice(const hr_lattice_desc *lat)
{
    if (!lat) { set_error("null lattice descriptor"); return HR_ERR_INVALID; }
    if (lat->N < 2 || lat->N > HR_MAX_N) { set_error("N = %d outside 2..%d", lat->N, HR_MAX_N); return HR_ERR_INVALID; }
    if (lat->rep < HR_FUND || lat->rep > HR_ASYM_REAL) { set_error("bad representation %d", (int)lat->rep); return HR_ERR_INVALID; }
    for (int mu = 0; mu < 4; mu++) {
        if (lat->dims[mu] < 2 || (lat->dims[mu] & 1)) {
            set_error("dims[%d] = %d must be even and >= 2", mu, lat->dims[mu]);
            return HR_ERR_INVALID;
        }
        if (lat->bc[mu] != 1 && lat->bc[mu] != -1) {
            set_error("bc[%d] = %d must be +1 or -1", mu, lat->bc[mu]);
            return HR_ERR_INVALID;
        }
    }
    if (!pair_supported(lat->N, lat->rep)) {
        set_error("SU(%d) representation %d is not compiled into this library", lat->N, (int)lat->rep);
        return HR_ERR_UNSUPPORTED;
    }
    return HR_OK;
}

Geom make_geom(const hr_lattice_desc &l)
{
    Geom g;
    g.T = l.dims[0];
    g.X = l.dims[1];
    g.Y = l.dims[2];
    g.Z = l.dims[3];
    g.hz = g.Z / 2;
    g.vh = lat_volume(l) / 2;
    g.ntiles = (g.vh + HR_TILE - 1) / HR_TILE;
    for (int mu = 0; mu < 4; mu++) g.bc[mu] = l.bc[mu];
    return g;
}

FieldView make_view(void *ptr, long nsites, int D, int P)
{
    FieldView f;
    f.data = reinterpret_cast<char *>(ptr);
    f.scale = (P == HR_F16 || P == HR_BF16) ? f.data + field_scale_offset(nsites, D, P) : nullptr;
    f.rhs_stride = field_rhs_bytes(nsites, D, P);
    return f;
}

FieldView half_view(const FieldView &full, int parity, long vh, int D, int P)
{
    FieldView f = full;
    f.data += (size_t)parity * vh * 4 * D * prec_cbytes(P);
    if (f.scale) f.scale += (size_t)parity * vh * 4;
    return f;
}

hr_status ws_reserve(const hr_gauge *cg, size_t bytes, cudaStream_t stream)
{
    hr_gauge *g = const_cast<hr_gauge *>(cg);
    if (g->ws_bytes >= bytes) return HR_OK;
    if (g->ws) {
        HR_CUDA_CHECK(cudaStreamSynchronize(stream));
        HR_CUDA_CHECK(cudaDeviceSynchronize());
        HR_CUDA_CHECK(cudaFree(g->ws));
        g->ws = nullptr;
        g->ws_bytes = 0;
    }
    bytes = align_up(bytes + bytes / 8, 1 << 20);
    cudaError_t e = cudaMalloc(&g->ws, bytes);
    if (e != cudaSuccess) {
        g->ws = nullptr;
        return cuda_fail(e, "workspace cudaMalloc");
    }
    HR_CUDA_CHECK(cudaMemsetAsync(g->ws, 0, bytes, stream));
    g->ws_bytes = bytes;
    return HR_OK;
}

bool rebuild_for(const hr_gauge *g, int P)
{
    if (g->mode == HR_LINKS_AUTO) return g->auto_mode[P] == HR_LINKS_REBUILD && g->fund[P][0] != nullptr;
    return g->mode == HR_LINKS_REBUILD;
}

const void *links_for(const hr_gauge *g, int P, int parity, bool *rebuild)
{
    if (rebuild_for(g, P)) {
        *rebuild = true;
        return g->fund[P][parity];
    }
    *rebuild = false;
    return g->rep[P][parity];
}

Scratch carve_scratch(char *&p, int nrhs, long max_blocks)
{
    Scratch s;
    auto take = [&](size_t b) { char *q = p; p += align_up(b, 256); return q; };
    s.counters = reinterpret_cast<unsigned *>(take(sizeof(unsigned) * 8 * nrhs));
    s.state = reinterpret_cast<CgState *>(take(sizeof(CgState) * nrhs));
    s.red = reinterpret_cast<double *>(take(sizeof(double) * 4 * nrhs));
    s.carry = reinterpret_cast<double *>(take(sizeof(double) * 4 * nrhs));
    s.sv = reinterpret_cast<double *>(take(sizeof(double) * 2 * nrhs));
    s.partials = reinterpret_cast<double *>(take(sizeof(double) * 2 * nrhs * (size_t)max_blocks));
    return s;
}

size_t scratch_bytes(int nrhs, long max_blocks)
{
    return align_up(sizeof(unsigned) * 8 * nrhs, 256) + align_up(sizeof(CgState) * nrhs, 256) +
           2 * align_up(sizeof(double) * 4 * nrhs, 256) + align_up(sizeof(double) * 2 * nrhs, 256) +
           align_up(sizeof(double) * 2 * nrhs * (size_t)max_blocks, 256);
}

hr_status scratch_reserve(const hr_gauge *cg, int nrhs, cudaStream_t stream, Scratch *out)
{
    hr_gauge *g = const_cast<hr_gauge *>(cg);
    const long mb = max_blocks_for(g);
    const size_t need = scratch_bytes(nrhs, mb);
    if (g->scr_bytes < need) {
        if (g->scr) {
            HR_CUDA_CHECK(cudaStreamSynchronize(stream));
            HR_CUDA_CHECK(cudaDeviceSynchronize());
            HR_CUDA_CHECK(cudaFree(g->scr));
            g->scr = nullptr;
            g->scr_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&g->scr, need);
        if (e != cudaSuccess) {
            g->scr = nullptr;
            return cuda_fail(e, "scratch cudaMalloc");
        }
        HR_CUDA_CHECK(cudaMemsetAsync(g->scr, 0, need, stream));
        g->scr_bytes = need;
    }
    char *p = g->scr;
    *out = carve_scratch(p, nrhs, mb);
    return HR_OK;
}

hr_status pinned_reserve(const hr_gauge *cg, size_t bytes, cudaStream_t stream, char **host, char **dev)
{
    hr_gauge *g = const_cast<hr_gauge *>(cg);
    if (g->pinned_bytes < bytes) {
        if (g->pinned) {
            HR_CUDA_CHECK(cudaStreamSynchronize(stream));
            cudaFreeHost(g->pinned);
            g->pinned = nullptr;
            g->pinned_bytes = 0;
        }
        void *p = nullptr;
        cudaError_t e = cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc");
        memset(p, 0, bytes);
        g->pinned = p;
        g->pinned_bytes = bytes;
    }
    void *d = nullptr;
    HR_CUDA_CHECK(cudaHostGetDevicePointer(&d, g->pinned, 0));
    *host = static_cast<char *>(g->pinned);
    *dev = static_cast<char *>(d);
    return HR_OK;
}

long max_blocks_for(const hr_gauge *g)
{
    const long V = 2 * g->geom.vh;
    return std::max((V + 127) / 128, (V + BLAS_THREADS - 1) / BLAS_THREADS) + 1;
}

// One hopping-term launch: out(parity) = a * H in(other parity) + b * diag
hr_status hop(const hr_gauge *g, int P, int out_parity, int dagger, const FieldView &in, const FieldView &out,
              const FieldView *diag, double a, double b, int nrhs, cudaStream_t stream, int epi, const Scratch *sc,
              int fin, const double *carry, double *red_out, const FieldView *r, const FieldView *x,
              const FieldView *p, int variant)
{
    HopParams prm;
    memset(&prm, 0, sizeof prm);
    prm.g = g->geom;
    prm.out_parity = out_parity;
    prm.dagger = dagger;
    bool rebuild;
    prm.links = links_for(g, P, out_parity, &rebuild);
    if (!prm.links) {
        set_error("no %s links stored for precision %d", rebuild ? "fundamental" : "represented", P);
        return HR_ERR_INVALID;
    }
    prm.in = in;
    prm.out = out;
    if (diag) prm.diag = *diag;
    prm.a = a;
    prm.b = b;
    prm.nrhs = nrhs;
    if (sc) {
        prm.partials = sc->partials;
        prm.counters = sc->counters;
        prm.state = sc->state;   // solver launches: skip converged right-hand sides
    }
    prm.fin = fin;
    prm.carry = carry;
    prm.red_out = red_out;
    if (r) prm.r = *r;
    if (x) prm.x = *x;
    if (p) prm.p = *p;
    // a block of right-hand sides: right-hand-side-fastest block order, so the
    // links are fetched from HBM once and served from L2 to the other rhs
    if (nrhs >= 2) {
        prm.rhs_inner = 1;
        prm.nblk = (int)((g->geom.vh + 127) / 128);
    }
    if (variant < 0) variant = hop_variant(g, P, rebuild, epi, nrhs);
    return hop_dispatch(g->lat.N, g->lat.rep, P, prm, rebuild, epi, variant, stream);
}

unsigned hop_variants_of(const hr_gauge *g, int P)
{
    if (large_n(g)) return 0x1u;   // the colour-parallel kernel only
    if (P == HR_F64 || P == HR_DF64) return 0x1u;
    return g->D <= 4 ? 0x1Bu : 0x1Fu;   // as hop_variant_mask for the handle's pair
}

int hop_variant(const hr_gauge *g, int P, bool rebuild, int epi, int nrhs)
{
    const unsigned mask = hop_variants_of(g, P);
    auto compiled = [&](int v) {
        return v >= 0 && v < HOP_NVARIANTS && ((mask >> v) & 1u) && hop_variant_fits(v, nrhs);
    };
    if (g->force_variant >= 0) return compiled(g->force_variant) ? g->force_variant : HOP_DIRECT;
    const int t = g->tuned[P][rebuild ? 1 : 0][epi][nrhs > 1 ? 1 : 0];
    if (compiled(t)) return t;
    if (mask == 0x1u) return HOP_DIRECT;
    // untuned default, from measurements on GB300 (32^4 .. 64x32^3 lattices):
    // the staged kernel wins every fused CG update (r, x, p are read and
    // written at the warp's own sites) and the stores of the 8x8 real adjoint
    // and the SU(4) fundamental, where per-lane gathers saturate the L1
    // data pipe; the direct kernel wins the other stores
    if (epi == EPI_CG_UPDATE) return HOP_STAGED;
    if ((g->lat.rep == HR_ADJ && g->D >= 8) || (g->lat.rep == HR_FUND && g->lat.N >= 4)) return HOP_STAGED;
    return HOP_DIRECT;
}

}  // namespace hr

using namespace hr;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *hr_status_string(hr_status s)
{
    switch (s) {
    case HR_OK: return "HR_OK";
    case HR_ERR_INVALID: return "HR_ERR_INVALID: invalid argument";
    case HR_ERR_CUDA: return "HR_ERR_CUDA: CUDA runtime error";
    case HR_ERR_NOMEM: return "HR_ERR_NOMEM: device allocation failed";
    case HR_ERR_NOT_CONVERGED: return "HR_ERR_NOT_CONVERGED: solver did not reach the tolerance";
    case HR_ERR_NONFINITE: return "HR_ERR_NONFINITE: NaN or Inf in a reduction";
    case HR_ERR_TIMEOUT: return "HR_ERR_TIMEOUT: bounded device wait expired";
    case HR_ERR_UNSUPPORTED: return "HR_ERR_UNSUPPORTED: combination not compiled";
    }
    return "unknown hr_status";
}

const char *hr_last_error(void) { return g_last_error.c_str(); }

unsigned long long hr_launch_count(void) { return (unsigned long long)g_launches.load(); }

int hr_rep_dim(int N, hr_rep rep)
{
    if (N < 2 || N > HR_MAX_N || rep < HR_FUND || rep > HR_ASYM_REAL || (rep == HR_ASYM_REAL && N != 4)) return -1;
    return rep_dim(N, rep);
}

hr_status hr_generators(int N, double *T)
{
    if (N < 2 || N > HR_MAX_N || !T) {
        set_error("hr_generators: bad arguments");
        return HR_ERR_INVALID;
    }
    const int ng = N * N - 1;
    memset(T, 0, sizeof(double) * 2 * ng * N * N);
    for (int a = 0; a < ng; a++)
        for (int e = 0; e < gen_nent(N, a); e++) {
            cx<double> v = gen_val<double>(N, a, e);
            double *t = T + 2 * ((size_t)a * N * N + gen_row(N, a, e) * N + gen_col(N, a, e));
            t[0] = v.re;
            t[1] = v.im;
        }
    return HR_OK;
}

size_t hr_field_bytes(const hr_lattice_desc *lat, hr_parity par, hr_prec prec, int nrhs)
{
    if (check_lattice(lat) != HR_OK || prec < HR_F64 || prec > HR_DF64 || nrhs < 1) return 0;
    long V = lat_volume(*lat);
    long ns = par == HR_FULL ? V : V / 2;
    return field_rhs_bytes(ns, rep_dim(lat->N, lat->rep), prec) * (size_t)nrhs;
}

hr_status hr_represent_gauge(const hr_lattice_desc *lat, const void *U_fund, unsigned prec_mask,
                             unsigned link_modes, void *stream, hr_gauge **out)
{
    if (!out) { set_error("hr_represent_gauge: out is NULL"); return HR_ERR_INVALID; }
    *out = nullptr;
    hr_status st = check_lattice(lat);
    if (st != HR_OK) return st;
    if (!U_fund) { set_error("hr_represent_gauge: U_fund is NULL"); return HR_ERR_INVALID; }
    if (prec_mask == 0 || (prec_mask & ~0x1Fu)) { set_error("bad prec_mask 0x%x", prec_mask); return HR_ERR_INVALID; }
    if (link_modes == 0 || (link_modes & ~0x3u)) { set_error("bad link_modes 0x%x", link_modes); return HR_ERR_INVALID; }
    if (colour_pair(lat->N, lat->rep) && link_modes != (1u << HR_LINKS_STORED)) {
        set_error("SU(%d): the colour-parallel kernel reads stored links only (link_modes = STORED)", lat->N);
        return HR_ERR_UNSUPPORTED;
    }
    hr_gauge *g = new hr_gauge;
    memset(g, 0, sizeof *g);
    memset(g->tuned, -1, sizeof g->tuned);
    memset(g->auto_mode, -1, sizeof g->auto_mode);
    g->force_variant = -1;
    g->autotune = 1;
    g->lat = *lat;
    g->geom = make_geom(*lat);
    g->D = rep_dim(lat->N, lat->rep);
    g->real = rep_real(lat->rep);
    g->prec_mask = prec_mask;
    g->link_modes = link_modes;
    g->mode = (link_modes & (1u << HR_LINKS_STORED)) ? HR_LINKS_STORED : HR_LINKS_REBUILD;
    cudaGetDevice(&g->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto fail = [&](hr_status e) { hr_gauge_destroy(g); return e; };
    for (int P = 0; P < HR_NPREC; P++) {
        if (!(prec_mask & (1u << P))) continue;
        if (link_modes & (1u << HR_LINKS_STORED)) {
            size_t b = link_record_bytes(g->geom, P, g->real, g->D * link_row_stride(lat->N, lat->rep, P));
            g->rep_bytes[P] = b;
            for (int par = 0; par < 2; par++) {
                cudaError_t e = cudaMalloc(&g->rep[P][par], b);
                if (e != cudaSuccess) { g->rep[P][par] = nullptr; return fail(cuda_fail(e, "link cudaMalloc")); }
                e = cudaMemsetAsync(g->rep[P][par], 0, b, s);
                if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync"));
            }
        }
        // float-float is compiled for stored links only
        if ((link_modes & (1u << HR_LINKS_REBUILD)) && P != HR_DF64) {
            size_t b = link_record_bytes(g->geom, P, false, lat->N * lat->N);
            g->fund_bytes[P] = b;
            for (int par = 0; par < 2; par++) {
                cudaError_t e = cudaMalloc(&g->fund[P][par], b);
                if (e != cudaSuccess) { g->fund[P][par] = nullptr; return fail(cuda_fail(e, "link cudaMalloc")); }
                e = cudaMemsetAsync(g->fund[P][par], 0, b, s);
                if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync"));
            }
        }
    }
    // T_R^a tables for the force: (T_R^a)_{nm} = -i d/de R(exp(i e T^a))_{nm}
    {
        const int N = lat->N, D = g->D, ng = N * N - 1;
        std::vector<double> h((size_t)ng * D * D * 2, 0.0);
        rep_generator_table(N, lat->rep, h.data());
        cudaError_t e = cudaMalloc(&g->TR, h.size() * sizeof(double));
        if (e != cudaSuccess) { g->TR = nullptr; return fail(cuda_fail(e, "cudaMalloc")); }
        e = cudaMemcpy(g->TR, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy"));
    }
    {
        cudaError_t e = cudaMalloc(&g->err, sizeof(int));
        if (e != cudaSuccess) { g->err = nullptr; return fail(cuda_fail(e, "cudaMalloc")); }
        e = cudaMemsetAsync(g->err, 0, sizeof(int), s);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync"));
    }
    st = represent_dispatch(*g, reinterpret_cast<const double2 *>(U_fund), s);
    if (st != HR_OK) return fail(st);
    *out = g;
    return HR_OK;
}

hr_status hr_gauge_update(hr_gauge *g, const void *U_fund, void *stream)
{
    if (!g || !U_fund) { set_error("hr_gauge_update: NULL argument"); return HR_ERR_INVALID; }
    hr_status st = represent_dispatch(*g, reinterpret_cast<const double2 *>(U_fund), reinterpret_cast<cudaStream_t>(stream));
    // the clover term follows the links
    if (st == HR_OK && g->clover_mode) st = clover_build(g, U_fund, reinterpret_cast<cudaStream_t>(stream));
    return st;
}

hr_status hr_gauge_set_link_mode(hr_gauge *g, hr_link_mode mode)
{
    const unsigned need = mode == HR_LINKS_AUTO ? 0x3u : (mode == HR_LINKS_STORED || mode == HR_LINKS_REBUILD)
                                                              ? (1u << mode) : 0x4u;
    if (!g || (g->link_modes & need) != need) {
        set_error("hr_gauge_set_link_mode: mode %d not available", (int)mode);
        return HR_ERR_INVALID;
    }
    g->mode = mode;
    return HR_OK;
}

int hr_gauge_link_mode(const hr_gauge *g, hr_prec prec)
{
    if (!g || prec < HR_F64 || prec > HR_DF64) return -1;
    return rebuild_for(g, prec) ? HR_LINKS_REBUILD : HR_LINKS_STORED;
}

hr_status hr_gauge_destroy(hr_gauge *g)
{
    if (!g) return HR_OK;
    cudaDeviceSynchronize();
    for (int P = 0; P < HR_NPREC; P++)
        for (int par = 0; par < 2; par++) {
            if (g->rep[P][par]) cudaFree(g->rep[P][par]);
            if (g->fund[P][par]) cudaFree(g->fund[P][par]);
        }
    if (g->TR) cudaFree(g->TR);
    for (int P = 0; P < HR_NPREC; P++)
        if (g->cl[P]) cudaFree(g->cl[P]);
    if (g->err) cudaFree(g->err);
    if (g->ws) cudaFree(g->ws);
    if (g->scr) cudaFree(g->scr);
    if (g->pinned) cudaFreeHost(g->pinned);
    delete g;
    return HR_OK;
}

static hr_status check_apply(const hr_gauge *g, hr_parity par, hr_prec prec, const void *in, void *out, int nrhs)
{
    if (!g || !in || !out || nrhs < 1) { set_error("hr_dirac_apply: NULL argument or nrhs < 1"); return HR_ERR_INVALID; }
    if (prec < HR_F64 || prec > HR_DF64 || !(g->prec_mask & (1u << prec))) {
        set_error("precision %d not stored in this gauge handle (mask 0x%x)", (int)prec, g->prec_mask);
        return HR_ERR_INVALID;
    }
    if (par < HR_EVEN || par > HR_EO_PRECOND) { set_error("bad parity selector %d", (int)par); return HR_ERR_INVALID; }
    if (in == out) { set_error("in and out must not overlap"); return HR_ERR_INVALID; }
    return HR_OK;
}

static hr_status apply_impl(const hr_gauge *g, hr_parity par, hr_prec prec, const void *in, void *out, int nrhs,
                            void *stream, int dagger)
{
    hr_status st = check_apply(g, par, prec, in, out, nrhs);
    if (st != HR_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long vh = g->geom.vh;
    const int D = g->D;
    const double m4 = 4.0 + g->lat.m0;
    if (par == HR_EVEN || par == HR_ODD) {
        FieldView vi = make_view(const_cast<void *>(in), vh, D, prec), vo = make_view(out, vh, D, prec);
        return hop(g, prec, par == HR_EVEN ? 0 : 1, dagger, vi, vo, nullptr, -0.5, 0.0, nrhs, s, EPI_STORE);
    }
    if (g->clover_mode && prec != HR_F64 && prec != HR_F32) {
        set_error("with a clover term D_m and Dhat are available in FP64 and FP32 only");
        return HR_ERR_UNSUPPORTED;
    }
    if (par == HR_FULL) {
        FieldView fi = make_view(const_cast<void *>(in), 2 * vh, D, prec), fo = make_view(out, 2 * vh, D, prec);
        for (int p = 0; p < 2; p++) {
            FieldView ih = half_view(fi, 1 - p, vh, D, prec), dh = half_view(fi, p, vh, D, prec);
            FieldView oh = half_view(fo, p, vh, D, prec);
            if (g->clover_mode) {
                // out_p = C_pp in_p + hops (C is Hermitian: the same for D^dag)
                st = clover_apply(g, prec, p, 0, dh, oh, nrhs, s);
                if (st == HR_OK) st = hop(g, prec, p, dagger, ih, oh, &oh, -0.5, 1.0, nrhs, s, EPI_STORE);
            } else {
                st = hop(g, prec, p, dagger, ih, oh, &dh, -0.5, m4, nrhs, s, EPI_STORE);
            }
            if (st != HR_OK) return st;
        }
        return HR_OK;
    }
    // Dhat = (4+m)^2 - D_eo D_oe  (dagger: same with D^dag blocks)
    size_t tb = field_rhs_bytes(vh, D, prec) * nrhs;
    st = ws_reserve(g, tb, s);
    if (st != HR_OK) return st;
    FieldView vi = make_view(const_cast<void *>(in), vh, D, prec), vo = make_view(out, vh, D, prec);
    FieldView vt = make_view(g->ws, vh, D, prec);
    st = hop(g, prec, 1, dagger, vi, vt, nullptr, -0.5, 0.0, nrhs, s, EPI_STORE);
    if (st != HR_OK) return st;
    if (g->clover_mode) {
        // Dhat = C_ee - D_eo C_oo^-1 D_oe
        st = clover_apply(g, prec, 1, 1, vt, vt, nrhs, s);
        if (st == HR_OK) st = clover_apply(g, prec, 0, 0, vi, vo, nrhs, s);
        if (st != HR_OK) return st;
        return hop(g, prec, 0, dagger, vt, vo, &vo, 0.5, 1.0, nrhs, s, EPI_STORE);
    }
    return hop(g, prec, 0, dagger, vt, vo, &vi, 0.5, m4 * m4, nrhs, s, EPI_STORE);
}

hr_status hr_dirac_apply(const hr_gauge *g, hr_parity par, hr_prec prec, const void *in, void *out, int nrhs,
                         void *stream)
{
    return apply_impl(g, par, prec, in, out, nrhs, stream, 0);
}

hr_status hr_dirac_dagger(const hr_gauge *g, hr_parity par, hr_prec prec, const void *in, void *out, int nrhs,
                          void *stream)
{
    return apply_impl(g, par, prec, in, out, nrhs, stream, 1);
}

hr_status hr_field_convert(const hr_lattice_desc *lat, hr_parity par, hr_prec src_prec, const void *src,
                           hr_prec dst_prec, void *dst, int nrhs, void *stream)
{
    hr_status st = check_lattice(lat);
    if (st != HR_OK) return st;
    if (!src || !dst || nrhs < 1 || src == dst) { set_error("hr_field_convert: bad pointers or nrhs"); return HR_ERR_INVALID; }
    if (src_prec < HR_F64 || src_prec > HR_DF64 || dst_prec < HR_F64 || dst_prec > HR_DF64) {
        set_error("hr_field_convert: bad precision");
        return HR_ERR_INVALID;
    }
    const long V = lat_volume(*lat);
    const long ns = par == HR_FULL ? V : V / 2;
    const int D = rep_dim(lat->N, lat->rep);
    BlasParams bp;
    memset(&bp, 0, sizeof bp);
    bp.nsites = ns;
    bp.nrhs = nrhs;
    bp.a = make_view(dst, ns, D, dst_prec);
    bp.b = make_view(const_cast<void *>(src), ns, D, src_prec);
    bp.s = 1.0;
    return blas_convert(D, dst_prec, src_prec, bp, reinterpret_cast<cudaStream_t>(stream));
}

hr_status hr_field_dot(const hr_lattice_desc *lat, hr_parity par, hr_prec prec, const void *a, const void *b,
                       int nrhs, double *out, void *stream)
{
    hr_status st = check_lattice(lat);
    if (st != HR_OK) return st;
    if (!a || !b || !out || nrhs < 1 || prec < HR_F64 || prec > HR_DF64 || par < HR_EVEN || par > HR_EO_PRECOND) {
        set_error("hr_field_dot: bad arguments");
        return HR_ERR_INVALID;
    }
    const long V = lat_volume(*lat);
    const long ns = par == HR_FULL ? V : V / 2;
    const int D = rep_dim(lat->N, lat->rep);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long nblk = (ns + BLAS_THREADS - 1) / BLAS_THREADS + 1;
    char *buf = nullptr;
    size_t bytes = scratch_bytes(nrhs, nblk);
    HR_CUDA_CHECK(cudaMallocAsync((void **)&buf, bytes, s));
    HR_CUDA_CHECK(cudaMemsetAsync(buf, 0, bytes, s));
    char *p = buf;
    Scratch sc = carve_scratch(p, nrhs, nblk);
    BlasParams bp;
    memset(&bp, 0, sizeof bp);
    bp.nsites = ns;
    bp.nrhs = nrhs;
    bp.a = make_view(const_cast<void *>(a), ns, D, prec);
    bp.b = make_view(const_cast<void *>(b), ns, D, prec);
    bp.partials = sc.partials;
    bp.counters = sc.counters;
    bp.red_out = sc.red;
    st = blas_dot(D, prec, bp, s);
    if (st == HR_OK) {
        cudaError_t e = cudaMemcpyAsync(out, sc.red, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "hr_field_dot copy");
    }
    cudaFreeAsync(buf, s);
    return st;
}

hr_status hr_dirac_force(const hr_gauge *g, hr_parity sys, const void *X, const void *Y, double coeff, void *F,
                         void *stream)
{
    return hr_dirac_force_prec(g, sys, X, Y, coeff, F, HR_F64, stream);
}

hr_status hr_dirac_force_prec(const hr_gauge *g, hr_parity sys, const void *X, const void *Y, double coeff, void *F,
                              hr_prec arith, void *stream)
{
    if (g && g->clover_mode) {
        set_error("hr_dirac_force: the clover term's force is not provided");
        return HR_ERR_UNSUPPORTED;
    }
    if (!g || !X || !Y || !F) { set_error("hr_dirac_force: NULL argument"); return HR_ERR_INVALID; }
    if (arith != HR_F64 && arith != HR_DF64) {
        set_error("hr_dirac_force: arithmetic must be HR_F64 or HR_DF64");
        return HR_ERR_INVALID;
    }
    if (!(g->prec_mask & (1u << HR_F64)) || !g->rep[HR_F64][0]) {
        set_error("hr_dirac_force needs FP64 stored represented links in the handle");
        return HR_ERR_INVALID;
    }
    if (arith == HR_DF64 && !g->rep[HR_DF64][0]) {
        set_error("hr_dirac_force: the float-float force needs DF64 stored represented links in the handle");
        return HR_ERR_INVALID;
    }
    if (sys != HR_FULL && sys != HR_EO_PRECOND) { set_error("hr_dirac_force: sys must be FULL or EO_PRECOND"); return HR_ERR_INVALID; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long vh = g->geom.vh;
    const int D = g->D;
    hr_status st;
    FieldView fx, fy;
    double c = coeff;
    if (sys == HR_FULL) {
        fx = make_view(const_cast<void *>(X), 2 * vh, D, HR_F64);
        fy = make_view(const_cast<void *>(Y), 2 * vh, D, HR_F64);
    } else {
        // S = -2 Re <Y_e, Dhat X_e> = 2 Re <Y_e, D_eo D_oe X_e> + const: the full-operator
        // derivative with X' = (X_e, D_oe X_e), Y' = (Y_e, (D^dag)_oe Y_e) and coeff -> -coeff
        size_t fb = field_rhs_bytes(2 * vh, D, HR_F64);
        st = ws_reserve(g, 2 * fb, s);
        if (st != HR_OK) return st;
        fx = make_view(g->ws, 2 * vh, D, HR_F64);
        fy = make_view(g->ws + fb, 2 * vh, D, HR_F64);
        st = kernel_copy(fx.data, X, (size_t)vh * 4 * D * 16, s);
        if (st == HR_OK) st = kernel_copy(fy.data, Y, (size_t)vh * 4 * D * 16, s);
        if (st != HR_OK) return st;
        FieldView xe = half_view(fx, 0, vh, D, HR_F64), xo = half_view(fx, 1, vh, D, HR_F64);
        FieldView ye = half_view(fy, 0, vh, D, HR_F64), yo = half_view(fy, 1, vh, D, HR_F64);
        const hr_link_mode keep = g->mode;
        const_cast<hr_gauge *>(g)->mode = HR_LINKS_STORED;
        st = hop(g, HR_F64, 1, 0, xe, xo, nullptr, -0.5, 0.0, 1, s, EPI_STORE);
        if (st == HR_OK) st = hop(g, HR_F64, 1, 1, ye, yo, nullptr, -0.5, 0.0, 1, s, EPI_STORE);
        const_cast<hr_gauge *>(g)->mode = keep;
        if (st != HR_OK) return st;
        c = -coeff;
    }
    return force_full(g, fx, fy, c, reinterpret_cast<double *>(F), arith, s);
}

}  // extern "C"

namespace hr {

hr_status force_full(const hr_gauge *g, const FieldView &fx, const FieldView &fy, double c, double *F, int arith,
                     cudaStream_t s)
{
    const long vh = g->geom.vh;
    const int D = g->D;
    for (int p = 0; p < 2; p++) {
        ForceParams fp;
        fp.g = g->geom;
        fp.parity = p;
        fp.arith = arith;
        fp.links = g->rep[arith][p];
        fp.X_here = half_view(fx, p, vh, D, HR_F64);
        fp.Y_here = half_view(fy, p, vh, D, HR_F64);
        fp.X_nb = half_view(fx, 1 - p, vh, D, HR_F64);
        fp.Y_nb = half_view(fy, 1 - p, vh, D, HR_F64);
        fp.TR = g->TR;
        fp.coeff = c;
        fp.F = F;
        hr_status st = force_dispatch(*g, fp, s);
        if (st != HR_OK) return st;
    }
    return HR_OK;
}

}  // namespace hr

namespace hr {

// (T_R^a)_{nm} = -i d/de R(exp(i e T^a))_{nm} at e = 0, differentiating the
// same sparse formulas the represent kernel evaluates:
//   ADJ:  R_bc = 2 sum_{(i,j,be) in T_b} sum_{(k,l,ga) in T_c} be ga U_jk conj(U_il)
//         -> T_R = 2 sum be ga [T_jk delta_il - delta_jk conj(T_il)]
//   SYM/ASYM: R_nm = sum w v U_ik U_jl -> T_R = sum w v [T_ik delta_jl + delta_ik T_jl]
void rep_generator_table(int N, int rep, double *out)
{
    const int ng = N * N - 1, D = rep_dim(N, rep);
    std::vector<cx<double>> T((size_t)ng * N * N, cx<double>{0, 0});
    for (int a = 0; a < ng; a++)
        for (int e = 0; e < gen_nent(N, a); e++)
            T[(size_t)a * N * N + gen_row(N, a, e) * N + gen_col(N, a, e)] = gen_val<double>(N, a, e);
    for (int a = 0; a < ng; a++) {
        const cx<double> *Ta = &T[(size_t)a * N * N];
        for (int n = 0; n < D; n++)
            for (int m = 0; m < D; m++) {
                cx<double> v = {0, 0};
                if (rep == HR_FUND) {
                    v = Ta[n * N + m];
                } else if (rep == HR_ADJ) {
                    for (int e1 = 0; e1 < gen_nent(N, n); e1++) {
                        int i = gen_row(N, n, e1), j = gen_col(N, n, e1);
                        cx<double> be = gen_val<double>(N, n, e1);
                        for (int e2 = 0; e2 < gen_nent(N, m); e2++) {
                            int k = gen_row(N, m, e2), l = gen_col(N, m, e2);
                            cx<double> ga = gen_val<double>(N, m, e2);
                            cx<double> d = {0, 0};
                            if (i == l) d = d + Ta[j * N + k];
                            if (j == k) d = d - conj(Ta[i * N + l]);
                            v = v + 2.0 * ((be * ga) * d);
                        }
                    }
                } else if (rep == HR_ASYM_REAL) {
                    // R_nm = conj(c_n) c_m sum w v U_ik U_jl -> the same with
                    // [T_ik delta_jl + delta_ik T_jl]
                    for (int e1 = 0; e1 < 4; e1++) {
                        int i = rb_row(n, e1), j = rb_col(n, e1);
                        for (int e2 = 0; e2 < 4; e2++) {
                            int k = rb_row(m, e2), l = rb_col(m, e2);
                            cx<double> d = {0, 0};
                            if (j == l) d = d + Ta[i * N + k];
                            if (i == k) d = d + Ta[j * N + l];
                            v = v + (rb_val(n, e1) * rb_val(m, e2)) * d;
                        }
                    }
                    v = rb_cc(n, rb_c(m, v));
                } else {
                    for (int e1 = 0; e1 < sb_nent(N, rep, n); e1++) {
                        int i = sb_row(N, rep, n, e1), j = sb_col(N, rep, n, e1);
                        double w = sb_val(N, rep, n, e1);
                        for (int e2 = 0; e2 < sb_nent(N, rep, m); e2++) {
                            int k = sb_row(N, rep, m, e2), l = sb_col(N, rep, m, e2);
                            double vv = sb_val(N, rep, m, e2);
                            cx<double> d = {0, 0};
                            if (j == l) d = d + Ta[i * N + k];
                            if (i == k) d = d + Ta[j * N + l];
                            v = v + (w * vv) * d;
                        }
                    }
                }
                double *o = out + 2 * (((size_t)a * D + n) * D + m);
                o[0] = v.re;
                o[1] = v.im;
            }
    }
}

}  // namespace hr
