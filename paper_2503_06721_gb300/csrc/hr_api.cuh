// hr_api.cuh -- host-side internals shared by hr_api.cu and hr_cg.cu.
#pragma once

#include <algorithm>
#include <vector>

#include "hr_blas.cuh"
#include "hr_gauge.cuh"

namespace hr {

// device scratch for fused reductions and solver state
struct Scratch {
    double *partials;   // [nrhs][max_blocks][2]
    unsigned *counters; // [8 * nrhs] (zero between kernels)
    CgState *state;     // [nrhs]
    double *red;        // [nrhs][4]
    double *carry;      // [nrhs][4]
    double *sv;         // [nrhs][2] per-rhs scalars
};

long lat_volume(const hr_lattice_desc &l);
hr_status check_lattice(const hr_lattice_desc *lat);
bool pair_supported(int N, int rep);
Geom make_geom(const hr_lattice_desc &l);
FieldView make_view(void *ptr, long nsites, int D, int P);
FieldView half_view(const FieldView &full, int parity, long vh, int D, int P);
hr_status ws_reserve(const hr_gauge *g, size_t bytes, cudaStream_t stream);
Scratch carve_scratch(char *&p, int nrhs, long max_blocks);
size_t scratch_bytes(int nrhs, long max_blocks);
long max_blocks_for(const hr_gauge *g);
// the handle's host-mapped pinned buffer of at least `bytes` (grown on
// demand): host address in *host, device address in *dev
hr_status pinned_reserve(const hr_gauge *g, size_t bytes, cudaStream_t stream, char **host, char **dev);
// the handle's reduction scratch for nrhs right-hand sides (grown and zeroed on demand)
hr_status scratch_reserve(const hr_gauge *g, int nrhs, cudaStream_t stream, Scratch *out);

// variant < 0: the handle's tuned (or default) choice for this launch
hr_status hop(const hr_gauge *g, int P, int out_parity, int dagger, const FieldView &in, const FieldView &out,
              const FieldView *diag, double a, double b, int nrhs, cudaStream_t stream, int epi,
              const Scratch *sc = nullptr, int fin = FIN_WRITE, const double *carry = nullptr,
              double *red_out = nullptr, const FieldView *r = nullptr, const FieldView *x = nullptr,
              const FieldView *p = nullptr, int variant = -1);

// the large-N fundamental pairs (N >= 5), run by the colour-parallel hopping
// kernel without a fused CG-update epilogue
// pairs run by the colour-parallel hopping kernel (no fused CG update)
inline bool large_n(const hr_gauge *g) { return colour_pair(g->lat.N, g->lat.rep); }

// whether operator launches in precision P read fundamental links (rebuild)
bool rebuild_for(const hr_gauge *g, int P);

// kernel variants compiled for the handle's pair in precision P (bit v = variant v)
unsigned hop_variants_of(const hr_gauge *g, int P);
// the variant a launch would use (forced, tuned, or the fixed default)
int hop_variant(const hr_gauge *g, int P, bool rebuild, int epi, int nrhs);
// time every variant of every epilogue in precision P for the handle's
// lattice, link mode and nrhs, record the fastest (blocks the host)
hr_status tune_hops(hr_gauge *g, int P, int nrhs, cudaStream_t stream);

// F += c * (force of the full-operator action -2 Re <Y, D X>) for full FP64
// fields X = fx, Y = fy, in FP64 on the stored FP64 links (arith = HR_F64)
// or in float-float on the stored DF64 links (HR_DF64)
hr_status force_full(const hr_gauge *g, const FieldView &fx, const FieldView &fy, double c, double *F, int arith,
                     cudaStream_t s);

// the clover diagonal (hr_clover.cu): build C and C^-1 from U_F for the
// handle's clover_mode and csw (FP64 and, if the handle holds FP32, FP32);
// apply out = C_pp in (kind 0) or C_pp^-1 in (kind 1) on the sites of parity
// p (in == out allowed)
hr_status clover_build(hr_gauge *g, const void *U_fund, cudaStream_t s);
hr_status clover_apply(const hr_gauge *g, int P, int parity, int kind, const FieldView &in, const FieldView &out,
                       int nrhs, cudaStream_t s);

// number of kernel launches counted so far (graph contents counted when they run)
long long launch_counter();

// (T_R^a)_{nm} as complex double [(N*N-1)][D][D] (host)
void rep_generator_table(int N, int rep, double *out);

}  // namespace hr
