/*
 * hr.h -- C ABI of the GB300 (sm_103a) Wilson-Dirac library for fermions in
 * higher representations of SU(N): the hot path of HiRep v2
 * (arXiv 2503.06721).
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice (Sec. 2.1): dims = {T, X, Y, Z}, mu = 0 is time; every extent even
 * and >= 2.  Lexicographic site index lex = ((t*X + x)*Y + y)*Z + z.
 * Even sites have (t+x+y+z) mod 2 == 0 (Sec. 4.3.3).  A parity ("half")
 * field over V/2 sites is indexed by lex/2 inside its parity.  A FULL field
 * is the even half followed by the odd half (even sites indexed first, as in
 * Sec. 3.4.1).
 *
 * Spinor fields (Sec. 3.1.2, Table "elementary data types"):
 *   HR_F64 / HR_F32: [nrhs][nsites][spin 0..3][colour 0..D_R-1] interleaved
 *     complex (re, im) in double / float.
 *   HR_DF64: the same layout with every complex as four floats
 *     (re.hi, re.lo, im.hi, im.lo), value = hi + lo.
 *   HR_F16 / HR_BF16 (reduced storage with one scale per site):
 *     each right-hand side is a block of hr_field_bytes(..., 1) bytes holding
 *     [nsites][4][D_R] pairs (re, im) of half / bfloat16 values v/s_x,
 *     followed, at the next 256-byte boundary, by [nsites] float scales s_x
 *     (the largest |component| of site x).  The value is  s_x * stored.
 * Gauge field input (Sec. 3.1.3): U_F[lex][mu][row][col] complex double
 *   (SU(N) links in the positive directions), device memory.
 * Force output: F[lex][mu][a] double, a = 0..N*N-2 in the generator order
 *   of hr_generators() (generalised Gell-Mann matrices / 2).
 *
 * Memory and errors: all field pointers are DEVICE pointers owned by the
 * caller; the library never frees them.  hr_represent_gauge allocates the
 * internal link storage (freed by hr_gauge_destroy) and each hr_gauge holds
 * a lazily grown solver workspace.  Every call returns an hr_status and never
 * exits or throws; hr_last_error() gives a thread-local message for the last
 * failure.  Calls are asynchronous on the given CUDA stream (a cudaStream_t
 * passed as void*, NULL = legacy default stream) except where stated.
 */
#ifndef HR_H
#define HR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Supported representations, Table 1 (Sec. 2.3). HR_ASYM is "2AS".
 * HR_ASYM_REAL is the 2AS of SU(4) (the 6, a real representation) in a
 * basis where R(U) is real orthogonal, so its links are stored as reals
 * (Sec. 3.1.2): the orthonormal antisymmetric matrices
 *   f_2k = (e_P + s e_Q)/sqrt2,  f_2k+1 = i (e_P - s e_Q)/sqrt2,
 *   (P, Q; s) = ((0,1),(2,3);+1), ((0,2),(1,3);-1), ((0,3),(1,2);+1) for k = 0,1,2,
 * with e_(ij) = (E_ij - E_ji)/sqrt2 the HR_ASYM basis.  Colour components of
 * spinors are coordinates in this basis: psi_real = W^dag psi_2AS with
 * W_mn = Tr(e_m^dag f_n). */
typedef enum { HR_FUND = 0, HR_ADJ = 1, HR_SYM = 2, HR_ASYM = 3, HR_ASYM_REAL = 4 } hr_rep;

/* Storage precision of fields and links.  F64 computes in double, F32/F16/BF16
 * in float; F16/BF16 spinors carry one float scale per site.  DF64 holds every
 * FP64 value as an exact pair of floats (hi, lo), 16 bytes per complex like
 * F64, and computes in float-float arithmetic (about 48 significant bits). */
typedef enum { HR_F64 = 0, HR_F32 = 1, HR_F16 = 2, HR_BF16 = 3, HR_DF64 = 4 } hr_prec;

/* Output parity / operator selector (Sec. 4.3.3, Eq. dmeo and Eq. deo):
 *   HR_EVEN        out_e = D_eo in_o   (hopping block, includes the -1/2)
 *   HR_ODD         out_o = D_oe in_e
 *   HR_FULL        out   = D_m in      on FULL fields
 *   HR_EO_PRECOND  out_e = Dhat in_e,  Dhat = (4+m)^2 - D_eo D_oe          */
typedef enum { HR_EVEN = 0, HR_ODD = 1, HR_FULL = 2, HR_EO_PRECOND = 3 } hr_parity;

typedef enum {
    HR_OK = 0,
    HR_ERR_INVALID = -1,        /* bad argument (message in hr_last_error) */
    HR_ERR_CUDA = -2,           /* a CUDA runtime call failed */
    HR_ERR_NOMEM = -3,          /* device allocation failed */
    HR_ERR_NOT_CONVERGED = -4,  /* solver hit max_iter above tolerance */
    HR_ERR_NONFINITE = -5,      /* NaN/Inf met in a reduction */
    HR_ERR_TIMEOUT = -6,        /* a bounded device-side wait gave up */
    HR_ERR_UNSUPPORTED = -7     /* combination not compiled in */
} hr_status;

/* How the operator kernels obtain U_R (Sec. 3.1.3, represented field):
 *   HR_LINKS_STORED   read the D_R x D_R represented links kept in HBM
 *   HR_LINKS_REBUILD  read the N x N fundamental links and rebuild the action
 *                     of U_R inside the kernel (fewer bytes, more flops)
 *   HR_LINKS_AUTO     per precision, whichever of the two hr_tune measured
 *                     faster on the handle's lattice (STORED until tuned;
 *                     always STORED for F16 and BF16, whose rebuilt links
 *                     carry about twice the rounding error of the stored
 *                     ones); needs both storages (hr_gauge_set_link_mode only) */
typedef enum { HR_LINKS_STORED = 0, HR_LINKS_REBUILD = 1, HR_LINKS_AUTO = 2 } hr_link_mode;

typedef struct {
    int N;          /* SU(N): N = 2, 3, 4 with the representations FUND,
                       ADJ, SYM (N = 2, 3), ASYM (N = 3, 4), ASYM_REAL
                       (N = 4); the colour-parallel pairs -- FUND for
                       N = 5, 6, 8 and ADJ, SYM for N = 4 (D_R = 15, 10) --
                       run on the colour-parallel hopping kernel (Sec.
                       8.2): FP64 / FP32 stored links, solves on the
                       multi-shift engine, no batched or fused solve + force */
    hr_rep rep;
    int dims[4];    /* T, X, Y, Z (all even) */
    int bc[4];      /* +1 periodic, -1 antiperiodic fermion boundary (Sec. 5.3.1) */
    double m0;      /* bare mass m of D_m = D + m (Eq. D_m^R) */
} hr_lattice_desc;

typedef struct hr_gauge hr_gauge;   /* opaque: represented (and/or fund) links */

/* ------------------------------------------------------------------ */
/* Representation of the gauge field (Sec. 2.3 Eq. U^R = exp(i w T_R),   */
/* Sec. 3.1.3; boundary signs Sec. 5.3.1)                                */
/* ------------------------------------------------------------------ */
/* Builds U_R(x,mu) = R(U_F(x,mu)) for every link and applies the fermion
 * boundary condition as a -1 on the represented links of the last slice
 * (x_mu = L_mu - 1) of every antiperiodic direction.
 *   lat        lattice; copied into the handle.
 *   U_fund     device, complex double [V][4][N][N]; read only, not retained.
 *   prec_mask  OR of (1u << hr_prec) for every precision the operator will
 *              be applied in; links are stored once per precision.
 *   link_modes OR of (1u << hr_link_mode): STORED keeps D_R x D_R links,
 *              REBUILD keeps the N x N fundamental links for in-kernel
 *              rebuilding.  Both may be set (hr_gauge_set_link_mode picks).
 *   out        receives the new handle (NULL on failure).
 * Errors: HR_ERR_INVALID (bad N/rep/dims/mask), HR_ERR_NOMEM, HR_ERR_CUDA.
 * The links are ready once the work queued on `stream` completes. */
hr_status hr_represent_gauge(const hr_lattice_desc *lat, const void *U_fund,
                             unsigned prec_mask, unsigned link_modes,
                             void *stream, hr_gauge **out);

/* Re-represents a new U_F into the existing storage of g (after a gauge
 * update, Sec. 5.3.1: "only necessary after every gauge update"). */
hr_status hr_gauge_update(hr_gauge *g, const void *U_fund, void *stream);

/* Clover improvement (Sec. 5.1.2) and exponential clover (Sec. 5.1.3): the
 * diagonal of D_m becomes, per site,
 *   HR_CLOVER_PLAIN:  (4+m) + csw (i/4) sum_{mu,nu} sigma_mu_nu F_mu_nu
 *   HR_CLOVER_EXP:    (4+m) exp(csw/(4+m) (i/4) sum_{mu,nu} sigma_mu_nu F_mu_nu)
 * with sigma_mu_nu = (i/2)[gamma_mu, gamma_nu] and F_mu_nu = (Q - Q^dag)/8,
 * Q the four plaquettes of the (mu,nu) plane through x (Eq. clover-term),
 * each as the closed loop through x, in the fermion representation.
 * hr_gauge_set_clover builds the term (and its inverse) from U_fund (the
 * links g was built from; hr_gauge_update rebuilds it with the new links);
 * HR_CLOVER_NONE removes it.  With a clover term: hr_dirac_apply /
 * hr_dirac_dagger give D_m (HR_FULL) and Dhat = C_ee - D_eo C_oo^-1 D_oe
 * (HR_EO_PRECOND) in FP64 and FP32 (the hopping blocks HR_EVEN / HR_ODD
 * are unchanged); hr_cg_solve and hr_cg_solve_multishift solve with it
 * (inner FP64 or FP32, x started from 0); hr_cg_solve_batched,
 * hr_cg_solve_force and hr_dirac_force return HR_ERR_UNSUPPORTED (the
 * clover term's force is not provided).  Needs FP64 links in g; the FP32
 * records are built when g holds FP32 links.
 * Errors: HR_ERR_NONFINITE if a clover block is singular. */
typedef enum { HR_CLOVER_NONE = 0, HR_CLOVER_PLAIN = 1, HR_CLOVER_EXP = 2 } hr_clover_mode;
hr_status hr_gauge_set_clover(hr_gauge *g, const void *U_fund, double csw,
                              hr_clover_mode mode, void *stream);

/* Chooses STORED, REBUILD or AUTO links for later operator calls on g.
 * HR_ERR_INVALID if that storage (both, for AUTO) was not requested at
 * creation.  The force always reads stored links (FP64, or DF64 for the
 * float-float force). */
hr_status hr_gauge_set_link_mode(hr_gauge *g, hr_link_mode mode);

/* The link mode operator calls in precision prec use now (STORED or
 * REBUILD); -1 for bad arguments. */
int hr_gauge_link_mode(const hr_gauge *g, hr_prec prec);

/* Frees the link storage and solver workspace (synchronises the device). */
hr_status hr_gauge_destroy(hr_gauge *g);

/* ------------------------------------------------------------------ */
/* Kernel-variant autotuning                                             */
/* ------------------------------------------------------------------ */
/* The hopping kernel (Eq. D_m^R) is compiled in several variants that
 * produce bitwise identical results and differ in how a warp moves its
 * site records and in register budget:
 *   HR_HOP_DIRECT        each lane loads its own neighbour spinors;
 *   HR_HOP_STAGED        the warp gathers its 32 records cooperatively
 *                        through shared memory (cp.async, double-buffered);
 *   HR_HOP_STAGED_TIGHT  the staged kernel at a smaller register budget
 *                        (D_R > 4 only);
 *   HR_HOP_STAGED_LINKS  the staged kernel with the link records staged
 *                        through shared memory as well;
 *   HR_HOP_MRHS          for nrhs >= 2: a block of 4 right-hand sides shares
 *                        each loaded link record (a9).
 * FP64 and DF64 have the direct variant only.  Launches are identified by
 * their epilogue: HR_EPI_STORE (out = a H in), HR_EPI_STORE_NORM (the same
 * plus |out|^2), HR_EPI_CG_UPDATE (the fused r -= alpha A p, x += alpha p,
 * |r|^2 of a CG iteration). */
enum { HR_HOP_DIRECT = 0, HR_HOP_STAGED = 1, HR_HOP_STAGED_TIGHT = 2, HR_HOP_STAGED_LINKS = 3,
       HR_HOP_MRHS = 4 };
enum { HR_EPI_STORE = 0, HR_EPI_STORE_NORM = 1, HR_EPI_CG_UPDATE = 2 };

/* Times every compiled variant of every epilogue in precision prec for g's
 * lattice, current link mode and nrhs right-hand sides, on zero-filled
 * scratch fields that it allocates and frees, and records the fastest in g;
 * later launches with that (prec, link mode, epilogue, nrhs == 1 or > 1) use
 * the record.  In HR_LINKS_AUTO mode it does so for both link modes and
 * keeps, for prec, the mode whose best kernels make one CG iteration (two
 * stores, a store with |out|^2 and a fused update) faster.  BLOCKS the calling thread.  hr_cg_solve and
 * hr_cg_solve_batched call it for their inner precision when no record
 * exists yet, unless autotuning is switched off with hr_gauge_set_tuning.
 * Errors: HR_ERR_INVALID (precision not stored), HR_ERR_NOMEM, HR_ERR_CUDA. */
hr_status hr_tune(hr_gauge *g, hr_prec prec, int nrhs, void *stream);

/* autotune: 1 (default) lets the solvers tune before their first iteration
 * in a precision, 0 never tunes implicitly.  variant: -1 (default) uses the
 * tuned record, or a fixed default where none exists; HR_HOP_* forces that
 * variant for every launch on g (clamped to the variants compiled for a
 * precision), which is how the variants are compared. */
hr_status hr_gauge_set_tuning(hr_gauge *g, int autotune, int variant);

/* The variant a launch on g would use now; -1 for bad arguments. */
int hr_gauge_hop_variant(const hr_gauge *g, hr_prec prec, int epilogue, int nrhs);

/* ------------------------------------------------------------------ */
/* Field helpers                                                         */
/* ------------------------------------------------------------------ */
/* Bytes of a field of nrhs right-hand sides over the sites selected by par
 * (V/2 for EVEN/ODD/EO_PRECOND, V for FULL) in precision prec. */
size_t hr_field_bytes(const hr_lattice_desc *lat, hr_parity par, hr_prec prec,
                      int nrhs);

/* Converts a field between precisions (F64/F32 <-> F16/BF16 computes the
 * per-site scales).  src and dst must not overlap. */
hr_status hr_field_convert(const hr_lattice_desc *lat, hr_parity par,
                           hr_prec src_prec, const void *src,
                           hr_prec dst_prec, void *dst, int nrhs, void *stream);

/* <a, b> = sum conj(a_i) b_i over each right-hand side, accumulated with
 * compensated (double-double) sums (Sec. 4.1.1).  par: HR_EVEN, HR_ODD or
 * HR_EO_PRECOND (V/2 sites) or HR_FULL (V sites); other values give
 * HR_ERR_INVALID.  out is a HOST array of 2*nrhs doubles (re, im); the call
 * synchronises the stream. */
hr_status hr_field_dot(const hr_lattice_desc *lat, hr_parity par, hr_prec prec,
                       const void *a, const void *b, int nrhs, double *out,
                       void *stream);

/* hr_field_dot without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * -- e.g. when another allocator owns the device memory, or on a path that
 * cannot take the implicit synchronisation of cudaMalloc/cudaFree -- while
 * hr_field_dot takes its reduction scratch from cudaMallocAsync.
 * Same arguments as hr_field_dot (every precision and representation it
 * accepts); additionally nrhs must be 1..16 (HR_ERR_INVALID otherwise).  The
 * result equals hr_field_dot's up to rounding: both sum in FP64 with
 * compensated cross-block sums, but the summation order differs (a fixed
 * number of blocks, each thread summing several sites with TwoSum).  Its
 * scratch is a fixed ~312 KB array in device memory, present on every GPU
 * that loads the library until the process exits; every call shares it and
 * it keeps the last call's contents (each call zeroes the tickets it needs
 * first).  Calls that overlap on the GPU race on that array, so order them
 * on one stream.  The first call on a device looks up the array's device
 * address with that device current; make that first call before any stream
 * capture on the device.
 * Synchronises the stream. */
hr_status hr_field_dot_static(const hr_lattice_desc *lat, hr_parity par,
                              hr_prec prec, const void *a, const void *b,
                              int nrhs, double *out, void *stream);

/* ------------------------------------------------------------------ */
/* Wilson-Dirac operator (Eq. D_m^R in Sec. 2.3; Sec. 4.3.3)              */
/* ------------------------------------------------------------------ */
/* D_m psi(x) = (4+m) psi(x) - 1/2 sum_mu [(1 - g_mu) U_R(x,mu) psi(x+mu)
 *                                  + (1 + g_mu) U_R(x-mu,mu)^dag psi(x-mu)]
 * with the gamma basis of Sec. 2.2.  out_par selects the block (see
 * hr_parity).  in and out hold nrhs fields in precision prec; in and out
 * must not overlap; for HR_EO_PRECOND the handle's workspace holds the
 * intermediate odd field, so concurrent calls on one handle must be
 * stream-ordered.
 * Errors: HR_ERR_INVALID (null pointers, nrhs < 1, prec not in prec_mask). */
hr_status hr_dirac_apply(const hr_gauge *g, hr_parity out_par, hr_prec prec,
                         const void *in, void *out, int nrhs, void *stream);

/* The adjoint D_m^dag (= gamma5 D_m gamma5, Eq. Q_m), same blocks and
 * arguments: EVEN gives (D^dag)_eo = (D_oe)^dag, EO_PRECOND gives Dhat^dag. */
hr_status hr_dirac_dagger(const hr_gauge *g, hr_parity out_par, hr_prec prec,
                          const void *in, void *out, int nrhs, void *stream);

/* ------------------------------------------------------------------ */
/* Conjugate gradient on the normal equations (Sec. 4.1.2, Sec. 4.3.3)    */
/* ------------------------------------------------------------------ */
typedef struct {
    double tol_rel;       /* stop when |b - A x| / |b| <= tol_rel (true residual) */
    int max_iter;         /* total inner iterations allowed */
    hr_prec inner;        /* HR_F64: plain FP64 CG; F32/F16/BF16: FP64 defect
                             correction around an inner CG in that precision */
    double inner_tol;     /* relative reduction asked of each inner solve */
    int use_initial_guess;/* 1: x holds the start vector; 0: start from 0 */
    hr_prec residual;     /* arithmetic of the defect-correction true residuals
                             (inner != HR_F64 only): HR_F64 (0, the default) or
                             HR_DF64, float-float with the handle's DF64 links,
                             which must be stored.  With HR_DF64 the
                             intermediate residuals are float-float; the one
                             the last inner solve is expected to bring within
                             tol_rel, and any float-float one that meets it,
                             are formed in FP64, so the reported
                             true_rel_residual is always an FP64 one. */
} hr_cg_params;

typedef struct {
    int iters;                 /* inner (or plain) CG iterations */
    int outer_iters;           /* defect-correction steps (0 for plain FP64) */
    double true_rel_residual;  /* |b - A x| / |b| recomputed in FP64 */
    hr_status status;
} hr_cg_result;

/* Solves A x = b with A = D_m^dag D_m (sys = HR_FULL, FULL fields) or
 * A = Dhat^dag Dhat (sys = HR_EO_PRECOND, even half fields).  b and x are
 * FP64 fields of nrhs right-hand sides; res is a HOST array of nrhs results.
 * The gauge handle must hold F64 links, and the inner precision's links
 * when params->inner != HR_F64.  BLOCKS the calling thread until every
 * right-hand side has converged or failed.
 * With a clover term (hr_gauge_set_clover) or for a colour-parallel pair
 * (N >= 5, SU(4) ADJ and SYM) the solve runs on
 * the multi-shift engine with the single shift 0 (same CG iterates; inner
 * FP64 or FP32, x started from 0, FP64 residuals).
 * Errors: HR_ERR_NOT_CONVERGED (x holds the last iterate),
 *         HR_ERR_NONFINITE, HR_ERR_INVALID, HR_ERR_NOMEM, HR_ERR_CUDA. */
hr_status hr_cg_solve(const hr_gauge *g, hr_parity sys, const void *b,
                      void *x, int nrhs, const hr_cg_params *params,
                      hr_cg_result *res, void *stream);

/* Solves n_inst independent systems (different lattices, masses and
 * right-hand-side counts; all with the same N and representation) together:
 * every iteration of all unconverged instances is one CUDA-graph launch.
 *   g[i], b[i], x[i], nrhs[i]  as in hr_cg_solve for instance i
 *   res  HOST array of sum(nrhs) results, instance-major.
 * BLOCKS until all instances finish. */
hr_status hr_cg_solve_batched(int n_inst, const hr_gauge *const *g,
                              hr_parity sys, const void *const *b,
                              void *const *x, const int *nrhs,
                              const hr_cg_params *params, hr_cg_result *res,
                              void *stream);

/* The fermion force of S_f = b^dag A^{-1} b in one call (the HMC force step,
 * Sec. 2.5 with the solve of Sec. 4.1.2): solves A x = b as hr_cg_solve with
 * one right-hand side, then F += coeff * dS/dU with Y = D x (sys = HR_FULL)
 * or Y = Dhat x (HR_EO_PRECOND), exactly as hr_dirac_force(g, sys, x, Y,
 * coeff, F).  The operator applications the force needs (D x, and for the
 * even/odd system D_oe x and (D^dag)_oe Dhat x) are those of the solve's
 * final FP64 true residual, kept instead of recomputed.
 *   Y  optional DEVICE output of D x / Dhat x (NULL: not returned).
 * The handle needs stored FP64 links.  With params->residual = HR_DF64
 * the force kernel runs in float-float on the stored DF64 links
 * (hr_dirac_force_prec with HR_DF64); otherwise in FP64.  F is left
 * unchanged if the solve fails (its status is returned).  BLOCKS like
 * hr_cg_solve. */
hr_status hr_cg_solve_force(const hr_gauge *g, hr_parity sys, const void *b,
                            void *x, const hr_cg_params *params,
                            hr_cg_result *res, void *Y, double coeff,
                            void *F, void *stream);

/* Multi-shift CG (Sec. 4.1.2, Supported Inverters; Sec. 4.3.2, the RHMC's
 * (Q^2 + beta_k)^{-1} phi for every pole beta_k): solves
 *     (A + shifts[k]) x_k = b        for k = 0 .. nshift-1
 * with A = D_m^dag D_m (sys = HR_FULL, FULL fields) or Dhat^dag Dhat
 * (HR_EO_PRECOND, even half fields), all shifts in one Krylov space.
 *   b       DEVICE, FP64 fields of nrhs right-hand sides [nrhs][sites][4][D]
 *   x       DEVICE, FP64 output [nshift][nrhs][sites][4][D] (shift-major);
 *           overwritten, must not overlap b
 *   shifts  HOST array of nshift finite values >= 0, in any order (the
 *           smallest is the base system); 1 <= nshift <= 64,
 *           nrhs * nshift <= 4096
 *   params  tol_rel: every shift stops at |b - (A + shifts[k]) x_k| / |b|
 *           <= tol_rel, recomputed in FP64.  inner = HR_F64: FP64
 *           iterations; HR_F32: FP32 iterations to max(inner_tol, tol_rel),
 *           then FP64 defect correction of each shift by single-shift FP32
 *           solves of all unconverged shifts together.  max_iter bounds the
 *           multi-shift iterations and, separately, the correction
 *           iterations.  use_initial_guess must be 0 and residual HR_F64.
 *   res     HOST array [nshift][nrhs]: iters = iterations until the shift
 *           met its tolerance plus its correction iterations; outer_iters =
 *           corrections; true_rel_residual in FP64; status.
 * The handle needs FP64 links and those of the inner precision.  BLOCKS
 * until every shift has converged or failed.
 * Errors: HR_ERR_NOT_CONVERGED, HR_ERR_NONFINITE (a non-positive or
 * non-finite reduction), HR_ERR_INVALID, HR_ERR_NOMEM, HR_ERR_CUDA. */
hr_status hr_cg_solve_multishift(const hr_gauge *g, hr_parity sys,
                                 const void *b, void *x, int nrhs,
                                 const double *shifts, int nshift,
                                 const hr_cg_params *params,
                                 hr_cg_result *res, void *stream);

/* y = a0 b + sum_k a[k] x_k over FP64 fields of parity par: with the
 * multi-shift solutions x_k = (A + b_k)^{-1} b this is the RHMC's rational
 * function r(A) b = a0 b + sum_k a_k (A + b_k)^{-1} b (Sec. 4.3.2).
 *   b, y  DEVICE [nrhs][sites][4][D]; y may be b, must not overlap x
 *   x     DEVICE [nterms][nrhs][sites][4][D] (hr_cg_solve_multishift's layout)
 *   a     HOST array of nterms doubles; 0 <= nterms <= 64
 * Asynchronous on stream. */
hr_status hr_field_lincomb(const hr_lattice_desc *lat, hr_parity par,
                           double a0, const void *b, int nterms,
                           const double *a, const void *x, void *y, int nrhs,
                           void *stream);

/* RHMC rational approximation (Sec. 4.3.2: the rational functions of Q^2
 * whose poles become the multi-shift CG's shifts, with coefficients from the
 * Remez algorithm): the best relative approximation of degree (n, n),
 *     r(x) = a0 + sum_k res[k] / (x + poles[k])  ~  x^(-alpha)  on [lo, hi],
 * i.e. the one minimising max |r(x) x^alpha - 1|, found by a Remez exchange
 * (the error levelled on 2n + 2 alternating reference points by Newton's
 * method on the factored form, then the reference moved to the error's
 * extrema, with continuation in the degree).  Powers: alpha = 1/2 for the
 * one-flavour action and force ((Q^2)^(-1/2)), alpha = -1/4 for its heat
 * bath ((Q^2)^(1/4)), and any other 0 < |alpha| < 1.
 *   n          1..64
 *   0 < lo < hi  the interval (it must contain the spectrum of A)
 *   a0, max_rel_err  HOST doubles; res, poles  HOST arrays of n doubles,
 *              poles ascending and positive (pass them as the shifts of
 *              hr_cg_solve_multishift, then a0 and res to hr_field_lincomb)
 *   max_rel_err  max |r(x) x^alpha - 1| over [lo, hi] (evaluated in FP64;
 *              near 1e-13 the evaluation's rounding floor)
 * Host computation only (no GPU work, no stream).
 * Errors: HR_ERR_INVALID; HR_ERR_NOT_CONVERGED if the exchange cannot level
 * the error (a degree beyond what FP64 resolves on [lo, hi]). */
hr_status hr_rational_approx(double alpha, int n, double lo, double hi,
                             double *a0, double *res, double *poles,
                             double *max_rel_err);

/* ------------------------------------------------------------------ */
/* HMC building blocks (Sec. 2.4, Sec. 2.5, Sec. 4.2)                    */
/* ------------------------------------------------------------------ */
/* Conventions (Sec. 2.5): H = H_pi + S_g + S_f, H_pi = T_F/2 sum pi^2
 * (T_F = 1/2), dU/dtau = pi U with pi = i pi^a T^a, dpi^a/dtau = F^a =
 * -(1/T_F) dS/de^a, dS/de^a the derivative along exp(i e T^a) U_mu(x).
 * U_fund: DEVICE FP64 [V][4][N][N] complex (the layout of
 * hr_represent_gauge), periodic in every direction.  pi and forces: DEVICE
 * FP64 [V][4][N*N-1].  N = 2, 3 or 4. */

/* S_g = beta sum_{x, mu<nu} (1 - Re tr P_{mu nu}(x) / N), the Wilson action
 * of the plaquette P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag
 * U_nu(x)^dag (Eq. plaquette).  *S is a HOST double; synchronises stream. */
hr_status hr_gauge_action(const hr_lattice_desc *lat, const void *U_fund,
                          double beta, double *S, void *stream);

/* F[x][mu][a] += coeff * dS_g/de^a = coeff * (-(beta/N)) Re tr(i T^a
 * U_mu(x) W_mu(x)), W the sum of the six staples; coeff = -1/T_F gives the
 * gauge force F_G of Sec. 2.5, coeff = -h/T_F a momentum step of length h. */
hr_status hr_gauge_force(const hr_lattice_desc *lat, const void *U_fund,
                         double beta, double coeff, double *F, void *stream);

/* U_mu(x) <- exp(i eps pi^a(x,mu) T^a) U_mu(x) for every link (the gauge
 * step of Hamilton's equations, Sec. 2.5). */
hr_status hr_link_update(const hr_lattice_desc *lat, void *U_fund,
                         const double *pi, double eps, void *stream);

/* *H = T_F/2 sum pi^2 (HOST double; synchronises stream). */
hr_status hr_momenta_energy(const hr_lattice_desc *lat, const double *pi,
                            double *H, void *stream);

typedef enum { HR_MD_LEAPFROG = 0, HR_MD_OMELYAN2 = 1 } hr_md_integrator;

typedef struct {
    double beta;                 /* Wilson gauge coupling */
    double tau;                  /* trajectory length */
    int nsteps;                  /* integration steps */
    hr_md_integrator integrator; /* PQP, or P(l h) Q(h/2) P((1-2l)h) Q(h/2)
                                    P(l h) with l = 0.1931833... (Sec. 4.2) */
    hr_parity sys;               /* fermion action phi^dag A^-1 phi with
                                    A = Dhat^dag Dhat (HR_EO_PRECOND, phi
                                    even) or D^dag D (HR_FULL) */
    hr_cg_params cg;             /* the fermion-force solves */
} hr_md_params;

typedef struct {
    int force_evals;               /* fermion force evaluations */
    int cg_iters;                  /* summed over them */
    double max_true_rel_residual;  /* worst force solve */
    hr_status status;
} hr_md_stats;

/* One molecular-dynamics trajectory of length tau: updates U_fund and pi in
 * place, and leaves g representing the new U_fund.  phi (DEVICE pseudofermion,
 * FP64 field of sys) may be NULL for the pure gauge theory; otherwise g must
 * hold stored FP64 links (and those of p->cg.inner) and each momentum step
 * runs hr_cg_solve_force.  Adjacent momentum steps are merged (leapfrog
 * takes nsteps + 1 force evaluations, Omelyan 2 nsteps + 1).  BLOCKS. */
hr_status hr_md_trajectory(hr_gauge *g, void *U_fund, double *pi,
                           const void *phi, const hr_md_params *p,
                           hr_md_stats *stats, void *stream);

typedef struct {
    double H0[3], H1[3];   /* (H_pi, S_g, S_f) before and after the trajectory */
    double dH;             /* sum(H1) - sum(H0) */
    int accepted;          /* 1 if u_accept < exp(-dH) */
    hr_md_stats md;        /* the trajectory's statistics */
} hr_hmc_result;

/* One HMC update (Sec. 2.5): the pseudofermion heat bath phi = Dhat^dag eta
 * (D^dag eta for sys = HR_FULL), H = H_pi + S_g + S_f before, one MD
 * trajectory (hr_md_trajectory), H after, and the Metropolis test: the new
 * links are kept if u_accept < exp(-dH), otherwise U_fund is restored.  The
 * random draws are the caller's:
 *   pi        DEVICE heat-bath momenta pi^a ~ N(0, 1/T_F) (FP64 [V][4][N*N-1]);
 *             on return the trajectory's final momenta
 *   eta       DEVICE complex Gaussian field of p->sys (FP64, Re and Im each
 *             N(0, 1/2)); NULL for the pure gauge theory
 *   u_accept  uniform draw in [0, 1) (any finite value >= 1 rejects: a
 *             forced rejection)
 * S_f = phi^dag A^-1 phi is formed by a solve (p->cg with the tolerance
 * min(p->cg.tol_rel, 1e-11)) and hr_field_dot, before and after.  g
 * represents U_fund on return, accepted or not.  Takes device scratch for a
 * copy of U_fund and two fields (cudaMallocAsync on stream).  BLOCKS.
 * Errors: those of the calls it makes; HR_ERR_INVALID for bad arguments. */
hr_status hr_hmc_update(hr_gauge *g, void *U_fund, double *pi, const void *eta,
                        double u_accept, const hr_md_params *p,
                        hr_hmc_result *res, void *stream);

/* ------------------------------------------------------------------ */
/* Fermion force (Sec. 2.5)                                              */
/* ------------------------------------------------------------------ */
/* F[x][mu][a] += coeff * d/de S(U_F(x,mu) -> exp(i e T^a) U_F(x,mu)) at e=0
 * with X, Y held fixed, where
 *   sys = HR_FULL:        S = -2 Re <Y, D_m X>      (X, Y FULL FP64 fields)
 *   sys = HR_EO_PRECOND:  S = -2 Re <Y, Dhat X>     (X, Y even FP64 fields)
 * For X = A^{-1} phi and Y = D X (resp. Dhat X) this is the derivative of
 * S_f = phi^dag A^{-1} phi.  The derivative reaches the fundamental link
 * through dU_R = i e T_R^a U_R (T_R^a the generators in representation R).
 * F is a device array of V*4*(N*N-1) doubles. */
hr_status hr_dirac_force(const hr_gauge *g, hr_parity sys, const void *X,
                         const void *Y, double coeff, void *F, void *stream);

/* hr_dirac_force with a choice of arithmetic for the force kernel:
 *   arith = HR_F64   FP64 on the stored FP64 links (hr_dirac_force);
 *   arith = HR_DF64  float-float (about 48 significant bits) on the stored
 *                    DF64 links, which g must hold: the FP64 spinors are
 *                    projected in FP64 and split into float-float pairs, the
 *                    matrix products run on the FP32 units, and F (FP64) is
 *                    accumulated in FP64.  Each component agrees with the
 *                    FP64 force to about 1e-14 of max |F|.
 * The hops that form D_oe X and (D^dag)_oe Y for sys = HR_EO_PRECOND are
 * FP64 in both cases.  HR_ERR_INVALID for another arith or missing links. */
hr_status hr_dirac_force_prec(const hr_gauge *g, hr_parity sys, const void *X,
                              const void *Y, double coeff, void *F,
                              hr_prec arith, void *stream);

/* ------------------------------------------------------------------ */
/* Introspection                                                         */
/* ------------------------------------------------------------------ */
/* Dimension D_R of a representation (Table 1); -1 if unsupported. */
int hr_rep_dim(int N, hr_rep rep);
/* Writes the (N*N-1) generators T^a (Tr T^a T^b = delta/2) as complex double
 * [(N*N-1)][N][N] into the HOST array T. */
hr_status hr_generators(int N, double *T);
const char *hr_status_string(hr_status s);
const char *hr_last_error(void);
/* Number of kernel launches this library has issued in this process. */
unsigned long long hr_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* HR_H */
