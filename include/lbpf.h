/*
 * lbpf.h — C ABI of libgb_lbpf: the coupled phi-mu lattice Boltzmann time step
 * of the grand-potential phase-field model of dissolution and precipitation
 * (Boutin, Verdier & Cartalade, arXiv 2111.05960), on one GB300 GPU (sm_103a).
 *
 * What one time step computes (Sec. 3, in this order, all in lattice units):
 *   - closure mu = mu_eq + c - c^co(phi), c^co = c_l^co phi + c_s^co (1 - phi)
 *     (Eq. PotChim_Equilibirum, Eq. Coexistence_Interpol, h(phi) = phi);
 *   - grad(phi) by directional derivatives (Eq. DerivDirec_Grad, Eq. Grad) and
 *     the unit normal n = grad / sqrt(|grad|^2 + eps_n^2) (Eq. NormalVector);
 *   - the phi source G_k (Eq. TermG) with S_phi of Eq. SourceTerm_Coexistence and
 *     either the double-well term (Eq. SourceG_dw) or the counter term that
 *     cancels curvature-driven motion (Eq. SourceG_CT);
 *   - BGK collision and streaming of the phi populations (Eq. LBE_PhaseField_Eq,
 *     g^eq = w_k phi, Eq. Geq_Allen-Cahn_Eq-1), new phi (Eq. Moment_Phi);
 *   - dphi/dt by explicit Euler, anti-trapping current
 *     j_at = a W (c_s^co - c_l^co) dphi/dt n (Eq. Anti-trapping_Equilibrium);
 *   - the composition source H_k = gamma w_k e_k.(mu D' grad phi + j_at)
 *     (Eq. SourceTerm_LBE_h), equilibrium h^eq (Eq. Heq_Composition), BGK
 *     collision and streaming (Eq. LBE_Composition), c = sum_k h_k
 *     (Eq. Moment0_LBM_Concent).
 * Two variants of the composition scheme named in Sec. 3 are selectable: the
 * alternative equilibrium h^eq,alt that carries the flux with H_k = 0
 * (Eq. LBE_Concent_Alt, Eq. Seq_Concent_Alt), and h on the small lattice of the
 * paper's code (D2Q5 / D3Q7, Sec. 3.1) while g keeps D2Q9 / D3Q19.  The
 * free energies may also be parabolas of unequal curvature (Sec. 2.3:
 * Eq. Closure, Eq. SourceTerm, Eq. Anti-Trapping_Quadratic).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an lbpf_status and never throws across the ABI.
 *   - Fields crossing the ABI are FP64, row-major [nz][ny][nx] (x fastest),
 *     whatever the internal precision.  ptr_is_device = 0: host memory (any
 *     alignment; pinned memory makes the copies faster); 1: device memory of
 *     the context's GPU, 8-byte aligned.
 *   - The caller owns every array it passes; lbpf_create copies them.  The
 *     context owns its populations, fields and scratch; lbpf_destroy frees them.
 *   - Work is queued on the CUDA stream given at creation (NULL = legacy default
 *     stream).  lbpf_step returns once the kernels are queued; lbpf_mass,
 *     lbpf_get_fields and lbpf_get_populations synchronise that stream.  On a
 *     non-default stream, lbpf_step replays two steps captured once as a CUDA
 *     graph (when every step has the same kernels: mass_every <= 1); the first
 *     call that captures must not itself run inside another capture.
 *   - One context must not be used by two threads at once.
 *   - After LBPF_EUNSTABLE the context is poisoned: every later call except
 *     lbpf_last_error, lbpf_get_step and lbpf_destroy returns LBPF_ESTATE.
 */
#ifndef LBPF_H
#define LBPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBPF_OK = 0,
    LBPF_EINVAL = 1,      /* bad argument or parameter; nothing changed */
    LBPF_ENOMEM = 2,      /* device allocation failed; nothing leaked */
    LBPF_ECUDA = 3,       /* a CUDA call failed; message in lbpf_last_error */
    LBPF_EUNSTABLE = 4,   /* non-finite field or phi far outside [0, 1] */
                          /* 5 is unused: no kernel of this library waits on
                             another block, stream or device, so no call times out */
    LBPF_ESTATE = 6,      /* context poisoned by an earlier error */
    LBPF_EUNSUPPORTED = 7 /* option combination not built */
} lbpf_status;

/* Lattices of g (and by default of h): D2Q9, D3Q19.  D2Q5 and D3Q7 only carry
 * h (lbpf_params.h_lattice = 1) and are listed for lbpf_lattice_info. */
typedef enum { LBPF_D2Q9 = 0, LBPF_D3Q19 = 1, LBPF_D2Q5 = 2, LBPF_D3Q7 = 3 } lbpf_lattice;

/* Storage and arithmetic of the populations and fields.  FP64: all FP64.
 * FP32: FP32 storage and arithmetic.  The *DEV modes store each population as a
 * 16-bit deviation from its equilibrium (g^eq = w_k phi, h^eq of
 * Eq. Heq_Composition) and compute in FP32.  Mass sums are FP64 in every mode. */
typedef enum {
    LBPF_FP64 = 0,
    LBPF_FP32 = 1,
    LBPF_FP32_BF16DEV = 2,
    LBPF_FP32_FP16DEV = 3
} lbpf_precision;

typedef enum { LBPF_PERIODIC = 0, LBPF_BOUNCEBACK = 1 } lbpf_bc;

/* Model parameters.  With dx = dt = 1 everything is in lattice units; otherwise
 * W is a length and D_l, D_s are diffusivities in the same physical units, and
 * the library converts them (W/dx, D dt/dx^2).  The relaxation times are the
 * dimensionless tau-bar of Sec. 3.1:
 *   M_phi = tau_g dx^2 / (3 dt)           (Sec. 3.2)
 *   gamma = 3 dt / (tau_h dx^2)            (Sec. 3.3, Tab. 4)            */
typedef struct {
    int32_t nx, ny, nz;          /* nodes per axis; nz = 1 selects 2-D */
    int32_t lattice;             /* lbpf_lattice: D2Q9 needs nz == 1, D3Q19 nz >= 1 */
    int32_t bc[3];               /* lbpf_bc per axis (x, y, z); walls are half-way
                                    bounce-back with mirror ghosts for grad(phi) */
    int32_t precision;           /* lbpf_precision */
    double dx, dt;               /* 1, 1 for lattice units */
    double tau_g, tau_h;         /* > 0 */
    double W;                    /* interface width, > 0 */
    double lambda;               /* coupling constant of Eq. SourceG_ST */
    double D_l, D_s;             /* diffusivities of liquid and solid, >= 0 */
    double c_s_co, c_l_co;       /* coexistence compositions */
    double mu_eq;                /* equilibrium chemical potential */
    int32_t counter_term;        /* 1: counter term G^ct; 0: double-well G^dw */
    int32_t anti_trapping;       /* 1: j_at included in H_k */
    double a_at;                 /* a of j_at; < 0 selects (1 - D_s/D_l)/4 */
    double eps_n;                /* regularisation of |grad phi| in n; default 1e-12 */
    int32_t mass_every;          /* steps between FP64 mass corrections, 0 = off (see
                                    lbpf_solute_mass); FP32 and 16-bit modes want 1 */
    int32_t checkpoint_every;    /* 0: no adjoint; k > 0: record the state every k
                                    steps for lbpf_adjoint_step (FP64 and FP32 only) */
    int32_t h_lattice;           /* 0: h on the lattice of g; 1: h on the small lattice,
                                    D2Q5 with D2Q9 or D3Q7 with D3Q19 (Sec. 3.1), weights
                                    1/3, 1/6 and 0, 1/6 so that xi_s^2 = 1/3 and
                                    tau_h = 3 dt / (gamma dx^2) still hold */
    int32_t h_eq_alt;            /* 0: h^eq with the source H_k (Eq. Heq_Composition,
                                    Eq. SourceTerm_LBE_h); 1: the alternative
                                    equilibrium h^eq,alt_k = w_k [gamma D mu + e_k.F /
                                    xi_s^2] with H_k = 0 (Eq. Seq_Concent_Alt), F = mu D'
                                    grad phi + j_at */
    int32_t unequal_eps;         /* 0: parabolas of equal curvature (the closure and
                                    sources above); 1: curvature ratio eps_ratio, with
                                    e_s = sqrt(eps_ratio), e_l = 1/e_s:
                                      mu = [c - m_l phi - m_s (1-phi)] / [e_s phi + e_l (1-phi)]
                                      S_phi = p'(phi) [(e_l-e_s) mu^2/2 - (m_l-m_s) mu - df]
                                      j_at = a W [(e_l-e_s) mu + m_s - m_l] dphi/dt n
                                    where m_l = c_l^co - e_s mu_eq, m_s = c_s^co - e_l mu_eq
                                    and df = (e_l-e_s) mu_eq^2/2 - (m_l-m_s) mu_eq (equal
                                    chemical potentials at c_s^co, c_l^co and equal grand
                                    potentials at mu_eq, Sec. 2.3.2) */
    double eps_ratio;            /* eps_s / eps_l (> 0) when unequal_eps = 1 */
} lbpf_params;

typedef struct lbpf_ctx lbpf_ctx;

/* Fill *p with defaults: 2-D D2Q9 64x64 periodic, FP64, dx = dt = 1,
 * tau_g = tau_h = 0.36, W = 3, lambda = 0, D_l = D_s = 0.1, c_s^co = 1,
 * c_l^co = 0.5, mu_eq = 0.4, counter term on, anti-trapping off, a = -1 (auto),
 * eps_n = 1e-12, h on the lattice of g with H_k (h_lattice = h_eq_alt = 0),
 * equal curvatures (unequal_eps = 0, eps_ratio = 1).
 * Returns LBPF_EINVAL if p is NULL. */
lbpf_status lbpf_default_params(lbpf_params *p);

/* Create a context on the current CUDA device: validate p, allocate the
 * populations (two ping-pong sets of g and h, SoA [k][z][y][x]) and the fields
 * phi^n, phi^{n+1}, c^n, c^{n+1}, copy phi0 and c0 (FP64, [nz][ny][nx]) and set
 * the populations to g_k = w_k phi0 - G_k/2 and h_k = h^eq_k - H_k/2 (the
 * variable change of Sec. 3.1 at equilibrium, H at dphi/dt = 0), or
 * h_k = h^eq,alt_k with h_eq_alt = 1.
 * cuda_stream: a cudaStream_t (NULL = default stream).  On success *out owns
 * everything; on failure *out is NULL and nothing is leaked.
 * Errors: EINVAL (NULL pointers, sizes < 1, nz != 1 for D2Q9, a bounce-back
 * axis with fewer than 2 nodes, tau <= 0, W <= 0, D < 0, unknown enum,
 * h_lattice, h_eq_alt or unequal_eps not 0 / 1, eps_ratio <= 0), ENOMEM,
 * ECUDA, EUNSUPPORTED (checkpoint_every > 0 with h_lattice, h_eq_alt or
 * unequal_eps set: the adjoint covers the main scheme only). */
lbpf_status lbpf_create(const lbpf_params *p, const double *phi0, const double *c0,
                        int32_t ptr_is_device, void *cuda_stream, lbpf_ctx **out);

/* Queue nsteps coupled time steps (n -> n + nsteps) on the context's stream:
 * each step is the sequence of Sec. 3 listed at the top of this header (the phi
 * LBE of Sec. 3.2, then the composition LBE of Sec. 3.3 with dphi/dt from this
 * step's phi), followed by the FP64 mass correction when mass_every divides the
 * step count.  nsteps >= 0.  Errors: EINVAL, ECUDA (launch failure), ESTATE. */
lbpf_status lbpf_step(lbpf_ctx *ctx, int64_t nsteps);

/* Total solute sum_x c and phase sum_x phi, accumulated in FP64 on the GPU
 * (deterministic two-pass block reduction), copied to the host pointers
 * (either may be NULL).  Synchronises the stream.  Returns LBPF_EUNSTABLE and
 * poisons the context if a field value is non-finite or phi leaves
 * [-0.5, 1.5]. */
lbpf_status lbpf_mass(lbpf_ctx *ctx, double *total_c, double *total_phi);

/* Exact solute mass of the current state: the sum over nodes and directions of
 * the h populations (their zeroth moment, Eq. Moment0_LBM_Concent), accumulated
 * without rounding loss in FP64 (deviation modes add their references back).
 * With mass_every > 0, *target (optional) receives the mass the correction
 * holds: the exact population mass right after creation; else NaN.
 *
 * Mass correction (a build addition; the paper's FP64-free scheme has none):
 * FP32 arithmetic rounds each collision at ~1e-7 relative, and nodes sitting on
 * a binade boundary (c = 1 in the solid) round asymmetrically, so the total
 * solute drifts by ~1e-9 per step.  With mass_every = k > 0, every k-th step the
 * composition kernel also sums the exact mass it wrote (one FP64 value per
 * block), a one-block kernel compares it with the target in FP64, and a third
 * kernel adds the difference back to h_0 and c on a rotating subset of nodes
 * (about 1e-5 per node, so each node's rounding is ~1% of it).  The next
 * measurement sees any residual, so errors do not accumulate.  Synchronises. */
lbpf_status lbpf_solute_mass(lbpf_ctx *ctx, double *mass, double *target);

/* Copy phi, c and mu = mu_eq + c - c^co(phi) at the current step into FP64
 * arrays [nz][ny][nx] (any of them may be NULL).  Synchronises the stream. */
lbpf_status lbpf_get_fields(lbpf_ctx *ctx, double *phi, double *c, double *mu,
                            int32_t ptr_is_device);

/* Copy the populations g and h (post-streaming, before the next collision),
 * FP64 [q][nz][ny][nx]: g with q = 9 (D2Q9) or 19 (D3Q19), h with the q of its
 * lattice (9 / 19, or 5 / 7 with h_lattice = 1).  For the deviation-storage
 * modes the stored deviations are expanded back to full populations.  With
 * h_eq_alt = 0 the h returned are the shifted populations h~ of Sec. 3.3.
 * Either pointer may be NULL.  Synchronises the stream. */
lbpf_status lbpf_get_populations(lbpf_ctx *ctx, double *g, double *h, int32_t ptr_is_device);

/* Time the kernels of nsteps steps with CUDA events recorded on the context's
 * stream around each launch.  kernel_ms[0] accumulates the phi kernel,
 * kernel_ms[1] the composition kernel, kernel_ms[2] the mass-correction
 * kernels (0 when mass_every = 0), in milliseconds; kernel_ms has 3 entries.
 * Synchronises. */
lbpf_status lbpf_step_timed(lbpf_ctx *ctx, int64_t nsteps, double *kernel_ms);

/* How the context's step kernels read the populations they pull:
 * *tensor_maps = 1 when the copy engine brings each plane's rows of the links
 * with e_x = 0 into shared memory through tensor maps of the context's buffers
 * (the threads load the other links themselves), 0 when every thread loads all
 * of its own.  The tensor-map form is opt-in: the environment variable
 * LBPF_TMA=1 at creation, FP32 storage on D3Q19, every axis periodic, nx a
 * multiple of 4 and at least 32.  Its results are bit-identical to the load
 * form; it is slower on GB300 (1.31 against 1.02 ms per 256^3 step), so it is
 * not the default.  Needs no GPU work.
 * Errors: EINVAL (ctx or tensor_maps NULL). */
lbpf_status lbpf_pull_path(const lbpf_ctx *ctx, int32_t *tensor_maps);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (*tflops),
 * from a kernel of independent FMA chains on every SM (about a second of
 * work at 1 TFLOP/s scale), timed with CUDA events on cuda_stream (NULL =
 * default stream); synchronises it.  The FP64 step is bound by FP64
 * arithmetic rather than by memory on GPUs with a small FP64 rate, and this
 * is its roofline denominator.  The paper has no counterpart.
 * Errors: EINVAL (tflops NULL), ECUDA. */
lbpf_status lbpf_fp64_fma_rate(void *cuda_stream, double *tflops);

/* Lattice table of the population ordering used by lbpf_get_populations:
 * *q = 9, 19, 5 or 7; e (optional, int32 [q][3]) the link vectors; w
 * (optional, [q]) the weights.  D2Q9 follows Sec. 3.1 (e0 = 0, e1..e4 axis
 * links (1,0),(0,1),(-1,0),(0,-1), e5..e8 diagonals (1,1),(-1,1),(-1,-1),
 * (1,-1)); D2Q5 and D3Q7 are the first 5 / 7 links of D2Q9 / D3Q19.
 * Needs no GPU.  Errors: EINVAL for an unknown lattice or q == NULL. */
lbpf_status lbpf_lattice_info(int32_t lattice, int32_t *q, int32_t *e, double *w);

/* Batch of 2-D instances of uneven size in one context (a parameter sweep,
 * counter term on and off, ...), stepped together: each kernel phase is one
 * persistent launch over a flat list of row-marched tiles (BX columns x ROWS
 * rows, the shape picked by an autotuner at creation, see lbpf_batch_tile) of
 * all periodic instances, and one more over those of the instances with a
 * bounce-back axis (if any), so the work is balanced whatever the size mix.  p[i], phi0[i],
 * c0[i] describe instance i exactly as for lbpf_create (each with its own
 * sizes, walls and parameters); all instances must be D2Q9 with the same
 * precision, mass_every = 0, checkpoint_every = 0, h_lattice = h_eq_alt =
 * unequal_eps = 0
 * and 9 nx ny x (bytes per
 * stored value: 8 FP64, 4 FP32, 2 for 16-bit storage) < 2^31 (the kernels
 * address within an instance with 32-bit byte offsets).  The fields are copied;
 * ptr_is_device says where phi0[i] and c0[i] live.  lbpf_step,
 * lbpf_step_timed and lbpf_mass (sums over all instances) work on a batch;
 * lbpf_get_fields, lbpf_get_populations and lbpf_solute_mass return
 * LBPF_EUNSUPPORTED (use the calls below).
 * Errors: EINVAL (NULL pointers, n < 1, an invalid or oversized instance: the
 * message names it), EUNSUPPORTED (non-D2Q9 instance, mass_every != 0,
 * checkpoint_every != 0, h_lattice, h_eq_alt or unequal_eps != 0), ENOMEM,
 * ECUDA. */
lbpf_status lbpf_create_batch(const lbpf_params *p, int32_t n, const double *const *phi0,
                              const double *const *c0, int32_t ptr_is_device, void *cuda_stream,
                              lbpf_ctx **out);

/* Tile shape of a batch's step kernels: each persistent block walks tiles of
 * *tile_x columns x *tile_rows rows (row segments marched along y).  At
 * creation the library times one step with each built shape (32x32, 32x64,
 * 64x32, 64x64, 128x32) on the batch itself and keeps the fastest; the shape
 * changes the schedule only, never the results.  ms_per_step (optional, 5
 * doubles) receives the timed milliseconds per step of each shape in that
 * order.  Errors: EINVAL (NULL pointers, not a batch). */
lbpf_status lbpf_batch_tile(const lbpf_ctx *ctx, int32_t *tile_x, int32_t *tile_rows, double *ms_per_step);

/* Use one of the built tile shapes instead of the autotuned one.  Synchronises
 * the stream.  Errors: EINVAL (not a batch, or a shape that is not built),
 * ESTATE. */
lbpf_status lbpf_batch_set_tile(lbpf_ctx *ctx, int32_t tile_x, int32_t tile_rows);

/* Fields of instance i of a batch, as lbpf_get_fields (FP64 [ny][nx]). */
lbpf_status lbpf_batch_get_fields(lbpf_ctx *ctx, int32_t i, double *phi, double *c, double *mu,
                                  int32_t ptr_is_device);

/* Exact solute mass of every instance of a batch, as lbpf_solute_mass:
 * masses[i] for i < n (host memory).  Synchronises. */
lbpf_status lbpf_batch_solute_mass(lbpf_ctx *ctx, double *masses);

/* Largest n that lbpf_mass_noalloc accepts: 4096 blocks x 16384 elements. */
#define LBPF_NOALLOC_MAX_ELEMENTS 67108864LL

/* The sums of lbpf_mass (sum c, sum phi, count of bad nodes) over caller-owned
 * device arrays, without allocating anything.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, such as code
 * running inside a host callback where allocation is not allowed, a monitor that
 * must never block on the allocator, or an embedding runtime that owns all
 * device memory.
 *   c, phi      device arrays of n elements, FP64 (precision = LBPF_FP64) or FP32
 *               (precision = LBPF_FP32), e.g. fields from lbpf_get_fields.
 *   out_device  device array of 3 doubles: sum c, sum phi, and the number of
 *               elements that are non-finite or have phi outside [-0.5, 1.5].
 *   cuda_stream the stream the two kernels are queued on (NULL = default);
 *               the call returns without synchronising.
 * Scratch: a file-scope device array of 4096 x 3 doubles (96 KiB), present on
 * every GPU that loads the library until the process exits.  The first call in
 * each CUDA context (a device's primary context, a new one after
 * cudaDeviceReset, or a context the caller made current) looks up that array's
 * device address there (cudaGetSymbolAddress) and caches it under the
 * context's id, so make that first call before any stream capture.
 * Every call shares the array and leaves its partial sums in it; nothing in it
 * needs clearing, because each call overwrites the slots it reads.  Calls whose
 * kernels overlap on the GPU (other streams, other threads) race on the array
 * and must be serialised by the caller.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * Errors (message in lbpf_last_error(NULL)): EINVAL for NULL pointers, n < 0,
 * n > LBPF_NOALLOC_MAX_ELEMENTS or another precision; ECUDA. */
lbpf_status lbpf_mass_noalloc(const void *c, const void *phi, int64_t n, int32_t precision,
                              double *out_device, void *cuda_stream);

/* Number of parameter adjoints that lbpf_adjoint_step returns, in this order:
 * dL/dD_l, dL/dtau_g, dL/dtau_h, dL/dlambda, dL/da, dL/dD_s. */
#define LBPF_ADJ_NPARAMS 6

/* Discrete adjoint (reverse mode) of the whole trajectory since creation: the
 * gradient of a scalar loss L(phi_T, c_T) of the current fields with respect to
 * the initial fields and the parameters, exact for the discrete scheme (the
 * time step of Sec. 3 and the initialisation of lbpf_create, differentiated
 * by hand).  The paper does not differentiate its scheme; this makes the step a
 * differentiable layer.
 *   dL_dphi, dL_dc    FP64 [nz][ny][nx]: dL/dphi_T and dL/dc_T (NULL = zero).
 *   dL_dphi0, dL_dc0  FP64 [nz][ny][nx] outputs: dL/dphi0 and dL/dc0 (either
 *                     may be NULL).
 *   ptr_is_device     where those four arrays live (as for lbpf_get_fields).
 *   dL_dparams        host array of LBPF_ADJ_NPARAMS doubles, overwritten:
 *                     dL/dD_l, dL/dtau_g, dL/dtau_h, dL/dlambda, dL/da, dL/dD_s
 *                     in the units of lbpf_params (D_l, D_s physical when
 *                     dx, dt != 1).  When a_at < 0 selects a = (1 - D_s/D_l)/4,
 *                     the D_l and D_s entries include that dependence; dL/da is
 *                     the partial derivative at fixed D_l, D_s (0 without
 *                     anti-trapping).  The kinetic coefficient M_phi = tau_g/3
 *                     in lattice units, so dL/dM_phi = 3 dL/dtau_g.
 * Needs checkpoint_every = k > 0 at creation: the context then copies the
 * state (populations, fields, mass-correction state) every k steps.  The
 * sweep runs the segments in reverse: it restores a checkpoint, re-runs the
 * segment's forward steps into per-step storage (k + 1 states, allocated on the
 * first call and kept), then runs the adjoint steps back over it, three kernels
 * per step.  The mass correction (mass_every > 0) is replayed bit for bit and
 * treated as a constant shift (its derivative is not taken).  Parameter
 * adjoints are summed in FP64 in a fixed order (deterministic); the field
 * adjoints are computed in the context's precision.  The forward state is left
 * unchanged.  Synchronises the stream.
 * Errors: EINVAL (NULL ctx or dL_dparams), EUNSUPPORTED (checkpoint_every was
 * 0, a batch, or a 16-bit storage mode), ENOMEM, ECUDA, ESTATE. */
lbpf_status lbpf_adjoint_step(lbpf_ctx *ctx, const double *dL_dphi, const double *dL_dc,
                              double *dL_dphi0, double *dL_dc0, int32_t ptr_is_device,
                              double *dL_dparams);

/* Number of coupled steps taken since creation. */
lbpf_status lbpf_get_step(const lbpf_ctx *ctx, int64_t *step);

/* Free everything the context owns.  NULL-safe; returns LBPF_OK. */
lbpf_status lbpf_destroy(lbpf_ctx *ctx);

/* Last error message of ctx, or of the calling thread when ctx is NULL. */
const char *lbpf_last_error(const lbpf_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBPF_H */
