/*
 * sfrd.h -- C ABI of the GB300 (sm_103a) compact-MTT ETDRK4-P13 solver for
 * space-fractional reaction-diffusion equations (arXiv 2003.13569, "Fast and
 * accurate high-order method for high dimensional space-fractional
 * reaction-diffusion equation with general boundary conditions").
 *
 * Problem (Section 1, Eq. 1):
 *     du_s/dt = -kappa_s (-Delta)^{alpha_s/2} u_s + f_s(u, t),   1 < alpha_s <= 2,
 * on a box in R^d (d = 1, 2, 3) with periodic, homogeneous Dirichlet or homogeneous
 * Neumann boundary conditions, one to two species s.
 *
 * Space (Section 3): the fractional Laplacian is the matrix transfer technique
 * applied to the fourth-order compact Laplacian T = A^{-1}B (Eqs. Lap, MTT);
 * T is diagonalised per axis by the DFT (periodic, Eq. PP), DST-I (Dirichlet,
 * Eq. PD) or DCT-I (Neumann, Eq. PN), and the summed eigenvalue
 * Lambda = lambda_x + lambda_y (+ lambda_z) is raised to alpha/2 (Eqs. E16-E22).
 * Time (Section 4, Eq. ETDRK4P13, Algorithm 1): ETDRK4 with e^{-z} replaced by
 * its Pade-(1,3) approximant; the six coefficient arrays R13, Q13, phi, phi1,
 * phi2, phi3 of L = kappa tau Lambda^{alpha/2} are computed once in FP64 on the
 * GPU and stored in the run precision.
 *
 * Conventions shared by every call:
 *   - Grid: N[d] = number of intervals on [lo[d], hi[d]], axes listed x, y, z.
 *     Unknowns per axis: N (periodic: nodes 0..N-1), N-1 (Dirichlet: nodes
 *     1..N-1), N+1 (Neumann: nodes 0..N).
 *   - Field layout (device or host, as each call says): species-major, dense,
 *     row-major [S][n_z][n_y][n_x] (3D), [S][n_y][n_x] (2D) or [S][n_x] (1D), x fastest, in
 *     the plan's dtype (double for SFRD_F64, float for SFRD_F32).
 *   - Ownership: the caller owns every field buffer, the workspace and the
 *     stream; the plan owns only host metadata and its CUDA graph.  Device
 *     pointers are never freed by the library.
 *   - Errors: every call returns SFRD_OK (0) or a negative code; nothing aborts
 *     the process and no kernel traps.  SFRD_ECUDA carries the CUDA error
 *     string in sfrd_last_error().
 *   - Ordering: every device call is enqueued on the stream given to
 *     sfrd_bind and returns without synchronising, except those whose
 *     description says they synchronise.
 */
#ifndef SFRD_H
#define SFRD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define SFRD_OK            0
#define SFRD_EINVAL       -1  /* bad argument: alpha not in (1,2], kappa < 0, dt <= 0, N < 2, ... */
#define SFRD_EUNSUPPORTED -2  /* valid problem outside what the library handles (length not
                                 {2,3,5}-smooth, FFT length > 1024, a field
                                 array of 2^32 elements or more, ...) */
#define SFRD_ENOWS        -3  /* workspace missing, too small or not bound */
#define SFRD_ECUDA        -4  /* a CUDA runtime call failed; see sfrd_last_error() */
#define SFRD_ENONFINITE   -5  /* a non-finite value was detected in the state */
#define SFRD_ESTATE       -6  /* call out of order (e.g. advance before load) */

/* ---- enumerations ------------------------------------------------------ */
#define SFRD_BC_PERIODIC   0  /* Section 3.1.1: DFT eigenvectors (Eq. PP) */
#define SFRD_BC_DIRICHLET  1  /* Section 3.1.2: DST-I eigenvectors (Eq. PD) */
#define SFRD_BC_NEUMANN    2  /* Section 3.1.3: DCT-I eigenvectors (Eq. PN) */

#define SFRD_F64 0            /* fields, transforms and reaction in FP64 */
#define SFRD_F32 1            /* fields, transforms and reaction in FP32; coefficients and
                                 twiddles computed in FP64 and rounded once to FP32 */

/* Reaction terms f(u, t).  p[] and offset[] meanings per kind:
 *   NONE               f = 0                                   (1 or 2 species)
 *   LINEAR             f_s = p0 u_s                            (Eq. TEq test equation)
 *   FHN                p = [mu, eps, beta, gamma, delta]:      (Section 5.2, FitzHugh-Nagumo)
 *                      f_u = u(1-u)(u-mu) - v,  f_v = eps(beta u - gamma v - delta)
 *   GRAY_SCOTT         p = [F, K]:                             (Section 5.2, Eq. SG)
 *                      f_u = -u v^2 + F(1-u),   f_v = u v^2 - (F+K) v
 *   SCHNAKENBERG       p = [gamma, a, b]:                      (Section 5.2, Eq. SB)
 *                      f_u = gamma(a - U + U^2 V), f_v = gamma(b - U^2 V)
 *   GIERER_MEINHARDT   p = [c1, c2, c3, c4]:                   (Section 5.2, Eq. GM)
 *                      f_u = c1 U^2/V - c2 U,   f_v = c3 U^2 - c4 V
 *   HUXLEY_MMS         Example 2 (Section 5.1): u(1-u)(u-1) + the manufactured source
 *                      of u = t^alpha cos^3(2 pi x) cos^3(2 pi y); 1 species, 2D.
 *   FISHER_MMS         Example 1 (Section 5.1): u - u^2 + the manufactured source of
 *                      u = e^{-t} sin^3(2 pi x) (one kappa); 1 species, 1D.
 * For SCHNAKENBERG and GIERER_MEINHARDT, U = u + offset[0], V = v + offset[1]:
 * the solver integrates the perturbation about (offset[0], offset[1]); with
 * Dirichlet BCs the boundary condition applies to that perturbation.  The
 * Schnakenberg terms are evaluated expanded about the offset (their value at
 * the offset taken in FP64 at plan time, plus terms of the perturbation's
 * size), so that a small perturbation about the steady state keeps its
 * relative accuracy in FP32. */
#define SFRD_REACT_NONE              0
#define SFRD_REACT_LINEAR            1
#define SFRD_REACT_FHN               2
#define SFRD_REACT_GRAY_SCOTT        3
#define SFRD_REACT_SCHNAKENBERG      4
#define SFRD_REACT_GIERER_MEINHARDT  5
#define SFRD_REACT_HUXLEY_MMS        6
#define SFRD_REACT_FISHER_MMS        7

typedef struct sfrd_plan_s* sfrd_plan_t;

typedef struct {
    int32_t dim;      /* 1, 2 or 3 */
    int64_t N[3];     /* intervals per axis (x, y, z); unused entries ignored */
    double  lo[3];
    double  hi[3];
} sfrd_grid;

typedef struct {
    int32_t kind;       /* SFRD_REACT_* */
    int32_t nspecies;   /* 1 or 2 */
    double  p[8];
    double  offset[2];
} sfrd_reaction;

typedef struct {
    int32_t dim, bc, dtype, nspecies;
    int64_t n[3];            /* unknowns per axis (x, y, z) */
    int64_t fft_len[3];      /* complex FFT length per axis (N periodic, 2N otherwise) */
    int64_t dof;             /* unknowns x species */
    int64_t kernels_per_step;/* kernel launches of one ETDRK4 step */
    size_t  workspace_bytes;
} sfrd_info;

/* Create a plan (host only; no CUDA call).  Section 1 (Eq. 1) problem data:
 *   grid     : box and intervals;          bc    : SFRD_BC_*;
 *   alpha    : [nspecies] orders in (1,2]; kappa : [nspecies] diffusion >= 0;
 *   dt       : time step tau > 0;          dtype : SFRD_F64 or SFRD_F32;
 *   reaction : f(u, t), see above.
 * On success *out owns a new plan (release with sfrd_destroy).
 * Errors: SFRD_EINVAL, SFRD_EUNSUPPORTED. */
int sfrd_plan(sfrd_plan_t* out, const sfrd_grid* grid, int32_t bc,
              const double* alpha, const double* kappa, double dt,
              int32_t dtype, const sfrd_reaction* reaction);

/* How the slow-axis combination obtains the Padé(1,3) coefficients R13, Q13,
 * phi, phi1, phi2, phi3 of L = kappa tau Lambda^{alpha/2} (Algorithm 1,
 * precompute lines; Eq. 37 and the rational forms of its phi-functions):
 *   SFRD_COEF_STORED   : the six arrays are computed in FP64 at bind time and
 *                        stored in the run precision (default; 10 words per
 *                        unknown and step are read by the four combinations);
 *   SFRD_COEF_RATIONAL : only L is stored (computed in FP64 at bind time and
 *                        rounded to FP32; one array shared by both species when
 *                        their orders are equal, as tau Lambda^{alpha/2}); the
 *                        rationals are evaluated in FP32 inside the passes.
 *                        They have no cancellation for small L, so the
 *                        coefficients keep FP32 accuracy; 2 (shared) or 4 words
 *                        per unknown and step instead of 10.
 * Call before sfrd_bind (it changes sfrd_workspace_bytes).  SFRD_COEF_RATIONAL
 * needs an FP32 plan whose axes all run on the register engine (N a power of
 * two in [64, 1024], or 96, 200 or 384); such a
 * plan has no adjoint (sfrd_adjoint* return SFRD_EUNSUPPORTED) and
 * sfrd_coefficients evaluates the rationals from the stored L.
 * Errors: SFRD_EINVAL (mode), SFRD_EUNSUPPORTED, SFRD_ESTATE (already bound). */
#define SFRD_COEF_STORED   0
#define SFRD_COEF_RATIONAL 1
int sfrd_set_coefficients(sfrd_plan_t plan, int32_t mode);

/* Time-stepping scheme (Section 4).  SFRD_SCHEME_P13 (default) is the paper's
 * ETDRK4-P13: Algorithm 1 with the Padé(1,3) coefficients.  SFRD_SCHEME_COX_MATTHEWS
 * runs the same stages with the exact-exponential coefficients it approximates
 * (e^{-L} in the place of R13(L), and the phi-functions of e^{-L}, computed in
 * FP64 at bind time: Taylor series of the phi-functions for L < 1, closed forms
 * otherwise); a single eigenmode then decays by exactly exp(-kappa
 * Lambda^{alpha/2} t) under zero reaction.  Call before sfrd_bind.  The
 * Cox-Matthews scheme uses stored coefficient arrays (not SFRD_COEF_RATIONAL);
 * its adjoint runs the same reverse sweep over those arrays, with the kappa and
 * alpha gradients through dC/dL of the exact-exponential coefficients.
 * Errors: SFRD_EINVAL (scheme), SFRD_EUNSUPPORTED, SFRD_ESTATE (already bound). */
#define SFRD_SCHEME_P13           0
#define SFRD_SCHEME_COX_MATTHEWS  1
int sfrd_set_scheme(sfrd_plan_t plan, int32_t scheme);

/* Autotuner of the radix/tile schedule: for the axes on the shared-memory
 * engine (lengths other than the register engine's: powers of two 64..1024,
 * 96, 200, 384), times `steps` steps with every
 * tile width and radix-stage order (as factored, reversed, ascending,
 * descending) and keeps the fastest.  With the environment variable
 * SFRD_AUTOTUNE_CACHE naming a file, a choice recorded there for the same grid,
 * boundary condition, precision, species count and device name is reused
 * without timing, and a new choice is appended.  The plan must be bound; it is
 * bound again with the chosen schedule, so the resident state is lost (call
 * sfrd_load afterwards).  Plans whose axes all run on the register engine have
 * nothing to tune.  chosen (may be NULL) receives {tile width, order rule}.
 * Errors: SFRD_EINVAL, SFRD_ENOWS, SFRD_ECUDA. */
int sfrd_autotune(sfrd_plan_t plan, int32_t steps, int32_t* chosen);

/* Bytes of device workspace the plan needs (coefficient arrays, spectral state
 * and stored stage spectra, scratch, tables). */
int sfrd_workspace_bytes(sfrd_plan_t plan, size_t* bytes);

/* Static description of the plan (sizes, launches per step). */
int sfrd_get_info(sfrd_plan_t plan, sfrd_info* info);

/* Attach caller-owned device workspace (>= sfrd_workspace_bytes, 256-byte
 * aligned) and a cudaStream_t (NULL = legacy default stream).  Uploads the
 * FP64-computed eigenvalue, twiddle and permutation tables and runs the FP64
 * init kernel that fills the six Algorithm 1 coefficient arrays (Algorithm 1,
 * precompute lines).  May be called again to move the plan to new memory or a
 * new stream; the resident state is then invalid until the next sfrd_load.
 * Errors: SFRD_ENOWS (NULL, short or misaligned workspace), SFRD_ECUDA. */
int sfrd_bind(sfrd_plan_t plan, void* workspace, size_t bytes, void* stream);

/* Transform a physical device field u0 [S][...] to the resident spectral state
 * (Algorithm 1: u_h = fftn(u)) and set the clock to t0.  u0 is only read. */
int sfrd_load(sfrd_plan_t plan, const void* u0, double t0);

/* Advance the resident state by nsteps ETDRK4-P13 steps (Eq. ETDRK4P13;
 * Algorithm 1 loop body, four stages with reaction times t_k, t_k + tau/2,
 * t_k + tau/2, t_k + tau).  Launched as a captured CUDA graph.  nsteps >= 0. */
int sfrd_advance(sfrd_plan_t plan, int64_t nsteps);

/* Failure detection: SFRD_ENONFINITE when the resident spectral state holds a
 * NaN or an infinity (a blown-up run, or a non-finite initial field), else
 * SFRD_OK.  One reduction kernel writes a device flag that the host reads back
 * (synchronises the stream; nothing waits on the device).  With the environment
 * variable SFRD_DEBUG_CHECKS set (not "0") when the plan is created,
 * sfrd_advance (and so sfrd_run, sfrd_step) ends with this check and returns
 * its code.  Errors: SFRD_EINVAL, SFRD_ENOWS, SFRD_ESTATE (nothing loaded),
 * SFRD_ECUDA. */
int sfrd_check_finite(sfrd_plan_t plan);

/* Write the resident state to the physical device field u [S][...]
 * (Algorithm 1: u = ifftn(...)).  Does not change the resident state. */
int sfrd_store(sfrd_plan_t plan, void* u);

/* u <- u(t0 + nsteps tau): sfrd_load(u, t0); sfrd_advance(nsteps); sfrd_store(u).
 * u is a device field, overwritten in place. */
int sfrd_run(sfrd_plan_t plan, void* u, double t0, int64_t nsteps);

/* One step: sfrd_run(plan, u, t, 1). */
int sfrd_step(sfrd_plan_t plan, void* u, double t);

/* End-to-end run through host memory: copies u_in (host, [S][...]) to the
 * device, runs nsteps from t0, copies the result to u_out (host, may equal
 * u_in) and synchronises the stream.  Pinned host buffers give overlap-free
 * DMA at full speed; pageable buffers work but are slower. */
int sfrd_run_host(sfrd_plan_t plan, const void* u_in, void* u_out, double t0, int64_t nsteps);

/* The separable transform of Eqs. E19/E22 in this library's real form:
 * uhat = T_z T_y T_x u with T = discrete Hartley transform (periodic; it shares
 * the DFT's eigenvalues because lambda_k = lambda_{N-k}), DST-I (Dirichlet) or
 * DCT-I with endpoint weights (1/2, 1, ..., 1, 1/2) on the input (Neumann),
 * all unnormalised.  u and uhat are dense device fields [S][...]. */
int sfrd_forward(sfrd_plan_t plan, const void* u, void* uhat);

/* Inverse of sfrd_forward: u = T_z T_y T_x uhat / C with C = prod over axes of
 * (N for periodic, N/2 otherwise). */
int sfrd_inverse(sfrd_plan_t plan, const void* uhat, void* u);

/* Allocation-free form of sfrd_forward (no counterpart in the paper: an
 * implementation service).  For callers that must not allocate device memory
 * at all -- e.g. a component embedded in a host application that owns the GPU
 * memory budget and forbids allocations after start-up, or a latency-critical
 * loop that cannot absorb the implicit synchronisation of cudaMalloc/cudaFree.
 * The plan needs no workspace and no sfrd_bind: the scratch (one padded field
 * of the plan plus its twiddle and permutation tables) lives in a fixed device
 * array of 16 MiB that every GPU loading this library holds until exit.  u and
 * uhat are caller-owned device fields [S][...] (same layout and result as
 * sfrd_forward); stream is a cudaStream_t (NULL: legacy default stream).
 * The first call on a device looks up that array's device address (once per
 * device, with the device current).  Every call copies the plan's tables from
 * pageable host memory and synchronises the stream, so no call may be made on
 * a capturing stream or while a global-mode stream capture is in progress.
 * Every call shares the array and leaves its
 * contents behind; the call clears what must start at zero.  Calls that
 * overlap on the GPU (other streams, other threads) race on the array, and the
 * plan must not be used by another thread during the call.  Synchronises the
 * stream, also when a launch or copy failed part way.  A bound plan stays
 * bound: its workspace, stream and tables are untouched.  Errors: SFRD_EUNSUPPORTED when the plan's scratch exceeds 16 MiB,
 * SFRD_ECUDA, SFRD_EINVAL. */
int sfrd_forward_noalloc(sfrd_plan_t plan, const void* u, void* uhat, void* stream);

/* Copy coefficient array `which` (0 R13, 1 Q13, 2 phi, 3 phi1, 4 phi2, 5 phi3;
 * Algorithm 1) for every species into the dense device buffer out [S][...],
 * indexed like the spectral field (mode k per axis in eigenvalue order). */
int sfrd_coefficients(sfrd_plan_t plan, int32_t which, void* out);

/* Per-launch device times of one ETDRK4 step of the resident state (which it
 * advances): the step's kernels are launched individually (no graph) with a
 * CUDA event recorded on the bound stream before and after each launch; the
 * call synchronises.  For i < min(cap, kernels_per_step): ms[i] = duration of
 * launch i, kind[i] = pass kind (0: contiguous-axis pass with the reaction,
 * 1: middle-axis pass, 2..5: slow-axis pass of stage a, b, c, update).
 * Errors: SFRD_ESTATE before sfrd_load. */
int sfrd_profile_step(sfrd_plan_t plan, int32_t cap, float* ms, int32_t* kind);

/* ---- discrete adjoint (gradients through nsteps steps) ---------------------
 * Available when every axis runs on the register engine: N a power of two in
 * [64, 1024], or 96, 200 or 384 (SFRD_EUNSUPPORTED otherwise).  The adjoint is
 * the exact transpose of the library's own FP arithmetic path (transposed transforms, the same
 * coefficient arrays, the reaction Jacobian transposed), i.e. the gradient of
 * the discrete map u0 -> u(t0 + nsteps tau) of Eq. ETDRK4P13 (or of the
 * Cox-Matthews step of sfrd_set_scheme, whose coefficient arrays it then uses).
 *
 * Memory: a caller-owned device buffer of sfrd_adjoint_workspace_bytes(nsteps,
 * ckpt_every) bytes (256-byte aligned) holds one spectral checkpoint every
 * ckpt_every steps and, during the reverse sweep, the stage intermediates of
 * one segment of ckpt_every steps (recomputed from its checkpoint). */
int sfrd_adjoint_workspace_bytes(sfrd_plan_t plan, int64_t nsteps, int64_t ckpt_every, size_t* bytes);

/* u <- u(t0 + nsteps tau) like sfrd_run, also writing the checkpoints that
 * sfrd_adjoint needs into adj_ws.  u is a device field, overwritten. */
int sfrd_run_checkpointed(sfrd_plan_t plan, void* u, double t0, int64_t nsteps, int64_t ckpt_every,
                          void* adj_ws, size_t adj_bytes);

/* Gradients of a loss l(u_T), u_T = u(t0 + nsteps tau), after sfrd_run_checkpointed
 * with the same (t0, nsteps, ckpt_every, adj_ws):
 *   dLduT  (device, [S][...], read)  : dl/du_T
 *   dLdu0  (device, [S][...], write) : dl/du0
 *   dLdalpha, dLdkappa (host, [S])   : dl/dalpha_s, dl/dkappa_s (NULL to skip)
 *   dLdparams (host, [8])            : dl/dp of the reaction parameters p[0..4]
 *                                      (p[5..7] reported as 0; NULL to skip).
 * Synchronises the stream.  Leaves no resident state (call sfrd_load before
 * sfrd_advance again). */
int sfrd_adjoint(sfrd_plan_t plan, double t0, int64_t nsteps, int64_t ckpt_every, void* adj_ws, size_t adj_bytes,
                 const void* dLduT, void* dLdu0, double* dLdalpha, double* dLdkappa, double* dLdparams);

/* ---- batched instances ---------------------------------------------------
 * count independent problems of the same dimension, species count, reaction
 * kind/parameters, dtype and time step, each with its own grid (intervals per
 * axis <= 512), boundary condition bcs[i] and coefficients alpha[i*S+s],
 * kappa[i*S+s].  One ETDRK4-P13 step of all instances is replayed from a
 * captured CUDA graph: each pass (8 in 2D, 16 in 3D) is one persistent launch
 * per group of instances that share the pass axis's length (one kernel per
 * register-engine length, one for the shared-memory engine), the groups of a
 * pass issued as parallel branches; each launch's blocks draw (instance, tile)
 * work items, longest lines first.
 * Fields are passed as host arrays of count device pointers, field i laid out
 * [S][...] for instance i's grid.  Errors as for single plans. */
typedef struct sfrd_batch_s* sfrd_batch_t;

/* Host only.  grids, bcs: count entries; alpha, kappa: count * S entries
 * (S = reaction->nspecies), all read during the call only.  Every instance is
 * validated as by sfrd_plan; all share grids[0].dim, which must be 2 or 3
 * (1D: SFRD_EUNSUPPORTED; an instance of another dim: SFRD_EINVAL), and have
 * at most 512 intervals per axis (else SFRD_EUNSUPPORTED).  On success *out
 * owns a new batch (release with sfrd_batch_destroy). */
int sfrd_batch_plan(sfrd_batch_t* out, int64_t count, const sfrd_grid* grids, const int32_t* bcs,
                    const double* alpha, const double* kappa, double dt, int32_t dtype,
                    const sfrd_reaction* reaction);

/* Bytes of device workspace for all instances (their states, stage spectra,
 * coefficient arrays and tables) plus the work-item schedule. */
int sfrd_batch_workspace_bytes(sfrd_batch_t batch, size_t* bytes);

/* As sfrd_bind, for every instance at once: caller-owned workspace
 * (>= sfrd_batch_workspace_bytes, 256-byte aligned) and a cudaStream_t.
 * Errors: SFRD_ENOWS, SFRD_ECUDA. */
int sfrd_batch_bind(sfrd_batch_t batch, void* workspace, size_t bytes, void* stream);

/* u0: host array of count device pointers, u0[i] the physical field of
 * instance i laid out [S][...] on its own grid (only read).  Transforms every
 * instance to its resident spectral state and sets all clocks to t0. */
int sfrd_batch_load(sfrd_batch_t batch, const void* const* u0, double t0);

/* nsteps replays of the captured batched step (stream-ordered, no sync).
 * Errors: SFRD_ESTATE before sfrd_batch_load, SFRD_ECUDA. */
int sfrd_batch_advance(sfrd_batch_t batch, int64_t nsteps);

/* u: host array of count device pointers; writes each instance's physical
 * field (the resident state is kept). */
int sfrd_batch_store(sfrd_batch_t batch, void* const* u);

/* count, total unknowns over all instances and species, and kernel launches
 * per batched step (a NULL output pointer is skipped). */
int sfrd_batch_info(sfrd_batch_t batch, int64_t* count, int64_t* dof, int64_t* launches_per_step);
/* Autotuner of the batched schedule: times `steps` batched steps for each
 * number of resident blocks per SM (1..4) of the persistent column-pass launches
 * (the x-pass launches run at their kernel's full occupancy) and each
 * radix-stage order of the instances on the shared-memory engine, and keeps the
 * fastest.  The batch must be bound; it is bound again, so the instances must
 * be loaded afterwards.  chosen (may be NULL) receives {blocks per SM, order
 * rule}.  Errors: SFRD_EINVAL, SFRD_ENOWS, SFRD_ECUDA. */
int sfrd_batch_autotune(sfrd_batch_t batch, int32_t steps, int32_t* chosen);
void sfrd_batch_destroy(sfrd_batch_t batch);

/* Release the plan and its CUDA graph (not the workspace). */
void sfrd_destroy(sfrd_plan_t plan);

/* Static description of an error code; text of the last CUDA error seen by
 * this thread. */
const char* sfrd_strerror(int code);
const char* sfrd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SFRD_H */
