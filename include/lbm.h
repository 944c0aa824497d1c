/*
 * lbm.h - C ABI of the GB300 (sm_103a) implementation of the per-node time step
 * of the multiphase lattice Boltzmann model with self-tuning equation of state
 * (R. Huang, H. Wu, N. A. Adams, "Lattice Boltzmann model with self-tuning
 * equation of state for multiphase flows", arXiv:1809.02390).
 *
 * One time step on a periodic D2Q9 lattice (delta_x = 1) is: pull streaming
 * f_i(x) = fbar_i(x - e_i) (supplement Eq. 2), density rho = sum_i f_i,
 * the pairwise interaction force F = G^2 rho sum_i omega_i rho(x + e_i) e_i
 * (Eq. 12), and the collision of Eq. 13 in moment space (moment transform
 * of supplement Eq. 4, equilibrium of Eq. 3 with the self-tuning eta, forcing
 * of Eq. 4, non-diagonal collision matrix of Eq. 6, cubic-velocity correction
 * of Eq. 10-11 and the eps^3 term S Q_m of Eq. 14), executed in the sequence
 * of supplement Sec. IV, followed by the inverse transform.
 *
 * Units.  The library runs with lattice speed c = 1: pressures are carried as
 * p / c^2 and the interaction strength as G2 = G^2 / c^2 (the model is
 * invariant under this rescaling).  The physical -> lattice derivation follows
 * Eqs. 21-22 (G = K_INT sqrt(2 K_EOS a), c_s = K_INT sqrt(d(p_EOS + K_EOS a rho^2)/drho)
 * at rho_l, c = sqrt(3) c_s) unless the caller gives `lam` / `G2` directly.
 *
 * Memory.  The caller owns every buffer: the library never allocates device
 * memory for the lattice and never frees caller memory.  Populations are stored
 * structure-of-arrays, f[i][y][x] (LB_LAYOUT_PLANES, the default) or with a
 * row's nine population rows side by side, f[y][i][x] (LB_LAYOUT_ROWS), i = 0..8
 * in the velocity order of supplement Eq. 3 (rest, +x, +y, -x, -y, (+1,+1),
 * (-1,+1), (-1,-1), (+1,-1)), x fastest, no padding, as the deviation
 * fbar_i - w_i rho_ref from the rest state (w = 4/9, 1/9 x4, 1/36 x4;
 * rho_ref = 0 stores plain populations).
 * Element type: double (LB_FP64), float (LB_FP32) or IEEE half (LB_FP16S).
 * The stored state is always post-collision (after the last completed step).
 *
 * Streams.  `stream` is a cudaStream_t passed as void*; every call enqueues
 * its kernels on it and returns without synchronising (except where stated).
 *
 * Errors.  Every int-returning call returns LB_OK (0) or a negative code;
 * lb_last_error() gives a message.  Invalid parameters never reach the GPU.
 * There is no CPU fallback: without a CUDA device the calls fail with LB_ECUDA.
 */
#ifndef LBM_H_
#define LBM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LB_OK 0
#define LB_EINVAL (-1)     /* invalid argument or parameter */
#define LB_ECUDA (-2)      /* CUDA runtime error (message has the CUDA error string) */
#define LB_ENOMEM (-3)     /* caller-provided scratch too small */
#define LB_ENONFINITE (-4) /* non-finite density found by lb_reduce / lb_batch_status */
#define LB_ETIMEOUT (-5)   /* a bounded device-side wait gave up */
#define LB_ENOTSUP (-6)    /* combination not supported */

enum lb_precision { LB_FP64 = 0, LB_FP32 = 1, LB_FP16S = 2 };
enum lb_eos_kind { LB_EOS_VDW = 0, LB_EOS_CS = 1 };
enum lb_variant { LB_AUTO = 0, LB_FUSED = 1, LB_TWO_PASS = 2 };
enum lb_rounding { LB_ROUND_STOCHASTIC = 0, LB_ROUND_NEAREST = 1 };
/* Population layout of the state buffers (the arithmetic is the same in both;
 * results are bit-identical).  PLANES: f[9][ny][nx]; ROWS: f[ny][9][nx], one
 * lattice row's nine population rows contiguous, so that a step reads and writes
 * one region per row instead of nine planes far apart. */
enum lb_layout { LB_LAYOUT_PLANES = 0, LB_LAYOUT_ROWS = 1 };

/* Problem statement (main text Eqs. 6, 7, 16, 20-22; supplement Sec. V). */
typedef struct lb_params {
  int32_t nx, ny;    /* periodic lattice size, each >= 3 */
  int32_t precision; /* enum lb_precision: storage type; FP16S computes in FP32 */
  int32_t eos;       /* enum lb_eos_kind: van der Waals p = rho R T/(1 - b rho) - a rho^2,
                        or Carnahan-Starling (Eq. 20); both times K_EOS */
  int32_t variant;   /* enum lb_variant: fused single-kernel step or density pass + collision;
                        LB_AUTO selects the fused step (the faster one on this GPU) */
  int32_t rounding;  /* enum lb_rounding, FP16S only: rounding of the stored populations.
                        Stochastic (default): a pseudo-random dither below the half
                        mantissa, then truncation, so that rounding errors have zero mean
                        and mass does not drift in stationary states; nearest: IEEE
                        round-to-nearest-even (biased in a stationary state: the same
                        errors repeat every step) */
  double eos_a, eos_b, R_gas; /* EOS constants a, b, R (> 0) */
  double Tr;                  /* reduced temperature T/Tc, in (0, 1) for two phases */
  double K_eos, K_int;        /* scaling factors of Eqs. 20-22 (> 0) */
  double G2;    /* > 0: interaction strength G^2/c^2 given directly; <= 0: Eq. 21-22 */
  double lam;   /* > 0: pressure scale K_EOS/c^2 given directly; <= 0: c_s rule of Eq. 22 */
  double varpi; /* bulk-viscosity coefficient of Eq. 7; 0 selects the paper's 1/6;
                   1 and 1/3 are singular (main text after Eq. 9) and rejected */
  double s_p;   /* shear relaxation rate, in (0, 2) (relaxation time tau = 1/s_p) */
  double s_q, s_e, s_eps; /* <= 0: s_q and s_e from tau_p tau_q = (k+1) tau_e tau_q = 1/12
                             (Eq. 16), s_eps = s_e; otherwise in (0, 2) */
  double s_0, s_j;        /* rates of the conserved moments (act on zero); <= 0 selects 1 */
  double rho_ref;         /* storage shift: populations stored as fbar_i - w_i rho_ref
                             (rounded to float for FP32 and FP16 storage).  NaN: the mean
                             of the initial density, summed in FP64 on the device by
                             lb_init / lb_batch_init (lb_get_params, lb_batch_params
                             return the value taken); infinite values are rejected */
  int32_t layout;         /* enum lb_layout.  LB_LAYOUT_ROWS: forward step, moments, pressure,
                             reductions, batched solver (all lattices of a batch in one
                             layout); the adjoint calls take LB_LAYOUT_PLANES only
                             (LB_ENOTSUP) */
  int32_t reserved1;      /* must be 0 */
} lb_params;

/* Derived lattice-unit quantities (all FP64, computed on the host). */
typedef struct lb_derived {
  double Tc, T;          /* critical and actual temperature */
  double rho_g, rho_l;   /* Maxwell-construction coexistence densities of p_EOS */
  double p_star;         /* coexistence pressure (physical units, with K_EOS) */
  double lam, G2;        /* lattice pressure scale K_EOS/c^2 and G^2/c^2 in use */
  double c2;             /* c^2 = 3 c_s^2 of Eq. 22 (physical lattice speed squared) */
  double s_0, s_e, s_eps, s_j, s_q, s_p; /* relaxation rates in use */
  double k, h, b, beta2; /* coefficients of Eq. 7 with alpha_1 = -1, beta_1 = 1 */
  double W1, sigma1;     /* flat-interface thickness and surface tension predicted by the
                            pressure tensor (Eq. 17) at K_INT = 1, physical units */
} lb_derived;

typedef struct lb_handle lb_handle;

/* Version of this ABI (incremented on incompatible change). */
int lb_abi_version(void);

/* Derives the lattice-unit parameters of `p` on the host (FP64, no GPU use):
 * Maxwell construction for rho_g, rho_l (from the closed-form free energy
 * psi with p_EOS = rho psi' - psi, below Eq. 19), Eq. 21-22 for G2 and lam,
 * Eq. 16 for the rates, Eq. 7 for k, h, b, beta_2, and the pressure-tensor
 * interface thickness W1 and surface tension sigma1 (Eq. 17, 23) at K_INT = 1.
 * Returns LB_EINVAL for invalid parameters (message in lb_last_error(NULL)). */
int lb_derive(const lb_params* p, lb_derived* out);

/* Bytes of one population buffer: 9 * nx * ny * element size. */
size_t lb_state_bytes(const lb_params* p);

/* Bytes of device scratch memory: one density plane (two-pass variant, reductions),
 * the reduction workspace and 256 bytes of tile tickets (fused tensor-copy step). */
size_t lb_scratch_bytes(const lb_params* p);

/* Creates a handle bound to the caller's buffers and stream and initialises the
 * lattice at rest: fbar_i = (M^-1 m_eq(rho0, u = 0))_i - w_i rho_ref, with eta
 * from the EOS at rho0 (the stated initial condition; the paper does not give
 * one), computed in the step's compute type (FP64 for LB_FP64, FP32 otherwise).
 * Host densities are checked on the device as the state is built: the first node
 * that is not positive and finite (or, for vdW, not below 1/b) is reported.  f_a, f_b: device buffers of lb_state_bytes() each (ping-pong; f_a holds
 * the state after init).  scratch: device buffer of lb_scratch_bytes() bytes, or
 * NULL (the fused step then walks its tiles statically, and lb_reduce and the
 * two-pass variant are unavailable); it holds the tile tickets of the fused step,
 * so handles that step concurrently need scratch buffers of their own.  rho0: nx*ny doubles, row-major [y][x], on the host
 * (rho0_on_device = 0; copied through f_b, synchronously) or the device (1).
 * The handle keeps the pointers; the caller keeps ownership and must keep the
 * buffers alive until lb_free.  Fails with LB_EINVAL for bad parameters or
 * non-positive densities on the host path, LB_ENOMEM for a short scratch or when
 * 4096 handles are already live (each holds one slot of a static array of device
 * words for lb_status until lb_free). */
int lb_init(lb_handle** out, const lb_params* p, void* f_a, void* f_b, void* scratch,
            size_t scratch_bytes, const double* rho0, int rho0_on_device, void* stream);

/* Advances nsteps >= 0 time steps (Eq. 13 + supplement Eq. 2) on the stream.
 * Asynchronous.  Runs of 64 steps replay a CUDA graph that the handle captures on
 * first use (again after lb_set_step_blocks or lb_set_tile_dispatch change the
 * launch); the graph runs on a stream the handle owns, ordered after the caller's
 * stream's earlier work and before its later work, and gives the same bits as 64
 * separate launches (FP16 stores take their per-step seed from a device word with
 * the step count, written before each replay).  While the caller's stream is being
 * captured into a graph of its own, every step is a plain launch on that stream. */
int lb_step(lb_handle* h, int64_t nsteps);

/* Device pointer of the buffer holding the current state. */
void* lb_state(lb_handle* h);

/* Number of steps taken since lb_init. */
int64_t lb_steps_done(const lb_handle* h);

/* Macroscopic fields at the time level of the last collision (Eq. 5): the
 * collision conserves mass and adds F to the momentum, so
 * rho = sum_i fbar_i and rho u = sum_i e_i fbar_i - F/2.  rho, ux, uy: device
 * arrays of nx*ny elements ([y][x]), double for LB_FP64, float otherwise; ux and
 * uy may be NULL. */
int lb_moments(lb_handle* h, void* rho, void* ux, void* uy);

/* Pressure field p_EOS(rho)/c^2 of the current state (the EOS of Eq. 20 or van
 * der Waals, times K_EOS, in the lattice units of the step: multiply by c^2 of
 * lb_derived for the paper's units).  p: device array of nx*ny elements ([y][x]),
 * double for LB_FP64, float otherwise.  Asynchronous on the handle's stream. */
int lb_pressure(lb_handle* h, void* p);

/* FP64 reductions of the current state, synchronous (waits on the stream):
 * out[0] = total mass, out[1..2] = total momentum sum_x rho u,
 * out[3] = p_EOS/c^2 at the lattice centre (nx/2, ny/2), out[4] = p_EOS/c^2 at
 * node (0, 0), out[5] = number of nodes with rho > (rho_g + rho_l)/2,
 * out[6] = min rho, out[7] = max rho.  Returns LB_ENONFINITE if any density is
 * not finite (the values are still written). */
int lb_reduce(lb_handle* h, double out[8]);

/* lb_reduce for callers that cannot allocate device memory (the paper has no
 * counterpart).  Such callers exist: a host program whose own allocator has taken
 * the whole GPU and grants no further buffers, or a plugin inside such a program,
 * which receives the lattice from its host and has no allocator of its own.  Same
 * results as lb_reduce (same kernels, same block count, same order), but the
 * scratch is a file-scope static device array inside the library, of
 * LB_REDUCE_STATIC_MAX_NODES * 8 + 65600 bytes (about 8.1 MB).  lb_init commits
 * that array on its device (it looks up the array's address there, with the
 * device current, which loads the module holding it), so every GPU on which a
 * handle has been created holds it until the process exits, and a later call
 * cannot fail for want of memory.  Nothing is allocated by the call: no
 * cudaMalloc / cudaFree, no allocating library routine.  The handle may have been
 * created with scratch = NULL.
 * Limits: lattices above LB_REDUCE_STATIC_MAX_NODES nodes are rejected with
 * LB_ENOMEM (use lb_reduce).  All calls share the one array and each call writes
 * every element it reads, so nothing carries over between calls, but calls whose
 * GPU work overlaps (several streams or threads at once) race on it and must be
 * serialised by the caller.  Synchronous like lb_reduce: it waits on the handle's
 * stream, so it must not be called while that stream is being captured into a
 * CUDA graph. */
#define LB_REDUCE_STATIC_MAX_NODES 1048576
int lb_reduce_static(lb_handle* h, double out[8]);

/* Bytes of device scratch lb_adjoint_step needs: 11 planes of the compute type
 * (the population cotangents mu and the force-stencil cotangent) plus FP64
 * per-block partial sums of the parameter gradient. */
size_t lb_adjoint_scratch_bytes(const lb_params* p);

/* Adjoint (transposed Jacobian) of one time step.  The forward step maps the
 * post-collision state s to s' = Phi(s; theta): pull streaming (supplement
 * Eq. 2), rho, the force stencil of Eq. 12, the collision of Eq. 13 (execution
 * sequence of supplement Sec. IV).  Given lam_in = dL/ds' this computes
 * lam_out = (dPhi/ds)^T lam_in: the collision's vector-Jacobian product at every
 * node (hand-written reverse of the sequence, including the EOS, the force, S(u),
 * R(u), T(u), X(u) and Q_m), the transposed force stencil and the transposed pull.
 * dtheta (device, 3 doubles, or NULL) accumulates dL/dT, dL/dG2, dL/dlam, with
 * T the temperature, G2 = G^2/c^2 and lam = K_EOS/c^2 as in lb_derived.
 * f_state: the state s the step started from (storage type of the handle);
 * lam_in, lam_out: [9][ny][nx] device arrays in the compute type (double for
 * LB_FP64, float for LB_FP32), distinct.  Uses the handle's parameters and stream,
 * not its current state.  LB_ENOTSUP for LB_FP16S, LB_ENOMEM for a short scratch. */
int lb_adjoint_step(lb_handle* h, const void* f_state, const void* lam_in, void* lam_out, double* dtheta,
                    void* scratch, size_t scratch_bytes);

/* Adjoint of k consecutive steps in one call (a checkpoint segment): states[j]
 * (host array of k device pointers) is the state s^{n+j} each forward step
 * started from; lam holds dL/ds^{n+k} on entry and dL/ds^n on return (in place,
 * compute type).  Same mathematics as k calls of lb_adjoint_step, but the
 * transposed pull and stencil of step j+1 are fused into the local
 * vector-Jacobian product of step j, so each step is one kernel reading the
 * state, the cotangent populations and the stencil cotangent (124 B per node in
 * FP32).  dtheta as in lb_adjoint_step.  Scratch: lb_adjoint_steps_scratch_bytes. */
size_t lb_adjoint_steps_scratch_bytes(const lb_params* p);
int lb_adjoint_steps(lb_handle* h, const void* const* states, int k, void* lam, double* dtheta, void* scratch,
                     size_t scratch_bytes);

/* ---------------------------------------------------------------------------
 * Batched solver: n independent periodic lattices (each with its own size and
 * lb_params: Tr, K_int, rho_ref, ...) advanced together by one kernel launch per
 * time step over a flat list of tiles of all lattices; runs of 64 steps are
 * captured into CUDA graphs and replayed.  FP32 storage only.
 * Memory (all the caller's): two population pools of lb_batch_pool_bytes (lattice
 * i at element offset lb_batch_offset(i), layout f[9][ny][sx], or f[ny][9][sx] when
 * the lattices' lb_params.layout is LB_LAYOUT_ROWS (one layout per batch), with the
 * row stride sx = lb_batch_row_stride(i) = nx rounded up to a multiple of 4;
 * columns nx..sx-1 are padding, never read or written) and a metadata buffer of
 * lb_batch_meta_bytes (descriptors, coefficients, tensor maps, per-lattice
 * counters of the non-finite check; the maps hold the pools' addresses, so the
 * pools must not move while the batch lives).
 * rho0: the initial densities of all lattices concatenated ([y][x] each), host
 * (staged through pool_b, synchronous) or device.  A stream of NULL (the legacy
 * default stream) cannot be captured: lb_batch_run then launches step by step. */
typedef struct lb_batch lb_batch;
size_t lb_batch_pool_bytes(const lb_params* ps, int n);
size_t lb_batch_meta_bytes(const lb_params* ps, int n);
int lb_batch_init(lb_batch** out, const lb_params* ps, int n, void* pool_a, void* pool_b, void* meta,
                  size_t meta_bytes, const double* rho0, int rho0_on_device, void* stream);
/* Advances every lattice by nsteps.  While the batch's stream is being captured
 * into the caller's own CUDA graph, the steps go in as plain launches (a graph
 * of the library's own is never replayed into another capture); the results
 * are the same bits either way. */
int lb_batch_run(lb_batch* b, int64_t nsteps);
/* Autotuner: times each launch shape (plain loads: tile height 16 or 32, register
 * budget, and either one block per tile or a persistent grid of 1..max resident
 * blocks per SM; tensor copies: persistent grid of 1..max blocks per SM) for
 * trial_steps steps on the batch itself (advancing it) and keeps the fastest;
 * writes its time per step.  lb_batch_config reports blocks_per_sm = 0 for the
 * one-block-per-tile grid; lb_batch_uses_tma is 1 when the tensor-copy kernel is
 * the chosen shape. */
int lb_batch_tune(lb_batch* b, int trial_steps, double* best_ms_per_step);
int lb_batch_config(const lb_batch* b, int* tile_y, int* blocks_per_sm, int* grid);
int lb_batch_uses_tma(const lb_batch* b);
/* Sets the launch form by hand: shape 0, 1, 2 = plain loads with 32 x 16 tiles at
 * 64 registers, 32 x 16 at 80, 32 x 32 at 64 (blocks_per_sm 0 = one block per tile,
 * else a persistent grid); shape 3, 4 = the persistent tensor-copy kernel at 80 and
 * 128 registers walking the tile list statically (block b: tiles b, b + grid, ...);
 * shape 5, 6 = the same at 80 and 128 registers taking tiles by ticket, with two
 * tiles' windows in flight per block (blocks_per_sm >= 1 for 3 - 6).  LB_EINVAL
 * outside the ranges (blocks_per_sm at most the resident maximum), LB_ENOTSUP for
 * 3 - 6 when a lattice has no tensor map. */
int lb_batch_set_config(lb_batch* b, int shape, int blocks_per_sm);
/* Synchronous health check: LB_ETIMEOUT if a bounded wait of the tensor-copy
 * kernel gave up since the last call (the flag is cleared); else LB_ENONFINITE if
 * any lattice of the current state has a node whose density (the sum of its nine
 * populations) is not finite, with the lattice indices in lb_batch_last_error;
 * else LB_OK.  The check reads every population once (one kernel). */
int lb_batch_status(lb_batch* b);
/* Non-finite check of every lattice of the current state (synchronous, the
 * check of lb_batch_status): counts[i] (host array of n, or NULL) = number of
 * nodes of lattice i whose density is not finite.  Returns the number of
 * lattices with at least one such node (0 = all finite), or a negative error
 * code.  A lattice goes non-finite when the method itself is unstable for its
 * parameters (thin interfaces at low temperature); the others are unaffected. */
int lb_batch_nonfinite(lb_batch* b, uint32_t* counts);
/* Device pointer of the pool holding the current state; element offset of lattice i. */
void* lb_batch_state(lb_batch* b);
int64_t lb_batch_steps_done(const lb_batch* b);
int64_t lb_batch_offset(const lb_batch* b, int i);
int lb_batch_row_stride(const lb_batch* b, int i);
/* Density of lattice i at the time level of its last collision, rho = sum_i fbar_i
 * (Eq. 5; the collision conserves mass): rho, a device array of ny*nx floats
 * ([y][x]), written asynchronously on the batch's stream. */
int lb_batch_density(lb_batch* b, int i, void* rho);
int lb_batch_derived(const lb_batch* b, int i, lb_derived* out);
/* Parameters of lattice i as used (rho_ref as stored).  LB_EINVAL for a bad index. */
int lb_batch_params(const lb_batch* b, int i, lb_params* out);
const char* lb_batch_last_error(const lb_batch* b);
void lb_batch_free(lb_batch* b);

/* Sets the current state to the equilibrium of a density and velocity field, in
 * place of a caller-made state (no counterpart in the paper; lb_init's rest state is
 * the case u = 0): fbar_i = (M^-1 m_eq(rho, u))_i - w_i rho_ref, with m_eq of Eq. 3
 * (self-tuning eta from the EOS at rho; alpha_1 = -1, beta_1 = 1, alpha_2 = 1) and
 * momentum rho u, so u is the velocity before the half-force shift of Eq. 5 (the
 * first step's velocity is u + F/(2 rho)).  rho, ux, uy: nx*ny doubles each, [y][x],
 * on the device; ux or uy NULL means 0.  Asynchronous on the handle's stream; the
 * step count is unchanged. */
int lb_set_equilibrium(lb_handle* h, const double* rho, const double* ux, const double* uy);

/* Copies the current state to / from a caller device buffer of lb_state_bytes(). */
int lb_get_state(lb_handle* h, void* dst);
int lb_set_state(lb_handle* h, const void* src);

/* Synchronous health check of this handle: LB_ETIMEOUT if a bounded wait of one
 * of its kernels (step or adjoint) for an asynchronous tensor copy gave up since
 * the last call (the handle's own device flag is cleared), else LB_OK.  Each
 * handle has its own flag, so a give-up is reported on the handle whose kernel
 * had it.  Kernels never spin without a limit. */
int lb_status(lb_handle* h);

/* Check of the reporting above, for users and tests (no counterpart in the paper):
 * runs one block whose bounded wait can never succeed (an mbarrier expecting bytes
 * that no copy delivers), polling it `polls` times (1 .. 2^22; the kernels' waits
 * also give up after 1 s, whichever comes first), then returns what
 * lb_status returns: LB_ETIMEOUT when the give-up was recorded and read back (the
 * expected result; the flag is cleared), LB_OK if it was lost.  Synchronous.  No
 * memory is touched but the device flag, and the context stays usable. */
int lb_wait_selftest(lb_handle* h, long long polls);

/* 1 if the handle's fused step stages populations with tensor copies (TMA):
 * FP32 storage with nx a multiple of 4 and nx >= 104, or FP16 storage with nx a
 * multiple of 8 and nx >= 112; ny >= 50.  Else 0. */
int lb_uses_tma(const lb_handle* h);

/* How the tensor-copy step hands tiles to its persistent blocks.  1 (the default
 * when the handle has its scratch buffer): by ticket, one atomic add on a counter
 * in the scratch buffer per tile, so the tiles in flight are always the next ones
 * in row-major order across the grid, with two tiles' windows in flight per
 * block; 0: each block walks tiles b, b + grid, ... with one window in flight.
 * Results are the same bit for bit.  lb_set_tile_dispatch returns LB_ENOTSUP for
 * 1 when the step does not use tensor copies or the handle has no scratch. */
int lb_set_tile_dispatch(lb_handle* h, int dynamic);
int lb_tile_dispatch(const lb_handle* h);

/* Measurement aid (no counterpart in the paper): one pass with the step's memory
 * traffic and none of its arithmetic, a copy of the state into the other buffer
 * reading and writing every population in place, tile by tile as the step (32 x 16
 * tiles, one block per tile, the handle's layout).  The state is unchanged (the
 * copy is exact and becomes the current buffer).  Asynchronous on the handle's
 * stream; the pass's bandwidth is the ceiling quoted for the step's access pattern
 * (the fastest copy of that pattern measured). */
int lb_stream_copy(lb_handle* h);

/* Grid of the persistent tensor-copy step, in either tile dispatch (static walk:
 * each block steps tiles b, b + blocks, ...; tickets: tiles b and b + blocks, then
 * by ticket): blocks > 0 fixes it (at most the tile count), 0 restores the default
 * (as many blocks as can be resident).  LB_EINVAL if blocks < 0.  Results do not
 * depend on it; it exists for tuning and for tests of the per-block tile loop. */
int lb_set_step_blocks(lb_handle* h, int blocks);

/* Derived parameters in use by the handle. */
int lb_get_derived(const lb_handle* h, lb_derived* out);

/* The handle's parameters as used (rho_ref as stored: the mean initial density
 * when lb_init was given NaN).  LB_EINVAL for null arguments. */
int lb_get_params(const lb_handle* h, lb_params* out);

/* Message of the last error on this handle (h = NULL: of the last failed
 * lb_derive / lb_init on this thread).  Never NULL. */
const char* lb_last_error(const lb_handle* h);

/* Releases the handle (not the caller's buffers). */
void lb_free(lb_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H_ */
