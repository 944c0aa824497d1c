/* C ABI of the three-dimensional (D3Q19) time step of the self-tuning-EOS
 * multiphase lattice Boltzmann model (Huang, Wu & Adams, arXiv:1809.02390).
 *
 * The paper works on D2Q9 and states that the extension to a 3-D lattice is
 * straightforward though tedious (main text, after Eq. 2), without giving it.
 * The 3-D model of this library keeps every construction of the paper on the
 * D3Q19 lattice with orthogonal moments without weights (Eq. 2): the equilibrium
 * of Eq. 3 is the lattice's second-order Hermite equilibrium with eta in the
 * energy moment (p_LBE = c_s^2 (rho + eta), Eq. 9) and beta_2 eta in the
 * fourth-order moment; the force term of Eq. 4 is the second-order Hermite
 * force; S (Eq. 6) couples e to eps and to q, and the traceless second-order
 * moments to q, through velocity-dependent entries; Q_m (Eq. 14) has the
 * paper's second-order tensor (2 F~F~ + |F~|^2 I)/24.  The coefficients follow
 * from the same Chapman-Enskog conditions as Eqs. 7 and 16 on the D3Q19 moment
 * set:
 *   k = 38 (1 - varpi)/11, beta_2 = -19/k, b = 21 (1 - varpi)/(5 (7 - 18 varpi)),
 *   h = 798 varpi (1 - varpi)/(5 (7 - 18 varpi)),
 *   tau_p tau_q = (1 + 5k/19) tau_e tau_q = 1/12,
 * with varpi the ratio of the bulk viscosity to the plain lattice's
 * (2/3) c_s^2 (1/s_e - 1/2).  The recovered pressure tensor is Eq. 17, so
 * lb_derive's coexistence densities, G and c^2 (Eqs. 18-22) hold unchanged.  The
 * cubic-velocity corrections R, T, X (Eq. 10) are not part of the 3-D model.
 * The rates without a 2-D counterpart are fixed: s_m = s_q for the third-order
 * m moments, s_pi = s_eps for the anisotropic fourth-order moments, and
 * s_eps = 1.75 unless lb_params.s_eps gives it (s_eps = s_e lets the
 * checkerboard mode k = (pi, pi, pi) grow in the gas).
 *
 * Populations are stored as deviations fbar_i - w_i rho_ref in SoA layout
 * [19][nz][ny][nx] (x fastest), FP64 or FP32; lb_d3_velocities gives the order
 * of the 19 planes.  Errors: the codes of lbm.h, message in lb_last_error(NULL)
 * for calls without a handle and lb_d3_last_error(h) otherwise. */
#ifndef LBM3D_H
#define LBM3D_H

#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_d3_handle lb_d3_handle;

/* The 19 lattice velocities in plane order (ex[i], ey[i], ez[i]). */
void lb_d3_velocities(int* ex, int* ey, int* ez);

/* As lb_derive for the D3Q19 model: coexistence densities, lam, G2, c^2, W1 and
 * sigma1 as for D2Q9 (Eqs. 17-22); s_q, s_e from the 3-D closure above when
 * given as <= 0; k, h, b, beta2 the 3-D coefficients; s_eps = 1.75 when <= 0.
 * nx, ny, nz >= 1 and nx ny nz < 2^31 (32-bit node indices; population planes
 * are addressed with 64-bit offsets once 19 nx ny nz reaches 2^31).  precision:
 * LB_FP64 or LB_FP32 (FP16 storage: LB_ENOTSUP); layout must be
 * LB_LAYOUT_PLANES; variant LB_AUTO or LB_FUSED; varpi 7/18 (singular b and h)
 * and 1 are rejected. */
int lb_d3_derive(const lb_params* p, int32_t nz, lb_derived* out);

/* Bytes of one population buffer: 19 nx ny nz times the element size. */
size_t lb_d3_state_bytes(const lb_params* p, int32_t nz);

/* Creates a handle on the caller's device buffers f_a and f_b (lb_d3_state_bytes
 * each, distinct; ping-pong, f_a holds the state after init) and stream (NULL:
 * the legacy default stream), and initialises the lattice at rest:
 * fbar_i = (M^-1 m_eq(rho0, u = 0))_i - w_i rho_ref, computed in FP64 and rounded
 * to the storage type.  rho0: nx ny nz doubles [z][y][x], on the host
 * (rho0_on_device = 0; copied through f_b) or the device (1).  rho_ref = NaN takes
 * the mean of rho0 (computed in FP64).  Densities that are not positive and
 * finite, or for vdW not below 1/b, are reported as LB_EINVAL (checked on the
 * device; the handle is not created).  The handle owns a 33 KB device workspace
 * for lb_d3_reduce (LB_ENOMEM if it cannot be allocated), its graphs and a
 * private capture stream, all released by lb_d3_free.  Synchronous. */
int lb_d3_init(lb_d3_handle** out, const lb_params* p, int32_t nz, void* f_a, void* f_b, const double* rho0,
               int rho0_on_device, void* stream);

/* Advances nsteps >= 0 time steps on the handle's stream (asynchronous).  Runs of
 * 64 steps replay a CUDA graph captured on first use (one per starting buffer, on a
 * private stream); the remaining steps, and all steps while the handle's stream is
 * being captured into the caller's own graph, are plain launches; the results are
 * the same bits either way.  Each step is the fused kernel: pull streaming,
 * density with its one-node ring, force stencil (Eq. 12 with omega = 1/6 on the
 * axes, 1/12 on the edges), velocity (Eq. 5), EOS, equilibrium, forcing, Q_m,
 * collision (Eq. 13 without R, T, X) and store. */
int lb_d3_step(lb_d3_handle* h, int64_t nsteps);

/* rho (required) and the velocity components (each may be NULL) of the current
 * state as FP64 device arrays of nx ny nz, [z][y][x]:
 * rho = sum_i fbar_i + rho_ref, rho u = sum_i e_i fbar_i - F/2 (Eq. 5 for
 * post-collision populations).  Asynchronous on the handle's stream. */
int lb_d3_moments(lb_d3_handle* h, void* rho, void* ux, void* uy, void* uz);

/* FP64 diagnostics of the current state, computed on the device and copied to out
 * (synchronous): out[0] mass = sum rho, out[1..3] sum_i e_i fbar_i over the lattice
 * (the total momentum: the interaction forces sum to zero on a periodic lattice),
 * out[4] nodes with rho above (rho_g + rho_l)/2, out[5] min rho, out[6] max rho,
 * out[7] nodes whose density is not finite (excluded from 0-6).  Returns
 * LB_ENONFINITE when out[7] > 0 (out is filled).  Uses a workspace of about 33 KB
 * that lb_d3_init allocates. */
int lb_d3_reduce(lb_d3_handle* h, double out[8]);

/* Device buffer holding the current state (f_a or f_b). */
void* lb_d3_state(const lb_d3_handle* h);

/* Copies the current state to / from a device buffer of lb_d3_state_bytes
 * (asynchronous on the handle's stream). */
int lb_d3_get_state(lb_d3_handle* h, void* dst);
int lb_d3_set_state(lb_d3_handle* h, const void* src);

/* Parameters in use (with rho_ref as taken) and the derived quantities. */
int lb_d3_get_params(const lb_d3_handle* h, lb_params* out, lb_derived* derived);

/* Last error message of a handle (empty when none). */
const char* lb_d3_last_error(const lb_d3_handle* h);

/* Destroys the handle (the buffers stay the caller's). */
void lb_d3_free(lb_d3_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* LBM3D_H */
