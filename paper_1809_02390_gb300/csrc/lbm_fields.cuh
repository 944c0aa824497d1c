// Initial states and diagnostics of a lattice (sm_103a): the equilibrium state of a
// density and velocity field, the local density, the EOS pressure, the velocity
// of Eq. 5, and the FP64 reductions (mass, momentum, liquid area, extremes).
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int kReduceThreads = 256;
constexpr int kReduceSlots = 8;  // doubles per block partial
// Largest grid of k_reduce_partial: the partials buffer of lb_reduce (caller's
// scratch) and of lb_reduce_static (static array) both hold this many blocks, and
// both take min(2 x SMs, this) blocks, so the two calls sum in the same order.
constexpr int kMaxReduceBlocks = 1024;

// p_EOS / c^2 of one density in FP64 on the host (the probes of the reductions):
// vdW rho R T/(1 - b rho) - a rho^2, Carnahan-Starling (Eq. 20) with t = b rho / 4,
// both times K_EOS / c^2.
inline double p_eos_host(const VCoef<double>& c, double r) {
  if (c.eos == LB_EOS_VDW) return c.lam * (r * c.RT / (1.0 - c.bq * r) - c.a * r * r);
  const double t = c.bq * r, om = 1.0 - t;
  return c.lam * (r * c.RT * (1.0 + t + t * t - t * t * t) / (om * om * om) - c.a * r * r);
}

// The rest state of lb_init (u = 0) from an initial density field: f_i = (M^-1
// m_eq(rho, 0))_i - w_i rho_ref with m_eq of Eq. 3 and the self-tuning eta, in the
// compute type `real` (FP64 for FP64 storage; FP32 for FP32 and FP16 storage, where
// FP64 arithmetic on this GPU would cost more than the 20 steps after it), and, if
// bad is not null, the check of the density: bad[0] = smallest index of a density
// that is not positive and finite, bad[1] = smallest index of one at or above 1/b
// (vdW: 1 - b rho must stay positive); both start at 0xff..ff (none), and the
// check is done in FP64 on the given density.
template <typename store_t, typename real>
__global__ void k_init_rest(const double* __restrict__ rho0, store_t* __restrict__ f, int nx, int ny, Strides st,
                            VCoef<real> c, unsigned long long* __restrict__ bad, double vdw_b) {
  const size_t k = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= size_t(nx) * ny) return;
  const double r64 = rho0[k];
  if (bad) {
    if (!(r64 > 0.0) || !isfinite(r64)) atomicMin(&bad[0], static_cast<unsigned long long>(k));
    if (vdw_b > 0.0 && !(vdw_b * r64 < 1.0)) atomicMin(&bad[1], static_cast<unsigned long long>(k));
  }
  const size_t N = size_t(st.ps);                              // plane stride
  const size_t n = size_t(st.at(0, int(k % nx), int(k / nx)));  // node (x, y)
  const real rho = real(r64);
  real pe, dpe;
  eos(c, rho, pe, dpe);
  const real eta = real(3) * (pe + real(0.5) * c.G2 * rho * rho) - rho;
  const real n0 = (rho - c.rho_ref) / real(9);
  const real n1 = (real(-2) * rho + real(2) * eta + real(2) * c.rho_ref) / real(36);
  const real n2 = (rho + c.beta2 * eta - c.rho_ref) / real(36);
  const real axis = n0 - n1 - real(2) * n2, diag = n0 + real(2) * n1 + n2;
  const real o[9] = {n0 - real(4) * n1 + real(4) * n2, axis, axis, axis, axis, diag, diag, diag, diag};
#pragma unroll
  for (int i = 0; i < 9; ++i) st_st(f + (n + size_t(i) * N), o[i]);
}

// Equilibrium state from a density and a velocity field (computed in FP64, rounded
// once): m_eq(rho, u) of Eq. 3 with the self-tuning eta (alpha_1 = -1, beta_1 = 1,
// alpha_2 = 1), momentum rho u (c = 1), minus rho_ref M w, then the inverse
// transform M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
// ux = uy = null: the rest state (u = 0), without the velocity terms (FP64 is
// slow on this GPU: the rest state of a 4096^2 lattice takes 1.6 ms, 5.4 ms with
// them).
template <typename store_t>
__global__ void k_init_eq(const double* __restrict__ rho0, const double* __restrict__ ux0,
                          const double* __restrict__ uy0, store_t* __restrict__ f, int nx, int ny, Strides st,
                          VCoef<double> c) {
  const size_t k = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= size_t(nx) * ny) return;
  const size_t N = size_t(st.ps);                                    // plane stride
  const size_t n = size_t(st.at(0, int(k % nx), int(k / nx)));        // node (x, y)
  const double rho = rho0[k];
  double pe, dpe;
  eos(c, rho, pe, dpe);
  const double eta = 3.0 * (pe + 0.5 * c.G2 * rho * rho) - rho;
  double o[9];
  if (!ux0 && !uy0) {
    const double n0 = (rho - c.rho_ref) / 9.0;
    const double n1 = (-2.0 * rho + 2.0 * eta + 2.0 * c.rho_ref) / 36.0;
    const double n2 = (rho + c.beta2 * eta - c.rho_ref) / 36.0;
    const double axis = n0 - n1 - 2.0 * n2, diag = n0 + 2.0 * n1 + n2;
    o[0] = n0 - 4.0 * n1 + 4.0 * n2;
    o[1] = o[2] = o[3] = o[4] = axis;
    o[5] = o[6] = o[7] = o[8] = diag;
  } else {
    const double ux = ux0 ? ux0[k] : 0.0, uy = uy0 ? uy0[k] : 0.0;
    const double x2 = ux * ux, y2 = uy * uy, r3u2 = 3.0 * rho * (x2 + y2);
    const double m1 = 2.0 * (eta - rho) + r3u2;
    const double m2 = 9.0 * rho * x2 * y2 + (c.beta2 * eta + rho) - r3u2;
    const double n0 = (rho - c.rho_ref) / 9.0;
    const double n1 = (m1 + 2.0 * c.rho_ref) / 36.0;
    const double n2 = (m2 - c.rho_ref) / 36.0;
    const double sixth = 1.0 / 6.0, twelfth = 1.0 / 12.0;
    const double n3 = rho * ux * sixth, n5 = rho * uy * sixth;
    const double n4 = rho * ux * (3.0 * y2 - 1.0) * twelfth, n6 = rho * uy * (3.0 * x2 - 1.0) * twelfth;
    const double n7 = 0.25 * rho * (x2 - y2), n8 = 0.25 * rho * ux * uy;
    const double axis = n0 - n1 - 2.0 * n2, diag = n0 + 2.0 * n1 + n2;
    const double px = n3 - 2.0 * n4, py = n5 - 2.0 * n6, qx = n3 + n4, qy = n5 + n6;
    o[0] = n0 - 4.0 * n1 + 4.0 * n2;
    o[1] = axis + n7 + px;
    o[2] = axis - n7 + py;
    o[3] = axis + n7 - px;
    o[4] = axis - n7 - py;
    o[5] = diag + n8 + (qx + qy);
    o[6] = diag - n8 + (qy - qx);
    o[7] = diag + n8 - (qx + qy);
    o[8] = diag - n8 + (qx - qy);
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    if constexpr (sizeof(store_t) == 8)
      f[i * N + n] = o[i];
    else
      st_st(f + i * N + n, float(o[i]));
  }
}

// rho = sum_i fbar_i + rho_ref at every node (no pull: the stored state is post-collision).
template <typename real, typename store_t>
__global__ void k_rho_local(const store_t* __restrict__ f, real* __restrict__ rho, int nx, int ny, Strides st,
                            real rho_ref) {
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= size_t(nx) * ny) return;
  const int y = int(n / nx), o = st.at(0, int(n - size_t(y) * nx), y);
  real s = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) s += ld_st(f + (o + i * st.ps));
  rho[n] = s + rho_ref;
}

// p_EOS / c^2 at every node from rho = sum_i fbar_i + rho_ref (Eq. 20 or vdW, times K_EOS).
template <typename real, typename store_t>
__global__ void k_pressure(const store_t* __restrict__ f, real* __restrict__ p, int nx, int ny, Strides st,
                           VCoef<real> c) {
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= size_t(nx) * ny) return;
  const int y = int(n / nx), o = st.at(0, int(n - size_t(y) * nx), y);
  real s = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) s += ld_st(f + (o + i * st.ps));
  real pe, dpe;
  eos(c, s + c.rho_ref, pe, dpe);
  p[n] = pe;
}

// rho u = sum_i e_i fbar_i - F/2 with F from the density plane.
template <typename real, typename store_t>
__global__ void k_velocity(const store_t* __restrict__ f, const real* __restrict__ rho, real* __restrict__ ux,
                           real* __restrict__ uy, int nx, int ny, Strides st, real G2) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const size_t n = size_t(y) * nx + x;
  real d[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) d[i] = ld_st(f + st.at(i, x, y));
  real Sx, Sy;
  stencil(rho[size_t(ym) * nx + xm], rho[size_t(ym) * nx + x], rho[size_t(ym) * nx + xp], rho[n - x + xm],
          rho[n - x + xp], rho[size_t(yp) * nx + xm], rho[size_t(yp) * nx + x], rho[size_t(yp) * nx + xp], Sx,
          Sy);
  const real r = rho[n];
  const real jx = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
  const real jy = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
  if (ux) ux[n] = (jx - real(0.5) * G2 * r * Sx) / r;
  if (uy) uy[n] = (jy - real(0.5) * G2 * r * Sy) / r;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Per-block FP64 partials: mass, momentum x/y, count(rho > rho_mid), min, max,
// non-finite count.  rho: density plane (full density).
template <typename real, typename store_t>
__global__ void __launch_bounds__(kReduceThreads)
    k_reduce_partial(const store_t* __restrict__ f, const real* __restrict__ rho, int nx, int ny, Strides st,
                     real G2, double rho_mid, double* __restrict__ partial) {
  const size_t N = size_t(nx) * ny;
  double acc[kReduceSlots] = {0, 0, 0, 0, 1e300, -1e300, 0, 0};
  for (size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x; n < N; n += size_t(gridDim.x) * blockDim.x) {
    const int y = int(n / nx), x = int(n - size_t(y) * nx);
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    real d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = ld_st(f + st.at(i, x, y));
    real Sx, Sy;
    stencil(rho[size_t(ym) * nx + xm], rho[size_t(ym) * nx + x], rho[size_t(ym) * nx + xp], rho[n - x + xm],
            rho[n - x + xp], rho[size_t(yp) * nx + xm], rho[size_t(yp) * nx + x], rho[size_t(yp) * nx + xp],
            Sx, Sy);
    const double r = rho[n];
    const double jx = double(d[1] - d[3] + d[5] - d[6] - d[7] + d[8]) - 0.5 * double(G2) * r * double(Sx);
    const double jy = double(d[2] - d[4] + d[5] + d[6] - d[7] - d[8]) - 0.5 * double(G2) * r * double(Sy);
    if (isfinite(r)) {
      acc[0] += r;
      acc[1] += jx;
      acc[2] += jy;
      acc[3] += r > rho_mid ? 1.0 : 0.0;
      acc[4] = fmin(acc[4], r);
      acc[5] = fmax(acc[5], r);
    } else {
      acc[6] += 1.0;
    }
  }
  __shared__ double sh[kReduceThreads / 32][kReduceSlots];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kReduceSlots; ++k) {
    const double v = k == 4 ? warp_min(acc[k]) : k == 5 ? warp_max(acc[k]) : warp_sum(acc[k]);
    if (lane == 0) sh[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kReduceSlots) {
    const int k = threadIdx.x;
    double v = sh[0][k];
    for (int j = 1; j < kReduceThreads / 32; ++j)
      v = k == 4 ? fmin(v, sh[j][k]) : k == 5 ? fmax(v, sh[j][k]) : v + sh[j][k];
    partial[size_t(blockIdx.x) * kReduceSlots + k] = v;
  }
}

// Block sums of x[0 .. n) in FP64: partial[b] = the sum of block b's grid-stride
// share (a fixed order for a given grid, so that repeated calls agree bit for bit).
static __global__ void __launch_bounds__(kReduceThreads)
    k_sum_partial(const double* __restrict__ x, long long n, double* __restrict__ partial) {
  double s = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    s += x[k];
  __shared__ double sh[kReduceThreads / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = sh[0];
    for (int j = 1; j < kReduceThreads / 32; ++j) v += sh[j];
    partial[blockIdx.x] = v;
  }
}

// Folds the block partials in a fixed order (deterministic) into out[kReduceSlots].
static __global__ void k_reduce_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= kReduceSlots) return;
  double v = partial[k];
  for (int b = 1; b < nblocks; ++b) {
    const double u = partial[size_t(b) * kReduceSlots + k];
    v = k == 4 ? fmin(v, u) : k == 5 ? fmax(v, u) : v + u;
  }
  out[k] = v;
}

}  // namespace lbm
