// Kernels of the time step and its diagnostics (sm_103a).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

constexpr int kFusedThreads = 256;  // 8 warps; each warp owns a 32-column strip of rows
constexpr int kReduceThreads = 256;
constexpr int kReduceSlots = 8;     // doubles per block partial

__host__ __device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Pulls the nine populations of row r at columns (cm, cc, cp) = (x-1, x, x+1):
// f_i(x, r) = fbar_i(x - e_i, r - e_i) (supplement Eq. 2), periodic.
template <typename real, typename store_t>
__device__ __forceinline__ void pull_row(const store_t* __restrict__ fin, size_t plane, int nx, int ny, int r,
                                         int cm, int cc, int cp, real (&f)[9]) {
  const int rm = r == 0 ? ny - 1 : r - 1, rp = r == ny - 1 ? 0 : r + 1;
  const size_t oc = size_t(r) * nx, om = size_t(rm) * nx, op = size_t(rp) * nx;
  f[0] = ld_st(fin + oc + cc);
  f[1] = ld_st(fin + plane + oc + cm);
  f[2] = ld_st(fin + 2 * plane + om + cc);
  f[3] = ld_st(fin + 3 * plane + oc + cp);
  f[4] = ld_st(fin + 4 * plane + op + cc);
  f[5] = ld_st(fin + 5 * plane + om + cm);
  f[6] = ld_st(fin + 6 * plane + om + cp);
  f[7] = ld_st(fin + 7 * plane + op + cp);
  f[8] = ld_st(fin + 8 * plane + op + cm);
}

template <typename real>
__device__ __forceinline__ real sum9(const real (&f)[9]) {
  return ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
}

// Fused stream + force + collide step.  Each warp owns a strip of 32 columns
// [32*strip, 32*strip + 32) and a chunk of rows, and marches down the rows:
// lane l pulls the populations of its column, sums the density, exchanges the
// neighbour densities with warp shuffles (lanes 0 and 31 also compute the
// density of the column just outside the strip), and collides.  The pull of
// row y + 2 is issued before the collision of row y so that it is in flight
// while the warp computes.  No shared memory, no block barrier.
template <typename real, typename store_t>
__global__ void __launch_bounds__(kFusedThreads)
    k_step_fused(const store_t* __restrict__ fin, store_t* __restrict__ fout, int nx, int ny, int nstrips,
                 int rows_per_warp, int nwork, Coef<real> c) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kFusedThreads + threadIdx.x) >> 5;
  if (warp >= nwork) return;  // uniform per warp
  const int strip = warp % nstrips, chunk = warp / nstrips;
  const int xl = strip * 32 + lane;
  const int xc = wrap(xl, nx), xm = wrap(xl - 1, nx), xp = wrap(xl + 1, nx);
  const bool edge = lane == 0 || lane == 31;
  const int hl = lane == 0 ? xl - 1 : xl + 1;  // halo column of the edge lanes
  const int hc = wrap(hl, nx), hm = wrap(hl - 1, nx), hp = wrap(hl + 1, nx);
  const bool writer = xl < nx;
  const int y0 = chunk * rows_per_warp;
  const int y1 = min(y0 + rows_per_warp, ny);
  const size_t plane = size_t(nx) * ny;

  real fa[9], fb[9], ft[9];
  real rm, rc, rp, hmv = 0, hcv = 0, hpv = 0;
  pull_row(fin, plane, nx, ny, wrap(y0 - 1, ny), xm, xc, xp, ft);
  rm = sum9(ft);
  if (edge) {
    pull_row(fin, plane, nx, ny, wrap(y0 - 1, ny), hm, hc, hp, ft);
    hmv = sum9(ft);
  }
  pull_row(fin, plane, nx, ny, y0, xm, xc, xp, fa);
  rc = sum9(fa);
  if (edge) {
    pull_row(fin, plane, nx, ny, y0, hm, hc, hp, ft);
    hcv = sum9(ft);
  }
  pull_row(fin, plane, nx, ny, wrap(y0 + 1, ny), xm, xc, xp, fb);
  rp = sum9(fb);
  if (edge) {
    pull_row(fin, plane, nx, ny, wrap(y0 + 1, ny), hm, hc, hp, ft);
    hpv = sum9(ft);
  }

  for (int y = y0; y < y1; ++y) {
    const bool more = y + 1 < y1;
    real fc[9];
    if (more) {
      pull_row(fin, plane, nx, ny, wrap(y + 2, ny), xm, xc, xp, fc);
      if (edge) pull_row(fin, plane, nx, ny, wrap(y + 2, ny), hm, hc, hp, ft);
    }
    // Neighbour densities: left from lane - 1, right from lane + 1, halos at the ends.
    real l_m = __shfl_up_sync(0xffffffffu, rm, 1), r_m = __shfl_down_sync(0xffffffffu, rm, 1);
    real l_c = __shfl_up_sync(0xffffffffu, rc, 1), r_c = __shfl_down_sync(0xffffffffu, rc, 1);
    real l_p = __shfl_up_sync(0xffffffffu, rp, 1), r_p = __shfl_down_sync(0xffffffffu, rp, 1);
    if (lane == 0) {
      l_m = hmv;
      l_c = hcv;
      l_p = hpv;
    } else if (lane == 31) {
      r_m = hmv;
      r_c = hcv;
      r_p = hpv;
    }
    real Sx, Sy;
    stencil(l_m, rm, r_m, l_c, r_c, l_p, rp, r_p, Sx, Sy);
    real o[9];
    collide(c, fa, Sx, Sy, o);
    if (writer) {
      const size_t off = size_t(y) * nx + xc;
#pragma unroll
      for (int i = 0; i < 9; ++i) st_st(fout + i * plane + off, o[i]);
    }
    if (more) {
      rm = rc;
      rc = rp;
      rp = sum9(fc);
      hmv = hcv;
      hcv = hpv;
      if (edge) hpv = sum9(ft);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        fa[i] = fb[i];
        fb[i] = fc[i];
      }
    }
  }
}

// Two-pass variant, pass 1: density plane rho_dev(x) = sum_i fbar_i(x - e_i).
template <typename real, typename store_t>
__global__ void k_density(const store_t* __restrict__ fin, real* __restrict__ rho, int nx, int ny) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  real f[9];
  pull_row(fin, size_t(nx) * ny, nx, ny, y, x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1, f);
  rho[size_t(y) * nx + x] = sum9(f);
}

// Two-pass variant, pass 2: pull, force stencil from the density plane, collide.
template <typename real, typename store_t>
__global__ void k_collide_rho(const store_t* __restrict__ fin, store_t* __restrict__ fout,
                              const real* __restrict__ rho, int nx, int ny, Coef<real> c) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const size_t plane = size_t(nx) * ny;
  real f[9];
  pull_row(fin, plane, nx, ny, y, xm, x, xp, f);
  const real* rm = rho + size_t(ym) * nx;
  const real* rc = rho + size_t(y) * nx;
  const real* rpp = rho + size_t(yp) * nx;
  real Sx, Sy;
  stencil(__ldg(rm + xm), __ldg(rm + x), __ldg(rm + xp), __ldg(rc + xm), __ldg(rc + xp), __ldg(rpp + xm),
          __ldg(rpp + x), __ldg(rpp + xp), Sx, Sy);
  real o[9];
  collide(c, f, Sx, Sy, o);
  const size_t off = size_t(y) * nx + x;
#pragma unroll
  for (int i = 0; i < 9; ++i) st_st(fout + i * plane + off, o[i]);
}

// Rest equilibrium from an initial density (computed in FP64, rounded once):
// m_eq(rho, u = 0) = (rho, -2 rho + 2 eta, rho + beta_2 eta, 0, ...), minus rho_ref M w.
template <typename store_t>
__global__ void k_init_rest(const double* __restrict__ rho0, store_t* __restrict__ f, int nx, int ny,
                            Coef<double> c) {
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t N = size_t(nx) * ny;
  if (n >= N) return;
  const double rho = rho0[n];
  double pe, dpe;
  eos(c, rho, pe, dpe);
  const double eta = 3.0 * (pe + 0.5 * c.G2 * rho * rho) - rho;
  const double n0 = (rho - c.rho_ref) / 9.0;
  const double n1 = (-2.0 * rho + 2.0 * eta + 2.0 * c.rho_ref) / 36.0;
  const double n2 = (rho + c.beta2 * eta - c.rho_ref) / 36.0;
  const double axis = n0 - n1 - 2.0 * n2, diag = n0 + 2.0 * n1 + n2;
  if constexpr (sizeof(store_t) == 8) {
    f[n] = n0 - 4.0 * n1 + 4.0 * n2;
    for (int i = 1; i <= 4; ++i) f[i * N + n] = axis;
    for (int i = 5; i <= 8; ++i) f[i * N + n] = diag;
  } else {
    st_st(f + n, float(n0 - 4.0 * n1 + 4.0 * n2));
    for (int i = 1; i <= 4; ++i) st_st(f + i * N + n, float(axis));
    for (int i = 5; i <= 8; ++i) st_st(f + i * N + n, float(diag));
  }
}

// rho = sum_i fbar_i + rho_ref at every node (no pull: the stored state is post-collision).
template <typename real, typename store_t>
__global__ void k_rho_local(const store_t* __restrict__ f, real* __restrict__ rho, int nx, int ny, real rho_ref) {
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t N = size_t(nx) * ny;
  if (n >= N) return;
  real s = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) s += ld_st(f + i * N + n);
  rho[n] = s + rho_ref;
}

// rho u = sum_i e_i fbar_i - F/2 with F from the density plane.
template <typename real, typename store_t>
__global__ void k_velocity(const store_t* __restrict__ f, const real* __restrict__ rho, real* __restrict__ ux,
                           real* __restrict__ uy, int nx, int ny, real G2) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const size_t N = size_t(nx) * ny, n = size_t(y) * nx + x;
  real d[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) d[i] = ld_st(f + i * N + n);
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
    k_reduce_partial(const store_t* __restrict__ f, const real* __restrict__ rho, int nx, int ny, real G2,
                     double rho_mid, double* __restrict__ partial) {
  const size_t N = size_t(nx) * ny;
  double acc[kReduceSlots] = {0, 0, 0, 0, 1e300, -1e300, 0, 0};
  for (size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x; n < N; n += size_t(gridDim.x) * blockDim.x) {
    const int y = int(n / nx), x = int(n - size_t(y) * nx);
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    real d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = ld_st(f + i * N + n);
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

// Folds the block partials in a fixed order (deterministic) into out[kReduceSlots].
__global__ void k_reduce_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
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
