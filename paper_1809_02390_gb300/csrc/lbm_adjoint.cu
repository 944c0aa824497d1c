// Adjoint of one time step (lb_adjoint_step).
//
// Forward step: f = pull(s) (supplement Eq. 2), rho = sum_i f_i, S(x) = sum_j
// omega_j rho(x + e_j) e_j (Eq. 12), s'(x) = C(f(x), S(x); theta) (Eq. 13).
// Given lam' = dL/ds', the adjoint is
//   (mu, Sb, thetab)(x) = VJP of C at (f(x), S(x)) with lam'(x)      [k_adj_local]
//   rhob(y) = sum_j omega_j e_j . Sb(y - e_j)        (transposed stencil)
//   lam_i(z) = mu_i(z + e_i) + rhob(z + e_i)         (transposed pull) [k_adj_transpose]
// and dL/dtheta += sum_x thetab(x), reduced per block in FP64, folded in a
// fixed order (deterministic).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdio>

#include "lbm_adjoint.cuh"
#include "lbm_handle.cuh"
#include "lbm_tma.cuh"

namespace {

using namespace lbm;

constexpr int kAdjThreads = 256;

template <typename real, typename store_t>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_local(const store_t* __restrict__ s, const real* __restrict__ lam_in, real* __restrict__ mu,
                real* __restrict__ sbar, double* __restrict__ partial, int nx, int ny, VCoef<real> c) {
  __shared__ real rs[kTileY + 2][kTileX + 2];
  __shared__ double red[kAdjThreads / 32][3];
  const int tx = threadIdx.x & (kTileX - 1), ty = threadIdx.x / kTileX;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  const int plane = nx * ny;
  const int gx = x0 + tx;
  const int xc = wrap(gx, nx);
  const int xm = xc == 0 ? nx - 1 : xc - 1, xp = xc == nx - 1 ? 0 : xc + 1;
  real f[kTileRows][9];
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int gy = y0 + ty + k * kRowStride;
    pull_row(s, plane, nx, ny, wrap(gy, ny), xm, xc, xp, f[k]);
    rs[ty + k * kRowStride + 1][tx + 1] = sum9(f[k]);
  }
  for (int t = threadIdx.x; t < 2 * (kTileX + 2) + 2 * kTileY; t += kAdjThreads) {
    int wx, wy;
    if (t < kTileX + 2) {
      wx = t, wy = 0;
    } else if (t < 2 * (kTileX + 2)) {
      wx = t - (kTileX + 2), wy = kTileY + 1;
    } else if (t < 2 * (kTileX + 2) + kTileY) {
      wx = 0, wy = t - 2 * (kTileX + 2) + 1;
    } else {
      wx = kTileX + 1, wy = t - 2 * (kTileX + 2) - kTileY + 1;
    }
    const int hx = wrap(x0 - 1 + wx, nx), hy = wrap(y0 - 1 + wy, ny);
    real g[9];
    pull_row(s, plane, nx, ny, hy, hx == 0 ? nx - 1 : hx - 1, hx, hx == nx - 1 ? 0 : hx + 1, g);
    rs[wy][wx] = sum9(g);
  }
  __syncthreads();
  // Parameter cotangents summed in the compute type within a warp (FP64 arithmetic
  // is slow on this GPU); warp partials are folded in FP64.
  real acc[3] = {real(0), real(0), real(0)};
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int ly = ty + k * kRowStride + 1, lx = tx + 1;
    const int gy = y0 + ly - 1;
    if (gx >= nx || gy >= ny) continue;
    real Sx, Sy;
    stencil(rs[ly - 1][lx - 1], rs[ly - 1][lx], rs[ly - 1][lx + 1], rs[ly][lx - 1], rs[ly][lx + 1],
            rs[ly + 1][lx - 1], rs[ly + 1][lx], rs[ly + 1][lx + 1], Sx, Sy);
    const int off = gy * nx + gx;
    real ob[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) ob[i] = lam_in[i * plane + off];
    AdjOut<real> r;
    collide_vjp(c, f[k], Sx, Sy, ob, r);
#pragma unroll
    for (int i = 0; i < 9; ++i) mu[i * plane + off] = r.d[i];
    sbar[off] = r.Sx;
    sbar[plane + off] = r.Sy;
    acc[0] += r.RT;
    acc[1] += r.G2;
    acc[2] += r.lam;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    real v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][k] = double(v);
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int j = 0; j < kAdjThreads / 32; ++j) v += red[j][threadIdx.x];
    partial[(size_t(blockIdx.y) * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = v;
  }
}

// rhob(y) = sum_j omega_j e_j . Sb(y - e_j), read from the two Sb planes.
template <typename real>
__device__ __forceinline__ real stencil_t(const real* __restrict__ sbar, int plane, int nx, int ny, int x, int y) {
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const real* bx = sbar;
  const real* by = sbar + plane;
  const real third = real(1.0 / 3.0), twelfth = real(1.0 / 12.0);
  const real ax = bx[y * nx + xm] - bx[y * nx + xp];
  const real ay = by[ym * nx + x] - by[yp * nx + x];
  const real d5 = bx[ym * nx + xm] + by[ym * nx + xm];   // e = (+1, +1) from (x-1, y-1)
  const real d6 = by[ym * nx + xp] - bx[ym * nx + xp];   // e = (-1, +1) from (x+1, y-1)
  const real d7 = -bx[yp * nx + xp] - by[yp * nx + xp];  // e = (-1, -1) from (x+1, y+1)
  const real d8 = bx[yp * nx + xm] - by[yp * nx + xm];   // e = (+1, -1) from (x-1, y+1)
  return third * (ax + ay) + twelfth * ((d5 + d6) + (d7 + d8));
}

template <typename real>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_transpose(const real* __restrict__ mu, const real* __restrict__ sbar, real* __restrict__ lam_out, int nx,
                    int ny) {
  __shared__ real rb[kTileY + 2][kTileX + 2];
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  const int plane = nx * ny;
  for (int t = threadIdx.x; t < (kTileY + 2) * (kTileX + 2); t += kAdjThreads) {
    const int wy = t / (kTileX + 2), wx = t - wy * (kTileX + 2);
    rb[wy][wx] = stencil_t(sbar, plane, nx, ny, wrap(x0 - 1 + wx, nx), wrap(y0 - 1 + wy, ny));
  }
  __syncthreads();
  const int tx = threadIdx.x & (kTileX - 1), ty = threadIdx.x / kTileX;
  const int gx = x0 + tx;
  if (gx >= nx) return;
  const int xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int gy = y0 + ty + k * kRowStride;
    if (gy >= ny) continue;
    const int ym = gy == 0 ? ny - 1 : gy - 1, yp = gy == ny - 1 ? 0 : gy + 1;
    const int ly = ty + k * kRowStride + 1, lx = tx + 1;
    // lam_i(z) = mu_i(z + e_i) + rhob(z + e_i).
    const int oc = gy * nx, om = ym * nx, op = yp * nx;
    const int off = oc + gx;
    lam_out[off] = mu[off] + rb[ly][lx];
    lam_out[plane + off] = mu[plane + oc + xp] + rb[ly][lx + 1];
    lam_out[2 * plane + off] = mu[2 * plane + op + gx] + rb[ly + 1][lx];
    lam_out[3 * plane + off] = mu[3 * plane + oc + xm] + rb[ly][lx - 1];
    lam_out[4 * plane + off] = mu[4 * plane + om + gx] + rb[ly - 1][lx];
    lam_out[5 * plane + off] = mu[5 * plane + op + xp] + rb[ly + 1][lx + 1];
    lam_out[6 * plane + off] = mu[6 * plane + op + xm] + rb[ly + 1][lx - 1];
    lam_out[7 * plane + off] = mu[7 * plane + om + xm] + rb[ly - 1][lx - 1];
    lam_out[8 * plane + off] = mu[8 * plane + om + xp] + rb[ly - 1][lx + 1];
  }
}

// dtheta[k] += sum over blocks of partial[b][k], in a fixed order.
__global__ void k_adj_theta(const double* __restrict__ partial, int nblocks, double RT_over_T,
                            double* __restrict__ dtheta) {
  __shared__ double sh[256];
  for (int k = 0; k < 3; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) v += partial[size_t(b) * 3 + k];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) dtheta[k] += k == 0 ? sh[0] * RT_over_T : sh[0];
    __syncthreads();
  }
}

// Fused adjoint step on the (mu, Sb) representation of the cotangent: the
// cotangent of the state after step n+1 is lam(z) = mu'_i(z + e_i) + rhob'(z + e_i)
// with rhob' the transposed stencil of Sb'.  One kernel per step reads the state
// s^n (with its density ring), mu' (pulled backwards) and Sb' (with a two-node
// ring, staged in shared memory), forms lam at each node, and writes the local
// VJP (mu, Sb) of step n: 124 B per node in FP32 against 196 B for
// k_adj_local + k_adj_transpose.  The VJP runs node by node in scalar FP32: as a
// packed pair (two nodes per FFMA2) its live set needs 128 registers (2 blocks/SM)
// or spills 350 bytes per thread at 80, and either way the step was 20% slower.
// Resident blocks per SM: 3 for FP32 (<= 85 registers), 1 for FP64.
template <typename real>
constexpr int adj_min_blocks() {
  return sizeof(real) == 8 ? 1 : 3;
}

template <typename real, typename store_t>
__global__ void __launch_bounds__(kAdjThreads, adj_min_blocks<real>())
    k_adj_fused(const store_t* __restrict__ s, const real* __restrict__ mu_in, const real* __restrict__ sb_in,
                real* __restrict__ mu, real* __restrict__ sbar, double* __restrict__ partial, int accumulate, int nx,
                int ny, VCoef<real> c) {
  __shared__ real rs[kTileY + 2][kTileX + 2];   // density of s^n on tile + ring
  __shared__ real rb[kTileY + 2][kTileX + 2];   // rhob' on tile + ring
  __shared__ real sbx[kTileY + 4][kTileX + 4];  // Sb' on tile + two-node ring
  __shared__ real sby[kTileY + 4][kTileX + 4];
  // mu'_i(x + e_i) at the tile's nodes, staged for FP32 (in FP64 the 37 KB would
  // exceed the static shared-memory limit next to the rest; FP64 reads directly).
  constexpr bool kStageMu = sizeof(real) == 4;
  __shared__ real mus[kStageMu ? 9 : 1][kTileY][kTileX];
  __shared__ real red[kAdjThreads / 32][3];
  const int tx = threadIdx.x & (kTileX - 1), ty = threadIdx.x / kTileX;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  const int plane = nx * ny;
  // Every coordinate below lies in [-2, n + 33); one conditional wrap suffices
  // unless the lattice is smaller than a tile plus its two-node ring.
  const bool small = nx < kTileX + 4 || ny < kTileY + 4;
  auto wr = [&](int v, int n) { return small ? wrap(v, n) : wrap1(v, n); };
  const int gx = x0 + tx;
  const int xc = wr(gx, nx);
  const int xm = xc == 0 ? nx - 1 : xc - 1, xp = xc == nx - 1 ? 0 : xc + 1;
  // The cotangent reads go first, as asynchronous copies into shared memory, so
  // that they travel while the state is pulled: mu'_i at x + e_i for the thread's
  // nodes (wrapped coordinates also past a ragged edge: in bounds, unused), and Sb'
  // on the tile with its two-node ring.
#pragma unroll
  for (int k = 0; k < (kStageMu ? kTileRows : 0); ++k) {
    const int ly = ty + k * kRowStride;
    const int yc = wr(y0 + ly, ny);
    const int ym = yc == 0 ? ny - 1 : yc - 1, yp = yc == ny - 1 ? 0 : yc + 1;
    const int oc = yc * nx, om = ym * nx, op = yp * nx;
    cp_async_elem(&mus[0][ly][tx], mu_in + (oc + xc));
    cp_async_elem(&mus[1][ly][tx], mu_in + (plane + oc + xp));
    cp_async_elem(&mus[2][ly][tx], mu_in + (2 * plane + op + xc));
    cp_async_elem(&mus[3][ly][tx], mu_in + (3 * plane + oc + xm));
    cp_async_elem(&mus[4][ly][tx], mu_in + (4 * plane + om + xc));
    cp_async_elem(&mus[5][ly][tx], mu_in + (5 * plane + op + xp));
    cp_async_elem(&mus[6][ly][tx], mu_in + (6 * plane + op + xm));
    cp_async_elem(&mus[7][ly][tx], mu_in + (7 * plane + om + xm));
    cp_async_elem(&mus[8][ly][tx], mu_in + (8 * plane + om + xp));
  }
  for (int t = threadIdx.x; t < (kTileY + 4) * (kTileX + 4); t += kAdjThreads) {
    const int wy = t / (kTileX + 4), wx = t - wy * (kTileX + 4);
    const int o = wr(y0 - 2 + wy, ny) * nx + wr(x0 - 2 + wx, nx);
    cp_async_elem(&sbx[wy][wx], sb_in + o);
    cp_async_elem(&sby[wy][wx], sb_in + (plane + o));
  }
  cp_async_commit();
  real f[kTileRows][9];
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int gy = y0 + ty + k * kRowStride;
    pull_row(s, plane, nx, ny, wr(gy, ny), xm, xc, xp, f[k]);
  }
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) rs[ty + k * kRowStride + 1][tx + 1] = sum9(f[k]);
  for (int t = threadIdx.x; t < 2 * (kTileX + 2) + 2 * kTileY; t += kAdjThreads) {
    int wx, wy;
    if (t < kTileX + 2) {
      wx = t, wy = 0;
    } else if (t < 2 * (kTileX + 2)) {
      wx = t - (kTileX + 2), wy = kTileY + 1;
    } else if (t < 2 * (kTileX + 2) + kTileY) {
      wx = 0, wy = t - 2 * (kTileX + 2) + 1;
    } else {
      wx = kTileX + 1, wy = t - 2 * (kTileX + 2) - kTileY + 1;
    }
    const int hx = wr(x0 - 1 + wx, nx), hy = wr(y0 - 1 + wy, ny);
    real g[9];
    pull_row(s, plane, nx, ny, hy, hx == 0 ? nx - 1 : hx - 1, hx, hx == nx - 1 ? 0 : hx + 1, g);
    rs[wy][wx] = sum9(g);
  }
  cp_async_wait_all();
  __syncthreads();
  // rhob'(y) = sum_j omega_j e_j . Sb'(y - e_j) on tile + ring (smem index of y is (wy + 1, wx + 1)).
  const real third = real(1.0 / 3.0), twelfth = real(1.0 / 12.0);
  for (int t = threadIdx.x; t < (kTileY + 2) * (kTileX + 2); t += kAdjThreads) {
    const int wy = t / (kTileX + 2), wx = t - wy * (kTileX + 2);
    const int cy = wy + 1, cx = wx + 1;
    const real ax = sbx[cy][cx - 1] - sbx[cy][cx + 1];
    const real ay = sby[cy - 1][cx] - sby[cy + 1][cx];
    const real d5 = sbx[cy - 1][cx - 1] + sby[cy - 1][cx - 1];
    const real d6 = sby[cy - 1][cx + 1] - sbx[cy - 1][cx + 1];
    const real d7 = -sbx[cy + 1][cx + 1] - sby[cy + 1][cx + 1];
    const real d8 = sbx[cy + 1][cx - 1] - sby[cy + 1][cx - 1];
    rb[wy][wx] = third * (ax + ay) + twelfth * ((d5 + d6) + (d7 + d8));
  }
  __syncthreads();
  // Parameter cotangents summed in the compute type within a warp (FP64 arithmetic
  // is slow on this GPU); warp partials are folded in FP64.
  real acc[3] = {real(0), real(0), real(0)};
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int ly = ty + k * kRowStride + 1, lx = tx + 1;
    const int gy = y0 + ly - 1;
    if (gx >= nx || gy >= ny) continue;
    real Sx, Sy;
    stencil(rs[ly - 1][lx - 1], rs[ly - 1][lx], rs[ly - 1][lx + 1], rs[ly][lx - 1], rs[ly][lx + 1],
            rs[ly + 1][lx - 1], rs[ly + 1][lx], rs[ly + 1][lx + 1], Sx, Sy);
    const int off = gy * nx + gx;
    // lam_i(x) = mu'_i(x + e_i) + rhob'(x + e_i).
    real mu9[9];
    if constexpr (kStageMu) {
#pragma unroll
      for (int i = 0; i < 9; ++i) mu9[i] = mus[i][ly - 1][tx];
    } else {
      const int ym = gy == 0 ? ny - 1 : gy - 1, yp = gy == ny - 1 ? 0 : gy + 1;
      const int oc = gy * nx, om = ym * nx, op = yp * nx;
      mu9[0] = mu_in[off];
      mu9[1] = mu_in[plane + oc + xp];
      mu9[2] = mu_in[2 * plane + op + gx];
      mu9[3] = mu_in[3 * plane + oc + xm];
      mu9[4] = mu_in[4 * plane + om + gx];
      mu9[5] = mu_in[5 * plane + op + xp];
      mu9[6] = mu_in[6 * plane + op + xm];
      mu9[7] = mu_in[7 * plane + om + xm];
      mu9[8] = mu_in[8 * plane + om + xp];
    }
    real ob[9];
    ob[0] = mu9[0] + rb[ly][lx];
    ob[1] = mu9[1] + rb[ly][lx + 1];
    ob[2] = mu9[2] + rb[ly + 1][lx];
    ob[3] = mu9[3] + rb[ly][lx - 1];
    ob[4] = mu9[4] + rb[ly - 1][lx];
    ob[5] = mu9[5] + rb[ly + 1][lx + 1];
    ob[6] = mu9[6] + rb[ly + 1][lx - 1];
    ob[7] = mu9[7] + rb[ly - 1][lx - 1];
    ob[8] = mu9[8] + rb[ly - 1][lx + 1];
    AdjOut<real> r;
    collide_vjp(c, f[k], Sx, Sy, ob, r);
#pragma unroll
    for (int i = 0; i < 9; ++i) mu[i * plane + off] = r.d[i];
    sbar[off] = r.Sx;
    sbar[plane + off] = r.Sy;
    acc[0] += r.RT;
    acc[1] += r.G2;
    acc[2] += r.lam;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    real v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    // The block's partial in the compute type, widened once: one FP64 add per
    // block and parameter per step.
    real v = real(0);
    for (int j = 0; j < kAdjThreads / 32; ++j) v += red[j][threadIdx.x];
    // Each block owns its slot; successive steps on one stream accumulate in order.
    double* slot = partial + (size_t(blockIdx.y) * gridDim.x + blockIdx.x) * 3 + threadIdx.x;
    *slot = accumulate ? *slot + double(v) : double(v);
  }
}

// Staging of one FP32 adjoint tile in dynamic shared memory, for lattices with
// several waves of tiles: the state's pull window (the forward step's nine
// 40 x 18 windows), mu'_i at the tile's nodes shifted by e_i (nine 40 x 16 windows,
// plane i's from (x0 - 4, y0 + e_iy): node (tx, ly) reads column tx + 4 + e_ix of
// row ly) and Sb' on the tile with its two-node ring (two 40 x 20 windows from
// (x0 - 4, y0 - 2)).  An interior tile gets all twenty windows by tensor copies
// issued by one thread on one mbarrier; a tile whose windows wrap gets the same
// layout by per-thread asynchronous copies with periodic coordinates.
constexpr int kMuCols = kTileX + 8, kMuRows = kTileY;
constexpr int kMuPlane = kMuCols * kMuRows;  // 640 floats
constexpr int kSbCols = kTileX + 8, kSbRows = kTileY + 4;
constexpr int kSbPlane = kSbCols * kSbRows;  // 800 floats
constexpr int kAdjMuOff = 9 * kTmaPlane;     // after the state window
constexpr int kAdjSbOff = kAdjMuOff + 9 * kMuPlane;
constexpr int kAdjStageFloats = kAdjSbOff + 2 * kSbPlane;
constexpr unsigned kAdjStageSmem = unsigned(kAdjStageFloats) * 4 + 128;
constexpr unsigned kAdjCotBytes = unsigned(9 * kMuPlane + 2 * kSbPlane) * 4;  // mu' and Sb' windows
static_assert((kAdjMuOff * 4) % 128 == 0 && (kMuPlane * 4) % 128 == 0 && (kAdjSbOff * 4) % 128 == 0 &&
                  (kSbPlane * 4) % 128 == 0,
              "tensor-copy destinations start on 128-byte boundaries");

// All threads: the staging of a wrapping tile (lattice of at least 40 x 18) by
// per-thread asynchronous copies; commits one group.
__device__ __forceinline__ void stage_adj_async(float* base, const float* __restrict__ s,
                                                const float* __restrict__ mu_in, const float* __restrict__ sb_in,
                                                int nx, int ny, int x0, int y0) {
  const int plane = nx * ny;
  for (int e = threadIdx.x; e < 9 * kMuPlane; e += kAdjThreads) {
    const int i = e / kMuPlane, rc = e - i * kMuPlane, r = rc / kMuCols, cc = rc - r * kMuCols;
    const int y = wrap1(y0 + ey_of(i) + r, ny), x = wrap1(x0 - 4 + cc, nx);
    cp_async4(base + kAdjMuOff + e, mu_in + (i * plane + y * nx + x));
  }
  for (int e = threadIdx.x; e < 2 * kSbPlane; e += kAdjThreads) {
    const int p = e / kSbPlane, rc = e - p * kSbPlane, r = rc / kSbCols, cc = rc - r * kSbCols;
    const int y = wrap1(y0 - 2 + r, ny), x = wrap1(x0 - 4 + cc, nx);
    cp_async4(base + kAdjSbOff + e, sb_in + (p * plane + y * nx + x));
  }
  issue_window_async(base, s, nx, ny, planes_strides(nx, ny), x0, y0);  // commits the group
}

// One adjoint step of an FP32 tile from the staged windows above (the staged
// counterpart of k_adj_fused: same VJP, same sums, same outputs).  A wait for the
// tensor copies that gives up sets *err (reported by lb_status) and ends the block.
__global__ void __launch_bounds__(kAdjThreads, 3)
    k_adj_tma(const __grid_constant__ CUtensorMap tstate, const __grid_constant__ CUtensorMap tmu,
              const __grid_constant__ CUtensorMap tsb, const float* __restrict__ s, const float* __restrict__ mu_in,
              const float* __restrict__ sb_in, float* __restrict__ mu, float* __restrict__ sbar,
              double* __restrict__ partial, int accumulate, int nx, int ny, VCoef<float> c, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char dyn[];
  float* const base = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(dyn) + 127) & ~uintptr_t(127));
  const float* const muw = base + kAdjMuOff;
  const float* const sbx = base + kAdjSbOff;
  const float* const sby = sbx + kSbPlane;
  __shared__ float rs[kTileY + 2][kTileX + 2];  // density of s^n on tile + ring
  __shared__ float rb[kTileY + 2][kTileX + 2];  // rhob' on tile + ring
  __shared__ float red[kAdjThreads / 32][3];
  __shared__ __align__(8) unsigned long long bar;
  const int tx = threadIdx.x & (kTileX - 1), ty = threadIdx.x / kTileX;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  const int plane = nx * ny;
  const bool interior = tma_interior<float>(x0, y0, nx, ny);
  if (interior) {
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_proxy_async();
      issue_windows(base, &tstate, x0, y0, &bar, kAdjCotBytes);
#pragma unroll
      for (int i = 0; i < 9; ++i) tma_load_3d(base + kAdjMuOff + i * kMuPlane, &tmu, x0 - 4, y0 + ey_of(i), i, &bar);
      tma_load_3d(base + kAdjSbOff, &tsb, x0 - 4, y0 - 2, 0, &bar);
      tma_load_3d(base + kAdjSbOff + kSbPlane, &tsb, x0 - 4, y0 - 2, 1, &bar);
    }
    const bool late = !mbar_wait(&bar, 0);
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        mbar_wait(&bar, 0);
      }
      return;
    }
  } else {
    stage_adj_async(base, s, mu_in, sb_in, nx, ny, x0, y0);
    cp_async_wait_all();
    __syncthreads();
  }
  float f[kTileRows][9];
  window_tile(base, f, rs);
  // rhob'(y) = sum_j omega_j e_j . Sb'(y - e_j) on tile + ring; Sb' window column of
  // lattice column x0 - 2 + cx is cx + 2.
  const float third = float(1.0 / 3.0), twelfth = float(1.0 / 12.0);
  for (int t = threadIdx.x; t < (kTileY + 2) * (kTileX + 2); t += kAdjThreads) {
    const int wy = t / (kTileX + 2), wx = t - wy * (kTileX + 2);
    const int cy = wy + 1, cx = wx + 3;
    auto X = [&](int yy, int xx) { return sbx[yy * kSbCols + xx]; };
    auto Y = [&](int yy, int xx) { return sby[yy * kSbCols + xx]; };
    const float ax = X(cy, cx - 1) - X(cy, cx + 1);
    const float ay = Y(cy - 1, cx) - Y(cy + 1, cx);
    const float d5 = X(cy - 1, cx - 1) + Y(cy - 1, cx - 1);
    const float d6 = Y(cy - 1, cx + 1) - X(cy - 1, cx + 1);
    const float d7 = -X(cy + 1, cx + 1) - Y(cy + 1, cx + 1);
    const float d8 = X(cy + 1, cx - 1) - Y(cy + 1, cx - 1);
    rb[wy][wx] = third * (ax + ay) + twelfth * ((d5 + d6) + (d7 + d8));
  }
  __syncthreads();
  const int gx = x0 + tx;
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int ly = ty + k * kRowStride + 1, lx = tx + 1;
    const int gy = y0 + ly - 1;
    if (gx >= nx || gy >= ny) continue;
    float Sx, Sy;
    stencil(rs[ly - 1][lx - 1], rs[ly - 1][lx], rs[ly - 1][lx + 1], rs[ly][lx - 1], rs[ly][lx + 1],
            rs[ly + 1][lx - 1], rs[ly + 1][lx], rs[ly + 1][lx + 1], Sx, Sy);
    const int off = gy * nx + gx;
    // lam_i(x) = mu'_i(x + e_i) + rhob'(x + e_i).
    float ob[9];
#pragma unroll
    for (int i = 0; i < 9; ++i)
      ob[i] = muw[i * kMuPlane + (ly - 1) * kMuCols + tx + 4 + ex_of(i)] + rb[ly + ey_of(i)][lx + ex_of(i)];
    AdjOut<float> r;
    collide_vjp(c, f[k], Sx, Sy, ob, r);
#pragma unroll
    for (int i = 0; i < 9; ++i) mu[i * plane + off] = r.d[i];
    sbar[off] = r.Sx;
    sbar[plane + off] = r.Sy;
    acc[0] += r.RT;
    acc[1] += r.G2;
    acc[2] += r.lam;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float v = 0.f;
    for (int j = 0; j < kAdjThreads / 32; ++j) v += red[j][threadIdx.x];
    double* slot = partial + (size_t(blockIdx.y) * gridDim.x + blockIdx.x) * 3 + threadIdx.x;
    *slot = accumulate ? *slot + double(v) : double(v);
  }
}

// Cotangent lam of a state -> (mu, Sb) representation: mu_i(y) = lam_i(y - e_i), Sb = 0.
template <typename real>
__global__ void k_adj_push(const real* __restrict__ lam, real* __restrict__ mu, real* __restrict__ sbar, int nx,
                           int ny) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int plane = nx * ny;
  real v[9];
  pull_row(lam, plane, nx, ny, y, x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1, v);
  const int off = y * nx + x;
#pragma unroll
  for (int i = 0; i < 9; ++i) mu[i * plane + off] = v[i];
  sbar[off] = real(0);
  sbar[plane + off] = real(0);
}

size_t adj_scratch_bytes(const lb_params* p, size_t real_bytes) {
  const size_t N = size_t(p->nx) * p->ny;
  const size_t blocks = size_t((p->nx + kTileX - 1) / kTileX) * ((p->ny + kTileY - 1) / kTileY);
  return ((11 * N * real_bytes + 255) / 256) * 256 + blocks * 3 * sizeof(double);
}

// Two (mu, Sb) sets (ping-pong) + per-block partials.
size_t adj_steps_scratch_bytes(const lb_params* p, size_t real_bytes) {
  const size_t N = size_t(p->nx) * p->ny;
  const size_t blocks = size_t((p->nx + kTileX - 1) / kTileX) * ((p->ny + kTileY - 1) / kTileY);
  return 2 * ((11 * N * real_bytes + 255) / 256) * 256 + blocks * 3 * sizeof(double);
}

template <typename real, typename store_t>
int adjoint_steps(lb_handle* h, const void* const* states, int k, void* lam, double* dtheta, void* scratch) {
  const int nx = h->p.nx, ny = h->p.ny;
  const size_t N = size_t(nx) * ny;
  const size_t set = ((11 * N * sizeof(real) + 255) / 256) * 256;
  real* mu[2] = {static_cast<real*>(scratch), reinterpret_cast<real*>(static_cast<char*>(scratch) + set)};
  real* sb[2] = {mu[0] + 9 * N, mu[1] + 9 * N};
  double* partial = reinterpret_cast<double*>(static_cast<char*>(scratch) + 2 * set);
  const dim3 grd((nx + kTileX - 1) / kTileX, (ny + kTileY - 1) / kTileY);
  const VCoef<real>* c;
  if constexpr (sizeof(real) == 8)
    c = &h->cd;
  else
    c = &h->cf;
  const dim3 blk(32, 8), pgrd((nx + 31) / 32, (ny + 7) / 8);
  // FP32 on lattices with several waves of tiles: every input of a tile staged in
  // shared memory (k_adj_tma; tensor copies on interior tiles), so that all of a
  // block's reads are in flight before the first is used.  On small lattices (one
  // wave) waiting for the whole staging before any work measured slower (256^2:
  // 8.7 against 7.2 us per step), and k_adj_fused pulls the state directly.
  bool staged = false;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 0;
  if constexpr (sizeof(real) == 4 && sizeof(store_t) == 4) {
    if (h->use_tma && h->wait_error && async_window_ok(nx, ny) && nx % 4 == 0 && sms > 0 &&
        size_t(grd.x) * grd.y >= size_t(4) * 3 * sms) {
      const cudaError_t a =
          cudaFuncSetAttribute(k_adj_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kAdjStageSmem));
      if (a != cudaSuccess) {
        std::snprintf(h->err, sizeof(h->err), "adjoint kernels: %s", cudaGetErrorString(a));
        return LB_ECUDA;
      }
      staged = true;
    }
  }
  k_adj_push<real><<<pgrd, blk, 0, h->stream>>>(static_cast<const real*>(lam), mu[0], sb[0], nx, ny);
  int cur = 0;
  for (int j = k - 1; j >= 0; --j) {
    bool done = false;
    if constexpr (sizeof(real) == 4 && sizeof(store_t) == 4) {
      CUtensorMap ts, tm, tb;
      if (staged && encode_population_map(&ts, const_cast<void*>(states[j]), nx, ny, nx, 4) &&
          encode_plane_map(&tm, mu[cur], nx, ny, 9, kMuCols, kMuRows) &&
          encode_plane_map(&tb, sb[cur], nx, ny, 2, kSbCols, kSbRows)) {
        k_adj_tma<<<grd, kAdjThreads, kAdjStageSmem, h->stream>>>(
            ts, tm, tb, static_cast<const float*>(states[j]), mu[cur], sb[cur], mu[1 - cur], sb[1 - cur], partial,
            j < k - 1, nx, ny, *c, h->wait_error);
        done = true;
      }
    }
    if (!done)
      k_adj_fused<real, store_t><<<grd, kAdjThreads, 0, h->stream>>>(
          static_cast<const store_t*>(states[j]), mu[cur], sb[cur], mu[1 - cur], sb[1 - cur], partial, j < k - 1, nx,
          ny, *c);
    cur = 1 - cur;
  }
  if (dtheta) k_adj_theta<<<1, 256, 0, h->stream>>>(partial, int(grd.x * grd.y), h->p.R_gas, dtheta);
  k_adj_transpose<real><<<grd, kAdjThreads, 0, h->stream>>>(mu[cur], sb[cur], static_cast<real*>(lam), nx, ny);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::snprintf(h->err, sizeof(h->err), "adjoint kernels: %s", cudaGetErrorString(e));
    return LB_ECUDA;
  }
  return LB_OK;
}

template <typename real, typename store_t>
int adjoint(lb_handle* h, const void* f_state, const void* lam_in, void* lam_out, double* dtheta, void* scratch) {
  const int nx = h->p.nx, ny = h->p.ny;
  const size_t N = size_t(nx) * ny;
  real* mu = static_cast<real*>(scratch);
  real* sbar = mu + 9 * N;
  double* partial = reinterpret_cast<double*>(static_cast<char*>(scratch) + ((11 * N * sizeof(real) + 255) / 256) * 256);
  const dim3 grd((nx + kTileX - 1) / kTileX, (ny + kTileY - 1) / kTileY);
  const VCoef<real>* c;
  if constexpr (sizeof(real) == 8)
    c = &h->cd;
  else
    c = &h->cf;
  k_adj_local<real, store_t><<<grd, kAdjThreads, 0, h->stream>>>(
      static_cast<const store_t*>(f_state), static_cast<const real*>(lam_in), mu, sbar, partial, nx, ny, *c);
  k_adj_transpose<real><<<grd, kAdjThreads, 0, h->stream>>>(mu, sbar, static_cast<real*>(lam_out), nx, ny);
  if (dtheta) k_adj_theta<<<1, 256, 0, h->stream>>>(partial, int(grd.x * grd.y), h->p.R_gas, dtheta);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::snprintf(h->err, sizeof(h->err), "adjoint kernels: %s", cudaGetErrorString(e));
    return LB_ECUDA;
  }
  return LB_OK;
}

}  // namespace

extern "C" {

size_t lb_adjoint_scratch_bytes(const lb_params* p) {
  if (!p || p->nx < 1 || p->ny < 1) return 0;
  return adj_scratch_bytes(p, p->precision == LB_FP64 ? 8 : 4);
}

int lb_adjoint_step(lb_handle* h, const void* f_state, const void* lam_in, void* lam_out, double* dtheta,
                    void* scratch, size_t scratch_bytes) {
  if (!h) return LB_EINVAL;
  if (!f_state || !lam_in || !lam_out || lam_in == lam_out) {
    std::snprintf(h->err, sizeof(h->err), "lb_adjoint_step: null or aliased buffers");
    return LB_EINVAL;
  }
  if (h->p.layout != LB_LAYOUT_PLANES) {
    std::snprintf(h->err, sizeof(h->err), "lb_adjoint_step: the adjoint takes the planes layout");
    return LB_ENOTSUP;
  }
  const size_t need = lb_adjoint_scratch_bytes(&h->p);
  if (!scratch || scratch_bytes < need) {
    std::snprintf(h->err, sizeof(h->err), "lb_adjoint_step needs %zu bytes of scratch, got %zu", need,
                  scratch ? scratch_bytes : 0);
    return LB_ENOMEM;
  }
  switch (h->p.precision) {
    case LB_FP64: return adjoint<double, double>(h, f_state, lam_in, lam_out, dtheta, scratch);
    case LB_FP32: return adjoint<float, float>(h, f_state, lam_in, lam_out, dtheta, scratch);
    default:
      std::snprintf(h->err, sizeof(h->err), "lb_adjoint_step supports FP64 and FP32 storage");
      return LB_ENOTSUP;
  }
}

size_t lb_adjoint_steps_scratch_bytes(const lb_params* p) {
  if (!p || p->nx < 1 || p->ny < 1) return 0;
  return adj_steps_scratch_bytes(p, p->precision == LB_FP64 ? 8 : 4);
}

int lb_adjoint_steps(lb_handle* h, const void* const* states, int k, void* lam, double* dtheta, void* scratch,
                     size_t scratch_bytes) {
  if (!h) return LB_EINVAL;
  if (!states || k < 1 || !lam) {
    std::snprintf(h->err, sizeof(h->err), "lb_adjoint_steps: need k >= 1 states and a cotangent buffer");
    return LB_EINVAL;
  }
  if (h->p.layout != LB_LAYOUT_PLANES) {
    std::snprintf(h->err, sizeof(h->err), "lb_adjoint_steps: the adjoint takes the planes layout");
    return LB_ENOTSUP;
  }
  for (int j = 0; j < k; ++j)
    if (!states[j]) {
      std::snprintf(h->err, sizeof(h->err), "lb_adjoint_steps: state %d is null", j);
      return LB_EINVAL;
    }
  const size_t need = lb_adjoint_steps_scratch_bytes(&h->p);
  if (!scratch || scratch_bytes < need) {
    std::snprintf(h->err, sizeof(h->err), "lb_adjoint_steps needs %zu bytes of scratch, got %zu", need,
                  scratch ? scratch_bytes : 0);
    return LB_ENOMEM;
  }
  switch (h->p.precision) {
    case LB_FP64: return adjoint_steps<double, double>(h, states, k, lam, dtheta, scratch);
    case LB_FP32: return adjoint_steps<float, float>(h, states, k, lam, dtheta, scratch);
    default:
      std::snprintf(h->err, sizeof(h->err), "lb_adjoint_steps supports FP64 and FP32 storage");
      return LB_ENOTSUP;
  }
}

}  // extern "C"
