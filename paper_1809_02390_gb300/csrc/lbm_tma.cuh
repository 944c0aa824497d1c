// Fused FP32 step with TMA staging of the populations (sm_103a).
//
// For an interior 32 x 16 tile, one thread issues nine 3-D tensor copies
// (cp.async.bulk.tensor, one per population plane) of the 40 x 18 window that
// the pull and the density ring of the tile read, into shared memory, completing
// on one mbarrier.  The copy engine generates the memory requests, so a block's
// whole input is in flight at once without registers or address arithmetic; the
// threads then read their pulled populations and the ring densities from shared
// memory.  Plane i's window starts at (x0 - 4, y0 - 1 - e_iy): x0 - 4 keeps the
// innermost coordinate a multiple of 4 floats (16 bytes, as the tensor copy
// requires) and covers the columns x0 - 2 .. x0 + 33 that any direction reads.
// Tiles whose window would leave the lattice (the periodic wrap) take the
// plain loads of load_tile.
#pragma once

#include <cuda.h>

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int kTmaCols = kTileX + 8;                        // 40 floats
constexpr int kTmaRows = kTileY + 2;                        // 18 rows
constexpr int kTmaBox = kTmaCols * kTmaRows;                // floats copied per plane (2880 B)
constexpr int kTmaPlane = (kTmaBox * 4 + 127) / 128 * 32;   // plane stride in shared memory, floats (2944 B)
constexpr unsigned kTmaBytes = 9u * kTmaBox * 4;            // bytes a tile's nine copies deliver
constexpr unsigned kTmaSmem = 9u * kTmaPlane * 4 + 128;     // dynamic shared memory (+ alignment slack)
constexpr long long kWaitSpins = 1ll << 22;                 // bound of the mbarrier wait loop
// A tensor copy's shared-memory destination must be 128-byte aligned.
static_assert((kTmaPlane * 4) % 128 == 0, "plane windows must start on 128-byte boundaries");

__device__ __constant__ const int kEX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ const int kEY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Set when a bounded wait gave up (read and cleared by lb_status).
static __device__ int g_wait_error;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the barrier did not complete within kWaitSpins polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned phase) {
  for (long long i = 0; i < kWaitSpins; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
      "r"(smem_addr(bar))
      : "memory");
}

// Whether the TMA windows of the tile at (x0, y0) lie inside the lattice.
__device__ __forceinline__ bool tma_interior(int x0, int y0, int nx, int ny) {
  return x0 >= 4 && x0 + kTmaCols - 4 <= nx && y0 >= 2 && y0 + kTmaRows <= ny;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Resident blocks per SM the register budget must allow: 3 (80 registers).  At 4
// (64 registers) the collision spills about 150 bytes per thread and the step
// runs 30% slower on 4096^2.
#ifndef LBM_TMA_MIN_BLOCKS
#define LBM_TMA_MIN_BLOCKS 3
#endif
constexpr int kTmaMinBlocks = LBM_TMA_MIN_BLOCKS;

// Ring cell t (0 .. ring - 1) -> (wx, wy) in the (TY + 2) x (TX + 2) density tile.
__device__ __forceinline__ void ring_cell(int t, int& wx, int& wy) {
  if (t < kTileX + 2) {
    wx = t, wy = 0;
  } else if (t < 2 * (kTileX + 2)) {
    wx = t - (kTileX + 2), wy = kTileY + 1;
  } else if (t < 2 * (kTileX + 2) + kTileY) {
    wx = 0, wy = t - 2 * (kTileX + 2) + 1;
  } else {
    wx = kTileX + 1, wy = t - 2 * (kTileX + 2) - kTileY + 1;
  }
}

// Persistent form: block b takes tiles b, b + G, b + 2G, ... (G = gridDim.x, tiles
// row-major over the lattice, so the tiles in flight at one time are neighbours
// and their overlapping windows meet in L2).  One window buffer per block: once
// every thread holds its tile's populations in registers and the densities are
// in shared memory (the block barrier), the buffer is free and the nine copies
// of the block's next tile are issued into it, so that they travel while the
// block computes the force stencil and the collision of the current tile.  The
// density tile is double-buffered, which leaves one barrier per tile.  Tiles
// whose windows would wrap take the plain loads of load_tile.
template <typename V>
__global__ void __launch_bounds__(kFusedThreads, kTmaMinBlocks)
    k_step_tma(const __grid_constant__ CUtensorMap tin, const float* __restrict__ fin, float* __restrict__ fout,
               int nx, int ny, VCoef<V> c) {
  using real = float;
  extern __shared__ __align__(128) unsigned char dyn[];
  float* win = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(dyn) + 127) & ~uintptr_t(127));
  __shared__ real rs[2][kTileY + 2][kTileX + 2];
  __shared__ __align__(8) unsigned long long bar;
  const int tiles_x = (nx + kTileX - 1) / kTileX;
  const int total = tiles_x * ((ny + kTileY - 1) / kTileY);
  const int tx = threadIdx.x & (kTileX - 1), ty = threadIdx.x / kTileX;
  auto origin = [&](int t, int& x0, int& y0) {
    const int r = t / tiles_x;
    x0 = (t - r * tiles_x) * kTileX;
    y0 = r * kTileY;
  };
  // Thread 0: the nine copies of tile t's windows, if the tile is interior.
  auto issue = [&](int t) {
    int x0, y0;
    origin(t, x0, y0);
    if (t < total && tma_interior(x0, y0, nx, ny)) {
      mbar_expect_tx(&bar, kTmaBytes);
#pragma unroll
      for (int i = 0; i < 9; ++i) tma_load_3d(win + i * kTmaPlane, &tin, x0 - 4, y0 - 1 - kEY[i], i, &bar);
    }
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    issue(blockIdx.x);
  }
  __syncthreads();
  unsigned parity = 0;
  int buf = 0;
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int x0, y0;
    origin(t, x0, y0);
    real f[kTileRows][9];
    bool late = false;
    if (tma_interior(x0, y0, nx, ny)) {
      late = !mbar_wait(&bar, parity);
      parity ^= 1u;
      // Pulled population i of tile node (lx, ly): window row ly + 1, column lx + 4 - e_ix.
#pragma unroll
      for (int k = 0; k < kTileRows; ++k) {
        const int ly = ty + k * kRowStride;
#pragma unroll
        for (int i = 0; i < 9; ++i) f[k][i] = win[i * kTmaPlane + (ly + 1) * kTmaCols + tx + 4 - kEX[i]];
        rs[buf][ly + 1][tx + 1] = sum9(f[k]);
      }
      if (threadIdx.x < TileShape<kTileY>::ring) {
        int wx, wy;
        ring_cell(threadIdx.x, wx, wy);
        real g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = win[i * kTmaPlane + wy * kTmaCols + wx + 3 - kEX[i]];
        rs[buf][wy][wx] = sum9(g);
      }
    } else {
      load_tile<real, float, kTileY>(fin, nx, ny, x0, y0, f, rs[buf]);
    }
    // The window is consumed and the densities are in place.  A wait that gave up
    // (uniform decision through the barrier) ends the block: it records the
    // failure, waits once more (bounded) for the copies it issued, and returns.
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0) {
        atomicExch(&g_wait_error, 1);
        mbar_wait(&bar, parity ^ 1u);
      }
      return;
    }
    if (threadIdx.x == 0) {
      fence_proxy_async();
      issue(t + gridDim.x);
    }
    collide_tile<V, float, kTileY>(f, fout, nx, ny, c, lattice_part(c), x0, y0, rs[buf]);
    buf ^= 1;
  }
}

}  // namespace lbm
