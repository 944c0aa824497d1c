// Fused step with TMA staging of the populations (sm_103a), FP32 or FP16 storage.
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
// FP16 storage uses 48 x 18 windows from x0 - 8 (16 bytes of halves).  Tiles
// whose window would leave the lattice (the periodic wrap) take the plain loads
// of load_tile.  Rows layout (f[y][i][x]): the map's dimensions are (x, plane, y)
// and the same windows arrive in the same shared-memory arrangement.
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
constexpr long long kWaitSpins = 1ll << 22;                 // bound of the mbarrier wait loop (polls)
constexpr unsigned long long kWaitNs = 1000000000ull;      // and of its duration (1 s)
// A tensor copy's shared-memory destination must be 128-byte aligned.
static_assert((kTmaPlane * 4) % 128 == 0, "plane windows must start on 128-byte boundaries");
// FP16 storage: 48-half windows from x0 - 8 (the innermost coordinate a multiple of 8).
constexpr int kTmaColsH = kTileX + 16;
constexpr int kTmaBoxH = kTmaColsH * kTmaRows;              // halves per plane (1728 B)
constexpr int kTmaPlaneH = (kTmaBoxH * 2 + 127) / 128 * 64;  // plane stride in shared memory, halves (1792 B)
static_assert((kTmaPlaneH * 2) % 128 == 0, "plane windows must start on 128-byte boundaries");

// Window geometry per storage type: columns, column offset of x0, plane stride (elements),
// bytes a tile's nine copies deliver, dynamic shared memory of the kernel.
template <typename S>
struct Win;
template <>
struct Win<float> {
  static constexpr int cols = kTmaCols, xoff = 4, plane = kTmaPlane;
  static constexpr unsigned bytes = kTmaBytes, smem = kTmaSmem;
  __device__ static float get(float v) { return v; }
};
template <>
struct Win<__half> {
  static constexpr int cols = kTmaColsH, xoff = 8, plane = kTmaPlaneH;
  static constexpr unsigned bytes = 9u * kTmaBoxH * 2, smem = 9u * kTmaPlaneH * 2 + 128;
  __device__ static float get(__half v) { return __half2float(v); }
};

// D2Q9 velocity components e_ix, e_iy (folded to constants in unrolled loops).
__host__ __device__ constexpr int ex_of(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey_of(int i) {
  return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}

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

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: false if the barrier did not complete within `polls` polls or
// kWaitNs nanoseconds, whichever comes first (a poll may suspend the thread for a
// while, so the time bound is the one that holds in every case).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned phase, long long polls = kWaitSpins) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  for (long long i = 1; i < polls; ++i) {
    if (mbar_try_wait(bar, phase)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
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

// Plain bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory, completing on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Whether the TMA windows of the tile at (x0, y0) lie inside the lattice.
template <typename S = float>
__host__ __device__ __forceinline__ bool tma_interior(int x0, int y0, int nx, int ny) {
  return x0 >= Win<S>::xoff && x0 + Win<S>::cols - Win<S>::xoff <= nx && y0 >= 2 && y0 + kTmaRows <= ny;
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

// Windows of tiles that wrap, by per-thread asynchronous copies (cp.async): the
// window of such a tile gets the cells a tensor copy would deliver, with periodic
// source coordinates, so that every tile of a lattice of at least kTmaCols x
// kTmaRows nodes is staged ahead (every coordinate then lies in [-4, 2n) and one
// conditional wrap suffices).  180 threads, one per window row (18) and run of four
// columns (10); each copies its run in all nine planes.  A run is one 16-byte copy
// when its four source cells are contiguous and 16-byte aligned, i.e. when it does
// not cross the lattice's right edge and its start is a multiple of 4 after the
// wrap: always when nx is a multiple of 4, else for runs inside [0, nx); otherwise
// four 4-byte copies.  Row strides and plane strides are multiples of 4 floats in
// every layout that reaches here (the tensor-copy path needs them).
__host__ __device__ __forceinline__ bool async_window_ok(int nx, int ny) {
  return nx >= kTmaCols && ny >= kTmaRows;
}

constexpr int kAsyncRuns = kTmaCols / 4;                 // 10 runs of four columns per window row
constexpr int kAsyncThreads = kTmaRows * kAsyncRuns;     // 180
static_assert(kTmaCols % 4 == 0 && kAsyncThreads <= kFusedThreads, "window rows split in runs of four columns");

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
// 16 bytes (both addresses 16-byte aligned), bypassing L1.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
// One element (4 or 8 bytes, naturally aligned) by cp.async.
__device__ __forceinline__ void cp_async_elem(float* dst, const float* src) { cp_async4(dst, src); }
__device__ __forceinline__ void cp_async_elem(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// All but the newest committed group of this thread have completed.
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// All threads: the window of the (wrapping) tile at (x0, y0) of a lattice with
// populations at fin (16-byte aligned; layout st) into win.  Plane i's window row r
// holds lattice row y0 - 1 - e_iy + r, window column c lattice column x0 - 4 + c.
__device__ __forceinline__ void issue_window_async(float* win, const float* __restrict__ fin, int nx, int ny,
                                                   Strides st, int x0, int y0) {
  const int j = threadIdx.x;
  if (j < kAsyncThreads) {
    const int r = j / kAsyncRuns, c4 = 4 * (j - r * kAsyncRuns);
    const int col = x0 - 4 + c4;  // lattice column of the run's first cell, in [-4, 2 nx)
    const bool whole = (nx & 3) == 0 || (col >= 0 && col + 3 < nx);
    int row[3];  // [e_iy + 1]: element offset of lattice row y0 - 1 - e_iy + r
#pragma unroll
    for (int e = 0; e < 3; ++e) row[e] = wrap1(y0 - e + r, ny) * st.rs;
    float* dst = win + r * kTmaCols + c4;
    if (whole) {
      const int gx = wrap1(col, nx);
#pragma unroll
      for (int i = 0; i < 9; ++i) cp_async16(dst + i * kTmaPlane, fin + (i * st.ps + row[ey_of(i) + 1] + gx));
    } else {
      int gx[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) gx[q] = wrap1(col + q, nx);
#pragma unroll
      for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) cp_async4(dst + i * kTmaPlane + q, fin + (i * st.ps + row[ey_of(i) + 1] + gx[q]));
    }
  }
  cp_async_commit();
}

// Phase 1 of an interior tile from its staged windows: the populations of the
// thread's two nodes (window row ly + 1, column lx + xoff - e_ix for plane i) into
// f, the densities of tile + ring into rs.  XP: column pairs (NodeMap); with FP16
// storage a population's two cells are read as 4-byte half pairs (one for e_ix =
// 0, the two that hold it otherwise: window columns are even at the pairs).
template <typename S, bool XP = false>
__device__ __forceinline__ void window_tile(const S* __restrict__ win, float (&f)[kTileRows][9],
                                            float (*rs)[kTileX + 2]) {
  using W = Win<S>;
  using M = NodeMap<kTileY, XP>;
  if constexpr (XP && sizeof(S) == 2) {
    static_assert(W::plane % 2 == 0 && W::cols % 2 == 0 && W::xoff % 2 == 0, "half pairs start at even columns");
    const __half2* w2 = reinterpret_cast<const __half2*>(win);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int e = ex_of(i);
      const int h = (i * W::plane + (M::ly(0) + 1) * W::cols + M::lx(0) + W::xoff) / 2;  // cells lx, lx + 1 at e = 0
      if (e == 0) {
        const __half2 v = w2[h];
        f[0][i] = __low2float(v);
        f[1][i] = __high2float(v);
      } else {
        const __half2 u = w2[h - (e > 0 ? 1 : 0)], v = w2[h + (e > 0 ? 0 : 1)];
        f[0][i] = __high2float(u);
        f[1][i] = __low2float(v);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < kTileRows; ++k)
#pragma unroll
      for (int i = 0; i < 9; ++i)
        f[k][i] = W::get(win[i * W::plane + (M::ly(k) + 1) * W::cols + M::lx(k) + W::xoff - ex_of(i)]);
  }
  // Both densities as one packed sum (lane k = node k; the same additions in the
  // same order as the scalar sum).
  f2 d[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) d[i].v = make_float2(f[0][i], f[1][i]);
  const f2 rho = sum9(d);
  rs[M::ly(0) + 1][M::lx(0) + 1] = rho.v.x;
  rs[M::ly(1) + 1][M::lx(1) + 1] = rho.v.y;
  if (threadIdx.x < TileShape<kTileY>::ring) {
    int wx, wy;
    ring_cell(threadIdx.x, wx, wy);
    float g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = W::get(win[i * W::plane + wy * W::cols + wx + W::xoff - 1 - ex_of(i)]);
    rs[wy][wx] = sum9(g);
  }
}

// The nine copies of the interior tile at (x0, y0) into win, completing on bar
// (one thread).  rows: the map's dimensions are (x, plane, y) instead of (x, y, plane).
template <typename S>
__device__ __forceinline__ void issue_windows(S* win, const CUtensorMap* map, int x0, int y0,
                                              unsigned long long* bar, unsigned extra_bytes = 0, bool rows = false) {
  using W = Win<S>;
  mbar_expect_tx(bar, W::bytes + extra_bytes);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int wy = y0 - 1 - ey_of(i);
    tma_load_3d(win + i * W::plane, map, x0 - W::xoff, rows ? i : wy, rows ? wy : i, bar);
  }
}

// How a tile's window is staged: by tensor copies (interior), by per-thread
// asynchronous copies (wrapping tile of a lattice of at least 40 x 18), or not at
// all (plain loads in phase 1).
enum TileKind { kTensorCopy = 0, kAsyncCopy = 1, kPlainLoad = 2 };

template <bool ASYNC_EDGES = true, typename S = float>
__host__ __device__ __forceinline__ int tile_kind(int x0, int y0, int nx, int ny) {
  return tma_interior<S>(x0, y0, nx, ny) ? kTensorCopy
                                         : (ASYNC_EDGES && async_window_ok(nx, ny) ? kAsyncCopy : kPlainLoad);
}

// Persistent form: block b takes tiles b, b + G, b + 2G, ... (G = gridDim.x, tiles
// row-major over the lattice, so the tiles in flight at one time are neighbours
// and their overlapping windows meet in L2).  One window buffer per block: once
// every thread holds its tile's populations in registers and the densities are
// in shared memory (the block barrier), the buffer is free and the block's next
// tile is staged into it (tensor copies issued by thread 0 on the mbarrier, or
// the per-thread copies of a wrapping tile), so that it travels while the block
// computes the force stencil and the collision of the current tile.  The density
// tile is double-buffered, which leaves one barrier per tile (two for a wrapping
// tile: every thread's copies must have landed).  A wait that gives up sets *err.
// ASYNC_EDGES = false leaves wrapping tiles to plain loads: the per-thread copies
// cost registers (spills rise from 52 to 140 bytes per thread), which a lattice
// with few wrapping tiles does not win back (and they exist for FP32 only).
// S: storage type (float, or __half with the stores rounded as rnd says).
template <typename V, typename S, bool ASYNC_EDGES>
__global__ void __launch_bounds__(kFusedThreads, kTmaMinBlocks)
    k_step_tma(const __grid_constant__ CUtensorMap tin, const S* __restrict__ fin, S* __restrict__ fout, int nx,
               int ny, Strides st, VCoef<V> c, int* __restrict__ err, Rounding rnd) {
  static_assert(!ASYNC_EDGES || sizeof(S) == 4, "asynchronous edge windows exist for FP32 storage only");
  rnd = resolve(rnd);
  using real = float;
  extern __shared__ __align__(128) unsigned char dyn[];
  S* win = reinterpret_cast<S*>((reinterpret_cast<uintptr_t>(dyn) + 127) & ~uintptr_t(127));
  constexpr bool XP = xpairs<S>();
  __shared__ __align__(16) real rs[2][kTileY + 2][kTileX + 2];
  __shared__ __align__(8) unsigned long long bar;
  const int tiles_x = (nx + kTileX - 1) / kTileX;
  const int total = tiles_x * ((ny + kTileY - 1) / kTileY);
  const bool rows = st.ps == nx;  // rows layout (the planes one has ps = nx ny, ny >= 50 here)
  // Tile t sits at column t mod tiles_x, row t / tiles_x; the walk t -> t + G
  // advances the origin by a fixed step (two divisions per block, none per tile).
  const int step_r = gridDim.x / tiles_x, step_c = gridDim.x - step_r * tiles_x;
  auto advance = [&](int& c0, int& r0) {
    c0 += step_c;
    r0 += step_r;
    if (c0 >= tiles_x) {
      c0 -= tiles_x;
      ++r0;
    }
  };
  // All threads: stage the tile at tile column c0, row r0 (thread 0 the tensor
  // copies, everyone the per-thread ones).
  auto issue = [&](int c0, int r0) {
    const int x0 = c0 * kTileX, y0 = r0 * kTileY;
    const int kind = tile_kind<ASYNC_EDGES, S>(x0, y0, nx, ny);
    if (kind == kTensorCopy && threadIdx.x == 0) {
      fence_proxy_async();
      issue_windows(win, &tin, x0, y0, &bar, 0, rows);
    } else if (kind == kAsyncCopy) {
      if constexpr (ASYNC_EDGES) issue_window_async(win, fin, nx, ny, st, x0, y0);
    }
  };
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  int tr = blockIdx.x / tiles_x, tc = blockIdx.x - tr * tiles_x;  // current tile
  if (blockIdx.x < total) issue(tc, tr);
  unsigned parity = 0;
  int buf = 0;
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int x0 = tc * kTileX, y0 = tr * kTileY;
    const int kind = tile_kind<ASYNC_EDGES, S>(x0, y0, nx, ny);
    real f[kTileRows][9];
    bool late = false;
    if (kind == kTensorCopy) {
      late = !mbar_wait(&bar, parity);
      parity ^= 1u;
    } else if (kind == kAsyncCopy) {
      cp_async_wait_all();
      __syncthreads();
    }
    if (kind == kPlainLoad)
      load_tile<real, S, kTileY, XP>(fin, nx, ny, st, x0, y0, f, rs[buf]);
    else  // read even after a failed wait (in bounds; the block then returns)
      window_tile<S, XP>(win, f, rs[buf]);
    // The window is consumed and the densities are in place.  A wait that gave up
    // (uniform decision through the barrier) ends the block: it records the
    // failure, waits once more (bounded) for the copies it issued, and returns.
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        mbar_wait(&bar, parity ^ 1u);
      }
      return;
    }
    advance(tc, tr);
    if (t + gridDim.x < total) issue(tc, tr);
    collide_tile<V, S, kTileY, XP>(f, fout, nx, ny, st, c, lattice_part(c), x0, y0, rs[buf], rnd);
    buf ^= 1;
  }
}

// Dynamic form: block b starts with tiles b and b + G (G = gridDim.x); from then on
// the blocks take tiles 2G, 2G + 1, ... from a ticket counter (one atomic add per
// tile by the issuer thread, drawn two tiles ahead, off the critical path), so that the
// tiles in flight at any time are the next ones in row-major order across the
// whole grid, and each block keeps two tiles' windows in flight (two window
// buffers, two mbarriers): while tile k is collided, tiles k + 1 and k + 2 are
// being copied.  With the static
// walk above the tiles in flight drift apart as blocks run at different speeds;
// copies of the same tiles measured 7.0 TB/s with one block per tile or dynamic
// dispatch at 8 blocks per SM, against 5.9 - 6.2 TB/s for static walks.
// queue[0] is the ticket counter, queue[1] counts finished blocks; the last block
// to finish resets both to zero for the next launch (also after a wait that gave
// up).  Results do not depend on which block steps which tile.
// The thread that draws tickets and issues the copies of the dynamic forms: lane 0
// of the last warp, which has no density-ring work (threads 0 - 99 sum the ring),
// so that the bookkeeping does not lengthen the slowest warp before each barrier
// (1% on 4096^2 against thread 0).
constexpr int kIssuer = kFusedThreads - 32;

template <typename S>
struct Win2 {
  static constexpr unsigned buffer = 9u * Win<S>::plane * sizeof(S);  // one window buffer (128-byte multiple)
  static constexpr unsigned smem = 2 * buffer + 128;
};

template <typename V, typename S>
__global__ void __launch_bounds__(kFusedThreads, kTmaMinBlocks)
    k_step_tma_dyn(const __grid_constant__ CUtensorMap tin, const S* __restrict__ fin, S* __restrict__ fout, int nx,
                   int ny, Strides st, VCoef<V> c, int* __restrict__ err, Rounding rnd, unsigned* __restrict__ queue) {
  using real = float;
  rnd = resolve(rnd);
  static_assert(Win2<S>::buffer % 128 == 0, "window buffers start on 128-byte boundaries");
  extern __shared__ __align__(128) unsigned char dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dyn) + 127) & ~uintptr_t(127));
  constexpr bool XP = xpairs<S>();
  __shared__ __align__(16) real rs[2][kTileY + 2][kTileX + 2];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ int tq[2];   // tile staged in each window buffer (>= total: none)
  __shared__ int2 tp[2];  // its origin (x0, y0), written by the issuer with tq
  const int tiles_x = (nx + kTileX - 1) / kTileX;
  const int total = tiles_x * ((ny + kTileY - 1) / kTileY);
  const bool rows = st.ps == nx;  // rows layout (the planes one has ps = nx ny, ny >= 50 here)
  auto win = [&](int slot) { return reinterpret_cast<S*>(base + slot * Win2<S>::buffer); };
  // Origin of tile t (row-major over the lattice): one division, by the issuer only.
  auto origin = [&](int t) {
    const int r = t / tiles_x;
    return make_int2((t - r * tiles_x) * kTileX, r * kTileY);
  };
  // The issuer: tiles 2G + ticket in increasing order; after the first one past the
  // last tile no more tickets are drawn.
  const int first = 2 * int(gridDim.x);
  bool dry = first >= total;
  auto draw = [&]() {
    if (dry) return total;
    const int t = first + int(atomicAdd(queue, 1u));
    dry = t >= total;
    return dry ? total : t;
  };
  auto kind_at = [&](int2 o) { return tile_kind<false, S>(o.x, o.y, nx, ny); };
  auto issue = [&](int t, int2 o, int slot) {  // the issuer
    if (t < total && kind_at(o) == kTensorCopy) {
      fence_proxy_async();
      issue_windows(win(slot), &tin, o.x, o.y, &bar[slot], 0, rows);
    }
  };
  int pending = total;  // the issuer: the tile after the two staged ones
  if (threadIdx.x == kIssuer) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    const int b = int(blockIdx.x), g = int(gridDim.x);
    tq[0] = b < total ? b : total;
    tq[1] = b + g < total ? b + g : total;
    tp[0] = origin(tq[0]);
    tp[1] = origin(tq[1]);
    issue(tq[0], tp[0], 0);
    issue(tq[1], tp[1], 1);
    pending = tq[1] < total ? draw() : total;
  }
  __syncthreads();
  unsigned ph = 0u;  // bit s: parity of the next phase of bar[s]
  for (int k = 0;; ++k) {
    const int slot = k & 1;
    const int t = tq[slot];  // tickets rise, so the first past the end ends the loop
    if (t >= total) break;
    const int2 o = tp[slot];
    const int x0 = o.x, y0 = o.y;
    const int kind = kind_at(o);
    real f[kTileRows][9];
    bool late = false;
    if (kind == kTensorCopy) {
      late = !mbar_wait(&bar[slot], (ph >> slot) & 1u);
      ph ^= 1u << slot;
    }
    if (kind == kPlainLoad)
      load_tile<real, S, kTileY, XP>(fin, nx, ny, st, x0, y0, f, rs[slot]);
    else  // read even after a failed wait (in bounds; the block then stops)
      window_tile<S, XP>(win(slot), f, rs[slot]);
    if (__syncthreads_or(late)) {
      if (threadIdx.x == kIssuer) {
        atomicExch(err, 1);
        mbar_wait(&bar[slot], ((ph >> slot) & 1u) ^ 1u);
        const int to = tq[slot ^ 1];
        if (to < total && kind_at(tp[slot ^ 1]) == kTensorCopy) mbar_wait(&bar[slot ^ 1], (ph >> (slot ^ 1)) & 1u);
      }
      break;
    }
    // The buffer of this tile is free: stage the tile two ahead into it.
    if (threadIdx.x == kIssuer) {
      tq[slot] = pending;
      tp[slot] = origin(pending);
      issue(pending, tp[slot], slot);
      pending = draw();
    }
    collide_tile<V, S, kTileY, XP>(f, fout, nx, ny, st, c, lattice_part(c), x0, y0, rs[slot], rnd);
  }
  if (threadIdx.x == kIssuer) {
    __threadfence();
    if (atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
      atomicExch(queue, 0u);
      atomicExch(queue + 1, 0u);
    }
  }
}

}  // namespace lbm
