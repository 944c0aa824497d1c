// Kernels of the time step (sm_103a); initial states and diagnostics are in
// lbm_fields.cuh.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

constexpr int kFusedThreads = 256;  // 8 warps; each warp owns a 32-column strip of rows

// Where population i of node (x, y) lives: f[i * ps + y * rs + x].  Planes layout
// f[9][ny][sx] (sx = nx, or the batched pools' padded row stride): ps = sx ny,
// rs = sx; rows layout f[ny][9][nx] (a row's nine planes side by side): ps = nx,
// rs = 9 nx.  32-bit offsets: the library limits 9 nx ny to below 2^31.
struct Strides {
  int ps, rs;
  __host__ __device__ int at(int i, int x, int y) const { return i * ps + y * rs + x; }
};
__host__ __device__ inline Strides planes_strides(int sx, int ny) { return Strides{sx * ny, sx}; }
__host__ __device__ inline Strides rows_strides(int nx) { return Strides{nx, 9 * nx}; }

__host__ __device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Single periodic wrap of v in [-n, 2n).
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Pulls the nine populations of row r at columns (cm, cc, cp) = (x-1, x, x+1):
// f_i(x, r) = fbar_i(x - e_i, r - e_i) (supplement Eq. 2), periodic.  plane, sx:
// the population and row strides in elements (Strides ps, rs).  32-bit offsets:
// the library limits the buffer to below 2^31 elements.
template <typename real, typename store_t>
__device__ __forceinline__ void pull_row(const store_t* __restrict__ fin, int plane, int sx, int ny, int r, int cm,
                                         int cc, int cp, real (&f)[9]) {
  const int rm = r == 0 ? ny - 1 : r - 1, rp = r == ny - 1 ? 0 : r + 1;
  const int oc = r * sx, om = rm * sx, op = rp * sx;
  f[0] = ld_st(fin + (oc + cc));
  f[1] = ld_st(fin + (plane + oc + cm));
  f[2] = ld_st(fin + (2 * plane + om + cc));
  f[3] = ld_st(fin + (3 * plane + oc + cp));
  f[4] = ld_st(fin + (4 * plane + op + cc));
  f[5] = ld_st(fin + (5 * plane + om + cm));
  f[6] = ld_st(fin + (6 * plane + om + cp));
  f[7] = ld_st(fin + (7 * plane + op + cp));
  f[8] = ld_st(fin + (8 * plane + op + cm));
}

template <typename real>
__device__ __forceinline__ real sum9(const real (&f)[9]) {
  return ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
}

// Fused stream + force + collide step on a TX x TY tile (TX = 32 columns, TY
// rows, 16 TY threads, two nodes per thread in the same column, TY/2 rows apart).
// Phase 1: each thread pulls the nine populations of its two nodes into
// registers; the 2 (TX + 2) + 2 TY nodes of the one-node ring around the tile
// are pulled too (densities only).  All loads are issued before any is used.
// The densities of tile + ring go to shared memory.  Phase 2: each thread forms
// the force stencil of its nodes from shared memory and collides; with V = f2
// the two nodes are the two lanes of one packed FP32x2 collision.  DRAM traffic
// is one read and one write of every population; the ring re-reads hit L2.
constexpr int kTileX = 32, kTileY = 16, kTileRows = 2;
constexpr int kRowStride = kTileY / kTileRows;  // 8
#ifndef LBM_FUSED_MIN_BLOCKS
#define LBM_FUSED_MIN_BLOCKS 4
#endif
// Resident blocks per SM the register budget must allow: 4 for the FP32-pair
// kernels (64 registers; the kernel is latency-bound, so the extra resident warps
// outweigh a few spilled registers), 2 for FP64.
template <typename V>
constexpr int fused_min_blocks() {
  return sizeof(typename LaneType<V>::type) == 8 ? 2 : LBM_FUSED_MIN_BLOCKS;
}

template <int TY>
struct TileShape {
  static constexpr int threads = kTileX * TY / kTileRows;
  static constexpr int stride = TY / kTileRows;
  static constexpr int ring = 2 * (kTileX + 2) + 2 * TY;
};

// The two nodes of a TX x TY tile a thread owns (tile-local column lx(k), row
// ly(k), k = 0, 1).  Row pairs: (t mod 32, t / 32 + k TY / 2), one warp per
// 32-column strip.  Column pairs (XP; the FP16-storage kernels): (2 (t mod 16) + k,
// row(t)), so that the two nodes' populations are adjacent in memory and leave as
// one 4-byte half pair per population, and their stencils come from aligned
// 8-byte reads of the density tile.  Warp w covers rows r and r + 2, r = 4 (w / 2)
// + w mod 2: two rows of an FP16 window (24 words a row) are 48 words, 16 banks,
// apart, so the two half-warps' reads of a window row fall in different banks.
template <int TY, bool XP>
struct NodeMap {
  static_assert(!XP || TY % 4 == 0, "column pairs take rows in groups of four");
  __device__ static int lx(int k) { return XP ? 2 * int(threadIdx.x & 15u) + k : int(threadIdx.x & 31u); }
  __device__ static int ly(int k) {
    if constexpr (XP) {
      const int w = int(threadIdx.x >> 5);
      return 4 * (w >> 1) + (w & 1) + 2 * int((threadIdx.x >> 4) & 1u);
    } else {
      return int(threadIdx.x >> 5) + k * (TY / kTileRows);
    }
  }
};

// Column pairs for 2-byte storage.
template <typename S>
__host__ __device__ constexpr bool xpairs() {
  return sizeof(S) == 2;
}

// Phase 2 of a tile, arithmetic part: force stencil of each thread's two nodes
// from the shared densities and the collision (one packed FP32x2 evaluation for
// V = f2); out[k] = post-collision deviations of the thread's node k (NodeMap).
template <typename V, int TY, bool XP = false>
__device__ __forceinline__ void collide_nodes(const typename LaneType<V>::type (&f)[kTileRows][9], const VCoef<V>& c,
                                              const LatCoef<V>& l,
                                              const typename LaneType<V>::type (*rs)[kTileX + 2],
                                              typename LaneType<V>::type (&out)[kTileRows][9]) {
  using real = typename LaneType<V>::type;
  if constexpr (Lanes<V>::n == 2 && XP) {
    // Lanes = columns 2j + 1, 2j + 2 of density rows ly .. ly + 2 (j = t mod 16);
    // each row's cells 2j .. 2j + 3 arrive as two aligned float2 reads (rows of
    // 34 floats, the tile 8-byte aligned): the pairs at dx = -1 and +1 as they are,
    // the one at dx = 0 from their inner halves.
    const int j = threadIdx.x & 15u, ly = NodeMap<TY, XP>::ly(0);
    float2 a[3], b[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float2* q = reinterpret_cast<const float2*>(rs[ly + r]) + j;
      a[r] = q[0];
      b[r] = q[1];
    }
    auto mid = [&](int r) {
      V v;
      v.v = make_float2(a[r].y, b[r].x);
      return v;
    };
    const V ml{a[0]}, mc = mid(0), mr{b[0]}, cl{a[1]}, cr{b[1]}, pl{a[2]}, pc = mid(2), pr{b[2]};
    const V Sxp = fmav(c.third, cr - cl, c.twelfth * ((pr - pl) + (mr - ml)));
    const V Syp = fmav(c.third, pc - mc, c.twelfth * ((pr + pl) - (mr + ml)));
    V d[9], o[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i].v = make_float2(f[0][i], f[1][i]);
    collide(c, l, d, Sxp, Syp, o);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      out[0][i] = o[i].v.x;
      out[1][i] = o[i].v.y;
    }
  } else if constexpr (Lanes<V>::n == 2) {
    // Both nodes' stencils as one packed evaluation: lane k reads row ty + k stride.
    const int tx = threadIdx.x & (kTileX - 1), ty = threadIdx.x / kTileX;
    const int lx = tx + 1, l0 = ty + 1, l1 = ty + TileShape<TY>::stride + 1;
    auto pair = [&](int dy, int dx) {
      V v;
      v.v = make_float2(rs[l0 + dy][lx + dx], rs[l1 + dy][lx + dx]);
      return v;
    };
    const V ml = pair(-1, -1), mc = pair(-1, 0), mr = pair(-1, 1), cl = pair(0, -1), cr = pair(0, 1);
    const V pl = pair(1, -1), pc = pair(1, 0), pr = pair(1, 1);
    const V Sxp = fmav(c.third, cr - cl, c.twelfth * ((pr - pl) + (mr - ml)));
    const V Syp = fmav(c.third, pc - mc, c.twelfth * ((pr + pl) - (mr + ml)));
    V d[9], o[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i].v = make_float2(f[0][i], f[1][i]);
    collide(c, l, d, Sxp, Syp, o);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      out[0][i] = o[i].v.x;
      out[1][i] = o[i].v.y;
    }
  } else {
    using M = NodeMap<TY, XP>;
#pragma unroll
    for (int k = 0; k < kTileRows; ++k) {
      const int ly = M::ly(k) + 1, lx = M::lx(k) + 1;
      real Sx, Sy;
      stencil(rs[ly - 1][lx - 1], rs[ly - 1][lx], rs[ly - 1][lx + 1], rs[ly][lx - 1], rs[ly][lx + 1],
              rs[ly + 1][lx - 1], rs[ly + 1][lx], rs[ly + 1][lx + 1], Sx, Sy);
      collide(c, l, f[k], Sx, Sy, out[k]);
    }
  }
}

// Phase 2 of a tile, store part: the thread's two nodes of the tile at (x0, y0).
// FP16 column pairs of an even-width lattice leave as half pairs.
template <typename real, typename store_t, int TY, bool XP = false>
__device__ __forceinline__ void store_nodes(const real (&out)[kTileRows][9], store_t* __restrict__ fout, int nx,
                                            int ny, Strides st, int x0, int y0, Rounding rnd) {
  using M = NodeMap<TY, XP>;
  if constexpr (XP && sizeof(real) == 4 && sizeof(store_t) == 2) {
    const int gx = x0 + M::lx(0), gy = y0 + M::ly(0);
    if ((nx & 1) == 0) {  // gx even, so gx < nx implies gx + 1 < nx
      if (gx < nx && gy < ny) store9_pair(fout + (gy * st.rs + gx), st.ps, out[0], out[1], gx, gy, nx, rnd);
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int gx = x0 + M::lx(k), gy = y0 + M::ly(k);
    if (gx < nx && gy < ny) store9(fout + (gy * st.rs + gx), st.ps, out[k], gx, gy, nx, rnd);
  }
}

// Phase 2 of a tile: collide_nodes, then store_nodes.
template <typename V, typename store_t, int TY, bool XP = false>
__device__ __forceinline__ void collide_tile(const typename LaneType<V>::type (&f)[kTileRows][9],
                                             store_t* __restrict__ fout, int nx, int ny, Strides st, const VCoef<V>& c,
                                             const LatCoef<V>& l, int x0, int y0,
                                             const typename LaneType<V>::type (*rs)[kTileX + 2],
                                             Rounding rnd = Rounding{0u, 0}) {
  typename LaneType<V>::type out[kTileRows][9];
  collide_nodes<V, TY, XP>(f, c, l, rs, out);
  store_nodes<typename LaneType<V>::type, store_t, TY, XP>(out, fout, nx, ny, st, x0, y0, rnd);
}

struct NoHook {
  __device__ void operator()() const {}
};

// Phase 1 of a tile with plain loads: pulls the populations of the thread's two
// nodes into f and writes the densities of tile + ring to rs (shared array of
// (TY + 2) x (TX + 2) densities).  (x0, y0): tile origin; st: the layout.
// Periodic wrap.
template <typename real, typename store_t, int TY, bool XP = false>
__device__ __forceinline__ void load_tile(const store_t* __restrict__ fin, int nx, int ny, Strides st, int x0,
                                          int y0, real (&f)[kTileRows][9], real (*rs)[kTileX + 2]) {
  using Shape = TileShape<TY>;
  using M = NodeMap<TY, XP>;
  const bool small = nx <= kTileX || ny <= TY;  // tiles may wrap more than once
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int gx = x0 + M::lx(k), gy = y0 + M::ly(k);
    const int xc = small ? wrap(gx, nx) : wrap1(gx, nx);
    const int xm = xc == 0 ? nx - 1 : xc - 1, xp = xc == nx - 1 ? 0 : xc + 1;
    pull_row(fin, st.ps, st.rs, ny, small ? wrap(gy, ny) : wrap1(gy, ny), xm, xc, xp, f[k]);
  }
  // Ring: the row above, the row below, then the left and right columns.
  const int t = threadIdx.x;
  const bool ring = t < Shape::ring;
  int wx = 0, wy = 0;
  real g[9];
  if (ring) {
    if (t < kTileX + 2) {
      wx = t, wy = 0;
    } else if (t < 2 * (kTileX + 2)) {
      wx = t - (kTileX + 2), wy = TY + 1;
    } else if (t < 2 * (kTileX + 2) + TY) {
      wx = 0, wy = t - 2 * (kTileX + 2) + 1;
    } else {
      wx = kTileX + 1, wy = t - 2 * (kTileX + 2) - TY + 1;
    }
    const int hx = small ? wrap(x0 - 1 + wx, nx) : wrap1(x0 - 1 + wx, nx);
    const int hy = small ? wrap(y0 - 1 + wy, ny) : wrap1(y0 - 1 + wy, ny);
    pull_row(fin, st.ps, st.rs, ny, hy, hx == 0 ? nx - 1 : hx - 1, hx, hx == nx - 1 ? 0 : hx + 1, g);
  }
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) rs[M::ly(k) + 1][M::lx(k) + 1] = sum9(f[k]);
  if (ring) rs[wy][wx] = sum9(g);
}

// One fused step of a tile: load_tile, block barrier, collide_tile.
// before_sync() runs after all phase-1 loads are issued and before the block
// barrier (the batched kernel stores its lattice coefficients there).
template <typename V, typename store_t, int TY, typename Hook = NoHook, bool XP = false>
__device__ __forceinline__ void step_tile(const store_t* __restrict__ fin, store_t* __restrict__ fout, int nx,
                                          int ny, Strides st, const VCoef<V>& c, const LatCoef<V>& l, int x0, int y0,
                                          typename LaneType<V>::type (*rs)[kTileX + 2],
                                          const Hook& before_sync = Hook(), Rounding rnd = Rounding{0u, 0}) {
  using real = typename LaneType<V>::type;
  real f[kTileRows][9];
  load_tile<real, store_t, TY, XP>(fin, nx, ny, st, x0, y0, f, rs);
  before_sync();
  __syncthreads();
  collide_tile<V, store_t, TY, XP>(f, fout, nx, ny, st, c, l, x0, y0, rs, rnd);
}

template <typename V, typename store_t>
__global__ void __launch_bounds__(kFusedThreads, fused_min_blocks<V>())
    k_step_fused(const store_t* __restrict__ fin, store_t* __restrict__ fout, int nx, int ny, Strides st,
                 VCoef<V> c, Rounding rnd) {
  rnd = resolve(rnd);
  __shared__ __align__(16) typename LaneType<V>::type rs[kTileY + 2][kTileX + 2];
  constexpr bool XP = xpairs<store_t>() && Lanes<V>::n == 2;
  step_tile<V, store_t, kTileY, NoHook, XP>(fin, fout, nx, ny, st, c, lattice_part(c), blockIdx.x * kTileX,
                                            blockIdx.y * kTileY, rs, NoHook(), rnd);
}

// Two-pass variant, pass 1: density plane rho_dev(x) = sum_i fbar_i(x - e_i).
template <typename real, typename store_t>
__global__ void k_density(const store_t* __restrict__ fin, real* __restrict__ rho, int nx, int ny, Strides st) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  real f[9];
  pull_row(fin, st.ps, st.rs, ny, y, x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1, f);
  rho[y * nx + x] = sum9(f);
}

// Two-pass variant, pass 2: pull, force stencil from the density plane, collide.
template <typename real, typename store_t>
__global__ void k_collide_rho(const store_t* __restrict__ fin, store_t* __restrict__ fout,
                              const real* __restrict__ rho, int nx, int ny, Strides st, VCoef<real> c,
                              Rounding rnd) {
  rnd = resolve(rnd);
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  real f[9];
  pull_row(fin, st.ps, st.rs, ny, y, xm, x, xp, f);
  const real* rm = rho + ym * nx;
  const real* rc = rho + y * nx;
  const real* rpp = rho + yp * nx;
  real Sx, Sy;
  stencil(__ldg(rm + xm), __ldg(rm + x), __ldg(rm + xp), __ldg(rc + xm), __ldg(rc + xp), __ldg(rpp + xm),
          __ldg(rpp + x), __ldg(rpp + xp), Sx, Sy);
  real o[9];
  collide(c, f, Sx, Sy, o);
  store9(fout + st.at(0, x, y), st.ps, o, x, y, nx, rnd);
}

}  // namespace lbm
