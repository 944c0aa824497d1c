// Batched solver: many independent periodic lattices, each with its own size and
// parameters, advanced together.  One kernel launch per time step walks a flat
// list of 32 x TY tiles spanning all lattices, stages the coefficients of the
// tile's lattice in shared memory and runs the same tile code as the
// single-lattice fused step; the fastest form is the persistent tensor-copy
// kernel of the single-lattice FP32 step with one tensor map per lattice.  Rows
// are stored with a stride of nx rounded up to a multiple of 4 floats, as the
// tensor copies require.  Runs of steps are captured once into CUDA graphs and
// replayed.  The autotuner times every launch form on the batch itself and keeps
// the fastest.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_handle.cuh"
#include "lbm_fields.cuh"
#include "lbm_tma.cuh"

namespace lbm {
template <typename V>
VCoef<V> make_vcoef(const lb_params& p, const lb_derived& d);
}  // namespace lbm

namespace {

using namespace lbm;

struct BatchLattice {
  int nx, ny;
  int sx;            // row stride: nx rounded up to a multiple of 4
  long long offset;  // element offset of the lattice's plane 0 in a pool
  int tile_start;    // index of its first tile in the flat tile list
  int tiles_x;       // tiles per row of tiles
};

__host__ __device__ constexpr int row_stride(int nx) { return (nx + 3) / 4 * 4; }

// Strides of a lattice in the pools: planes f[9][ny][sx], or rows f[ny][9][sx]
// (every lattice of a batch in the same layout).
__host__ __device__ inline Strides lat_strides(int sx, int ny, int rows) {
  return rows ? Strides{sx, 9 * sx} : planes_strides(sx, ny);
}

// Launch shapes the autotuner chooses among: tile height and the register budget
// the kernel is compiled for (resident blocks per SM it must allow), plain loads;
// shapes 3 and 4 are the persistent tensor-copy kernel (32 x 16 tiles, the tile
// list of shape 0) at 80 and 128 registers walking the list statically, shapes 5
// and 6 the same taking tiles by ticket with two windows in flight.
constexpr int kShapes = 7;
constexpr int kShapeTMA = 3;  // first tensor-copy shape
constexpr int kShapeDyn = 5;  // first ticket-dispatch shape
constexpr int kShapeTY[kShapes] = {16, 16, 32, 16, 16, 16, 16};
__host__ __device__ constexpr bool is_tma(int shape) { return shape >= kShapeTMA; }
__host__ __device__ constexpr bool is_dyn(int shape) { return shape >= kShapeDyn; }
constexpr int kGraphSteps = 64;  // steps per captured graph (even: the pools end where they started)

// One record per tile: its lattice, origin, the lattice's size and strides (in the
// pool's layout), how the tensor-copy kernels stage it (TileKind, from the tile's
// position, fixed when the batch is built) and the lattice's pool offset.
struct TileRec {
  int lat, x0, y0, nx, ny;
  int ps, rs;  // population and row strides of the lattice in its pool (Strides)
  int kind;
  long long offset;
};

// The coefficients shared by all lattices (varpi, rates, EOS constants) come from
// the kernel parameters; the ten that depend on each lattice's Tr, K_int, G2 and
// storage shift are staged in shared memory when the block moves to a new lattice,
// one 32-bit word per thread, stored after the tile's pulls are issued.  In the
// persistent mode the next tile's record and coefficient word are fetched while
// the current tile is processed.
constexpr int kCoefWords = int(sizeof(LatCoef<f2>) / sizeof(int));

struct StoreCoef {
  LatCoef<f2>* cs;
  int word;
  bool store;
  __device__ void operator()() const {
    if (store && threadIdx.x < kCoefWords) reinterpret_cast<int*>(cs)[threadIdx.x] = word;
  }
};

template <typename store_t, int TY, int MINB, bool PERSIST>
__global__ void __launch_bounds__(TileShape<TY>::threads, MINB)
    k_step_batch(const store_t* __restrict__ pool_in, store_t* __restrict__ pool_out,
                 const TileRec* __restrict__ tiles, const LatCoef<f2>* __restrict__ coef, int total_tiles,
                 VCoef<f2> common, int rows) {
  static_assert(kCoefWords <= TileShape<TY>::threads, "one coefficient word per thread");
  __shared__ float rs[TY + 2][kTileX + 2];
  __shared__ LatCoef<f2> cs;
  int t = blockIdx.x;
  if (t >= total_tiles) return;
  TileRec ti = tiles[t];
  int word = threadIdx.x < kCoefWords ? reinterpret_cast<const int*>(coef + ti.lat)[threadIdx.x] : 0;
  if constexpr (!PERSIST) {  // one block per tile
    step_tile<f2, store_t, TY>(pool_in + ti.offset, pool_out + ti.offset, ti.nx, ti.ny,
                               Strides{ti.ps, ti.rs}, common, cs, ti.x0, ti.y0, rs,
                               StoreCoef{&cs, word, true});
    return;
  }
  int last = -1;
  for (;;) {
    const int tn = t + gridDim.x;
    TileRec tin = ti;
    int wordn = word;
    if (tn < total_tiles) {
      tin = tiles[tn];
      if (threadIdx.x < kCoefWords) wordn = reinterpret_cast<const int*>(coef + tin.lat)[threadIdx.x];
    }
    const StoreCoef hook{&cs, word, ti.lat != last};
    last = ti.lat;
    step_tile<f2, store_t, TY>(pool_in + ti.offset, pool_out + ti.offset, ti.nx, ti.ny,
                               Strides{ti.ps, ti.rs}, common, cs, ti.x0, ti.y0, rs, hook);
    if (tn >= total_tiles) break;
    __syncthreads();  // shared densities and coefficients are reused by the next tile
    t = tn;
    ti = tin;
    word = wordn;
  }
}

// Persistent tensor-copy form (the single-lattice k_step_tma over the tile list of
// all lattices).  Per tile: thread 0 bulk-copies the lattice's coefficients into
// shared memory on the mbarrier and, for an interior tile, issues the nine window
// copies through that lattice's tensor map (maps[lat]); for a wrapping tile every
// thread issues its asynchronous copies of the window.  The next tile is staged
// once the current window is in registers, so it travels during the collision.
// Tile records (written by thread 0 one tile ahead), coefficients and densities
// are double-buffered in shared memory.  A wait that gives up sets *err.
static_assert(sizeof(LatCoef<f2>) % 16 == 0, "bulk copies move multiples of 16 bytes");

template <int MINB>
__global__ void __launch_bounds__(kFusedThreads, MINB)
    k_step_batch_tma(const float* __restrict__ pool_in, float* __restrict__ pool_out,
                     const TileRec* __restrict__ tiles, const LatCoef<f2>* __restrict__ coef,
                     const CUtensorMap* __restrict__ maps, int total_tiles, VCoef<f2> common, int* __restrict__ err,
                     int rows) {
  extern __shared__ __align__(128) unsigned char dyn[];
  float* win = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(dyn) + 127) & ~uintptr_t(127));
  __shared__ float rs[2][kTileY + 2][kTileX + 2];
  __shared__ __align__(16) LatCoef<f2> cs[2];
  __shared__ TileRec rec[2];
  __shared__ __align__(8) unsigned long long bar;
  if (blockIdx.x >= total_tiles) return;
  auto kind_of = [](const TileRec& r) { return r.kind; };
  // All threads: stage the tile of record r, its coefficients into cs[slot].
  auto issue = [&](const TileRec& r, int slot) {
    const int kind = kind_of(r);
    if (threadIdx.x == 0) {
      fence_proxy_async();
      if (kind == kTensorCopy)
        issue_windows(win, maps + r.lat, r.x0, r.y0, &bar, sizeof(LatCoef<f2>), rows != 0);
      else
        mbar_expect_tx(&bar, sizeof(LatCoef<f2>));
      bulk_load(&cs[slot], coef + r.lat, sizeof(LatCoef<f2>), &bar);
    }
    if (kind == kAsyncCopy) issue_window_async(win, pool_in + r.offset, r.nx, r.ny, Strides{r.ps, r.rs}, r.x0, r.y0);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    rec[0] = tiles[blockIdx.x];
  }
  __syncthreads();
  issue(rec[0], 0);
  unsigned parity = 0;
  int buf = 0;
  for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    const int tn = t + gridDim.x;
    // The next record, for everyone after the barrier below (its slot was last read
    // before the previous barrier).
    if (threadIdx.x == 0 && tn < total_tiles) rec[buf ^ 1] = tiles[tn];
    const TileRec ti = rec[buf];
    const int kind = kind_of(ti);
    const bool late = !mbar_wait(&bar, parity);
    parity ^= 1u;
    if (kind == kAsyncCopy) {
      cp_async_wait_all();
      __syncthreads();
    }
    float f[kTileRows][9];
    if (kind == kPlainLoad)
      load_tile<float, float, kTileY>(pool_in + ti.offset, ti.nx, ti.ny, Strides{ti.ps, ti.rs}, ti.x0,
                                      ti.y0, f, rs[buf]);
    else  // read even after a failed wait (in bounds; the block then returns)
      window_tile(win, f, rs[buf]);
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        mbar_wait(&bar, parity ^ 1u);
      }
      return;
    }
    if (tn < total_tiles) issue(rec[buf ^ 1], buf ^ 1);
    collide_tile<f2, float, kTileY>(f, pool_out + ti.offset, ti.nx, ti.ny, Strides{ti.ps, ti.rs}, common,
                                    cs[buf], ti.x0, ti.y0, rs[buf]);
    buf ^= 1;
  }
}

// Ticket form of the kernel above (the single-lattice k_step_tma_dyn over the tile
// list): block b starts with list entries b and b + G, then takes 2G, 2G + 1, ...
// by ticket (queue[0]; queue[1] counts finished blocks, and the last one resets
// both).  Tile k of a block has its window in buffer k mod 2, its coefficients in
// slot k mod 3 and its record in slot k mod 4: the record of tile k + 2 is written
// by the issuer before the barrier of tile k, and its window, coefficients (bulk
// copy on the buffer's mbarrier) and, for a wrapping tile, the per-thread
// asynchronous copies are issued after it.  The record's fields are read from
// shared memory where they are used (the store after the collision reads the
// lattice's origin, size and strides), so they hold no registers during the
// collision; the fourth record slot keeps a record until its tile is stored.  Every staged tile commits one group of asynchronous copies
// (empty unless it wraps), so waiting for all but the newest group completes tile
// k's.  A wait that gives up sets *err.
template <int MINB>
__global__ void __launch_bounds__(kFusedThreads, MINB)
    k_step_batch_tma_dyn(const float* __restrict__ pool_in, float* __restrict__ pool_out,
                         const TileRec* __restrict__ tiles, const LatCoef<f2>* __restrict__ coef,
                         const CUtensorMap* __restrict__ maps, int total_tiles, VCoef<f2> common,
                         int* __restrict__ err, unsigned* __restrict__ queue, int rows) {
  extern __shared__ __align__(128) unsigned char dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dyn) + 127) & ~uintptr_t(127));
  __shared__ float rs[2][kTileY + 2][kTileX + 2];
  __shared__ __align__(16) LatCoef<f2> cs[3];
  __shared__ TileRec rec[4];  // tile k's record in slot k mod 4, read until its store
  __shared__ int tq[4];
  __shared__ __align__(8) unsigned long long bar[2];
  const int total = total_tiles;
  auto win = [&](int slot) { return reinterpret_cast<float*>(base + slot * Win2<float>::buffer); };
  auto kind_of = [](const TileRec& r) { return r.kind; };
  const int first = 2 * int(gridDim.x);
  bool dry = first >= total;  // the issuer: no more tickets
  auto draw = [&]() {
    if (dry) return total;
    const int t = first + int(atomicAdd(queue, 1u));
    dry = t >= total;
    return dry ? total : t;
  };
  // All threads: stage tile j of the block (record in slot j mod 4, coefficients in
  // slot j mod 3).
  auto issue = [&](int j) {
    const int q = j % 3, slot = j & 1;
    const TileRec& r = rec[j & 3];
    const bool live = tq[j & 3] < total;
    const int kind = live ? kind_of(r) : kPlainLoad;
    if (live && threadIdx.x == kIssuer) {
      fence_proxy_async();
      if (kind == kTensorCopy)
        issue_windows(win(slot), maps + r.lat, r.x0, r.y0, &bar[slot], sizeof(LatCoef<f2>), rows != 0);
      else
        mbar_expect_tx(&bar[slot], sizeof(LatCoef<f2>));
      bulk_load(&cs[q], coef + r.lat, sizeof(LatCoef<f2>), &bar[slot]);
    }
    if (live && kind == kAsyncCopy)
      issue_window_async(win(slot), pool_in + r.offset, r.nx, r.ny, Strides{r.ps, r.rs}, r.x0, r.y0);
    else
      cp_async_commit();
  };
  int pending = total;  // the issuer: the tile after the staged ones
  if (threadIdx.x == kIssuer) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    const int b = int(blockIdx.x), g = int(gridDim.x);
    tq[0] = b < total ? b : total;
    tq[1] = b + g < total ? b + g : total;
    if (tq[0] < total) rec[0] = tiles[tq[0]];
    if (tq[1] < total) rec[1] = tiles[tq[1]];
    pending = tq[1] < total ? draw() : total;
  }
  __syncthreads();
  issue(0);
  issue(1);
  unsigned ph = 0u;  // bit s: parity of the next phase of bar[s]
  for (int k = 0;; ++k) {
    const int q = k % 3, slot = k & 1, rq = k & 3;
    if (tq[rq] >= total) break;  // uniform; tiles rise, so no later tile is staged
    const TileRec& ti = rec[rq];  // read where used: the fields stay in shared memory
    const int kind = kind_of(ti);
    if (threadIdx.x == kIssuer) {  // the record of tile k + 2 (its slot's last reader was tile k - 2,
      const int q2 = (k + 2) & 3;   // which every thread finished before the barrier of tile k - 1)
      tq[q2] = pending;
      if (pending < total) rec[q2] = tiles[pending];
      pending = draw();
    }
    const bool late = !mbar_wait(&bar[slot], (ph >> slot) & 1u);
    ph ^= 1u << slot;
    if (kind == kAsyncCopy) {
      cp_async_wait_all_but_one();
      __syncthreads();
    }
    float f[kTileRows][9];
    if (kind == kPlainLoad)
      load_tile<float, float, kTileY>(pool_in + ti.offset, ti.nx, ti.ny, Strides{ti.ps, ti.rs}, ti.x0,
                                      ti.y0, f, rs[slot]);
    else  // read even after a failed wait (in bounds; the block then stops)
      window_tile(win(slot), f, rs[slot]);
    if (__syncthreads_or(late)) {
      if (threadIdx.x == kIssuer) {
        atomicExch(err, 1);
        mbar_wait(&bar[slot], ((ph >> slot) & 1u) ^ 1u);
        if (tq[(k + 1) & 3] < total) mbar_wait(&bar[slot ^ 1], (ph >> (slot ^ 1)) & 1u);
      }
      cp_async_wait_all();
      break;
    }
    issue(k + 2);
    float out[kTileRows][9];
    collide_nodes<f2, kTileY>(f, common, cs[q], rs[slot], out);
    store_nodes<float, float, kTileY>(out, pool_out + ti.offset, ti.nx, ti.ny, Strides{ti.ps, ti.rs}, ti.x0,
                                      ti.y0, Rounding{0u, 0});
  }
  cp_async_wait_all();
  if (threadIdx.x == kIssuer) {
    __threadfence();
    if (atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
      atomicExch(queue, 0u);
      atomicExch(queue + 1, 0u);
    }
  }
}

// Non-finite check of every lattice of a batch: one block per tile of the
// 32 x 16 tile list, each thread the two nodes (x0 + tx, y0 + ty) and
// (x0 + tx, y0 + ty + 8); a node counts when the sum of its nine stored
// populations is not finite.  The block's count goes to bad[lattice].
__global__ void __launch_bounds__(kFusedThreads) k_batch_nonfinite(const float* __restrict__ pool,
                                                                    const TileRec* __restrict__ tiles, int rows,
                                                                    unsigned* __restrict__ bad) {
  const TileRec t = tiles[blockIdx.x];
  const int x = t.x0 + (threadIdx.x & (kTileX - 1));
  const Strides st{t.ps, t.rs};
  int n = 0;
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int y = t.y0 + int(threadIdx.x / kTileX) + k * kRowStride;
    if (x < t.nx && y < t.ny) {
      const float* f = pool + t.offset;
      float sum = 0.f;
#pragma unroll
      for (int i = 0; i < 9; ++i) sum += f[st.at(i, x, y)];
      n += isfinite(sum) ? 0 : 1;
    }
  }
  const int total = __syncthreads_count(n > 0) + __syncthreads_count(n > 1);
  if (threadIdx.x == 0 && total > 0) atomicAdd(bad + t.lat, unsigned(total));
}

template <int TY, int MINB>
void launch_shape(const float* in, float* out, const TileRec* tiles, const LatCoef<f2>* coef, int total, int bps,
                  int sms, const VCoef<f2>& common, cudaStream_t st, int rows) {
  if (bps > 0)
    k_step_batch<float, TY, MINB, true><<<bps * sms, TileShape<TY>::threads, 0, st>>>(in, out, tiles, coef, total,
                                                                                        common, rows);
  else
    k_step_batch<float, TY, MINB, false><<<total, TileShape<TY>::threads, 0, st>>>(in, out, tiles, coef, total,
                                                                                     common, rows);
}

const void* batch_kernel(int shape) {
  switch (shape) {
    case 0: return reinterpret_cast<const void*>(k_step_batch<float, 16, 4, true>);
    case 1: return reinterpret_cast<const void*>(k_step_batch<float, 16, 3, true>);
    case 2: return reinterpret_cast<const void*>(k_step_batch<float, 32, 2, true>);
    case 3: return reinterpret_cast<const void*>(k_step_batch_tma<3>);
    case 4: return reinterpret_cast<const void*>(k_step_batch_tma<2>);
    case 5: return reinterpret_cast<const void*>(k_step_batch_tma_dyn<3>);
    default: return reinterpret_cast<const void*>(k_step_batch_tma_dyn<2>);
  }
}

}  // namespace

struct lb_batch {
  int n;
  std::vector<lb_params> p;
  std::vector<lb_derived> d;
  std::vector<BatchLattice> desc[kShapes];
  int total_tiles[kShapes];
  void* pool[2];
  int cur;
  BatchLattice* d_desc[kShapes];
  TileRec* d_tiles[kShapes];
  LatCoef<f2>* d_coef;
  CUtensorMap* d_maps;  // [2][n]: lattice maps in pool 0, then in pool 1
  int* d_err;           // set by a bounded wait of the tensor-copy kernel that gave up
  unsigned* d_queue;    // tickets of the dispatch shapes (two words)
  unsigned* d_bad;      // per lattice: nodes whose density is not finite (lb_batch_nonfinite)
  std::vector<unsigned> h_bad;
  bool tma_ok;          // every lattice large enough to have interior tiles has its maps
  int rows;             // pools in the rows layout f[ny][9][sx] (else planes f[9][ny][sx])
  VCoef<f2> common;
  cudaStream_t stream;
  int sms;
  int shape;          // index into kShapeTY
  int blocks_per_sm;  // persistent grid = blocks_per_sm * sms
  int64_t steps;
  cudaGraphExec_t graph[2];  // starting from pool 0 / pool 1
  int graph_cfg[2];          // configuration the graph was captured with
  char err[512];
};

namespace {

int berr(lb_batch* b, int code, const char* fmt, const char* detail = "") {
  if (b) std::snprintf(b->err, sizeof(b->err), fmt, detail);
  else {
    char buf[512];
    std::snprintf(buf, sizeof(buf), fmt, detail);
    set_thread_error(buf);
  }
  return code;
}

size_t lattice_elems(const lb_params& p) { return ((9 * size_t(row_stride(p.nx)) * p.ny + 63) / 64) * 64; }

int max_blocks(lb_batch* b, int shape, int* out) {
  const void* k = batch_kernel(shape);
  const int threads = kShapeTY[shape] == 16 ? TileShape<16>::threads : TileShape<32>::threads;
  const int smem = is_dyn(shape) ? int(Win2<float>::smem) : (is_tma(shape) ? int(kTmaSmem) : 0);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, threads, smem);
  if (e != cudaSuccess) return berr(b, LB_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
  if (*out < 1) *out = 1;
  return LB_OK;
}

void launch_one(lb_batch* b, int from) {
  const float* in = static_cast<const float*>(b->pool[from]);
  float* out = static_cast<float*>(b->pool[1 - from]);
  // blocks_per_sm = 0: one block per tile (the hardware schedules the tiles);
  // otherwise a persistent grid whose blocks walk the tile list.
  const int s = b->shape;
  const TileRec* tiles = b->d_tiles[s];
  const int total = b->total_tiles[s];
  if (is_tma(s)) {
    const int grid = std::min(b->blocks_per_sm * b->sms, total);
    const CUtensorMap* maps = b->d_maps + from * b->n;
    if (s == kShapeDyn)
      k_step_batch_tma_dyn<3><<<grid, kFusedThreads, Win2<float>::smem, b->stream>>>(
          in, out, tiles, b->d_coef, maps, total, b->common, b->d_err, b->d_queue, b->rows);
    else if (s == kShapeDyn + 1)
      k_step_batch_tma_dyn<2><<<grid, kFusedThreads, Win2<float>::smem, b->stream>>>(
          in, out, tiles, b->d_coef, maps, total, b->common, b->d_err, b->d_queue, b->rows);
    else if (s == kShapeTMA)
      k_step_batch_tma<3><<<grid, kFusedThreads, kTmaSmem, b->stream>>>(in, out, tiles, b->d_coef, maps, total,
                                                                         b->common, b->d_err, b->rows);
    else
      k_step_batch_tma<2><<<grid, kFusedThreads, kTmaSmem, b->stream>>>(in, out, tiles, b->d_coef, maps, total,
                                                                         b->common, b->d_err, b->rows);
  } else if (s == 0)
    launch_shape<16, 4>(in, out, tiles, b->d_coef, total, b->blocks_per_sm, b->sms, b->common, b->stream, b->rows);
  else if (s == 1)
    launch_shape<16, 3>(in, out, tiles, b->d_coef, total, b->blocks_per_sm, b->sms, b->common, b->stream, b->rows);
  else
    launch_shape<32, 2>(in, out, tiles, b->d_coef, total, b->blocks_per_sm, b->sms, b->common, b->stream, b->rows);
}

int config_id(const lb_batch* b) { return b->shape * 64 + b->blocks_per_sm; }

int ensure_graph(lb_batch* b, int from) {
  if (b->graph[from] && b->graph_cfg[from] == config_id(b)) return LB_OK;
  if (b->graph[from]) {
    cudaGraphExecDestroy(b->graph[from]);
    b->graph[from] = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return berr(b, LB_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
  int side = from;
  for (int s = 0; s < kGraphSteps; ++s) {
    launch_one(b, side);
    side = 1 - side;
  }
  e = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess) return berr(b, LB_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph[from], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return berr(b, LB_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  b->graph_cfg[from] = config_id(b);
  return LB_OK;
}

}  // namespace

extern "C" {

size_t lb_batch_pool_bytes(const lb_params* ps, int n) {
  if (!ps || n < 1) return 0;
  size_t e = 0;
  for (int i = 0; i < n; ++i) e += lattice_elems(ps[i]);
  return e * sizeof(float);
}

size_t total_tiles_of(const lb_params* ps, int n, int TY) {
  size_t t = 0;
  for (int i = 0; i < n; ++i) t += size_t((ps[i].nx + kTileX - 1) / kTileX) * ((ps[i].ny + TY - 1) / TY);
  return t;
}

// The tensor-copy shape walks the tile list of shape 0; the other shapes own one.
constexpr int kTileLists = kShapeTMA;

size_t lb_batch_meta_bytes(const lb_params* ps, int n) {
  if (!ps || n < 1) return 0;
  size_t tiles = 0;
  for (int s = 0; s < kTileLists; ++s) tiles += total_tiles_of(ps, n, kShapeTY[s]);
  return size_t(n) * (kTileLists * sizeof(BatchLattice) + sizeof(LatCoef<f2>) + 2 * sizeof(CUtensorMap) +
                      sizeof(unsigned)) +
         tiles * sizeof(TileRec) + 4096 + 512;
}

int lb_batch_init(lb_batch** out, const lb_params* ps, int n, void* pool_a, void* pool_b, void* meta,
                  size_t meta_bytes, const double* rho0, int rho0_on_device, void* stream) {
  if (!out) return berr(nullptr, LB_EINVAL, "null output%s");
  *out = nullptr;
  if (!ps || n < 1 || !pool_a || !pool_b || pool_a == pool_b || !meta || !rho0)
    return berr(nullptr, LB_EINVAL, "lb_batch_init: invalid arguments%s");
  if (meta_bytes < lb_batch_meta_bytes(ps, n)) return berr(nullptr, LB_ENOMEM, "lb_batch_init: meta buffer too small%s");
  lb_batch* b = new (std::nothrow) lb_batch();
  if (!b) return berr(nullptr, LB_EINVAL, "out of host memory%s");
  b->n = n;
  b->rows = ps[0].layout == LB_LAYOUT_ROWS ? 1 : 0;
  b->p.assign(ps, ps + n);
  b->d.resize(n);
  b->stream = static_cast<cudaStream_t>(stream);
  b->pool[0] = pool_a;
  b->pool[1] = pool_b;
  b->cur = 0;
  b->graph[0] = b->graph[1] = nullptr;
  b->graph_cfg[0] = b->graph_cfg[1] = -1;
  auto bail = [&](int code, const char* msg) {
    set_thread_error(msg);
    delete b;
    return code;
  };
  // rho_ref = NaN: that lattice's storage shift is its mean initial density (as in
  // lb_init), from the densities staged in pool_b, block sums in pool_a.
  std::vector<double> mean(n, 0.0);
  bool staged = false;
  {
    bool any = false;
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
      if (ps[i].nx < 1 || ps[i].ny < 1) return bail(LB_EINVAL, "lb_batch_init: lattice sides must be positive");
      total += size_t(ps[i].nx) * ps[i].ny;
      any = any || std::isnan(ps[i].rho_ref);
    }
    if (any) {
      // Invalid parameters never reach the GPU: check every lattice first.
      for (int i = 0; i < n; ++i) {
        lb_derived tmp;
        char err[512] = {0};
        if (ps[i].precision != LB_FP32 || ps[i].layout != ps[0].layout ||
            derive(&ps[i], &tmp, err, sizeof(err)) != LB_OK) {
          any = false;  // the loop below reports the error
          break;
        }
      }
    }
    if (any) {
      cudaError_t e = cudaSuccess;
      const double* x = rho0;
      if (!rho0_on_device) {
        e = cudaMemcpyAsync(pool_b, rho0, total * sizeof(double), cudaMemcpyHostToDevice, b->stream);
        x = static_cast<const double*>(pool_b);
        staged = true;
      }
      size_t at = 0;
      for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const size_t N = size_t(ps[i].nx) * ps[i].ny;
        if (std::isnan(ps[i].rho_ref)) e = device_mean(x + at, N, pool_a, lb_batch_pool_bytes(ps, n), b->stream, &mean[i]);
        at += N;
      }
      if (e != cudaSuccess) {
        char msg[512];
        std::snprintf(msg, sizeof(msg), "lb_batch_init: mean initial density: %s", cudaGetErrorString(e));
        return bail(LB_ECUDA, msg);
      }
    }
  }
  std::vector<LatCoef<f2>> h_coef(n);
  size_t off = 0, total_nodes = 0;
  for (int i = 0; i < n; ++i) {
    char err[512] = {0};
    if (ps[i].precision != LB_FP32) return bail(LB_ENOTSUP, "lb_batch_init: the batched solver stores FP32");
    if (ps[i].layout != ps[0].layout)
      return bail(LB_ENOTSUP, "lb_batch_init: the lattices of one batch share the layout");
    if (derive(&ps[i], &b->d[i], err, sizeof(err)) != LB_OK) {
      char m[600];
      std::snprintf(m, sizeof(m), "lattice %d: %s", i, err);
      return bail(LB_EINVAL, m);
    }
    b->p[i].rho_ref = double(float(std::isnan(ps[i].rho_ref) ? mean[i] : ps[i].rho_ref));
    const VCoef<f2> full = make_vcoef<f2>(b->p[i], b->d[i]);
    if (i == 0) b->common = full;
    // Everything but the per-lattice part must agree across the batch.
    const lb_derived& d0 = b->d[0];
    const lb_derived& di = b->d[i];
    if (ps[i].eos != ps[0].eos || ps[i].eos_a != ps[0].eos_a || ps[i].eos_b != ps[0].eos_b || di.k != d0.k ||
        di.s_e != d0.s_e || di.s_eps != d0.s_eps || di.s_q != d0.s_q || di.s_p != d0.s_p)
      return bail(LB_ENOTSUP,
                  "lb_batch_init: lattices of one batch must share the EOS (kind, a, b), varpi and the relaxation rates");
    h_coef[i] = LatCoef<f2>{full.G2,        full.rho_ref, full.m2rr, full.lam_RT, full.neg_lam_a,
                            full.neg_2lam_a, full.g15,     full.Q1G2, full.Q2G2,   full.Q78G2};
    for (int s = 0; s < kTileLists; ++s) {
      BatchLattice L;
      L.nx = ps[i].nx;
      L.ny = ps[i].ny;
      L.sx = row_stride(ps[i].nx);
      L.offset = (long long)off;
      L.tiles_x = (ps[i].nx + kTileX - 1) / kTileX;
      L.tile_start = 0;
      b->desc[s].push_back(L);
    }
    off += lattice_elems(ps[i]);
    total_nodes += size_t(ps[i].nx) * ps[i].ny;
  }
  for (int s = 0; s < kTileLists; ++s) {
    int start = 0;
    for (int i = 0; i < n; ++i) {
      b->desc[s][i].tile_start = start;
      start += b->desc[s][i].tiles_x * ((ps[i].ny + kShapeTY[s] - 1) / kShapeTY[s]);
    }
    b->total_tiles[s] = start;
  }
  for (int s = kShapeTMA; s < kShapes; ++s) b->total_tiles[s] = b->total_tiles[0];
  // Metadata in the caller's buffer: descriptors and tile records per tile list,
  // coefficients, tensor maps, the wait-error word, each 256-byte aligned.
  auto align = [](uintptr_t v) { return (v + 255) / 256 * 256; };
  std::vector<TileRec> h_tiles[kTileLists];
  for (int s = 0; s < kTileLists; ++s) {
    h_tiles[s].reserve(b->total_tiles[s]);
    for (int i = 0; i < n; ++i) {
      const BatchLattice& L = b->desc[s][i];
      const Strides st = lat_strides(L.sx, L.ny, b->rows);
      const int tyn = (ps[i].ny + kShapeTY[s] - 1) / kShapeTY[s];
      for (int r = 0; r < tyn; ++r)
        for (int q = 0; q < L.tiles_x; ++q)
          h_tiles[s].push_back(TileRec{i, q * kTileX, r * kShapeTY[s], L.nx, L.ny, st.ps, st.rs,
                                       tile_kind(q * kTileX, r * kShapeTY[s], L.nx, L.ny), L.offset});
    }
  }
  uintptr_t m = align(reinterpret_cast<uintptr_t>(meta));
  for (int s = 0; s < kTileLists; ++s) {
    b->d_desc[s] = reinterpret_cast<BatchLattice*>(m);
    m = align(m + n * sizeof(BatchLattice));
    b->d_tiles[s] = reinterpret_cast<TileRec*>(m);
    m = align(m + h_tiles[s].size() * sizeof(TileRec));
  }
  for (int s = kShapeTMA; s < kShapes; ++s) {
    b->d_desc[s] = b->d_desc[0];
    b->d_tiles[s] = b->d_tiles[0];
  }
  b->d_coef = reinterpret_cast<LatCoef<f2>*>(m);
  m = align(m + n * sizeof(LatCoef<f2>));
  b->d_maps = reinterpret_cast<CUtensorMap*>(m);
  m = align(m + 2 * size_t(n) * sizeof(CUtensorMap));
  b->d_err = reinterpret_cast<int*>(m);
  m = align(m + sizeof(int));
  b->d_queue = reinterpret_cast<unsigned*>(m);
  m = align(m + 2 * sizeof(unsigned));
  b->d_bad = reinterpret_cast<unsigned*>(m);
  b->h_bad.assign(size_t(n), 0u);
  // Tensor maps of every lattice in both pools.  A lattice below 40 x 18 has no
  // interior tile (those need nx >= 68, ny >= 34) and keeps a zero map it never uses.
  std::vector<CUtensorMap> h_maps(2 * size_t(n));
  std::memset(h_maps.data(), 0, h_maps.size() * sizeof(CUtensorMap));
  b->tma_ok = true;
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < n; ++i) {
      const BatchLattice& L = b->desc[0][i];
      if (L.nx < kTmaCols || L.ny < kTmaRows) continue;
      float* base = static_cast<float*>(side ? pool_b : pool_a) + L.offset;
      if (!encode_population_map(&h_maps[side * size_t(n) + i], base, L.nx, L.ny, L.sx, 4, b->rows != 0))
        b->tma_ok = false;
    }
  cudaError_t e = cudaSuccess;
  e = cudaMemcpyAsync(b->d_maps, h_maps.data(), h_maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                      b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(unsigned), b->stream);
  // The ticket shapes hold two window buffers (above the 48 KB default).
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_step_batch_tma_dyn<3>),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(Win2<float>::smem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_step_batch_tma_dyn<2>),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(Win2<float>::smem));
  for (int s = 0; s < kTileLists && e == cudaSuccess; ++s) {
    e = cudaMemcpyAsync(b->d_desc[s], b->desc[s].data(), n * sizeof(BatchLattice), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_tiles[s], h_tiles[s].data(), h_tiles[s].size() * sizeof(TileRec),
                          cudaMemcpyHostToDevice, b->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_coef, h_coef.data(), n * sizeof(LatCoef<f2>), cudaMemcpyHostToDevice, b->stream);
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  // Initial state: rest equilibrium of each lattice's density (host path staged in pool_b).
  const double* rd = staged ? static_cast<const double*>(pool_b) : rho0;
  if (e == cudaSuccess && !rho0_on_device && !staged) {
    e = cudaMemcpyAsync(pool_b, rho0, total_nodes * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    rd = static_cast<const double*>(pool_b);
  }
  size_t node_off = 0;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const size_t N = size_t(ps[i].nx) * ps[i].ny;
    // FP32 arithmetic with the coefficients a single lattice of the same parameters
    // gets (b->p holds the storage shift rounded to float, as lb_init does), so that
    // every lattice starts bit-identical to its single-lattice run.
    k_init_rest<float, float><<<unsigned((N + 255) / 256), 256, 0, b->stream>>>(
        rd + node_off, static_cast<float*>(pool_a) + b->desc[0][i].offset, ps[i].nx, ps[i].ny,
        lat_strides(b->desc[0][i].sx, ps[i].ny, b->rows), make_vcoef<float>(b->p[i], b->d[i]), nullptr, 0.0);
    e = cudaGetLastError();
    node_off += N;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    char msg[512];
    std::snprintf(msg, sizeof(msg), "lb_batch_init: %s", cudaGetErrorString(e));
    return bail(LB_ECUDA, msg);
  }
  b->shape = 0;
  int mb = 1;
  if (max_blocks(b, 0, &mb) != LB_OK) return bail(LB_ECUDA, b->err);
  b->blocks_per_sm = mb;
  b->steps = 0;
  *out = b;
  return LB_OK;
}

int lb_batch_run(lb_batch* b, int64_t nsteps) {
  if (!b) return LB_EINVAL;
  if (nsteps < 0) return berr(b, LB_EINVAL, "nsteps must be >= 0%s");
  // The legacy default stream cannot be captured, and a stream that the caller is
  // capturing records plain launches in its own graph: plain launches there.
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  if (b->stream != nullptr && cudaStreamIsCapturing(b->stream, &capture) != cudaSuccess) {
    cudaGetLastError();
    capture = cudaStreamCaptureStatusActive;
  }
  while (b->stream != nullptr && capture == cudaStreamCaptureStatusNone && nsteps >= kGraphSteps) {
    const int rc = ensure_graph(b, b->cur);
    if (rc != LB_OK) return rc;
    const cudaError_t e = cudaGraphLaunch(b->graph[b->cur], b->stream);
    if (e != cudaSuccess) return berr(b, LB_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    nsteps -= kGraphSteps;
    b->steps += kGraphSteps;
  }
  for (; nsteps > 0; --nsteps) {
    launch_one(b, b->cur);
    b->cur = 1 - b->cur;
    ++b->steps;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return berr(b, LB_ECUDA, "batch step: %s", cudaGetErrorString(e));
  return LB_OK;
}

int lb_batch_tune(lb_batch* b, int trial_steps, double* best_ms_per_step) {
  if (!b || trial_steps < 1) return LB_EINVAL;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return berr(b, LB_ECUDA, "cudaEventCreate%s");
  float best = 1e30f;
  int best_shape = b->shape, best_bps = b->blocks_per_sm;
  int64_t tuned_steps = 0;
  for (int s = 0; s < kShapes; ++s) {
    if (is_tma(s) && !b->tma_ok) continue;
    int mb = 1;
    if (max_blocks(b, s, &mb) != LB_OK) return LB_ECUDA;
    for (int bps = is_tma(s) ? 1 : 0; bps <= mb; ++bps) {  // the tensor-copy kernel is persistent only
      b->shape = s;
      b->blocks_per_sm = bps;
      launch_one(b, b->cur);  // warm-up (two launches keep the pool parity)
      launch_one(b, 1 - b->cur);
      cudaEventRecord(e0, b->stream);
      for (int k = 0; k < 2 * ((trial_steps + 1) / 2); ++k) launch_one(b, (b->cur + k) & 1);
      tuned_steps += 2 + 2 * ((trial_steps + 1) / 2);
      cudaEventRecord(e1, b->stream);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return berr(b, LB_ECUDA, "autotune: %s", cudaGetErrorString(e));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= float(2 * ((trial_steps + 1) / 2));
      if (ms < best) {
        best = ms;
        best_shape = s;
        best_bps = bps;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->shape = best_shape;
  b->blocks_per_sm = best_bps;
  if (best_ms_per_step) *best_ms_per_step = best;
  // The trial launches advance every lattice by an even number of steps (the
  // pools end where they started); the state stays a valid trajectory.
  b->steps += tuned_steps;
  return LB_OK;
}

int lb_batch_config(const lb_batch* b, int* tile_y, int* blocks_per_sm, int* grid) {
  if (!b) return LB_EINVAL;
  if (tile_y) *tile_y = kShapeTY[b->shape];
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  if (grid) *grid = b->blocks_per_sm > 0 ? b->blocks_per_sm * b->sms : b->total_tiles[b->shape];
  return LB_OK;
}

int lb_batch_set_config(lb_batch* b, int shape, int blocks_per_sm) {
  if (!b) return LB_EINVAL;
  if (shape < 0 || shape >= kShapes) return berr(b, LB_EINVAL, "lb_batch_set_config: shape out of range%s");
  if (is_tma(shape) && !b->tma_ok)
    return berr(b, LB_ENOTSUP, "lb_batch_set_config: a lattice of the batch has no tensor map%s");
  int mb = 1;
  if (max_blocks(b, shape, &mb) != LB_OK) return LB_ECUDA;
  if (blocks_per_sm < (is_tma(shape) ? 1 : 0) || blocks_per_sm > mb)
    return berr(b, LB_EINVAL, "lb_batch_set_config: blocks_per_sm out of range for the shape%s");
  b->shape = shape;
  b->blocks_per_sm = blocks_per_sm;
  return LB_OK;
}

int lb_batch_uses_tma(const lb_batch* b) { return b && is_tma(b->shape) ? 1 : 0; }

}  // extern "C"

namespace {

// Counts the non-finite densities of every lattice of the current state into
// b->h_bad (synchronous); returns the number of lattices with any, or an error.
int count_nonfinite(lb_batch* b) {
  cudaError_t e = cudaMemsetAsync(b->d_bad, 0, size_t(b->n) * sizeof(unsigned), b->stream);
  if (e == cudaSuccess && b->total_tiles[0] > 0) {
    k_batch_nonfinite<<<unsigned(b->total_tiles[0]), kFusedThreads, 0, b->stream>>>(
        static_cast<const float*>(b->pool[b->cur]), b->d_tiles[0], b->rows, b->d_bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_bad.data(), b->d_bad, size_t(b->n) * sizeof(unsigned), cudaMemcpyDeviceToHost,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return berr(b, LB_ECUDA, "non-finite check: %s", cudaGetErrorString(e));
  int lattices = 0;
  for (unsigned v : b->h_bad) lattices += v ? 1 : 0;
  return lattices;
}

}  // namespace

extern "C" {

int lb_batch_status(lb_batch* b) {
  if (!b) return LB_EINVAL;
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess && v) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
  if (e != cudaSuccess) return berr(b, LB_ECUDA, "lb_batch_status: %s", cudaGetErrorString(e));
  if (v) return berr(b, LB_ETIMEOUT, "a bounded wait for a tensor copy gave up%s");
  const int bad = count_nonfinite(b);
  if (bad < 0) return bad;
  if (bad > 0) {
    char list[256] = {0};
    size_t used = 0;
    int shown = 0;
    for (int i = 0; i < b->n && shown < 16; ++i)
      if (b->h_bad[i]) {
        used += size_t(std::snprintf(list + used, sizeof(list) - used, "%s%d", shown ? ", " : "", i));
        ++shown;
        if (used >= sizeof(list)) break;
      }
    std::snprintf(b->err, sizeof(b->err), "%d lattice(s) have non-finite densities: %s%s", bad, list,
                  bad > shown ? ", ..." : "");
    return LB_ENONFINITE;
  }
  return LB_OK;
}

int lb_batch_nonfinite(lb_batch* b, uint32_t* counts) {
  if (!b) return LB_EINVAL;
  const int bad = count_nonfinite(b);
  if (bad < 0) return bad;
  if (counts) std::memcpy(counts, b->h_bad.data(), size_t(b->n) * sizeof(uint32_t));
  return bad;
}

void* lb_batch_state(lb_batch* b) { return b ? b->pool[b->cur] : nullptr; }

int64_t lb_batch_steps_done(const lb_batch* b) { return b ? b->steps : -1; }

int64_t lb_batch_offset(const lb_batch* b, int i) {
  if (!b || i < 0 || i >= b->n) return -1;
  return b->desc[0][i].offset;
}

int lb_batch_row_stride(const lb_batch* b, int i) {
  if (!b || i < 0 || i >= b->n) return -1;
  return b->desc[0][i].sx;
}

int lb_batch_density(lb_batch* b, int i, void* rho) {
  if (!b || i < 0 || i >= b->n || !rho) return LB_EINVAL;
  const BatchLattice& L = b->desc[0][i];
  const size_t N = size_t(L.nx) * L.ny;
  k_rho_local<float, float><<<unsigned((N + 255) / 256), 256, 0, b->stream>>>(
      static_cast<const float*>(b->pool[b->cur]) + L.offset, static_cast<float*>(rho), L.nx, L.ny,
      lat_strides(L.sx, L.ny, b->rows), float(b->p[i].rho_ref));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return berr(b, LB_ECUDA, "lb_batch_density: %s", cudaGetErrorString(e));
  return LB_OK;
}

int lb_batch_derived(const lb_batch* b, int i, lb_derived* out) {
  if (!b || i < 0 || i >= b->n || !out) return LB_EINVAL;
  *out = b->d[i];
  return LB_OK;
}

int lb_batch_params(const lb_batch* b, int i, lb_params* out) {
  if (!b || i < 0 || i >= b->n || !out) return LB_EINVAL;
  *out = b->p[i];
  return LB_OK;
}

const char* lb_batch_last_error(const lb_batch* b) { return b ? b->err : thread_error(); }

void lb_batch_free(lb_batch* b) {
  if (!b) return;
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
  delete b;
}

}  // extern "C"
