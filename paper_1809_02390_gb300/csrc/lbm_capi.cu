// C ABI of the library: handles, parameter checking, launches.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "lbm_handle.cuh"
#include "lbm_fields.cuh"
#include "lbm_tma.cuh"

namespace lbm {

template <typename V>
V bc(double x);
template <>
double bc<double>(double x) {
  return x;
}
template <>
float bc<float>(double x) {
  return float(x);
}
template <>
f2 bc<f2>(double x) {
  return f2{make_float2(float(x), float(x))};
}

// Collision constants (FP64 on the host, then rounded to V).
template <typename V>
VCoef<V> make_vcoef(const lb_params& p, const lb_derived& d) {
  VCoef<V> c;
  const double w = 1.0 - d.k;  // varpi
  const double k = d.k, h = d.h, b = d.b;
  const double se = d.s_e, seps = d.s_eps, sq = d.s_q, sp = d.s_p;
  const double lam = d.lam, RT = p.R_gas * d.T, a = p.eos_a;
  const double bq = p.eos == LB_EOS_VDW ? p.eos_b : p.eos_b / 4.0;
  c.eos = p.eos;
  c.G2 = bc<V>(d.G2);
  c.rho_ref = bc<V>(p.rho_ref);
  c.neg_bq = bc<V>(-bq);
  c.bq = bc<V>(bq);
  c.RT = bc<V>(RT);
  c.lam_RT = bc<V>(lam * RT);
  c.neg_lam_a = bc<V>(-lam * a);
  c.neg_2lam_a = bc<V>(-2.0 * lam * a);
  c.lam = bc<V>(lam);
  c.a = bc<V>(a);
  c.beta2 = bc<V>(d.beta2);
  // Step (2) and (3) of the execution sequence.
  c.hk_seps = bc<V>(0.5 * k * seps);
  c.hh_sq = bc<V>(0.5 * h * sq);
  c.b_sq = bc<V>(b * sq);
  c.hb_sq = bc<V>(0.5 * b * sq);
  c.om_e = bc<V>(1.0 - 0.5 * se);
  c.om_eps = bc<V>(1.0 - 0.5 * seps);
  c.om_q = bc<V>(1.0 - 0.5 * sq);
  c.om_p = bc<V>(1.0 - 0.5 * sp);
  // Step (4): supplement Eqs. 34, 37, 40.
  c.R11 = bc<V>(-se / (4.0 * w) * (9.0 * (1.0 - k) - 2.0 * (3.0 * k + h)));
  c.R17 = bc<V>(-3.0 * sp * (2.0 - se) / (4.0 * (2.0 - sp)) * (9.0 * (1.0 - k) + 2.0 * (3.0 * k + h)));
  c.R18 = bc<V>(12.0 * sp * (2.0 - se) / (2.0 - sp) * (3.0 * k + h));
  c.R71 = bc<V>(-se * (2.0 - sp) / (4.0 * w * (2.0 - se)) * (3.0 - 4.0 * b));
  c.R77 = bc<V>(-3.0 * sp / 4.0 * (3.0 + 4.0 * b));
  c.R81 = bc<V>(se * (2.0 - sp) / (w * (2.0 - se)) * b);
  c.R88 = bc<V>(6.0 * sp * b);
  c.T1a = bc<V>(3.0 * (2.0 - se) / 2.0 * (1.0 - k));
  c.negT1b = bc<V>(-3.0 * (2.0 - se) / 2.0 * (2.0 * k + h));
  c.X1 = bc<V>(9.0 * (2.0 - se) / 2.0 * (2.0 * k + h));
  c.T7 = bc<V>((2.0 - sp) / 2.0);
  c.T7b = bc<V>((2.0 - sp) * b);
  c.X7 = bc<V>(-3.0 * (2.0 - sp) * b);
  c.T8 = bc<V>(-(2.0 - sp) * b / 2.0);
  c.X8 = bc<V>(3.0 * (2.0 - sp) * b / 2.0);
  // Step (6): s_e Q1 + k (s_e/2 - 1) s_eps Q2 with Q1 = -Q2 = G^2 |S|^2 / 2; s_p Q7, s_p Q8.
  c.Q1G2 = bc<V>(0.5 * (se - k * (0.5 * se - 1.0) * seps) * d.G2);
  c.Q2G2 = bc<V>(-0.5 * seps * d.G2);
  c.Q78G2 = bc<V>(sp / 12.0 * d.G2);
  c.Q1 = bc<V>(0.5 * (se - k * (0.5 * se - 1.0) * seps));
  c.Q2 = bc<V>(-0.5 * seps);
  c.Q78 = bc<V>(sp / 12.0);
  c.neg_a = bc<V>(-a);
  c.h15 = bc<V>(1.5);
  c.m3 = bc<V>(-3.0);
  c.mhalf = bc<V>(-0.5);
  c.two_om_eps = bc<V>(2.0 - seps);
  c.two_om_q = bc<V>(2.0 - sq);
  c.eight = bc<V>(8.0);
  c.twenty = bc<V>(20.0);
  c.third = bc<V>(1.0 / 3.0);
  c.twelfth = bc<V>(1.0 / 12.0);
  c.one = bc<V>(1.0);
  c.mone = bc<V>(-1.0);
  c.two = bc<V>(2.0);
  c.three = bc<V>(3.0);
  c.four = bc<V>(4.0);
  c.six = bc<V>(6.0);
  c.m6 = bc<V>(-6.0);
  c.nine = bc<V>(9.0);
  c.eighteen = bc<V>(18.0);
  c.half = bc<V>(0.5);
  c.m2 = bc<V>(-2.0);
  c.m4 = bc<V>(-4.0);
  c.m2rr = bc<V>(-2.0 * p.rho_ref);
  c.g15 = bc<V>(1.5 * d.G2);
  c.ninth = bc<V>(1.0 / 9.0);
  c.i36 = bc<V>(1.0 / 36.0);
  c.sixth = bc<V>(1.0 / 6.0);
  c.i12 = bc<V>(1.0 / 12.0);
  c.quarter = bc<V>(0.25);
  return c;
}

template VCoef<float> make_vcoef<float>(const lb_params&, const lb_derived&);
template VCoef<f2> make_vcoef<f2>(const lb_params&, const lb_derived&);
template VCoef<double> make_vcoef<double>(const lb_params&, const lb_derived&);

}  // namespace lbm

using namespace lbm;

namespace {

int fail(lb_handle* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h)
    std::snprintf(h->err, sizeof(h->err), "%s", buf);
  else
    set_thread_error(buf);
  return code;
}

#define LB_CUDA(h, call)                                                                     \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail((h), LB_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t elem_bytes(int precision) { return precision == LB_FP64 ? 8 : precision == LB_FP32 ? 4 : 2; }
size_t real_bytes(int precision) { return precision == LB_FP64 ? 8 : 4; }

size_t rho_plane_bytes(const lb_params* p) {
  return (size_t(p->nx) * p->ny * real_bytes(p->precision) + 255) / 256 * 256;
}

size_t reduce_bytes() { return size_t(kMaxReduceBlocks) * kReduceSlots * sizeof(double) + 256; }
constexpr size_t kQueueBytes = 256;  // tile tickets of the dynamic tensor-copy step

template <typename V, typename real, typename store_t>
void launch_step(lb_handle* h, const VCoef<V>& cv, const VCoef<real>& c) {
  const store_t* fin = static_cast<const store_t*>(h->f[h->cur]);
  store_t* fout = static_cast<store_t*>(h->f[1 - h->cur]);
  const int nx = h->p.nx, ny = h->p.ny;
  // FP16 stores: a fresh dither sequence every step (seed from the step count; a
  // launch captured into a graph reads the count from the handle's step word).
  Rounding rnd{step_seed(unsigned(h->steps)), h->p.rounding == LB_ROUND_STOCHASTIC, nullptr, 0};
  if (h->graph_k >= 0) {
    rnd.step = h->step_word;
    rnd.k = h->graph_k;
  }
  if (h->variant == LB_FUSED) {
    const dim3 grd((nx + kTileX - 1) / kTileX, (ny + kTileY - 1) / kTileY);
    if constexpr (sizeof(store_t) <= 4 && std::is_same<V, f2>::value) {
      if (h->use_tma && h->use_dyn) {
        k_step_tma_dyn<V, store_t><<<h->dyn_grid, kFusedThreads, Win2<store_t>::smem, h->stream>>>(
            h->tmap[h->cur], fin, fout, nx, ny, h->st, cv, h->wait_error, rnd, h->queue);
        return;
      }
      if (h->use_tma) {
        k_step_tma<V, store_t, false><<<h->tma_grid, kFusedThreads, Win<store_t>::smem, h->stream>>>(
            h->tmap[h->cur], fin, fout, nx, ny, h->st, cv, h->wait_error, rnd);
        return;
      }
    }
    k_step_fused<V, store_t><<<grd, kFusedThreads, 0, h->stream>>>(fin, fout, nx, ny, h->st, cv, rnd);
  } else {
    real* rho = static_cast<real*>(h->scratch);
    const dim3 blk(32, 8), grd((nx + 31) / 32, (ny + 7) / 8);
    k_density<real, store_t><<<grd, blk, 0, h->stream>>>(fin, rho, nx, ny, h->st);
    k_collide_rho<real, store_t><<<grd, blk, 0, h->stream>>>(fin, fout, rho, nx, ny, h->st, c, rnd);
  }
}

int configure_device(lb_handle* h) {
  int dev = 0, sms = 0;
  LB_CUDA(h, cudaGetDevice(&dev));
  LB_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  h->reduce_blocks = sms * 2 < kMaxReduceBlocks ? sms * 2 : kMaxReduceBlocks;
  return LB_OK;
}

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

namespace lbm {

cudaError_t device_mean(const double* x, size_t n, void* work, size_t work_bytes, cudaStream_t stream, double* mean) {
  size_t blocks = (n + 8 * kReduceThreads - 1) / (8 * kReduceThreads);
  if (blocks > size_t(kMaxReduceBlocks)) blocks = kMaxReduceBlocks;
  if (blocks > work_bytes / sizeof(double)) blocks = work_bytes / sizeof(double);
  if (blocks < 1) blocks = 1;
  double* partial = static_cast<double*>(work);
  k_sum_partial<<<unsigned(blocks), kReduceThreads, 0, stream>>>(x, (long long)n, partial);
  cudaError_t e = cudaGetLastError();
  std::vector<double> h(blocks);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), partial, blocks * sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return e;
  double sum = 0.0;
  for (double v : h) sum += v;
  *mean = sum / double(n);
  return cudaSuccess;
}

// 3-D map of one FP32 (elem_bytes 4) or FP16 (2) population buffer: x (nx), y (ny,
// row stride sx), plane (9); box of one plane window (40 x 18 floats or 48 x 18
// halves).  Rows layout: x (nx), plane (9, stride sx), y (ny, stride 9 sx), box
// (cols, 1, 18), which lands in shared memory as the same 18 x cols window.  False
// if the layout does not allow it (base not 16-byte aligned, row stride not a
// multiple of 16 bytes).
static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return nullptr;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool encode_population_map(CUtensorMap* map, void* base, int nx, int ny, int sx, int elem_bytes, bool rows) {
  const EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if (elem_bytes != 4 && elem_bytes != 2) return false;
  const size_t eb = size_t(elem_bytes);
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || (size_t(sx) * eb) % 16 != 0 || sx < nx) return false;
  const int cols = elem_bytes == 4 ? Win<float>::cols : Win<__half>::cols;
  if (nx < cols || ny < kTmaRows) return false;
  const cuuint64_t dims[3] = {cuuint64_t(nx), cuuint64_t(rows ? 9 : ny), cuuint64_t(rows ? ny : 9)};
  const cuuint64_t strides[2] = {cuuint64_t(sx) * eb, cuuint64_t(sx) * (rows ? 9 : ny) * eb};
  const cuuint32_t box[3] = {cuuint32_t(cols), rows ? 1u : cuuint32_t(kTmaRows), rows ? cuuint32_t(kTmaRows) : 1u};
  const cuuint32_t estride[3] = {1, 1, 1};
  const CUtensorMapDataType dt = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  return fn(map, dt, 3, base, dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D map (x, y, plane) of `planes` FP32 planes of nx x ny (row stride nx), box
// of cols x rows x 1: one copy delivers a window of one plane.
bool encode_plane_map(CUtensorMap* map, const void* base, int nx, int ny, int planes, int cols, int rows) {
  const EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || (size_t(nx) * 4) % 16 != 0 || nx < cols || ny < rows)
    return false;
  const cuuint64_t dims[3] = {cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(planes)};
  const cuuint64_t strides[2] = {cuuint64_t(nx) * 4, cuuint64_t(nx) * ny * 4};
  const cuuint32_t box[3] = {cuuint32_t(cols), cuuint32_t(rows), 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace lbm

namespace {

// One word per live handle, set by a bounded wait of that handle's tensor-copy
// step or adjoint that gave up (read and cleared by lb_status on the handle).
// Slots are handed out by lb_init and returned by lb_free; the same slot index
// serves the handle on whichever device it lives (each device has its own array).
constexpr int kWaitSlots = 4096;
__device__ int g_wait_flags[kWaitSlots];
// Per handle slot: the step count that the FP16 steps of a replayed graph seed from.
__device__ unsigned g_step_words[kWaitSlots];

__global__ void k_set_word(unsigned* w, unsigned v) { *w = v; }
std::mutex g_slot_mu;
bool g_slot_used[kWaitSlots] = {false};

int take_wait_slot() {
  std::lock_guard<std::mutex> lock(g_slot_mu);
  for (int i = 0; i < kWaitSlots; ++i)
    if (!g_slot_used[i]) {
      g_slot_used[i] = true;
      return i;
    }
  return -1;
}

void release_wait_slot(lb_handle* h) {
  if (!h || h->wait_slot < 0) return;
  std::lock_guard<std::mutex> lock(g_slot_mu);
  g_slot_used[h->wait_slot] = false;
  h->wait_slot = -1;
}

void destroy(lb_handle* h) {
  if (!h) return;
  release_wait_slot(h);
  for (int k = 0; k < 2; ++k) {
    if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    if (h->gev[k]) cudaEventDestroy(h->gev[k]);
  }
  if (h->gstream) cudaStreamDestroy(h->gstream);
  delete h;
}

// The step's memory traffic without its arithmetic: one block per 32 x 16 tile
// (the step's tiles), each thread moving the nine populations of its two nodes
// (rows ty and ty + 8) to the same places of the other buffer, in the handle's
// layout.  With one block per tile the hardware hands tiles out in order as
// blocks finish and eight blocks per SM keep 147 KB of loads in flight: of the
// forms of this copy measured (grid-stride loops over nodes with 4-, 8- and
// 16-byte accesses, persistent tile walks), this one moves the most bytes, so its
// bandwidth is the ceiling quoted for the step's access pattern.
template <typename T>
__global__ void __launch_bounds__(256) k_stream_tiles(const T* __restrict__ in, T* __restrict__ out, int nx, int ny,
                                                      Strides st) {
  const int tiles_x = (nx + kTileX - 1) / kTileX;
  const int x = (blockIdx.x % tiles_x) * kTileX + (threadIdx.x & (kTileX - 1));
  const int y0 = (blockIdx.x / tiles_x) * kTileY + threadIdx.x / kTileX;
  if (x >= nx) return;
  T v[kTileRows][9];
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int y = y0 + k * kRowStride;
    if (y < ny) {
#pragma unroll
      for (int i = 0; i < 9; ++i) v[k][i] = in[st.at(i, x, y)];
    }
  }
#pragma unroll
  for (int k = 0; k < kTileRows; ++k) {
    const int y = y0 + k * kRowStride;
    if (y < ny) {
#pragma unroll
      for (int i = 0; i < 9; ++i) out[st.at(i, x, y)] = v[k][i];
    }
  }
}

template <typename T>
void launch_stream_copy(const lb_handle* h, const void* in, void* out) {
  const unsigned tiles = unsigned(((h->p.nx + kTileX - 1) / kTileX) * ((h->p.ny + kTileY - 1) / kTileY));
  k_stream_tiles<<<tiles, kFusedThreads, 0, h->stream>>>(static_cast<const T*>(in), static_cast<T*>(out), h->p.nx,
                                                         h->p.ny, h->st);
}

// A bounded wait that cannot succeed: the mbarrier's single arrival comes with 16
// expected bytes that no copy delivers, so its phase never completes.  Every thread
// polls it `polls` times, the block agrees through the barrier that the wait gave
// up, and thread 0 reports it the way the step kernels do.  No copy is in flight.
__global__ void k_wait_selftest(long long polls, int* __restrict__ err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, 16);
  }
  __syncthreads();
  const bool done = mbar_wait(&bar, 0, polls);
  if (__syncthreads_or(!done) && threadIdx.x == 0) atomicExch(err, 1);
}

int configure(lb_handle* h) {
  int rc = configure_device(h);
  if (rc != LB_OK) return rc;
  // This handle's wait word (cleared: a slot may come from a freed handle).
  h->wait_slot = take_wait_slot();
  if (h->wait_slot < 0) return fail(h, LB_ENOMEM, "more than %d live handles", kWaitSlots);
  void* w = nullptr;
  LB_CUDA(h, cudaGetSymbolAddress(&w, g_wait_flags));
  h->wait_error = static_cast<int*>(w) + h->wait_slot;
  LB_CUDA(h, cudaMemsetAsync(h->wait_error, 0, sizeof(int), h->stream));
  LB_CUDA(h, cudaGetSymbolAddress(&w, g_step_words));
  h->step_word = static_cast<unsigned*>(w) + h->wait_slot;
  // lb_reduce_static's array is committed now, while the caller can still spare
  // the memory, rather than at its first call.
  void* st = nullptr;
  rc = static_scratch_address(h, &st);
  if (rc != LB_OK) return rc;
  // The tensor-copy path needs FP32 or FP16 storage, rows of a multiple of 16
  // bytes and a lattice holding at least one interior tile; otherwise the plain
  // fused kernel runs.
  const bool fp32 = h->p.precision == LB_FP32, fp16 = h->p.precision == LB_FP16S;
  const bool rows = h->p.layout == LB_LAYOUT_ROWS;
  const int eb = fp32 ? 4 : 2, cols = fp32 ? Win<float>::cols : Win<__half>::cols;
  h->use_tma = (fp32 || fp16) && h->variant == LB_FUSED && (h->p.nx * eb) % 16 == 0 &&
               h->p.nx >= 2 * kTileX + cols && h->p.ny >= 2 * kTileY + kTmaRows &&
               encode_population_map(&h->tmap[0], h->f[0], h->p.nx, h->p.ny, h->p.nx, eb, rows) &&
               encode_population_map(&h->tmap[1], h->f[1], h->p.nx, h->p.ny, h->p.nx, eb, rows);
  if (h->use_tma) {
    // Persistent grid: as many blocks as can be resident.
    const void* k = fp32 ? reinterpret_cast<const void*>(k_step_tma<f2, float, false>)
                         : reinterpret_cast<const void*>(k_step_tma<f2, __half, false>);
    const int smem = int(fp32 ? Win<float>::smem : Win<__half>::smem);
    LB_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0, dev = 0, sms = 0;
    LB_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFusedThreads, smem));
    LB_CUDA(h, cudaGetDevice(&dev));
    LB_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int tiles = ((h->p.nx + kTileX - 1) / kTileX) * ((h->p.ny + kTileY - 1) / kTileY);
    h->tma_grid_auto = per_sm < 1 ? sms : per_sm * sms;
    if (h->tma_grid_auto > tiles) h->tma_grid_auto = tiles;
    h->tma_grid = h->tma_grid_auto;
  }
  // Dynamic tile dispatch: needs the ticket words at the end of the scratch buffer.
  h->use_dyn = false;
  h->queue = h->scratch ? reinterpret_cast<unsigned*>(static_cast<char*>(h->scratch) + rho_plane_bytes(&h->p) +
                                                      reduce_bytes())
                        : nullptr;
  if (h->use_tma && h->queue) {
    const void* k = fp32 ? reinterpret_cast<const void*>(k_step_tma_dyn<f2, float>)
                         : reinterpret_cast<const void*>(k_step_tma_dyn<f2, __half>);
    const int smem = int(fp32 ? Win2<float>::smem : Win2<__half>::smem);
    LB_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0, dev = 0, sms = 0;
    LB_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFusedThreads, smem));
    LB_CUDA(h, cudaGetDevice(&dev));
    LB_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int tiles = ((h->p.nx + kTileX - 1) / kTileX) * ((h->p.ny + kTileY - 1) / kTileY);
    h->dyn_grid_auto = per_sm < 1 ? sms : per_sm * sms;
    if (h->dyn_grid_auto > tiles) h->dyn_grid_auto = tiles;
    h->dyn_grid = h->dyn_grid_auto;
    LB_CUDA(h, cudaMemsetAsync(h->queue, 0, 2 * sizeof(unsigned), h->stream));
    h->use_dyn = true;
  }
  return LB_OK;
}

template <typename real, typename store_t>
void launch_moments(lb_handle* h, real* rho, real* ux, real* uy, real rho_ref, real G2) {
  const store_t* f = static_cast<const store_t*>(h->f[h->cur]);
  const int nx = h->p.nx, ny = h->p.ny;
  const size_t N = size_t(nx) * ny;
  k_rho_local<real, store_t><<<unsigned((N + 255) / 256), 256, 0, h->stream>>>(f, rho, nx, ny, h->st, rho_ref);
  if (ux || uy) {
    const dim3 blk(32, 8), grd((nx + 31) / 32, (ny + 7) / 8);
    k_velocity<real, store_t><<<grd, blk, 0, h->stream>>>(f, rho, ux, uy, nx, ny, h->st, G2);
  }
}

template <typename real, typename store_t>
int run_reduce(lb_handle* h, double out[8]) {
  const int nx = h->p.nx, ny = h->p.ny;
  const size_t N = size_t(nx) * ny;
  real* rho = static_cast<real*>(h->scratch);
  double* partial = reinterpret_cast<double*>(static_cast<char*>(h->scratch) + rho_plane_bytes(&h->p));
  double* dout = partial + size_t(kMaxReduceBlocks) * kReduceSlots;
  const store_t* f = static_cast<const store_t*>(h->f[h->cur]);
  const real rho_ref = real(h->p.rho_ref);
  k_rho_local<real, store_t><<<unsigned((N + 255) / 256), 256, 0, h->stream>>>(f, rho, nx, ny, h->st, rho_ref);
  const double rho_mid = 0.5 * (h->d.rho_g + h->d.rho_l);
  k_reduce_partial<real, store_t><<<h->reduce_blocks, kReduceThreads, 0, h->stream>>>(
      f, rho, nx, ny, h->st, real(h->d.G2), std::isfinite(rho_mid) ? rho_mid : 1e300, partial);
  k_reduce_final<<<1, 32, 0, h->stream>>>(partial, h->reduce_blocks, dout);
  double res[kReduceSlots];
  real probe[2];
  LB_CUDA(h, cudaGetLastError());
  LB_CUDA(h, cudaMemcpyAsync(res, dout, sizeof(res), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(h, cudaMemcpyAsync(&probe[0], rho + size_t(ny / 2) * nx + nx / 2, sizeof(real), cudaMemcpyDeviceToHost,
                             h->stream));
  LB_CUDA(h, cudaMemcpyAsync(&probe[1], rho, sizeof(real), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(h, cudaStreamSynchronize(h->stream));
  // p_EOS / c^2 at the two probe nodes, FP64 on the host.
  out[0] = res[0];
  out[1] = res[1];
  out[2] = res[2];
  out[3] = p_eos_host(h->cd, double(probe[0]));
  out[4] = p_eos_host(h->cd, double(probe[1]));
  out[5] = res[3];
  out[6] = res[4];
  out[7] = res[5];
  if (res[6] > 0) return fail(h, LB_ENONFINITE, "%.0f nodes have a non-finite density", res[6]);
  return LB_OK;
}

}  // namespace

extern "C" {

int lb_abi_version(void) { return 2; }

int lb_derive(const lb_params* p, lb_derived* out) {
  if (!out) return fail(nullptr, LB_EINVAL, "null output");
  char err[512] = {0};
  const int rc = derive(p, out, err, sizeof(err));
  if (rc != LB_OK) return fail(nullptr, rc, "%s", err);
  return LB_OK;
}

size_t lb_state_bytes(const lb_params* p) {
  if (!p || p->nx < 1 || p->ny < 1) return 0;
  return 9 * size_t(p->nx) * p->ny * elem_bytes(p->precision);
}

size_t lb_scratch_bytes(const lb_params* p) {
  if (!p || p->nx < 1 || p->ny < 1) return 0;
  return rho_plane_bytes(p) + reduce_bytes() + kQueueBytes;
}

int lb_init(lb_handle** out, const lb_params* p, void* f_a, void* f_b, void* scratch, size_t scratch_bytes,
            const double* rho0, int rho0_on_device, void* stream) {
  if (!out) return fail(nullptr, LB_EINVAL, "null handle pointer");
  *out = nullptr;
  lb_derived d;
  char err[512] = {0};
  int rc = derive(p, &d, err, sizeof(err));
  if (rc != LB_OK) return fail(nullptr, rc, "%s", err);
  if (!f_a || !f_b || f_a == f_b) return fail(nullptr, LB_EINVAL, "f_a and f_b must be two distinct device buffers");
  if (!rho0) return fail(nullptr, LB_EINVAL, "null initial density");
  const int variant = p->variant == LB_TWO_PASS ? LB_TWO_PASS : LB_FUSED;
  if (scratch && scratch_bytes < lb_scratch_bytes(p))
    return fail(nullptr, LB_ENOMEM, "scratch of %zu bytes is below the %zu needed", scratch_bytes,
                lb_scratch_bytes(p));
  if (variant == LB_TWO_PASS && !scratch)
    return fail(nullptr, LB_ENOMEM, "the two-pass variant needs %zu bytes of scratch", lb_scratch_bytes(p));
  const size_t N = size_t(p->nx) * p->ny;
  lb_handle* h = new (std::nothrow) lb_handle();
  if (!h) return fail(nullptr, LB_EINVAL, "out of host memory");
  h->p = *p;
  // The FP32 kernels add the shift back in float: store exactly that value.
  if (p->precision != LB_FP64) h->p.rho_ref = double(float(p->rho_ref));
  h->d = d;
  h->f[0] = f_a;
  h->f[1] = f_b;
  h->cur = 0;
  h->scratch = scratch;
  h->scratch_bytes = scratch_bytes;
  h->stream = static_cast<cudaStream_t>(stream);
  h->steps = 0;
  h->variant = variant;
  h->st = p->layout == LB_LAYOUT_ROWS ? rows_strides(p->nx) : planes_strides(p->nx, p->ny);
  h->cf = make_vcoef<float>(h->p, d);
  h->c2 = make_vcoef<f2>(h->p, d);
  h->cd = make_vcoef<double>(h->p, d);
  h->wait_slot = -1;
  h->graph_k = -1;
  rc = configure(h);
  if (rc != LB_OK) {
    set_thread_error(h->err);
    destroy(h);
    return rc;
  }
  const double* rho_dev = rho0;
  auto bail = [&](cudaError_t e, const char* what) {
    fail(nullptr, LB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    destroy(h);
    return LB_ECUDA;
  };
  cudaError_t e;
  // Host densities: staged in the second population buffer (9 x >= 2 bytes per
  // node hold the 8 of the density and, after them, the two words of the check)
  // and checked by the init kernel as it reads them (positive, finite, below 1/b
  // for vdW).
  unsigned long long* bad = nullptr;
  if (!rho0_on_device) {
    bad = reinterpret_cast<unsigned long long*>(static_cast<char*>(f_b) + N * sizeof(double));
    e = cudaMemsetAsync(bad, 0xff, 2 * sizeof(unsigned long long), h->stream);
    if (e != cudaSuccess) return bail(e, "cudaMemsetAsync(check)");
    e = cudaMemcpyAsync(f_b, rho0, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return bail(e, "cudaMemcpyAsync(rho0)");
    rho_dev = static_cast<const double*>(f_b);
  }
  // rho_ref = NaN: the storage shift is the mean initial density (block sums in
  // f_a, which the initial state overwrites next), rounded to float for FP32 and
  // FP16 storage; the coefficients that hold it are made again.
  if (std::isnan(p->rho_ref)) {
    double mean = 0.0;
    e = device_mean(rho_dev, N, f_a, lb_state_bytes(p), h->stream, &mean);
    if (e != cudaSuccess) return bail(e, "mean initial density");
    h->p.rho_ref = p->precision != LB_FP64 ? double(float(mean)) : mean;
    h->cf = make_vcoef<float>(h->p, d);
    h->c2 = make_vcoef<f2>(h->p, d);
    h->cd = make_vcoef<double>(h->p, d);
  }
  const unsigned blocks = unsigned((N + 255) / 256);
  const double vdw_b = p->eos == LB_EOS_VDW ? p->eos_b : 0.0;
  switch (p->precision) {
    case LB_FP64:
      k_init_rest<double, double><<<blocks, 256, 0, h->stream>>>(rho_dev, static_cast<double*>(f_a), p->nx, p->ny,
                                                                  h->st, h->cd, bad, vdw_b);
      break;
    case LB_FP32:
      k_init_rest<float, float><<<blocks, 256, 0, h->stream>>>(rho_dev, static_cast<float*>(f_a), p->nx, p->ny, h->st,
                                                                h->cf, bad, vdw_b);
      break;
    default:
      k_init_rest<__half, float><<<blocks, 256, 0, h->stream>>>(rho_dev, static_cast<__half*>(f_a), p->nx, p->ny,
                                                                 h->st, h->cf, bad, vdw_b);
      break;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return bail(e, "init kernel launch");
  if (!rho0_on_device) {
    unsigned long long first[2] = {0, 0};
    e = cudaMemcpyAsync(first, bad, sizeof(first), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return bail(e, "cudaMemcpyAsync(check)");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bail(e, "cudaStreamSynchronize");
    if (first[0] != ~0ull || first[1] != ~0ull) {
      destroy(h);
      if (first[0] != ~0ull)
        return fail(nullptr, LB_EINVAL, "initial density at node %llu is not positive and finite", first[0]);
      return fail(nullptr, LB_EINVAL, "initial density at node %llu exceeds 1/b of the vdW EOS", first[1]);
    }
  }
  *out = h;
  return LB_OK;
}

}  // extern "C"

namespace {

// Steps per captured graph (even, so a replay ends on the buffer it started from).
constexpr int kStepGraph = 64;

void launch_one_step(lb_handle* h) {
  switch (h->p.precision) {
    case LB_FP64: launch_step<double, double, double>(h, h->cd, h->cd); break;
    case LB_FP32: launch_step<f2, float, float>(h, h->c2, h->cf); break;
    default: launch_step<f2, float, __half>(h, h->c2, h->cf); break;
  }
}

// The launch configuration a graph bakes in: kernel form and grid sizes.
long long step_config(const lb_handle* h) {
  return (long long)h->variant | ((long long)h->use_tma << 2) | ((long long)h->use_dyn << 3) |
         ((long long)h->tma_grid << 4) | ((long long)h->dyn_grid << 34);
}

// Captures (once per starting buffer and configuration) kStepGraph steps into a
// graph on the internal stream.  False, with the handle left as it was, when the
// graph cannot be made (then the steps are launched directly).
bool ensure_step_graph(lb_handle* h) {
  const int from = h->cur;
  const long long cfg = step_config(h);
  if (h->graph[from] && h->graph_cfg[from] == cfg) return true;
  if (h->graph[from]) {
    cudaGraphExecDestroy(h->graph[from]);
    h->graph[from] = nullptr;
  }
  if (!h->gstream) {
    if (cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking) != cudaSuccess) return false;
    for (int k = 0; k < 2; ++k)
      if (cudaEventCreateWithFlags(&h->gev[k], cudaEventDisableTiming) != cudaSuccess) return false;
  }
  cudaStream_t caller = h->stream;
  h->stream = h->gstream;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int s = 0; s < kStepGraph; ++s) {
      h->graph_k = s;
      launch_one_step(h);
      h->cur = 1 - h->cur;
    }
    e = cudaStreamEndCapture(h->gstream, &g);
  }
  h->graph_k = -1;
  h->stream = caller;
  h->cur = from;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph[from], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear a capture error; the direct launches report anything lasting
    h->graph[from] = nullptr;
    return false;
  }
  h->graph_cfg[from] = cfg;
  return true;
}

}  // namespace

extern "C" {

int lb_step(lb_handle* h, int64_t nsteps) {
  if (!h) return fail(nullptr, LB_EINVAL, "null handle");
  if (nsteps < 0) return fail(h, LB_EINVAL, "nsteps must be >= 0");
  // Runs of kStepGraph steps replay a captured graph on the handle's internal
  // stream, ordered after the caller's stream's earlier work and before its later
  // work by two events.  FP16 stores seed from the step count: before each replay
  // a one-thread launch writes it to the handle's step word, which the graph's
  // steps read (step k of the graph adds k).
  // A caller capturing its own stream gets plain launches, which its graph records.
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(h->stream, &capture) != cudaSuccess) {
    cudaGetLastError();
    capture = cudaStreamCaptureStatusActive;  // unknown: take the plain launches
  }
  if (nsteps >= kStepGraph && !h->graph_off && capture == cudaStreamCaptureStatusNone) {
    if (!ensure_step_graph(h)) {
      h->graph_off = true;
    } else {
      LB_CUDA(h, cudaEventRecord(h->gev[0], h->stream));
      LB_CUDA(h, cudaStreamWaitEvent(h->gstream, h->gev[0], 0));
      while (nsteps >= kStepGraph) {
        if (!ensure_step_graph(h)) return fail(h, LB_ECUDA, "step graph capture failed");
        if (h->p.precision == LB_FP16S) {
          k_set_word<<<1, 1, 0, h->gstream>>>(h->step_word, unsigned(h->steps));
          LB_CUDA(h, cudaGetLastError());
        }
        LB_CUDA(h, cudaGraphLaunch(h->graph[h->cur], h->gstream));
        h->steps += kStepGraph;
        nsteps -= kStepGraph;
      }
      LB_CUDA(h, cudaEventRecord(h->gev[1], h->gstream));
      LB_CUDA(h, cudaStreamWaitEvent(h->stream, h->gev[1], 0));
    }
  }
  for (int64_t s = 0; s < nsteps; ++s) {
    launch_one_step(h);
    LB_CUDA(h, cudaGetLastError());
    h->cur = 1 - h->cur;
    ++h->steps;
  }
  return LB_OK;
}

void* lb_state(lb_handle* h) { return h ? h->f[h->cur] : nullptr; }

int64_t lb_steps_done(const lb_handle* h) { return h ? h->steps : -1; }

int lb_moments(lb_handle* h, void* rho, void* ux, void* uy) {
  if (!h) return fail(nullptr, LB_EINVAL, "null handle");
  if (!rho) return fail(h, LB_EINVAL, "rho output is required");
  if (h->p.precision == LB_FP64)
    launch_moments<double, double>(h, static_cast<double*>(rho), static_cast<double*>(ux), static_cast<double*>(uy),
                                   h->cd.rho_ref, h->cd.G2);
  else if (h->p.precision == LB_FP32)
    launch_moments<float, float>(h, static_cast<float*>(rho), static_cast<float*>(ux), static_cast<float*>(uy),
                                 h->cf.rho_ref, h->cf.G2);
  else
    launch_moments<float, __half>(h, static_cast<float*>(rho), static_cast<float*>(ux), static_cast<float*>(uy),
                                  h->cf.rho_ref, h->cf.G2);
  LB_CUDA(h, cudaGetLastError());
  return LB_OK;
}

int lb_pressure(lb_handle* h, void* p) {
  if (!h) return fail(nullptr, LB_EINVAL, "null handle");
  if (!p) return fail(h, LB_EINVAL, "null output");
  const size_t N = size_t(h->p.nx) * h->p.ny;
  const unsigned blocks = unsigned((N + 255) / 256);
  const void* f = h->f[h->cur];
  if (h->p.precision == LB_FP64)
    k_pressure<double, double><<<blocks, 256, 0, h->stream>>>(static_cast<const double*>(f), static_cast<double*>(p),
                                                              h->p.nx, h->p.ny, h->st, h->cd);
  else if (h->p.precision == LB_FP32)
    k_pressure<float, float><<<blocks, 256, 0, h->stream>>>(static_cast<const float*>(f), static_cast<float*>(p),
                                                            h->p.nx, h->p.ny, h->st, h->cf);
  else
    k_pressure<float, __half><<<blocks, 256, 0, h->stream>>>(static_cast<const __half*>(f), static_cast<float*>(p),
                                                             h->p.nx, h->p.ny, h->st, h->cf);
  LB_CUDA(h, cudaGetLastError());
  return LB_OK;
}

int lb_reduce(lb_handle* h, double out[8]) {
  if (!h) return fail(nullptr, LB_EINVAL, "null handle");
  if (!out) return fail(h, LB_EINVAL, "null output");
  if (!h->scratch) return fail(h, LB_ENOMEM, "lb_reduce needs the scratch buffer (lb_scratch_bytes)");
  switch (h->p.precision) {
    case LB_FP64: return run_reduce<double, double>(h, out);
    case LB_FP32: return run_reduce<float, float>(h, out);
    default: return run_reduce<float, __half>(h, out);
  }
}

int lb_set_equilibrium(lb_handle* h, const double* rho, const double* ux, const double* uy) {
  if (!h) return fail(nullptr, LB_EINVAL, "null handle");
  if (!rho) return fail(h, LB_EINVAL, "rho is required");
  const size_t N = size_t(h->p.nx) * h->p.ny;
  const unsigned blocks = unsigned((N + 255) / 256);
  void* f = h->f[h->cur];
  const int nx = h->p.nx, ny = h->p.ny;
  switch (h->p.precision) {
    case LB_FP64:
      k_init_eq<double><<<blocks, 256, 0, h->stream>>>(rho, ux, uy, static_cast<double*>(f), nx, ny, h->st, h->cd);
      break;
    case LB_FP32:
      k_init_eq<float><<<blocks, 256, 0, h->stream>>>(rho, ux, uy, static_cast<float*>(f), nx, ny, h->st, h->cd);
      break;
    default:
      k_init_eq<__half><<<blocks, 256, 0, h->stream>>>(rho, ux, uy, static_cast<__half*>(f), nx, ny, h->st, h->cd);
  }
  LB_CUDA(h, cudaGetLastError());
  return LB_OK;
}

int lb_get_state(lb_handle* h, void* dst) {
  if (!h || !dst) return fail(h, LB_EINVAL, "null argument");
  LB_CUDA(h, cudaMemcpyAsync(dst, h->f[h->cur], lb_state_bytes(&h->p), cudaMemcpyDeviceToDevice, h->stream));
  return LB_OK;
}

int lb_set_state(lb_handle* h, const void* src) {
  if (!h || !src) return fail(h, LB_EINVAL, "null argument");
  LB_CUDA(h, cudaMemcpyAsync(h->f[h->cur], src, lb_state_bytes(&h->p), cudaMemcpyDeviceToDevice, h->stream));
  return LB_OK;
}

int lb_get_derived(const lb_handle* h, lb_derived* out) {
  if (!h || !out) return LB_EINVAL;
  *out = h->d;
  return LB_OK;
}

int lb_get_params(const lb_handle* h, lb_params* out) {
  if (!h || !out) return LB_EINVAL;
  *out = h->p;
  return LB_OK;
}

int lb_status(lb_handle* h) {
  if (!h) return fail(nullptr, LB_EINVAL, "null handle");
  int v = 0;
  LB_CUDA(h, cudaMemcpyAsync(&v, h->wait_error, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(h, cudaStreamSynchronize(h->stream));
  if (v) {
    LB_CUDA(h, cudaMemsetAsync(h->wait_error, 0, sizeof(int), h->stream));
    LB_CUDA(h, cudaStreamSynchronize(h->stream));
    return fail(h, LB_ETIMEOUT, "a bounded wait for a tensor copy gave up");
  }
  return LB_OK;
}

int lb_wait_selftest(lb_handle* h, long long polls) {
  if (!h) return fail(nullptr, LB_EINVAL, "null handle");
  if (polls < 1 || polls > (1ll << 22)) return fail(h, LB_EINVAL, "polls must be in [1, 2^22]");
  k_wait_selftest<<<1, 128, 0, h->stream>>>(polls, h->wait_error);
  LB_CUDA(h, cudaGetLastError());
  return lb_status(h);
}

int lb_stream_copy(lb_handle* h) {
  if (!h) return fail(nullptr, LB_EINVAL, "null handle");
  const void* in = h->f[h->cur];
  void* out = h->f[1 - h->cur];
  switch (h->p.precision) {
    case LB_FP64: launch_stream_copy<double>(h, in, out); break;
    case LB_FP32: launch_stream_copy<float>(h, in, out); break;
    default: launch_stream_copy<__half>(h, in, out);
  }
  LB_CUDA(h, cudaGetLastError());
  h->cur = 1 - h->cur;  // same data in the other buffer: the state is unchanged
  return LB_OK;
}

int lb_uses_tma(const lb_handle* h) { return h && h->use_tma ? 1 : 0; }

int lb_set_step_blocks(lb_handle* h, int blocks) {
  if (!h) return fail(nullptr, LB_EINVAL, "null handle");
  if (blocks < 0) return fail(h, LB_EINVAL, "negative block count");
  const int tiles = ((h->p.nx + kTileX - 1) / kTileX) * ((h->p.ny + kTileY - 1) / kTileY);
  h->tma_grid = blocks == 0 ? h->tma_grid_auto : (blocks < tiles ? blocks : tiles);
  h->dyn_grid = blocks == 0 ? h->dyn_grid_auto : (blocks < tiles ? blocks : tiles);
  return LB_OK;
}

int lb_set_tile_dispatch(lb_handle* h, int dynamic) {
  if (!h) return fail(nullptr, LB_EINVAL, "null handle");
  if (dynamic && !(h->use_tma && h->queue))
    return fail(h, LB_ENOTSUP, "dynamic dispatch needs the tensor-copy step and the scratch buffer");
  h->use_dyn = dynamic != 0;
  return LB_OK;
}

int lb_tile_dispatch(const lb_handle* h) { return h && h->use_tma && h->use_dyn ? 1 : 0; }

const char* lb_last_error(const lb_handle* h) { return h ? h->err : thread_error(); }

void lb_free(lb_handle* h) { destroy(h); }

}  // extern "C"
