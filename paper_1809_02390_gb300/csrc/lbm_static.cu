// lb_reduce_static: the diagnostics of lb_reduce for callers that cannot
// allocate device memory.  Some callers cannot call cudaMalloc at all: a host
// program whose own allocator has taken every byte of the GPU and hands out no
// more buffers, or a plugin loaded into such a program, which gets the lattice
// from its host and has no allocator of its own.  lb_reduce needs the caller's
// scratch buffer; this variant keeps its scratch in the file-scope device array
// below instead, so nothing is allocated by the caller, by this library or by
// any library it calls.  The call is synchronous (it copies the sums to the host
// and waits on the handle's stream), so it must not be made on a stream that is
// being captured into a CUDA graph.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "lbm_handle.cuh"
#include "lbm_fields.cuh"

namespace {

using namespace lbm;

constexpr size_t kPlaneBytes = size_t(LB_REDUCE_STATIC_MAX_NODES) * sizeof(double);
constexpr size_t kPartialBytes = size_t(kMaxReduceBlocks) * kReduceSlots * sizeof(double);
constexpr size_t kOutBytes = kReduceSlots * sizeof(double);

// Density plane (as double or float) | block partials | final sums.  The driver
// loads the module that holds this array, and so commits the array's memory,
// when lb_init first looks up its address on a device (static_scratch_address);
// from then on that GPU holds it until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kPlaneBytes + kPartialBytes + kOutBytes];

// Device address of g_static_scratch for each device, looked up once per device
// with that device current (in host code the symbol is only a host-side stand-in).
std::mutex g_mu;
void* g_addr[256] = {nullptr};

int set_err(lb_handle* h, int code, const char* msg, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess)
    std::snprintf(h->err, sizeof(h->err), "%s: %s", msg, cudaGetErrorString(e));
  else
    std::snprintf(h->err, sizeof(h->err), "%s", msg);
  return code;
}

}  // namespace

namespace lbm {

// Looks up (once per device, with that device current) the device address of the
// static scratch, which loads its module and commits the array on this device.
// lb_init calls it, so that the memory is taken when a handle is created and a
// later lb_reduce_static cannot fail for want of device memory.
int static_scratch_address(lb_handle* h, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_err(h, LB_ECUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= 256) return set_err(h, LB_ENOTSUP, "device ordinal above 255");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return set_err(h, LB_ECUDA, "cudaGetSymbolAddress(static scratch)", e);
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return LB_OK;
}

}  // namespace lbm

namespace {

template <typename real, typename store_t>
int reduce_static(lb_handle* h, unsigned char* base, double out[8]) {
  const int nx = h->p.nx, ny = h->p.ny;
  const size_t N = size_t(nx) * ny;
  // Every element read below is first written by this same call (density plane
  // by k_rho_local, each block's partial by k_reduce_partial, the sums by
  // k_reduce_final), so nothing left by an earlier call is ever used.
  real* rho = reinterpret_cast<real*>(base);
  double* partial = reinterpret_cast<double*>(base + kPlaneBytes);
  double* dout = reinterpret_cast<double*>(base + kPlaneBytes + kPartialBytes);
  const store_t* f = static_cast<const store_t*>(h->f[h->cur]);
  const int blocks = h->reduce_blocks;  // at most kMaxReduceBlocks (configure_device), as in lb_reduce
  k_rho_local<real, store_t><<<unsigned((N + 255) / 256), 256, 0, h->stream>>>(f, rho, nx, ny, h->st,
                                                                                real(h->p.rho_ref));
  const double rho_mid = 0.5 * (h->d.rho_g + h->d.rho_l);
  k_reduce_partial<real, store_t><<<blocks, kReduceThreads, 0, h->stream>>>(
      f, rho, nx, ny, h->st, real(h->d.G2), rho_mid == rho_mid ? rho_mid : 1e300, partial);
  k_reduce_final<<<1, 32, 0, h->stream>>>(partial, blocks, dout);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(h, LB_ECUDA, "reduce kernels", e);
  double res[kReduceSlots];
  real probe[2];
  e = cudaMemcpyAsync(res, dout, sizeof(res), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&probe[0], rho + size_t(ny / 2) * nx + nx / 2, sizeof(real), cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&probe[1], rho, sizeof(real), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return set_err(h, LB_ECUDA, "reading the reduction", e);
  out[0] = res[0];
  out[1] = res[1];
  out[2] = res[2];
  out[3] = p_eos_host(h->cd, double(probe[0]));
  out[4] = p_eos_host(h->cd, double(probe[1]));
  out[5] = res[3];
  out[6] = res[4];
  out[7] = res[5];
  if (res[6] > 0) {
    std::snprintf(h->err, sizeof(h->err), "%.0f nodes have a non-finite density", res[6]);
    return LB_ENONFINITE;
  }
  return LB_OK;
}

}  // namespace

extern "C" int lb_reduce_static(lb_handle* h, double out[8]) {
  if (!h) return LB_EINVAL;
  if (!out) return set_err(h, LB_EINVAL, "null output");
  const size_t N = size_t(h->p.nx) * h->p.ny;
  if (N > size_t(LB_REDUCE_STATIC_MAX_NODES)) {
    std::snprintf(h->err, sizeof(h->err),
                  "lb_reduce_static: lattice of %zu nodes exceeds its static scratch of %d nodes (use lb_reduce)", N,
                  LB_REDUCE_STATIC_MAX_NODES);
    return LB_ENOMEM;
  }
  void* base = nullptr;
  const int rc = static_scratch_address(h, &base);
  if (rc != LB_OK) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  switch (h->p.precision) {
    case LB_FP64: return reduce_static<double, double>(h, b, out);
    case LB_FP32: return reduce_static<float, float>(h, b, out);
    default: return reduce_static<float, __half>(h, b, out);
  }
}
