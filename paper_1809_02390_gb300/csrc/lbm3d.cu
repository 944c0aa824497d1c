// D3Q19 form of the self-tuning-EOS multiphase lattice Boltzmann time step
// (Huang, Wu & Adams, arXiv:1809.02390, extended to three dimensions) and the
// lb_d3_* C ABI of include/lbm3d.h.
//
// The step kernel and its device code are in lbm3d_step.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm3d.h"
#include "lbm_internal.h"

#include "lbm3d_step.cuh"

namespace {

// Initial state at rest from FP64 densities: deviations of M^-1 m_eq(rho, 0).
// Invalid densities record the first offending node in bad[0] (not positive and
// finite) or bad[1] (vdW: rho >= 1/b).
template <typename T>
__global__ void k_d3_init(const double* __restrict__ rho0, T* __restrict__ f, int N, C3<double> c,
                          unsigned long long* bad) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double rho = rho0[n];
  if (!(rho > 0.0) || !isfinite(rho)) {
    atomicMin(bad, (unsigned long long)n);
    return;
  }
  if (c.eos == LB_EOS_VDW && !(c.b * rho < 1.0)) {
    atomicMin(bad + 1, (unsigned long long)n);
    return;
  }
  const double delta = rho - c.rho_ref;
  const double eta = 3.0 * (p_eos(c, rho) + 0.5 * c.G2 * rho * rho) - rho;
  const double r_ = delta / 19.0, e_ = (-11.0 * delta + 19.0 * eta) / 2394.0, p_ = (3.0 * delta + c.beta2 * eta) / 252.0;
  double o[Q];
  o[0] = r_ - 30.0 * e_ + 12.0 * p_;
  const double ax = r_ - 11.0 * e_ - 4.0 * p_, ce = r_ + 8.0 * e_ + p_;
  for (int i = 1; i < 7; ++i) o[i] = ax;
  for (int i = 7; i < Q; ++i) o[i] = ce;
  for (int i = 0; i < Q; ++i) f[size_t(i) * N + n] = T(o[i]);
}

// rho = sum_i fbar_i + rho_ref into an FP64 array.
template <typename T>
__global__ void k_d3_rho(const T* __restrict__ f, double* __restrict__ rho, int N, double rho_ref) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double a = 0.0;
  for (int i = 0; i < Q; ++i) a += double(f[size_t(i) * N + n]);
  rho[n] = a + rho_ref;
}

// rho u = sum_i e_i fbar_i - F/2 with F = G^2 rho sum_i omega_i rho(x + e_i) e_i.
template <typename T>
__global__ void k_d3_vel(const T* __restrict__ f, const double* __restrict__ rho, double* ux, double* uy, double* uz,
                         int nx, int ny, int nz, double G2) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = nx * ny * nz;
  if (n >= N) return;
  const int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
  double s[3] = {0.0, 0.0, 0.0}, j[3] = {0.0, 0.0, 0.0};
  for (int i = 1; i < Q; ++i) {
    const int xx = wrap(x + cEX[i], nx), yy = wrap(y + cEY[i], ny), zz = wrap(z + cEZ[i], nz);
    const double w = (cEX[i] * cEX[i] + cEY[i] * cEY[i] + cEZ[i] * cEZ[i]) == 1 ? 1.0 / 6.0 : 1.0 / 12.0;
    const double r = rho[(zz * ny + yy) * nx + xx];
    s[0] += w * r * cEX[i];
    s[1] += w * r * cEY[i];
    s[2] += w * r * cEZ[i];
    const double v = double(f[size_t(i) * N + n]);
    j[0] += cEX[i] * v;
    j[1] += cEY[i] * v;
    j[2] += cEZ[i] * v;
  }
  const double r0 = rho[n];
  if (ux) ux[n] = (j[0] - 0.5 * G2 * r0 * s[0]) / r0;
  if (uy) uy[n] = (j[1] - 0.5 * G2 * r0 * s[1]) / r0;
  if (uz) uz[n] = (j[2] - 0.5 * G2 * r0 * s[2]) / r0;
}

// FP64 diagnostics, first stage: block b sums nodes b, b + G, ... in a fixed order
// and writes kReduceSlots3 values: mass, the three components of sum_i e_i fbar_i,
// the number of nodes with rho above `mid`, min rho, max rho, the number of nodes
// whose density is not finite.  Second stage: k_d3_reduce_final (one block).
constexpr int kReduceBlocks3 = 512, kReduceSlots3 = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_d3_reduce_partial(const T* __restrict__ f, int N, double rho_ref, double mid,
                                                            double* __restrict__ part) {
  __shared__ double sh[kReduceSlots3][256];
  double a[kReduceSlots3] = {0.0, 0.0, 0.0, 0.0, 0.0, INFINITY, -INFINITY, 0.0};
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int i = 0; i < Q; ++i) {
      const double v = double(f[size_t(i) * N + n]);
      r += v;
      jx += cEX[i] * v;
      jy += cEY[i] * v;
      jz += cEZ[i] * v;
    }
    r += rho_ref;
    if (!isfinite(r)) {
      a[7] += 1.0;
      continue;
    }
    a[0] += r;
    a[1] += jx;
    a[2] += jy;
    a[3] += jz;
    a[4] += r > mid ? 1.0 : 0.0;
    a[5] = fmin(a[5], r);
    a[6] = fmax(a[6], r);
  }
  for (int k = 0; k < kReduceSlots3; ++k) sh[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < kReduceSlots3; ++k) {
        const double x = sh[k][threadIdx.x], y = sh[k][threadIdx.x + w];
        sh[k][threadIdx.x] = k == 5 ? fmin(x, y) : (k == 6 ? fmax(x, y) : x + y);
      }
    __syncthreads();
  }
  if (threadIdx.x < kReduceSlots3) part[blockIdx.x * kReduceSlots3 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_d3_reduce_final(const double* __restrict__ part, int blocks, double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= kReduceSlots3) return;
  double a = k == 5 ? INFINITY : (k == 6 ? -INFINITY : 0.0);
  for (int b = 0; b < blocks; ++b) {
    const double x = part[b * kReduceSlots3 + k];
    a = k == 5 ? fmin(a, x) : (k == 6 ? fmax(a, x) : a + x);
  }
  out[k] = a;
}

}  // namespace

struct lb_d3_handle {
  lb_params p;
  lb_derived d;
  int nz;
  void* f[2];
  int cur;
  cudaStream_t stream;
  C3<double> c64;
  C3<float> c32;
  int tz;  // planes per z-chunk of the step kernel
  // Graphs of kD3GraphSteps steps starting from buffer 0 and 1 (captured on first
  // use on the handle's private stream, launched on `stream`); graph_failed: a
  // capture failed once, so plain launches are used from then on.
  cudaStream_t cstream = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  bool graph_failed = false;
  double* part = nullptr;  // reduction partials (kReduceBlocks3 x kReduceSlots3) and the result
  char err[512];
};

namespace {

using namespace lbm;

int fail3(lb_d3_handle* h, int code, const char* fmt, ...) {
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

size_t nodes(const lb_params* p, int nz) { return size_t(p->nx) * size_t(p->ny) * size_t(nz); }

// 3-D parameters: the thermodynamics of lb_derive (Eqs. 17-22 hold unchanged),
// the 3-D coefficients of Eq. 7 and the 3-D closure of Eq. 16.
int derive3(const lb_params* p, int nz, lb_derived* d, char* err, size_t n) {
  auto bad = [&](int code, const char* m) {
    std::snprintf(err, n, "%s", m);
    return code;
  };
  if (!p || !d) return bad(LB_EINVAL, "null argument");
  if (p->nx < 1 || p->ny < 1 || nz < 1) return bad(LB_EINVAL, "nx, ny and nz must be >= 1");
  if (int64_t(p->nx) * p->ny * nz >= (int64_t(1) << 31))
    return bad(LB_EINVAL, "lattice too large: nx ny nz must be below 2^31");
  if (p->precision == LB_FP16S) return bad(LB_ENOTSUP, "the D3Q19 step stores FP64 or FP32 populations");
  if (p->layout != LB_LAYOUT_PLANES) return bad(LB_ENOTSUP, "the D3Q19 step uses the planes layout");
  if (p->variant != LB_AUTO && p->variant != LB_FUSED) return bad(LB_ENOTSUP, "the D3Q19 step is the fused one");
  const double w = p->varpi == 0.0 ? 1.0 / 6.0 : p->varpi;
  if (!(w > 0) || w == 1.0 || std::fabs(w - 7.0 / 18.0) < 1e-12)
    return bad(LB_EINVAL, "varpi must be > 0 and not 1 or 7/18 (singular 3-D coefficients)");
  lb_params q = *p;
  q.nx = q.nx < 3 ? 3 : q.nx;
  q.ny = q.ny < 3 ? 3 : q.ny;
  q.varpi = 1.0 / 6.0;  // validated above; the 2-D coefficients are replaced below
  q.s_q = q.s_e = q.s_eps = 1.0;
  const int rc = derive(&q, d, err, n);
  if (rc != LB_OK) return rc;
  const double k = 38.0 * (1.0 - w) / 11.0;
  d->k = k;
  d->beta2 = -19.0 / k;
  d->b = 21.0 * (1.0 - w) / (5.0 * (7.0 - 18.0 * w));
  d->h = 798.0 * w * (1.0 - w) / (5.0 * (7.0 - 18.0 * w));
  const double tau_p = 1.0 / p->s_p - 0.5;
  const double tau_q = 1.0 / (12.0 * tau_p);
  const double tau_e = 1.0 / (12.0 * (1.0 + 5.0 * k / 19.0) * tau_q);
  d->s_q = p->s_q > 0 ? p->s_q : 1.0 / (tau_q + 0.5);
  d->s_e = p->s_e > 0 ? p->s_e : 1.0 / (tau_e + 0.5);
  d->s_eps = p->s_eps > 0 ? p->s_eps : kSEps3;
  auto ok = [](double s) { return s > 0.0 && s < 2.0; };
  if (!ok(d->s_q) || !ok(d->s_e) || !ok(d->s_eps)) return bad(LB_EINVAL, "relaxation rates must lie in (0, 2)");
  return LB_OK;
}

template <typename T>
C3<T> make_c3(const lb_params& p, const lb_derived& d) {
  C3<T> c;
  c.eos = p.eos;
  c.rho_ref = T(p.rho_ref);
  c.G2 = T(d.G2);
  c.lam_RT = T(d.lam * p.R_gas * d.T);
  c.lam_a = T(d.lam * p.eos_a);
  c.b = T(p.eos_b);
  c.bq = T(p.eos_b / 4.0);
  c.se = T(d.s_e);
  c.seps = T(d.s_eps);
  c.sq = T(d.s_q);
  c.sp = T(d.s_p);
  c.sm = T(d.s_q);
  c.spi = T(d.s_eps);
  c.k_seps_ome = T(d.k * d.s_eps * (d.s_e / 2.0 - 1.0));
  c.h_sq_ome = T(d.h * d.s_q * (d.s_e / 2.0 - 1.0));
  c.b_sq_omp = T(d.b * d.s_q * (d.s_p / 2.0 - 1.0));
  c.beta2 = T(d.beta2);
  return c;
}

// Planes per z-chunk: 32 (fewest halo planes) unless that leaves fewer than two
// waves of resident blocks (3 per SM); then halved down to 2, because a block walks
// its chunk plane after plane and a short grid leaves the GPU waiting on that chain.
int chunk_planes(int nx, int ny, int nz, int sms) {
  const long long xy = (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
  int tz = TZ;
  while (tz > 2 && xy * ((nz + tz - 1) / tz) < 2LL * 3 * sms) tz /= 2;
  return tz;
}

void launch_step(lb_d3_handle* h) {
  const lb_params& p = h->p;
  const int tz = h->tz;
  const dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, (h->nz + tz - 1) / tz), block(TX, TY);
  const void* in = h->f[h->cur];
  void* out = h->f[1 - h->cur];
  // 32-bit plane offsets while 19 nx ny nz < 2^31 (the common case), 64-bit above.
  const bool wide = int64_t(Q) * p.nx * p.ny * h->nz >= (int64_t(1) << 31);
  const double* i64 = static_cast<const double*>(in);
  const float* i32 = static_cast<const float*>(in);
  if (p.precision == LB_FP64) {
    if (wide)
      k_d3_step<double, false, long long><<<grid, block, 0, h->stream>>>(i64, static_cast<double*>(out), p.nx, p.ny,
                                                                         h->nz, tz, h->c64);
    else
      k_d3_step<double, false, int><<<grid, block, 0, h->stream>>>(i64, static_cast<double*>(out), p.nx, p.ny, h->nz,
                                                                   tz, h->c64);
  } else {
    if (wide)
      k_d3_step<float, true, long long><<<grid, block, 0, h->stream>>>(i32, static_cast<float*>(out), p.nx, p.ny,
                                                                       h->nz, tz, h->c32);
    else
      k_d3_step<float, true, int><<<grid, block, 0, h->stream>>>(i32, static_cast<float*>(out), p.nx, p.ny, h->nz, tz,
                                                                 h->c32);
  }
  h->cur = 1 - h->cur;
}

constexpr int64_t kD3GraphSteps = 64;
static_assert(kD3GraphSteps % 2 == 0, "a graph must end in the buffer it starts from");

// Captures (once) the graph of kD3GraphSteps steps that starts from buffer h->cur.
// Returns false, and leaves plain launches in use, if the capture fails.
bool ensure_graph(lb_d3_handle* h) {
  const int c = h->cur;
  if (h->exec[c]) return true;
  if (h->graph_failed) return false;
  bool ok = h->cstream || cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) ok = cudaStreamBeginCapture(h->cstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    cudaStream_t keep = h->stream;
    h->stream = h->cstream;
    for (int64_t k = 0; k < kD3GraphSteps; ++k) launch_step(h);
    h->stream = keep;
    ok = cudaStreamEndCapture(h->cstream, &h->graph[c]) == cudaSuccess && h->graph[c];
    if (ok) ok = cudaGraphInstantiate(&h->exec[c], h->graph[c], 0) == cudaSuccess;
  }
  h->cur = c;  // the captured launches flipped it an even number of times
  if (!ok) {
    cudaGetLastError();
    h->graph_failed = true;
  }
  return ok;
}

}  // namespace

extern "C" {

void lb_d3_velocities(int* ex, int* ey, int* ez) {
  for (int i = 0; i < Q; ++i) {
    if (ex) ex[i] = kEX[i];
    if (ey) ey[i] = kEY[i];
    if (ez) ez[i] = kEZ[i];
  }
}

int lb_d3_derive(const lb_params* p, int32_t nz, lb_derived* out) {
  char err[256];
  lb_derived d;
  const int rc = derive3(p, nz, &d, err, sizeof(err));
  if (rc != LB_OK) return fail3(nullptr, rc, "%s", err);
  if (!out) return fail3(nullptr, LB_EINVAL, "null output");
  *out = d;
  return LB_OK;
}

size_t lb_d3_state_bytes(const lb_params* p, int32_t nz) {
  if (!p || nz < 1) return 0;
  return Q * nodes(p, nz) * (p->precision == LB_FP64 ? 8 : 4);
}

int lb_d3_init(lb_d3_handle** out, const lb_params* p, int32_t nz, void* f_a, void* f_b, const double* rho0,
               int rho0_on_device, void* stream) {
  if (!out) return fail3(nullptr, LB_EINVAL, "null handle pointer");
  *out = nullptr;
  char err[256];
  lb_derived d;
  int rc = derive3(p, nz, &d, err, sizeof(err));
  if (rc != LB_OK) return fail3(nullptr, rc, "%s", err);
  if (!f_a || !f_b || f_a == f_b) return fail3(nullptr, LB_EINVAL, "f_a and f_b must be two distinct device buffers");
  if (!rho0) return fail3(nullptr, LB_EINVAL, "null initial density");
  const size_t N = nodes(p, nz);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto cuda_fail = [&](cudaError_t e, const char* what) {
    return fail3(nullptr, LB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  };
  lb_params q = *p;
  const double* rho_dev = rho0;
  if (!rho0_on_device) {
    cudaError_t e = cudaMemcpyAsync(f_b, rho0, N * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy of the initial density");
    rho_dev = static_cast<const double*>(f_b);
  }
  if (std::isnan(q.rho_ref)) {
    std::vector<double> host;
    const double* hp = rho0;
    if (rho0_on_device) {
      host.resize(N);
      cudaError_t e = cudaMemcpyAsync(host.data(), rho0, N * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(e, "read of the initial density");
      hp = host.data();
    }
    double sum = 0.0;
    for (size_t n = 0; n < N; ++n) sum += hp[n];
    q.rho_ref = sum / double(N);
  }
  if (q.precision == LB_FP32) q.rho_ref = double(float(q.rho_ref));
  unsigned long long* bad = nullptr;
  cudaError_t e = cudaMalloc(&bad, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc of the status words");
  e = cudaMemsetAsync(bad, 0xff, 2 * sizeof(unsigned long long), s);
  const C3<double> c = make_c3<double>(q, d);
  const int threads = 256, blocks = int((N + threads - 1) / threads);
  if (e == cudaSuccess) {
    if (q.precision == LB_FP64)
      k_d3_init<double><<<blocks, threads, 0, s>>>(rho_dev, static_cast<double*>(f_a), int(N), c, bad);
    else
      k_d3_init<float><<<blocks, threads, 0, s>>>(rho_dev, static_cast<float*>(f_a), int(N), c, bad);
    e = cudaGetLastError();
  }
  unsigned long long first[2] = {~0ull, ~0ull};
  if (e == cudaSuccess) e = cudaMemcpyAsync(first, bad, sizeof(first), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bad);
  if (e != cudaSuccess) return cuda_fail(e, "initial state");
  if (first[0] != ~0ull)
    return fail3(nullptr, LB_EINVAL, "initial density at node %llu is not positive and finite", first[0]);
  if (first[1] != ~0ull) return fail3(nullptr, LB_EINVAL, "initial density at node %llu exceeds 1/b of the vdW EOS", first[1]);
  lb_d3_handle* h = new (std::nothrow) lb_d3_handle();
  if (!h) return fail3(nullptr, LB_EINVAL, "out of host memory");
  h->p = q;
  h->d = d;
  h->nz = nz;
  h->f[0] = f_a;
  h->f[1] = f_b;
  h->cur = 0;
  h->stream = s;
  h->c64 = c;
  h->c32 = make_c3<float>(q, d);
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  h->tz = chunk_planes(q.nx, q.ny, nz, sms);
  h->err[0] = 0;
  if (cudaMalloc(&h->part, (kReduceBlocks3 + 1) * kReduceSlots3 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail3(nullptr, LB_ENOMEM, "cudaMalloc of the %zu-byte reduction workspace",
                 size_t(kReduceBlocks3 + 1) * kReduceSlots3 * sizeof(double));
  }
  *out = h;
  return LB_OK;
}

int lb_d3_step(lb_d3_handle* h, int64_t nsteps) {
  if (!h) return fail3(nullptr, LB_EINVAL, "null handle");
  if (nsteps < 0) return fail3(h, LB_EINVAL, "nsteps must be >= 0");
  // Runs of kD3GraphSteps steps replay a graph, unless the caller's stream is being
  // captured itself (then the steps go into the caller's graph as plain launches).
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  if (h->stream != nullptr && cudaStreamIsCapturing(h->stream, &capture) != cudaSuccess) {
    cudaGetLastError();
    capture = cudaStreamCaptureStatusActive;
  }
  while (capture == cudaStreamCaptureStatusNone && nsteps >= kD3GraphSteps && ensure_graph(h)) {
    const cudaError_t e = cudaGraphLaunch(h->exec[h->cur], h->stream);
    if (e != cudaSuccess) return fail3(h, LB_ECUDA, "step graph launch: %s", cudaGetErrorString(e));
    nsteps -= kD3GraphSteps;  // an even number of steps: the state is back in the same buffer
  }
  for (int64_t k = 0; k < nsteps; ++k) launch_step(h);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail3(h, LB_ECUDA, "step launch: %s", cudaGetErrorString(e));
  return LB_OK;
}

int lb_d3_moments(lb_d3_handle* h, void* rho, void* ux, void* uy, void* uz) {
  if (!h) return fail3(nullptr, LB_EINVAL, "null handle");
  if (!rho) return fail3(h, LB_EINVAL, "rho output is required");
  const int N = int(nodes(&h->p, h->nz));
  const int threads = 256, blocks = (N + threads - 1) / threads;
  double* r = static_cast<double*>(rho);
  const void* f = h->f[h->cur];
  if (h->p.precision == LB_FP64)
    k_d3_rho<double><<<blocks, threads, 0, h->stream>>>(static_cast<const double*>(f), r, N, h->p.rho_ref);
  else
    k_d3_rho<float><<<blocks, threads, 0, h->stream>>>(static_cast<const float*>(f), r, N, h->p.rho_ref);
  if (ux || uy || uz) {
    double *a = static_cast<double*>(ux), *b = static_cast<double*>(uy), *c = static_cast<double*>(uz);
    if (h->p.precision == LB_FP64)
      k_d3_vel<double><<<blocks, threads, 0, h->stream>>>(static_cast<const double*>(f), r, a, b, c, h->p.nx, h->p.ny,
                                                          h->nz, h->d.G2);
    else
      k_d3_vel<float><<<blocks, threads, 0, h->stream>>>(static_cast<const float*>(f), r, a, b, c, h->p.nx, h->p.ny,
                                                         h->nz, h->d.G2);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail3(h, LB_ECUDA, "moments launch: %s", cudaGetErrorString(e));
  return LB_OK;
}

int lb_d3_reduce(lb_d3_handle* h, double out[8]) {
  if (!h) return fail3(nullptr, LB_EINVAL, "null handle");
  if (!out) return fail3(h, LB_EINVAL, "null output");
  const int N = int(nodes(&h->p, h->nz));
  const double mid = 0.5 * (h->d.rho_g + h->d.rho_l);
  const int blocks = std::min(kReduceBlocks3, (N + 255) / 256);
  const void* f = h->f[h->cur];
  if (h->p.precision == LB_FP64)
    k_d3_reduce_partial<double><<<blocks, 256, 0, h->stream>>>(static_cast<const double*>(f), N, h->p.rho_ref, mid,
                                                                h->part);
  else
    k_d3_reduce_partial<float><<<blocks, 256, 0, h->stream>>>(static_cast<const float*>(f), N, h->p.rho_ref, mid,
                                                               h->part);
  double* res = h->part + kReduceBlocks3 * kReduceSlots3;
  k_d3_reduce_final<<<1, 32, 0, h->stream>>>(h->part, blocks, res);
  cudaError_t e = cudaMemcpyAsync(out, res, kReduceSlots3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail3(h, LB_ECUDA, "reduction: %s", cudaGetErrorString(e));
  if (out[7] > 0) return fail3(h, LB_ENONFINITE, "%.0f nodes have a non-finite density", out[7]);
  return LB_OK;
}

void* lb_d3_state(const lb_d3_handle* h) { return h ? h->f[h->cur] : nullptr; }

int lb_d3_get_state(lb_d3_handle* h, void* dst) {
  if (!h || !dst) return fail3(h, LB_EINVAL, "null argument");
  const cudaError_t e = cudaMemcpyAsync(dst, h->f[h->cur], lb_d3_state_bytes(&h->p, h->nz), cudaMemcpyDeviceToDevice,
                                        h->stream);
  if (e != cudaSuccess) return fail3(h, LB_ECUDA, "state copy: %s", cudaGetErrorString(e));
  return LB_OK;
}

int lb_d3_set_state(lb_d3_handle* h, const void* src) {
  if (!h || !src) return fail3(h, LB_EINVAL, "null argument");
  const cudaError_t e = cudaMemcpyAsync(h->f[h->cur], src, lb_d3_state_bytes(&h->p, h->nz), cudaMemcpyDeviceToDevice,
                                        h->stream);
  if (e != cudaSuccess) return fail3(h, LB_ECUDA, "state copy: %s", cudaGetErrorString(e));
  return LB_OK;
}

int lb_d3_get_params(const lb_d3_handle* h, lb_params* out, lb_derived* derived) {
  if (!h) return fail3(nullptr, LB_EINVAL, "null handle");
  if (out) *out = h->p;
  if (derived) *derived = h->d;
  return LB_OK;
}

const char* lb_d3_last_error(const lb_d3_handle* h) { return h ? h->err : thread_error(); }

void lb_d3_free(lb_d3_handle* h) {
  if (!h) return;
  for (int c = 0; c < 2; ++c) {
    if (h->exec[c]) cudaGraphExecDestroy(h->exec[c]);
    if (h->graph[c]) cudaGraphDestroy(h->graph[c]);
  }
  if (h->cstream) cudaStreamDestroy(h->cstream);
  if (h->part) cudaFree(h->part);
  delete h;
}

}  // extern "C"
