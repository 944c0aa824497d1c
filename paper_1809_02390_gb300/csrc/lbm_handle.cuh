// Handle of one lattice (shared by the library's CUDA translation units).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_kernels.cuh"

struct lb_handle {
  lb_params p;
  lb_derived d;
  void* f[2];
  int cur;
  void* scratch;
  size_t scratch_bytes;
  cudaStream_t stream;
  int64_t steps;
  int variant;  // LB_FUSED or LB_TWO_PASS
  int reduce_blocks;
  lbm::Strides st;        // population layout (planes or rows)
  bool use_tma;           // FP32 fused step with tensor-copy staging (interior tiles)
  int tma_grid;           // persistent grid of that kernel
  int tma_grid_auto;      // its default: resident capacity, at most the tile count
  unsigned* queue;        // tile tickets of the dynamic form (end of the scratch buffer), or null
  bool use_dyn;           // the tensor-copy step takes tiles by ticket (k_step_tma_dyn)
  int dyn_grid, dyn_grid_auto;
  CUtensorMap tmap[2];    // 3-D maps of f[0] and f[1]: (x, y, plane), rows layout (x, plane, y)
  int* wait_error;        // this handle's device word, set by a bounded wait that gave up
  int wait_slot;          // its index in the library's array of such words (-1: none taken)
  // Replay of runs of steps (lb_step): graphs of kStepGraph steps captured on an
  // internal stream, one per starting buffer, with the launch configuration they
  // were captured for; events order them after and before the caller's stream.
  cudaStream_t gstream;
  cudaEvent_t gev[2];
  cudaGraphExec_t graph[2];
  long long graph_cfg[2];
  bool graph_off;         // capture failed once: direct launches only
  unsigned* step_word;    // device word with the step count a replayed FP16 graph seeds from
  int graph_k;            // while capturing: the place of the launch in the graph (else -1)
  lbm::VCoef<float> cf;  // FP32 scalar (two-pass variant, moments)
  lbm::VCoef<lbm::f2> c2;     // FP32 pairs (fused variant)
  lbm::VCoef<double> cd;
  char err[512];
};

namespace lbm {
// 3-D tensor map of an FP32 (elem_bytes 4) or FP16 (2) population buffer, box =
// one plane window of the tensor-copy step: dimensions (x, y, plane) with row
// stride sx, or (x, plane, y) for the rows layout (sx = nx); false if the layout
// does not allow one (lbm_capi.cu).
bool encode_population_map(CUtensorMap* map, void* base, int nx, int ny, int sx, int elem_bytes = 4,
                           bool rows = false);
// 3-D map (x, y, plane) of `planes` FP32 planes of nx x ny, box cols x rows x 1
// (lbm_capi.cu); false if the buffer does not allow one.
bool encode_plane_map(CUtensorMap* map, const void* base, int nx, int ny, int planes, int cols, int rows);
// Device address of lb_reduce_static's static scratch on the current device
// (looked up once per device, which commits the array there; lbm_static.cu).
int static_scratch_address(lb_handle* h, void** out);
// Mean of the n doubles at x (device memory), summed in FP64 on `stream` with
// block partials written to `work` (device memory of work_bytes >= 8), folded on
// the host in a fixed order; synchronous.  cudaSuccess or the CUDA error
// (lbm_capi.cu).
cudaError_t device_mean(const double* x, size_t n, void* work, size_t work_bytes, cudaStream_t stream, double* mean);
}  // namespace lbm
