// Internal: the solver context behind the opaque mhd_ctx of include/mhd.h, shared by the
// C-ABI implementation (mhd_capi.cu) and the batched persistent form (mhd_batch.cu).
#pragma once

#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/mhd.h"
#include "mhd_kernels.cuh"

using mhd::DevScalars;
using mhd::FieldSet;
using mhd::GridDesc;

// axis order of the forward sweep for each phase (Eq. "eq:L_sequence")
static constexpr int kOrder[3][3] = {{0, 1, 2}, {2, 0, 1}, {1, 2, 0}};

struct mhd_ctx {
  mhd_config cfg{};
  GridDesc g{};
  long long N = 0;
  size_t esz = 4;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* buf[2][8] = {};
  int cur[8] = {};
  void* staging = nullptr;      // N doubles, host <-> device conversions
  DevScalars* ds = nullptr;     // device
  DevScalars* hs = nullptr;     // pinned host mirror
  double* partial = nullptr;
  double* sums_out = nullptr;   // device, 8 doubles
  double* sums_host = nullptr;  // pinned, 8 doubles
  int sum_blocks = 0;
  int phase = 0;
  int step = 0;
  int steps_base = 0;           // ds->steps_done at the last synchronisation point
  int status = 0;               // sticky ST_* bits seen at synchronisation points
  // captured steps: per phase, up to two buffer states (a step whose middle CT pair runs as
  // one launch flips the B buffers once, so the state alternates); sig_in / sig_out: the
  // buffer assignment (cur[]) before and after the step
  struct StepGraph { cudaGraphExec_t exec = nullptr; unsigned sig_in = 0, sig_out = 0; };
  StepGraph graph[3][2];
  int graph_next[3] = {0, 0, 0};
  // tensor maps of the 16 state buffers for the TMA-staged x/y fluid sweeps (FP32 grids
  // with nz a multiple of 128; tma false otherwise), per buffer b and field k: boxes of 128 z
  // positions of one row (one), of kTmaG rows along x (gx) and along y (gy)
  bool tma = false;
  CUtensorMap tmap_one[2][8], tmap_gx[2][8], tmap_gy[2][8];
  long long dev_bytes = 0;
  std::string err;
  // kernel timing mode: steps are launched kernel by kernel with CUDA events around each
  bool profile = false;
  struct Pending { int kind; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;
  double prof_ms[8] = {};
  long long prof_n[8] = {};
};

