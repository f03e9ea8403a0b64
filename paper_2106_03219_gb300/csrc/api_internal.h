// Internal host-side declarations shared by the C-ABI translation units.
#pragma once

#include <atomic>
#include <cstdint>

#include "launch.h"
#include "omprt.h"

struct omprt_ctx {
  int device = 0;
  int sm_count = 0;
  int l2_bytes = 0;
  int max_smem_optin = 0;
  int smem_per_sm = 0;
  uint32_t* status_dev = nullptr;
  unsigned char* slots_dev = nullptr;
  unsigned char* pool_dev = nullptr;
  float* mlp_rows_dev = nullptr;   // MLP per-sample scratch, kMlpMaxBatch rows
  uint32_t stack_bytes = 0;
  uint32_t stage_bytes = 32768;    // per-team shared memory for staged dynamic schedules
  uint32_t stencil_stage_bytes = 0;  // per-CTA shared memory for the staged 2-D stencil windows
  uint32_t slab_floats = 0;   // 2-D stencil slabs: floats a line (16 / 32; 0 the default)
  uint32_t slab_buffers = 0;  // and buffers a warp (2 .. 4; 0 the default)
  bool launch_overlap = true;  // executor launches overlap the previous grid's tail
  std::atomic<uint32_t> next_slot{0};
  // learned schedule (host copy of the model)
  bool has_model = false;
  float model[OMPRT_MLP_NPARAM];
  float feat_mean[OMPRT_MLP_IN];
  float feat_std[OMPRT_MLP_IN];
};

// MLP training batch limit and per-sample scratch row (floats).
constexpr int kMlpMaxBatch = 16384;
constexpr int kMlpRowFloats = 272;

struct DeviceGuard {
  int prev = 0;
  bool changed = false;
  explicit DeviceGuard(int dev);
  ~DeviceGuard();
};

struct ScratchSlot {
  uint32_t* ticket;
  unsigned char* partials;
  unsigned long long* dyn_next;
};
ScratchSlot ctx_next_slot(omprt_ctx* ctx);

omprt_status loop_trip_count(const omprt_loop_desc* d, uint64_t* n, int64_t* wide_lb);

struct LearnedConfig {
  int32_t sched;
  int64_t chunk;
  int32_t teams_per_sm;
  int32_t threads;
};
LearnedConfig learned_config(int k);
