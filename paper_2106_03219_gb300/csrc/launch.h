// Host-side entry points of the executor translation units (internal).
#pragma once

#include <utility>

#include <cuda_runtime.h>

#include "region.cuh"

namespace rt {

// A launch gets 48 KB of shared memory, static and dynamic together, without
// the kernel's opt-in; beyond that the opt-in must cover the dynamic part.
// The kernel's static part is looked up once per kernel by the caller.
template <class K>
inline size_t static_smem_of(K kern) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
    cudaGetLastError();
    return 48 * 1024;  // unknown: always opt in
  }
  return fa.sharedSizeBytes;
}
template <class K>
inline cudaError_t smem_optin(K kern, size_t dyn, size_t static_bytes) {
  if (dyn + static_bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

// Launch overlap, per host thread: whether executor launches may overlap
// the tail of the previous grid on their stream (programmatic stream
// serialisation; on by default), the shared memory of one SM (0: unknown),
// and the dynamic shared memory of the last executor launch on each of the
// last kStreams streams this thread launched on.  An API call on a context
// sets the first two from the context for its duration (OverlapScope).
struct OverlapState {
  static constexpr int kStreams = 8;
  bool on = true;
  size_t smem_per_sm = 0;
  cudaStream_t stream[kStreams] = {};
  size_t smem[kStreams] = {};
  int used = 0, next = 0;  // entries filled; the one to replace next
  int find(cudaStream_t st) const {
    for (int i = 0; i < used; ++i)
      if (stream[i] == st) return i;
    return -1;
  }
  void record(cudaStream_t st, size_t bytes) {
    int i = find(st);
    if (i < 0) {
      i = next;
      next = (next + 1) % kStreams;
      if (used < kStreams) ++used;
      stream[i] = st;
    }
    smem[i] = bytes;
  }
};
inline OverlapState& overlap_state() {
  thread_local OverlapState s;
  return s;
}
struct OverlapScope {
  bool prev_on;
  size_t prev_per_sm;
  OverlapScope(bool on, size_t smem_per_sm) {
    OverlapState& s = overlap_state();
    prev_on = s.on;
    prev_per_sm = s.smem_per_sm;
    s.on = on;
    s.smem_per_sm = smem_per_sm;
  }
  ~OverlapScope() {
    overlap_state().on = prev_on;
    overlap_state().smem_per_sm = prev_per_sm;
  }
  OverlapScope(const OverlapScope&) = delete;
  OverlapScope& operator=(const OverlapScope&) = delete;
};

// A grid scheduled early lands beside the previous grid's blocks, and an SM
// that keeps running blocks keeps the split of its on-chip memory between L1
// and shared memory that the previous grid set.  A grid asking for much less
// shared memory than the one before it (a streaming loop after a staged
// stencil) would then run all its blocks with the small L1 of that split:
// measured on GB300, an axpy of 2^26 floats after a 200 KB-a-block copy lost
// 15 us that way, against 3 us gained by the overlap.  Such a launch is made
// plain, so the SMs drain and take the new split; where the two grids cannot
// share an SM, or ask for about the same, the launch overlaps.
constexpr size_t kOverlapSmemStep = 16 * 1024;
inline bool overlap_this_launch(cudaStream_t st, size_t smem) {
  const OverlapState& s = overlap_state();
  if (!s.on) return false;
  const int i = s.find(st);
  if (i < 0) return true;
  const size_t last = s.smem[i];
  const bool can_share = s.smem_per_sm == 0 || last + smem <= s.smem_per_sm;
  return !(can_share && last >= smem + kOverlapSmemStep);
}

// Launch an executor kernel (one that starts with enter_region_grid).  The
// launch error, if any, is returned and cleared.
template <class... KArgs, class... Args>
inline cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                 cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = overlap_this_launch(st, smem) ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  overlap_state().record(st, smem);
  return e;
}

// Reduction accumulator selected for a launch.
enum AccKind : int {
  kAccNone = 0,
  kAccSumI64,
  kAccCompF32,
  kAccNaiveF32,
  kAccMaxF32,
  kAccMinF32,
  kAccMaxI64,
  kAccMinI64,
};

// Launch one region kernel instance.  Returns cudaErrorNotSupported for a
// (body, data type, accumulator) combination that has no instance.
cudaError_t launch_region_f32(int body, int dtype, int acc, int sched, unsigned grid,
                              unsigned block, size_t smem, cudaStream_t st, const RegionArgs& a);
cudaError_t launch_region_int(int body, int dtype, int acc, int sched, unsigned grid,
                              unsigned block, size_t smem, cudaStream_t st, const RegionArgs& a);

// Per-body instance units.
cudaError_t launch_axpy(int dtype, int acc, int sched, unsigned grid, unsigned block, size_t smem,
                        cudaStream_t st, const RegionArgs& a);
cudaError_t launch_stencil(int body, int acc, int sched, unsigned grid, unsigned block,
                           size_t smem, cudaStream_t st, const RegionArgs& a);
cudaError_t launch_dot_load(int body, int dtype, int acc, int sched, unsigned grid,
                            unsigned block, size_t smem, cudaStream_t st, const RegionArgs& a);

// schedule(auto) 2-D stencil on tensor tiles (k_stencil_tiles.cu);
// cudaErrorNotSupported (nothing launched) where that form does not apply.
cudaError_t launch_stencil2d_tiles(const void* in, float* out, uint64_t nx, uint64_t ny, float c0,
                                   float c1, unsigned teams, unsigned threads, uint32_t* status,
                                   cudaStream_t st);

// static(c) 2-D stencil with the team's rows staged through a ring in shared
// memory (k_stencil_rows.cu): c in [4, 8) and [32, 128], where it beats the
// plain form; cudaErrorNotSupported (nothing launched) elsewhere.
cudaError_t launch_stencil2d_rows(const void* in, float* out, uint64_t nx, uint64_t ny,
                                  uint64_t chunk, float c0, float c1, unsigned teams,
                                  unsigned threads, int max_smem, uint32_t* status,
                                  cudaStream_t st);

// static, static(c) and dynamic(c) 2-D stencil with each team's rows staged
// in shared memory by bulk copies, `budget` bytes per CTA
// (k_stencil_owner.cu); cudaErrorNotSupported (nothing launched) where that
// form does not apply.
cudaError_t launch_stencil2d_owner(const void* in, float* out, uint64_t nx, uint64_t ny, int sched,
                                   uint64_t chunk, float c0, float c1, unsigned teams,
                                   unsigned threads, uint32_t budget, int sm_count, int max_smem,
                                   uint32_t* status, cudaStream_t st);

// static(c) and dynamic(c) 2-D stencil with teams of one warp whose blocks are
// the 32 / m rows that hold 32 chunks (m = nx / c < 32): the CTA's warps play
// adjacent teams, one tensor copy a step for all of them (k_stencil_colring.cu); cudaErrorNotSupported
// (nothing launched) for other launches.
cudaError_t launch_stencil2d_colring(const void* in, float* out, uint64_t nx, uint64_t ny,
                                     int sched, uint64_t chunk, float c0, float c1,
                                     unsigned teams, unsigned threads, uint32_t buffers,
                                     int sm_count, int max_smem, uint32_t* status,
                                     cudaStream_t st);

// static(c) and dynamic(c) 2-D stencil, c a multiple of 16 dividing nx, team
// blocks of whole rows: each warp's chunks arrive slab by slab as swizzled
// tensor copies (k_stencil_slabs.cu); cudaErrorNotSupported (nothing
// launched) for other launches.
cudaError_t launch_stencil2d_slabs(const void* in, float* out, uint64_t nx, uint64_t ny, int sched,
                                   uint64_t chunk, float c0, float c1, unsigned teams,
                                   unsigned threads, uint32_t slab_floats, uint32_t buffers,
                                   int sm_count, int max_smem, uint32_t* status,
                                   cudaStream_t st);

// dynamic(c) 2-D stencil, team blocks of whole rows, streamed through a ring
// of row slots in shared memory, `budget` bytes per CTA
// (k_stencil_rowring.cu); cudaErrorNotSupported (nothing launched) for other
// launches.
cudaError_t launch_stencil2d_rowring(const void* in, float* out, uint64_t nx, uint64_t ny,
                                     int sched, uint64_t chunk, float c0, float c1,
                                     unsigned teams, unsigned threads, uint32_t budget,
                                     int sm_count, int max_smem, uint32_t* status,
                                     cudaStream_t st);

// static(1) 2-D stencil, team size dividing nx, team blocks of whole rows:
// each warp's strips a band of rows at a time from tensor copies
// (k_stencil_bands.cu); cudaErrorNotSupported (nothing launched) for other
// launches.
cudaError_t launch_stencil2d_bands(const void* in, float* out, uint64_t nx, uint64_t ny, float c0,
                                   float c1, unsigned teams, unsigned threads, uint32_t buffers,
                                   int sm_count, int max_smem, uint32_t* status,
                                   cudaStream_t st);

// static(1), static(4/8) and static 2-D stencil whose owner map repeats row
// by row, walked as vertical strips (k_stencil_strips.cu);
// cudaErrorNotSupported (nothing launched) for other launches.
cudaError_t launch_stencil2d_strips(const void* in, float* out, uint64_t nx, uint64_t ny, int sched,
                                    uint64_t chunk, float c0, float c1, unsigned teams,
                                    unsigned threads, int sm_count, cudaStream_t st);

// Support kernels (k_support.cu).
cudaError_t launch_static_table(uint64_t n, int64_t lb, int64_t incr, uint64_t chunk, unsigned G,
                                unsigned T, int64_t* table, cudaStream_t st);
cudaError_t launch_test_atomics(unsigned G, unsigned T, int reps, uint32_t e, uint32_t* words,
                                uint32_t* returned, uint32_t* status, cudaStream_t st);
cudaError_t launch_test_barrier(unsigned G, unsigned T, unsigned sub, int rounds, uint32_t* errors,
                                cudaStream_t st);
cudaError_t launch_test_wait(unsigned G, const uint32_t* flag, uint32_t expect, uint64_t max_ns,
                             int32_t* out, uint32_t* status, cudaStream_t st);
cudaError_t launch_test_stack(unsigned G, uint32_t S, uint32_t Q, unsigned char* pool,
                              const int64_t* ops, int64_t nops, int64_t* out, int64_t* status_out,
                              uint32_t* status, cudaStream_t st);

}  // namespace rt
