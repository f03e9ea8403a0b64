// Support kernels: the static worksharing table, and device self-tests of the
// runtime atomics, team barriers and the team shared-memory stack.
#include "launch.h"

namespace rt {

__device__ __forceinline__ int64_t wadd(int64_t a, int64_t b) {
  return (int64_t)((uint64_t)a + (uint64_t)b);
}
__device__ __forceinline__ int64_t wmul(uint64_t a, int64_t b) {
  return (int64_t)(a * (uint64_t)b);
}

// One thread per (team g, thread t): the tuple __kmpc_for_static_init would
// return at both levels of the composite construct.
__global__ void static_table_kernel(uint64_t n, int64_t lb, int64_t incr, uint64_t chunk,
                                    uint32_t G, uint32_t T, int64_t* table) {
  const uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (uint64_t)G * T) return;
  const uint32_t g = (uint32_t)(row / T), t = (uint32_t)(row % T);
  uint64_t bs, bn;
  split_even(n, G, g, bs, bn);
  int64_t* r = table + 8 * row;
  // level 1: team block over [0, n)
  {
    const uint64_t s = bn ? bs : n;
    const int64_t LB = wadd(lb, wmul(s, incr));
    r[0] = LB;
    r[1] = bn ? wadd(LB, wmul(bn - 1, incr)) : wadd(LB, -incr);
    r[2] = wmul(n, incr);
    r[3] = (bn > 0 && bs + bn == n) ? 1 : 0;
  }
  // level 2: thread t inside the block
  uint64_t s, cnt;
  int64_t stride;
  bool last;
  if (chunk == 0) {
    split_even(bn, T, t, s, cnt);
    stride = wmul(bn, incr);
    last = cnt > 0 && s + cnt == bn;
  } else {
    const uint64_t nch = bn ? (bn - 1) / chunk + 1 : 0;
    if (t < nch) {
      s = (uint64_t)t * chunk;
      cnt = bn - s > chunk ? chunk : bn - s;
    } else {
      s = bn;
      cnt = 0;
    }
    stride = wmul((uint64_t)T * chunk, incr);
    last = nch > 0 && (nch - 1) % T == t;
  }
  if (cnt == 0) s = bn;
  const int64_t LB = wadd(lb, wmul(bs + s, incr));
  r[4] = LB;
  r[5] = cnt ? wadd(LB, wmul(cnt - 1, incr)) : wadd(LB, -incr);
  r[6] = stride;
  r[7] = last ? 1 : 0;
}

cudaError_t launch_static_table(uint64_t n, int64_t lb, int64_t incr, uint64_t chunk, unsigned G,
                                unsigned T, int64_t* table, cudaStream_t st) {
  const uint64_t rows = (uint64_t)G * T;
  const unsigned blocks = (unsigned)((rows + 255) / 256);
  static_table_kernel<<<blocks, 256, 0, st>>>(n, lb, incr, chunk, G, T, table);
  return cudaGetLastError();
}

// Each thread applies the five atomics `reps` times.  The cas word is used
// as a counter advanced by a bounded cas loop.
__global__ void test_atomics_kernel(int reps, uint32_t e, uint32_t* w, uint32_t* returned,
                                    uint32_t* status) {
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int r = 0; r < reps; ++r) {
    atomic_add(&w[0], 1u);
    const uint32_t v = atomic_inc(&w[1], e);
    if (returned) returned[(uint64_t)gid * reps + r] = v;
    atomic_max(&w[2], gid);
    atomic_exchange(&w[3], gid);
    bool done = false;
    for (int tries = 0; tries < (1 << 20) && !done; ++tries) {
      const uint32_t old = *(volatile uint32_t*)&w[4];
      done = atomic_cas(&w[4], old, old + 1u) == old;
    }
    if (!done) set_status(status, OMPRT_DEV_TIMEOUT);
  }
}

cudaError_t launch_test_atomics(unsigned G, unsigned T, int reps, uint32_t e, uint32_t* words,
                                uint32_t* returned, uint32_t* status, cudaStream_t st) {
  test_atomics_kernel<<<G, T, 0, st>>>(reps, e, words, returned, status);
  return cudaGetLastError();
}

// Barrier invariant: after a barrier every thread sees every slot at the
// current round; a second barrier keeps the next round's writes out.
__global__ void test_barrier_kernel(uint32_t sub, int rounds, uint32_t* errors) {
  extern __shared__ uint32_t slots[];
  const uint32_t t = threadIdx.x, T = blockDim.x;
  uint32_t bad = 0;
  for (int r = 1; r <= rounds; ++r) {
    slots[t] = (uint32_t)r;
    team_barrier();
    for (uint32_t k = 0; k < T; ++k) bad += slots[(t + k) % T] != (uint32_t)r;
    team_barrier();
  }
  if (sub) {
    // sub-teams of `sub` threads, each on its own named barrier 1 .. T/sub
    const uint32_t team = t / sub, base = team * sub, id = 1 + team;
    for (int r = 1; r <= rounds; ++r) {
      slots[t] = (uint32_t)(1000 + r + team);
      named_barrier(id, sub);
      for (uint32_t k = 0; k < sub; ++k)
        bad += slots[base + (t - base + k) % sub] != (uint32_t)(1000 + r + team);
      named_barrier(id, sub);
    }
  }
  if (bad) atomicAdd(errors, bad);
}

cudaError_t launch_test_barrier(unsigned G, unsigned T, unsigned sub, int rounds, uint32_t* errors,
                                cudaStream_t st) {
  test_barrier_kernel<<<G, T, T * sizeof(uint32_t), st>>>(sub, rounds, errors);
  return cudaGetLastError();
}

// Trace replay through the team stack, serialised in thread 0 of each team.
// A free names the op index of the alloc whose block it releases.
__global__ void test_stack_kernel(uint32_t S, uint32_t Q, unsigned char* pool, const int64_t* ops,
                                  int64_t nops, int64_t* out, int64_t* status_out,
                                  uint32_t* status) {
  if (threadIdx.x != 0) return;
  const uint32_t g = blockIdx.x;
  unsigned char* slice = pool ? pool + (uint64_t)g * Q : nullptr;
  stack_init(S, slice, Q);
  int64_t* o = out + 2 * nops * (int64_t)g;
  int64_t st = 0;
  for (int64_t i = 0; i < nops; ++i) {
    const int64_t kind = ops[2 * i], arg = ops[2 * i + 1];
    if (kind == 0) {
      void* p = alloc_shared((uint64_t)arg, status);
      int64_t reg = 2, off = 0;
      if (p) {
        reg = stack_region(p);
        off = reg == 0 ? (const unsigned char*)p - rt_dyn_smem
                       : (const unsigned char*)p - slice;
      } else {
        st |= OMPRT_DEV_STACK_NOMEM;
      }
      o[2 * i] = reg;
      o[2 * i + 1] = off;
    } else {
      int64_t bits = 0;
      if (arg < 0 || arg >= i || ops[2 * arg] != 0) {
        bits = OMPRT_DEV_STACK_ORDER;
        set_status(status, OMPRT_DEV_STACK_ORDER);
      } else {
        const int64_t reg = o[2 * arg], off = o[2 * arg + 1];
        if (reg != 2) {
          void* p = reg == 0 ? (void*)(rt_dyn_smem + off) : (void*)(slice + off);
          bits = free_shared(p, (uint64_t)ops[2 * arg + 1], status);
        }
      }
      st |= bits;
      o[2 * i] = bits;
      o[2 * i + 1] = 0;
    }
  }
  status_out[g] = st;
}

cudaError_t launch_test_stack(unsigned G, uint32_t S, uint32_t Q, unsigned char* pool,
                              const int64_t* ops, int64_t nops, int64_t* out, int64_t* status_out,
                              uint32_t* status, cudaStream_t st) {
  static const size_t static_bytes = static_smem_of(test_stack_kernel);
  const cudaError_t e = smem_optin(test_stack_kernel, S, static_bytes);
  if (e != cudaSuccess) return e;
  test_stack_kernel<<<G, 32, S, st>>>(S, Q, pool, ops, nops, out, status_out, status);
  return cudaGetLastError();
}

// One thread per team waits on a flag; out[g] = 1 if it was seen, 0 on timeout.
__global__ void test_wait_kernel(const uint32_t* flag, uint32_t expect, uint64_t max_ns,
                                 int32_t* out, uint32_t* status) {
  if (threadIdx.x != 0) return;
  out[blockIdx.x] = bounded_wait_eq(flag, expect, max_ns, status) ? 1 : 0;
}

cudaError_t launch_test_wait(unsigned G, const uint32_t* flag, uint32_t expect, uint64_t max_ns,
                             int32_t* out, uint32_t* status, cudaStream_t st) {
  test_wait_kernel<<<G, 32, 0, st>>>(flag, expect, max_ns, out, status);
  return cudaGetLastError();
}

}  // namespace rt
