// MLP cost model 16 -> 64 -> 64 -> 12 (fp32): forward, loss + gradient, Adam.
//
// Kernel A runs one sample per warp: the forward pass, and for training the
// output error and the back-propagated deltas, which it leaves in a per-sample
// scratch row.  Kernel B gives each parameter one thread that sums its
// gradient over the batch in sample order (deterministic, no atomics).
// Weights sit in shared memory with rows padded to an odd stride, so both the
// forward (row) and backward (column) reads are free of bank conflicts.
#include <cmath>

#include "api_internal.h"

namespace rt {

constexpr int kIn = OMPRT_MLP_IN, kHid = OMPRT_MLP_HID, kOut = OMPRT_MLP_OUT;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid,
              kOffB3 = kOffW3 + kOut * kHid, kNParam = kOffB3 + kOut;
static_assert(kNParam == OMPRT_MLP_NPARAM, "parameter layout");

// per-sample scratch row: h1, h2, dh1, dh2 (64 each), dy (12), loss term
constexpr int kRowH1 = 0, kRowH2 = 64, kRowD1 = 128, kRowD2 = 192, kRowDy = 256, kRowLoss = 268;
constexpr int kRowStride = 272;
constexpr int kWarps = 8;

// Padded strides: 17 and 65 are odd, so lane u reading row u and lane i
// reading column i both touch 32 different banks.
constexpr int kP1 = kIn + 1, kP2 = kHid + 1;

struct MlpShared {
  float w1[kHid * kP1];
  float w2[kHid * kP2];
  float w3[kOut * kP2];
  float b1[kHid], b2[kHid], b3[kOut];
  float h1[kWarps][kHid], h2[kWarps][kHid], d2[kWarps][kHid], y[kWarps][16];
};

__device__ void load_weights(MlpShared& S, const float* p) {
  for (int k = threadIdx.x; k < kHid * kIn; k += blockDim.x)
    S.w1[(k / kIn) * kP1 + k % kIn] = p[kOffW1 + k];
  for (int k = threadIdx.x; k < kHid * kHid; k += blockDim.x)
    S.w2[(k / kHid) * kP2 + k % kHid] = p[kOffW2 + k];
  for (int k = threadIdx.x; k < kOut * kHid; k += blockDim.x)
    S.w3[(k / kHid) * kP2 + k % kHid] = p[kOffW3 + k];
  for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
    S.b1[k] = p[kOffB1 + k];
    S.b2[k] = p[kOffB2 + k];
  }
  for (int k = threadIdx.x; k < kOut; k += blockDim.x) S.b3[k] = p[kOffB3 + k];
}

// train == false: write y; train == true: also the deltas and loss term.
template <bool kTrain>
__global__ void __launch_bounds__(kWarps * 32) mlp_sample_kernel(const float* __restrict__ p,
                                                                 const float* __restrict__ X,
                                                                 const float* __restrict__ Yt,
                                                                 int B, float scale,
                                                                 float* __restrict__ Y,
                                                                 float* __restrict__ rows) {
  __shared__ MlpShared S;
  load_weights(S, p);
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int b = blockIdx.x * kWarps + w; b < B; b += gridDim.x * kWarps) {
    float x[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) x[i] = X[(size_t)b * kIn + i];
    // layer 1: units l and l + 32
    float h1a = S.b1[l], h1b = S.b1[l + 32];
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
      h1a = __fmaf_rn(S.w1[l * kP1 + i], x[i], h1a);
      h1b = __fmaf_rn(S.w1[(l + 32) * kP1 + i], x[i], h1b);
    }
    h1a = fmaxf(h1a, 0.f);
    h1b = fmaxf(h1b, 0.f);
    S.h1[w][l] = h1a;
    S.h1[w][l + 32] = h1b;
    __syncwarp();
    // layer 2
    float h2a = S.b2[l], h2b = S.b2[l + 32];
    for (int k = 0; k < kHid; ++k) {
      const float hk = S.h1[w][k];
      h2a = __fmaf_rn(S.w2[l * kP2 + k], hk, h2a);
      h2b = __fmaf_rn(S.w2[(l + 32) * kP2 + k], hk, h2b);
    }
    h2a = fmaxf(h2a, 0.f);
    h2b = fmaxf(h2b, 0.f);
    S.h2[w][l] = h2a;
    S.h2[w][l + 32] = h2b;
    __syncwarp();
    // layer 3: lanes 0..11
    float yo = 0.f, dyo = 0.f, lt = 0.f;
    if (l < kOut) {
      yo = S.b3[l];
      for (int k = 0; k < kHid; ++k) yo = __fmaf_rn(S.w3[l * kP2 + k], S.h2[w][k], yo);
      if constexpr (!kTrain) {
        Y[(size_t)b * kOut + l] = yo;
      } else {
        const float d = __fsub_rn(yo, Yt[(size_t)b * kOut + l]);
        lt = __fmul_rn(d, d);
        dyo = __fmul_rn(__fmul_rn(2.f, d), scale);
        S.y[w][l] = dyo;
      }
    }
    if constexpr (kTrain) {
      __syncwarp();
      float* row = rows + (size_t)b * kRowStride;
      // loss term of this sample, summed over outputs in order by lane 0
      float ls = 0.f;
#pragma unroll
      for (int o = 0; o < kOut; ++o) ls = __fadd_rn(ls, __shfl_sync(0xffffffffu, lt, o));
      if (l == 0) row[kRowLoss] = ls;
      if (l < kOut) row[kRowDy + l] = dyo;
      // dh2 = relu'(h2) * W3^T dy
      float sa = 0.f, sb = 0.f;
      for (int o = 0; o < kOut; ++o) {
        const float dy = S.y[w][o];
        sa = __fmaf_rn(S.w3[o * kP2 + l], dy, sa);
        sb = __fmaf_rn(S.w3[o * kP2 + l + 32], dy, sb);
      }
      const float d2a = h2a > 0.f ? sa : 0.f, d2b = h2b > 0.f ? sb : 0.f;
      S.d2[w][l] = d2a;
      S.d2[w][l + 32] = d2b;
      __syncwarp();
      // dh1 = relu'(h1) * W2^T dh2
      float ta = 0.f, tb = 0.f;
      for (int k = 0; k < kHid; ++k) {
        const float dk = S.d2[w][k];
        ta = __fmaf_rn(S.w2[k * kP2 + l], dk, ta);
        tb = __fmaf_rn(S.w2[k * kP2 + l + 32], dk, tb);
      }
      row[kRowH1 + l] = h1a;
      row[kRowH1 + l + 32] = h1b;
      row[kRowH2 + l] = h2a;
      row[kRowH2 + l + 32] = h2b;
      row[kRowD1 + l] = h1a > 0.f ? ta : 0.f;
      row[kRowD1 + l + 32] = h1b > 0.f ? tb : 0.f;
      row[kRowD2 + l] = d2a;
      row[kRowD2 + l + 32] = d2b;
    }
    __syncwarp();
  }
}

// One thread per parameter: its gradient summed over the batch in order.
// The extra last thread sums the per-sample loss terms.
__global__ void mlp_grad_kernel(const float* __restrict__ X, const float* __restrict__ rows, int B,
                                float scale, float* __restrict__ grad, float* __restrict__ loss) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == kNParam) {
    if (loss) {
      float s = 0.f;
      for (int b = 0; b < B; ++b) s = __fadd_rn(s, rows[(size_t)b * kRowStride + kRowLoss]);
      *loss = __fmul_rn(s, scale);
    }
    return;
  }
  if (q > kNParam) return;
  int a_off, o, i = -1;  // delta column a_off + o times input column (i or bias)
  const float* in_base = nullptr;
  int in_stride = 0, in_off = 0;
  if (q < kOffB1) {
    o = q / kIn; i = q % kIn; a_off = kRowD1; in_base = X; in_stride = kIn; in_off = 0;
  } else if (q < kOffW2) {
    o = q - kOffB1; a_off = kRowD1;
  } else if (q < kOffB2) {
    const int r = q - kOffW2;
    o = r / kHid; i = r % kHid; a_off = kRowD2; in_base = rows; in_stride = kRowStride;
    in_off = kRowH1;
  } else if (q < kOffW3) {
    o = q - kOffB2; a_off = kRowD2;
  } else if (q < kOffB3) {
    const int r = q - kOffW3;
    o = r / kHid; i = r % kHid; a_off = kRowDy; in_base = rows; in_stride = kRowStride;
    in_off = kRowH2;
  } else {
    o = q - kOffB3; a_off = kRowDy;
  }
  float s = 0.f;
  if (i < 0) {
    for (int b = 0; b < B; ++b) s = __fadd_rn(s, rows[(size_t)b * kRowStride + a_off + o]);
  } else {
    for (int b = 0; b < B; ++b)
      s = __fmaf_rn(rows[(size_t)b * kRowStride + a_off + o],
                    in_base[(size_t)b * in_stride + in_off + i], s);
  }
  grad[q] = s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = __fadd_rn(__fmul_rn(b1, m[k]), __fmul_rn(__fsub_rn(1.f, b1), gk));
  const float vk =
      __fadd_rn(__fmul_rn(b2, v[k]), __fmul_rn(__fmul_rn(__fsub_rn(1.f, b2), gk), gk));
  m[k] = mk;
  v[k] = vk;
  const float mh = __fdiv_rn(mk, c1), vh = __fdiv_rn(vk, c2);
  p[k] = __fsub_rn(p[k], __fdiv_rn(__fmul_rn(lr, mh), __fadd_rn(__fsqrt_rn(vh), eps)));
}

}  // namespace rt

using namespace rt;

namespace {
constexpr int kMaxBatch = kMlpMaxBatch;
static_assert(kRowStride == kMlpRowFloats, "scratch row size");

// Per-sample scratch rows live in the context (allocated by omprt_init).
float* mlp_rows(omprt_ctx* c) { return c->mlp_rows_dev; }
}  // namespace

extern "C" {

omprt_status omprt_mlp_forward(omprt_ctx* c, const float* params, const float* x, int32_t B,
                               float* y, void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!params || B < 0 || (B && (!x || !y))) return OMPRT_ERR_INVALID;
  if (B == 0) return OMPRT_OK;
  DeviceGuard guard(c->device);
  const int grid = (B + kWarps - 1) / kWarps;
  mlp_sample_kernel<false><<<grid < 1024 ? grid : 1024, kWarps * 32, 0, (cudaStream_t)stream>>>(
      params, x, nullptr, B, 0.f, y, nullptr);
  return cudaGetLastError() == cudaSuccess ? OMPRT_OK : OMPRT_ERR_CUDA;
}

omprt_status omprt_mlp_loss_grad(omprt_ctx* c, const float* params, const float* x,
                                 const float* target, int32_t B, float* grad, float* loss,
                                 void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!params || !x || !target || !grad || B < 1 || B > kMaxBatch) return OMPRT_ERR_INVALID;
  DeviceGuard guard(c->device);
  const float scale = 1.0f / ((float)B * kOut);
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = (B + kWarps - 1) / kWarps;
  mlp_sample_kernel<true><<<grid < 1024 ? grid : 1024, kWarps * 32, 0, st>>>(
      params, x, target, B, scale, nullptr, mlp_rows(c));
  mlp_grad_kernel<<<(kNParam + 1 + 255) / 256, 256, 0, st>>>(x, mlp_rows(c), B, scale, grad, loss);
  return cudaGetLastError() == cudaSuccess ? OMPRT_OK : OMPRT_ERR_CUDA;
}

omprt_status omprt_mlp_adam(omprt_ctx* c, float* params, const float* grad, float* m, float* v,
                            int32_t n, int32_t t, float lr, float beta1, float beta2, float eps,
                            void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!params || !grad || !m || !v || n < 1 || t < 1) return OMPRT_ERR_INVALID;
  DeviceGuard guard(c->device);
  const float c1 = (float)(1.0 - std::pow((double)beta1, (double)t));
  const float c2 = (float)(1.0 - std::pow((double)beta2, (double)t));
  adam_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, lr, beta1,
                                                                 beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? OMPRT_OK : OMPRT_ERR_CUDA;
}

}  // extern "C"
