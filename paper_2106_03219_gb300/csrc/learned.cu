// Learned schedule selection (host side): the 12 candidate configurations, the
// 16 loop features, and inference of the installed cost model with the plain
// heuristic as fallback.  The model itself is trained by the MLP kernels.
#include <cmath>
#include <cstring>

#include "api_internal.h"

namespace {

// {static c=1, static c=8, static no chunk, dynamic c=256, auto, auto T=1024}
// x {teams = SMs, teams = 4 x SMs}; 256 threads unless stated.
const LearnedConfig kConfigs[12] = {
    {OMPRT_SCHED_STATIC_CHUNKED, 1, 1, 256}, {OMPRT_SCHED_STATIC_CHUNKED, 1, 4, 256},
    {OMPRT_SCHED_STATIC_CHUNKED, 8, 1, 256}, {OMPRT_SCHED_STATIC_CHUNKED, 8, 4, 256},
    {OMPRT_SCHED_STATIC, 0, 1, 256},         {OMPRT_SCHED_STATIC, 0, 4, 256},
    {OMPRT_SCHED_DYNAMIC, 256, 1, 256},      {OMPRT_SCHED_DYNAMIC, 256, 4, 256},
    {OMPRT_SCHED_AUTO, 0, 1, 256},           {OMPRT_SCHED_AUTO, 0, 4, 256},
    {OMPRT_SCHED_AUTO, 0, 1, 1024},          {OMPRT_SCHED_AUTO, 0, 4, 1024},
};
// The plain heuristic: auto mapping, 4 teams per SM, 256 threads.
constexpr int kHeuristic = 9;

int body_kind(int32_t body) {
  switch (body) {
    case OMPRT_BODY_AXPY: return 0;
    case OMPRT_BODY_DOT: return 1;
    case OMPRT_BODY_STENCIL1D3: return 2;
    case OMPRT_BODY_STENCIL2D5: return 3;
    case OMPRT_BODY_NONE: return 4;
  }
  return -1;
}

double dtype_bytes(int32_t t) {
  switch (t) {
    case OMPRT_BF16: return 2;
    case OMPRT_I64: case OMPRT_U64: case OMPRT_F64: return 8;
  }
  return 4;
}

}  // namespace

LearnedConfig learned_config(int k) { return kConfigs[k]; }

extern "C" {

omprt_status omprt_learned_configs(int32_t* sched, int64_t* chunk, int32_t* tps, int32_t* thr) {
  for (int k = 0; k < 12; ++k) {
    if (sched) sched[k] = kConfigs[k].sched;
    if (chunk) chunk[k] = kConfigs[k].chunk;
    if (tps) tps[k] = kConfigs[k].teams_per_sm;
    if (thr) thr[k] = kConfigs[k].threads;
  }
  return OMPRT_OK;
}

omprt_status omprt_set_cost_model(omprt_ctx* c, const float* params, const float* mean,
                                  const float* stdv) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!params) {
    c->has_model = false;
    return OMPRT_OK;
  }
  if (!mean || !stdv) return OMPRT_ERR_INVALID;
  std::memcpy(c->model, params, sizeof(c->model));
  std::memcpy(c->feat_mean, mean, sizeof(c->feat_mean));
  std::memcpy(c->feat_std, stdv, sizeof(c->feat_std));
  c->has_model = true;
  return OMPRT_OK;
}

// Features: log2 n, bytes/iter, flops/iter, one-hot kind (axpy, dot,
// stencil1d3, stencil2d5, reduce), reduction flag, element bytes,
// log2(n * bytes/iter), n / (SMs * 1024), log2(L2 bytes / (n * bytes/iter)),
// three zeros.
omprt_status omprt_loop_features(const omprt_ctx* c, const omprt_loop_desc* d, int32_t has_red,
                                 float* f) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!d || !f) return OMPRT_ERR_INVALID;
  uint64_t n;
  int64_t lb;
  omprt_status s = loop_trip_count(d, &n, &lb);
  if (s) return s;
  const int kind = body_kind(d->body);
  const double eb = dtype_bytes(d->data_type);
  double bpi, fpi;
  switch (kind) {
    case 0: bpi = 3 * eb; fpi = 2; break;
    case 1: bpi = 2 * eb; fpi = 2; break;
    case 2: bpi = 2 * eb; fpi = 4; break;
    case 3: bpi = 2 * eb; fpi = 6; break;
    case 4: bpi = eb; fpi = 1; break;
    default: bpi = 4; fpi = 0; break;
  }
  const double nn = n ? (double)n : 1.0;
  std::memset(f, 0, sizeof(float) * OMPRT_MLP_IN);
  f[0] = (float)std::log2(nn);
  f[1] = (float)bpi;
  f[2] = (float)fpi;
  if (kind >= 0) f[3 + kind] = 1.f;
  f[8] = has_red ? 1.f : 0.f;
  f[9] = (float)eb;
  f[10] = (float)std::log2(nn * bpi);
  f[11] = (float)(nn / ((double)c->sm_count * 1024.0));
  f[12] = (float)std::log2((double)c->l2_bytes / (nn * bpi));
  return OMPRT_OK;
}

omprt_status omprt_choose_config(const omprt_ctx* c, const omprt_loop_desc* d, int32_t has_red,
                                 int32_t* out) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!out) return OMPRT_ERR_INVALID;
  *out = kHeuristic;
  if (!c->has_model) return OMPRT_OK;
  float f[OMPRT_MLP_IN];
  omprt_status s = omprt_loop_features(c, d, has_red, f);
  if (s) return s;
  for (int i = 0; i < OMPRT_MLP_IN; ++i)
    f[i] = (f[i] - c->feat_mean[i]) / (c->feat_std[i] > 0.f ? c->feat_std[i] : 1.f);
  const float* W1 = c->model;
  const float* b1 = W1 + OMPRT_MLP_HID * OMPRT_MLP_IN;
  const float* W2 = b1 + OMPRT_MLP_HID;
  const float* b2 = W2 + OMPRT_MLP_HID * OMPRT_MLP_HID;
  const float* W3 = b2 + OMPRT_MLP_HID;
  const float* b3 = W3 + OMPRT_MLP_OUT * OMPRT_MLP_HID;
  float h1[OMPRT_MLP_HID], h2[OMPRT_MLP_HID];
  for (int o = 0; o < OMPRT_MLP_HID; ++o) {
    float s1 = b1[o];
    for (int i = 0; i < OMPRT_MLP_IN; ++i) s1 += W1[o * OMPRT_MLP_IN + i] * f[i];
    h1[o] = s1 > 0.f ? s1 : 0.f;
  }
  for (int o = 0; o < OMPRT_MLP_HID; ++o) {
    float s2 = b2[o];
    for (int i = 0; i < OMPRT_MLP_HID; ++i) s2 += W2[o * OMPRT_MLP_HID + i] * h1[i];
    h2[o] = s2 > 0.f ? s2 : 0.f;
  }
  int best = -1;
  float bv = 0.f;
  for (int o = 0; o < OMPRT_MLP_OUT; ++o) {
    float y = b3[o];
    for (int i = 0; i < OMPRT_MLP_HID; ++i) y += W3[o * OMPRT_MLP_HID + i] * h2[i];
    if (!std::isfinite(y)) return OMPRT_OK;  // heuristic
    if (best < 0 || y < bv) {
      best = o;
      bv = y;
    }
  }
  *out = best;
  return OMPRT_OK;
}

}  // extern "C"
