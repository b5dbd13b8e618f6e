// Launch-parameter selection on the host.
//
// 1. The learned predictor: the fp32 MLP of mlp.cu evaluated on the CPU with
//    the same multiply-add order (so it reproduces the GPU forward pass
//    bit for bit), its weights read from a file written by the training
//    driver.  Outputs are rounded to the parameter grid.
// 2. The paper's rule (Sec. 2.4): the sum model of Eq. 4 and the overhead
//    models of Eq. 7 fed into the optimum condition of Eq. 6, over
//    S in {1, 2, 4, 8, 16, 32} (Sec. 2.1).  Coefficients default to the
//    paper's RTX 2080 Ti fit and can be refit for this machine.
#include <dlfcn.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "tps_internal.h"

namespace {

constexpr int kIn = TPS_MLP_IN, kH = TPS_MLP_HIDDEN, kOut = TPS_MLP_OUT;
constexpr int kN = TPS_MLP_NPARAMS;

struct Weights {
  bool loaded = false;
  bool tried = false;
  float fmean[kIn], fscale[kIn];  // feature normalisation: (f - mean) * scale
  float oscale[kOut];             // output y * oscale = log2 of (m, S, chunk)
  float p[kN];
};

Weights g_w;
std::mutex g_mu;

// File layout: "TPSMLP1\0", int32 nparams, fmean[4], fscale[4], oscale[3],
// params[nparams] (all little-endian fp32).
bool read_weights(const char* path, Weights& w) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  char magic[8];
  int32_t np = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "TPSMLP1", 8) == 0 &&
            std::fread(&np, 4, 1, f) == 1 && np == kN &&
            std::fread(w.fmean, 4, kIn, f) == (size_t)kIn &&
            std::fread(w.fscale, 4, kIn, f) == (size_t)kIn &&
            std::fread(w.oscale, 4, kOut, f) == (size_t)kOut &&
            std::fread(w.p, 4, kN, f) == (size_t)kN;
  std::fclose(f);
  return ok;
}

// Weights: $TPS_PREDICTOR_WEIGHTS, else predictor/weights.bin next to libtps.so.
const Weights* weights() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_w.tried) {
    g_w.tried = true;
    std::string path;
    if (const char* e = std::getenv("TPS_PREDICTOR_WEIGHTS")) {
      path = e;
    } else {
      Dl_info info;
      if (dladdr((void*)&read_weights, &info) && info.dli_fname) {
        path = info.dli_fname;
        const size_t cut = path.find_last_of('/');
        path = (cut == std::string::npos ? std::string(".") : path.substr(0, cut)) +
               "/predictor/weights.bin";
      }
    }
    g_w.loaded = !path.empty() && read_weights(path.c_str(), g_w);
  }
  return g_w.loaded ? &g_w : nullptr;
}

// One layer, same accumulation order as the GPU kernel k_linear.
void linear(const float* x, int in, int out, const float* W, const float* b, float* z,
            bool relu) {
  for (int o = 0; o < out; ++o) {
    float s = b[o];
    for (int i = 0; i < in; ++i) s = std::fmaf(x[i], W[o * in + i], s);
    z[o] = relu ? (s > 0.0f ? s : 0.0f) : s;
  }
}

int clamp_pow2(double lg, int lo, int hi) {
  double r = std::nearbyint(lg);
  if (r < lo) r = lo;
  if (r > hi) r = hi;
  return (int)r;
}

}  // namespace

extern "C" {

void tps_mlp_forward_host(const float* params, const float* x, float* y) {
  float h1[kH], h2[kH];
  const float* p = params;
  linear(x, kIn, kH, p, p + kH * kIn, h1, true);
  p += kH * kIn + kH;
  linear(h1, kH, kH, p, p + kH * kH, h2, true);
  p += kH * kH + kH;
  linear(h2, kH, kOut, p, p + kOut * kH, y, false);
}

int tps_predict_params(const tps_plan_desc* desc, int32_t* m, int32_t* streams,
                       int64_t* chunk) {
  if (!desc || !m || !streams || !chunk) return 2;
  const Weights* w = weights();
  if (!w) return 1;
  const double n = desc->n_max > 1 ? (double)desc->n_max : 2.0;
  const double batch = desc->batch_max > 1 ? (double)desc->batch_max : 1.0;
  const float f[kIn] = {(float)std::log2(n), (float)std::log2(batch),
                        desc->dtype == TPS_F32 ? 1.0f : 0.0f,
                        desc->residency == TPS_HOST_PINNED ? 1.0f : 0.0f};
  float x[kIn], y[kOut];
  for (int i = 0; i < kIn; ++i) x[i] = (f[i] - w->fmean[i]) * w->fscale[i];
  tps_mlp_forward_host(w->p, x, y);
  *m = 1 << clamp_pow2(y[0] * w->oscale[0], 3, 10);
  *streams = 1 << clamp_pow2(y[1] * w->oscale[1], 0, 5);
  const int lc = clamp_pow2(y[2] * w->oscale[2], 10, 40);
  int64_t c = (int64_t)1 << lc;
  // one chunk per stream when the chunk exceeds n; and on a single stream
  // chunks run back to back with nothing to overlap, so none at all
  if (c > (int64_t)n || *streams == 1) c = 0;
  *chunk = c;
  return 0;
}

int tps_predict_available(void) { return weights() ? 1 : 0; }

int tps_predict_load(const char* path) {
  if (!path) return 2;
  Weights w;
  if (!read_weights(path, w)) return 1;
  std::lock_guard<std::mutex> lk(g_mu);
  std::memcpy(g_w.fmean, w.fmean, sizeof(w.fmean));
  std::memcpy(g_w.fscale, w.fscale, sizeof(w.fscale));
  std::memcpy(g_w.oscale, w.oscale, sizeof(w.oscale));
  std::memcpy(g_w.p, w.p, sizeof(w.p));
  g_w.loaded = true;
  g_w.tried = true;
  return 0;
}

int32_t tps_paper_predict_streams(double size, const double* sum_model, const double* small,
                                  const double* big, double split) {
  // Eq. 4 and Eq. 7 with the paper's RTX 2080 Ti coefficients by default
  static const double kSum[2] = {2.1890017149e-6, 0.1470644998564126};
  static const double kSmall[3] = {2.245645331e-7, 0.6009426920043296, -0.0605183610625299};
  static const double kBig[3] = {3.56594859e-8, 0.0522781620855163, 0.3941472844770443};
  const double* sm = sum_model ? sum_model : kSum;
  const double* ps = small ? small : kSmall;
  const double* pb = big ? big : kBig;
  if (!(split > 0.0)) split = 1e6;
  const double sum = sm[0] * size + sm[1];
  int32_t best = 1;
  double best_slack = 0.0;
  bool any = false;
  for (int32_t S = 1; S <= 32; S *= 2) {
    const double ov = size <= split ? ps[0] * size + ps[1] * std::log10((double)S) + ps[2]
                                    : (pb[0] * size + pb[1]) * (4.0 / 3.0) *
                                              std::log2((double)S) +
                                          pb[2];
    const double rhs = (double)(S - 1) / S * sum;
    if (ov < rhs) {
      const double slack = rhs - ov;
      if (!any || slack > best_slack) {
        best = S;
        best_slack = slack;
        any = true;
      }
    }
  }
  return best;
}

}  // extern "C"
