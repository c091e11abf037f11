// dc_smooth.cu -- the Gaussian filter layer on the learned redundancy weight
// (Ye et al., DRACO, Sec. 3.1: sigma 20, kernel size 121), and its transpose
// for the reverse mode.
//
// Per view the weight map W[mu][k] is filtered along mu and along s over the
// valid half-grid entries k < n_s - 1 (entry n_s - 1 is unused by the filter
// chain and passes through).  Taps exp(-t^2 / (2 sigma^2)), |t| <= radius,
// normalised to unit sum; each line is extended by mirroring about its end
// samples (index -1 reads 1, index n reads n - 2, repeated for short lines).
// The two axis filters act on different axes and commute.
//
// One kernel serves both axes: a CTA stages `cw` neighbouring lines of one
// view in shared memory (cw = 16 columns for the mu axis, whose elements are
// n_s apart; one contiguous row for the s axis).  The forward pass gathers
// from a mirror-extended copy of the line; the transpose computes the
// zero-padded correlation c(p) for every extended position p and folds it
// back onto the sample p mirrors to.
#include <algorithm>
#include <cmath>
#include <string>

#include "dc_common.cuh"

namespace {

constexpr int SM_THREADS = 256;
constexpr size_t SM_SMEM_BUDGET = 200 * 1024;

struct SmoothLines {
  const float *in;
  float *out;
  int n;            // samples per line
  int lines;        // lines per view
  size_t vstride;   // floats between views
  int es;           // floats between samples of a line
  int ls;           // floats between neighbouring lines
  int lcw;          // log2 of the lines per CTA
  int R;            // radius
  float sigma;
  int adjoint;
};

__device__ __forceinline__ int mirror_of(int p, int n) {
  if (n == 1) return 0;
  const int T = 2 * (n - 1);
  p %= T;
  if (p < 0) p += T;
  return p < n ? p : T - p;
}

__global__ void __launch_bounds__(SM_THREADS) k_smooth_lines(SmoothLines a) {
  extern __shared__ float sm[];
  const int R = a.R, n = a.n, cw = 1 << a.lcw, cm = cw - 1;
  const int ntap = 2 * R + 1;
  float *w = sm;                              // taps
  float *xe = sm + ((ntap + 3) & ~3);         // staged lines
  const int v = blockIdx.y, l0 = blockIdx.x * cw;
  const float *src = a.in + (size_t)v * a.vstride + (size_t)l0 * a.ls;
  float *dst = a.out + (size_t)v * a.vstride + (size_t)l0 * a.ls;
  const int tid = threadIdx.x;

  for (int t = tid; t < ntap; t += SM_THREADS) {
    const float d = (float)(t - R);
    w[t] = expf(-0.5f * d * d / (a.sigma * a.sigma));
  }
  __syncthreads();
  if (tid == 0) {  // normalise to unit sum (one thread: at most a few thousand taps)
    float s = 0.0f;
    for (int t = 0; t < ntap; ++t) s += w[t];
    const float inv = 1.0f / s;
    for (int t = 0; t < ntap; ++t) w[t] *= inv;
  }

  if (!a.adjoint) {
    // xe[(p + R) * cw + c] = line c at mirror(p), p in [-R, n - 1 + R]
    const int ne = n + 2 * R;
    for (int idx = tid; idx < ne * cw; idx += SM_THREADS) {
      const int pp = idx >> a.lcw, c = idx & cm;
      float val = 0.0f;
      if (l0 + c < a.lines) val = src[(size_t)mirror_of(pp - R, n) * a.es + (size_t)c * a.ls];
      xe[idx] = val;
    }
    __syncthreads();
    for (int idx = tid; idx < n * cw; idx += SM_THREADS) {
      const int i = idx >> a.lcw, c = idx & cm;
      if (l0 + c >= a.lines) continue;
      const float *x = xe + (size_t)i * cw + c;
      float acc = 0.0f;
      for (int t = 0; t < ntap; ++t) acc = fmaf(w[t], x[t * cw], acc);
      dst[(size_t)i * a.es + (size_t)c * a.ls] = acc;
    }
    return;
  }

  // transpose: y zero-padded by 2R on each side, then c(p) = sum_t w_t
  // y(p - t) for p in [-R, n - 1 + R], folded onto mirror(p)
  const int ny = n + 4 * R, nc = n + 2 * R;
  float *ye = xe;
  float *ce = xe + (size_t)ny * cw;
  for (int idx = tid; idx < ny * cw; idx += SM_THREADS) {
    const int q = (idx >> a.lcw) - 2 * R, c = idx & cm;
    float val = 0.0f;
    if (q >= 0 && q < n && l0 + c < a.lines) val = src[(size_t)q * a.es + (size_t)c * a.ls];
    ye[idx] = val;
  }
  __syncthreads();
  for (int idx = tid; idx < nc * cw; idx += SM_THREADS) {
    const int pp = idx >> a.lcw, c = idx & cm;  // p = pp - R: y(p - t) sits at ye[pp + 2R - t']
    const float *y = ye + (size_t)(pp + 2 * R) * cw + c;
    float acc = 0.0f;
    for (int t = 0; t < ntap; ++t) acc = fmaf(w[t], y[-(t * cw)], acc);
    ce[idx] = acc;
  }
  __syncthreads();
  for (int idx = tid; idx < n * cw; idx += SM_THREADS) {
    const int j = idx >> a.lcw, c = idx & cm;
    if (l0 + c >= a.lines) continue;
    float acc = 0.0f;
    if (n == 1) {
      for (int pp = 0; pp < nc; ++pp) acc += ce[(size_t)pp * cw + c];
    } else {
      // extended positions p in [-R, n - 1 + R] with mirror(p) = j:
      // p = j or p = -j modulo T = 2(n - 1) (one class at both ends)
      const int T = 2 * (n - 1);
      const int ncls = (j == 0 || j == n - 1) ? 1 : 2;
      for (int cl = 0; cl < ncls; ++cl) {
        const int p0 = cl ? -j : j;
        const int off = p0 + R;  // first p >= -R congruent to p0
        const int k = off >= 0 ? off / T : -((-off + T - 1) / T);
        for (int p = p0 - k * T; p <= n - 1 + R; p += T) acc += ce[(size_t)(p + R) * cw + c];
      }
    }
    dst[(size_t)j * a.es + (size_t)c * a.ls] = acc;
  }
}

size_t smem_floats(int n, int R, int lcw, int adjoint) {
  return (size_t)((2 * R + 1 + 3) & ~3) +
         ((size_t)1 << lcw) * (size_t)(adjoint ? (2 * n + 6 * R) : (n + 2 * R));
}

int launch_lines(const SmoothLines &a, int views, cudaStream_t st) {
  const int cw = 1 << a.lcw;
  const size_t smem = smem_floats(a.n, a.R, a.lcw, a.adjoint) * sizeof(float);
  static bool attr_done = false;
  if (!attr_done) {
    DC_CUDA(cudaFuncSetAttribute(k_smooth_lines, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SM_SMEM_BUDGET));
    attr_done = true;
  }
  dim3 grid((unsigned)((a.lines + cw - 1) / cw), (unsigned)views);
  dc::ProfScope ps(dc::KID_SMOOTH, st);
  k_smooth_lines<<<grid, SM_THREADS, smem, st>>>(a);
  DC_CHECK_LAUNCH("k_smooth_lines");
  return DC_OK;
}

// lines per CTA along mu: the widest power of two (<= 16) whose staging fits
int mu_log_width(int n_mu, int R, int adjoint) {
  for (int l = 4; l >= 0; --l)
    if (smem_floats(n_mu, R, l, adjoint) * sizeof(float) <= SM_SMEM_BUDGET) return l;
  return -1;
}

}  // namespace

extern "C" int dc_gauss_smooth(int V, int n_mu, int n_s, float sigma, int radius, int adjoint,
                               const float *in, float *out, float *work, void *stream) {
  if (V < 1 || n_mu < 1 || n_s < 2)
    return dc::fail(DC_ERR_ARG, "dc_gauss_smooth: sizes must be positive (n_s >= 2)");
  if (!in || !out || !work) return dc::fail(DC_ERR_ARG, "dc_gauss_smooth: NULL array");
  if (in == out || in == work || out == work)
    return dc::fail(DC_ERR_ARG, "dc_gauss_smooth: in, out and work must not alias");
  if (!(sigma > 0.0f) || !std::isfinite(sigma) || radius < 0 || radius > 1024)
    return dc::fail(DC_ERR_ARG, "dc_gauss_smooth: sigma > 0 and 0 <= radius <= 1024");
  const int ns1 = n_s - 1;
  const int ad = adjoint ? 1 : 0;
  const int lmu = mu_log_width(n_mu, radius, ad);
  if (lmu < 0 || smem_floats(ns1, radius, 0, ad) * sizeof(float) > SM_SMEM_BUDGET)
    return dc::fail(DC_ERR_UNSUPPORTED, "dc_gauss_smooth: lines too long for shared memory");
  cudaStream_t st = (cudaStream_t)stream;

  SmoothLines s_axis;  // rows: n_mu lines of ns1 contiguous samples
  s_axis.n = ns1;
  s_axis.lines = n_mu;
  s_axis.vstride = (size_t)n_mu * n_s;
  s_axis.es = 1;
  s_axis.ls = n_s;
  s_axis.lcw = 0;
  s_axis.R = radius;
  s_axis.sigma = sigma;
  s_axis.adjoint = ad;
  SmoothLines mu_axis = s_axis;  // columns: ns1 lines of n_mu samples, n_s apart
  mu_axis.n = n_mu;
  mu_axis.lines = ns1;
  mu_axis.es = n_s;
  mu_axis.ls = 1;
  mu_axis.lcw = lmu;

  // in -> work along s, work -> out along mu (the axis filters commute, and
  // so do their transposes); the unused entry n_s - 1 is copied through
  s_axis.in = in;
  s_axis.out = work;
  int rc = launch_lines(s_axis, V, st);
  if (rc != DC_OK) return rc;
  mu_axis.in = work;
  mu_axis.out = out;
  rc = launch_lines(mu_axis, V, st);
  if (rc != DC_OK) return rc;
  DC_CUDA(cudaMemcpy2DAsync(out + ns1, sizeof(float) * n_s, in + ns1, sizeof(float) * n_s,
                            sizeof(float), (size_t)V * n_mu, cudaMemcpyDeviceToDevice, st));
  return DC_OK;
}
