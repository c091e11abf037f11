// dc_crofton.cu -- smooth Crofton weights of Eq. 9 (Ye et al., DRACO, Sec.
// 2.3), the analytic redundancy weight for an arbitrary discrete orbit:
//
//   M(theta, lambda_i) = |a'(lambda_i).theta|^m c(lambda_i)
//                        / sum_alpha |a'(lambda_alpha).theta|^m c(lambda_alpha)
//
// for every view i and plane (mu, s_{k+1/2}) through the source a_i.  The
// intersections lambda_alpha of the plane with the orbit are view i itself
// and every sign change of f_j = (a_j - a_i).theta between consecutive views
// of a segment (wrapping for a closed segment; pairs containing i are
// skipped), where the tangent and the taper c are interpolated linearly.
// With m >= 1 the weight is continuous across tangencies, so FP32 suffices.
#include <cstring>
#include <string>

#include "dc_common.cuh"

namespace {

constexpr int CR_THREADS = 128;

struct CroftonArgs {
  const dc::MuRec *mu;      // cos, sin per angle
  const dc::FView *fv;      // D per view
  const double *geo;        // FP64 records (frame, tangent)
  int V, n_mu, n_s, m, taper;
  float ds;
  int n_seg;
  int seg_start[DC_MAX_SEGMENTS];
  int seg_closed[DC_MAX_SEGMENTS];
  float *W;
};

__device__ float taper_of(int j, const CroftonArgs &a) {
  if (a.taper <= 0) return 1.0f;
  for (int q = 0; q < a.n_seg; ++q) {
    int lo = a.seg_start[q], hi = (q + 1 < a.n_seg) ? a.seg_start[q + 1] : a.V;
    if (j < lo || j >= hi) continue;
    if (a.seg_closed[q]) return 1.0f;
    int d = min(j - lo, hi - 1 - j);
    if (d >= a.taper) return 1.0f;
    float x = sinpif(0.5f * ((float)d + 0.5f) / (float)a.taper);
    return x * x;
  }
  return 1.0f;
}

__device__ __forceinline__ float powi(float x, int m) {
  float r = 1.0f;
  for (int e = 0; e < m; ++e) r *= x;
  return r;
}

// grid (k blocks, mu, view); the orbit relative to a_i lives in shared memory
__global__ void __launch_bounds__(CR_THREADS) k_crofton(CroftonArgs a) {
  extern __shared__ float4 orb[];  // [V] (a_j - a_i, c_j), then [V] (v_j, 0)
  const int i = blockIdx.z, m = blockIdx.y;
  const int k = blockIdx.x * CR_THREADS + threadIdx.x;
  const double *gi = a.geo + (size_t)DC_VIEW_GEO_N * i;
  float4 *vt = orb + a.V;
  for (int j = threadIdx.x; j < a.V; j += CR_THREADS) {
    const double *gj = a.geo + (size_t)DC_VIEW_GEO_N * j;
    orb[j] = make_float4((float)(gj[0] - gi[0]), (float)(gj[1] - gi[1]), (float)(gj[2] - gi[2]),
                         taper_of(j, a));
    vt[j] = make_float4((float)gj[15], (float)gj[16], (float)gj[17], 0.0f);
  }
  __syncthreads();
  if (k >= a.n_s) return;
  float *out = a.W + ((size_t)i * a.n_mu + m) * a.n_s + k;
  if (k == a.n_s - 1) {
    *out = 0.0f;
    return;
  }
  const dc::MuRec mr = a.mu[m];
  const float D = a.fv[i].D;
  const float sh = ((float)k - 0.5f * (float)(a.n_s - 1) + 0.5f) * a.ds;
  const float nrm = rsqrtf(fmaf(sh, sh, D * D));
  float th[3];
  for (int c = 0; c < 3; ++c)
    th[c] = (D * mr.c * (float)gi[3 + c] + D * mr.s * (float)gi[6 + c] + sh * (float)gi[9 + c]) * nrm;
  const float4 vi = vt[i];
  float own = powi(fabsf(vi.x * th[0] + vi.y * th[1] + vi.z * th[2]), a.m) * orb[i].w;
  if (!(own > 0.0f)) {
    *out = 0.0f;
    return;
  }
  float sum = own;
  for (int q = 0; q < a.n_seg; ++q) {
    int lo = a.seg_start[q], hi = (q + 1 < a.n_seg) ? a.seg_start[q + 1] : a.V;
    int npair = a.seg_closed[q] ? hi - lo : hi - lo - 1;
    if (npair <= 0) continue;
    float4 o0 = orb[lo];
    float f0 = o0.x * th[0] + o0.y * th[1] + o0.z * th[2];
    for (int e = 0; e < npair; ++e) {
      int j0 = lo + e, j1 = (j0 + 1 < hi) ? j0 + 1 : lo;
      float4 o1 = orb[j1];
      float f1 = o1.x * th[0] + o1.y * th[1] + o1.z * th[2];
      if (j0 != i && j1 != i && ((f0 < 0.0f) != (f1 < 0.0f))) {
        float t = f0 / (f0 - f1);
        float4 v0 = vt[j0], v1 = vt[j1];
        float vx = fmaf(t, v1.x - v0.x, v0.x), vy = fmaf(t, v1.y - v0.y, v0.y),
              vz = fmaf(t, v1.z - v0.z, v0.z);
        float ca = fmaf(t, o1.w - orb[j0].w, orb[j0].w);
        sum += powi(fabsf(vx * th[0] + vy * th[1] + vz * th[2]), a.m) * ca;
      }
      f0 = f1;
      o0 = o1;
    }
  }
  *out = own / sum;
}

}  // namespace

extern "C" int dc_crofton_weights(const dc_geometry *g, int n_seg, const int *seg_start,
                                  const int *seg_closed, int m, int taper, float *W,
                                  void *stream) {
  if (!g || !W) return dc::fail(DC_ERR_ARG, "dc_crofton_weights: NULL argument");
  const dc_geometry_desc &d = g->d;
  CroftonArgs a;
  memset(&a, 0, sizeof(a));
  if (n_seg == 0) {
    a.n_seg = 1;
    a.seg_start[0] = 0;
    a.seg_closed[0] = d.closed_orbit ? 1 : 0;
  } else {
    if (n_seg < 0 || n_seg > DC_MAX_SEGMENTS || !seg_start || !seg_closed)
      return dc::fail(DC_ERR_ARG, "dc_crofton_weights: 1 <= n_seg <= " +
                                      std::to_string(DC_MAX_SEGMENTS) + " with both arrays");
    if (seg_start[0] != 0) return dc::fail(DC_ERR_ARG, "dc_crofton_weights: first segment must start at view 0");
    for (int q = 0; q < n_seg; ++q) {
      int hi = (q + 1 < n_seg) ? seg_start[q + 1] : d.n_views;
      if (seg_start[q] >= hi)
        return dc::fail(DC_ERR_ARG, "dc_crofton_weights: segment starts must increase below V");
      a.seg_start[q] = seg_start[q];
      a.seg_closed[q] = seg_closed[q] ? 1 : 0;
    }
    a.n_seg = n_seg;
  }
  if (m < 0 || m > 8) return dc::fail(DC_ERR_ARG, "dc_crofton_weights: 0 <= m <= 8");
  if (taper < 0) return dc::fail(DC_ERR_ARG, "dc_crofton_weights: taper must be >= 0");
  size_t smem = sizeof(float4) * 2 * (size_t)d.n_views;
  if (smem > 200 * 1024)
    return dc::fail(DC_ERR_UNSUPPORTED, "dc_crofton_weights: too many views for shared memory");
  a.mu = g->mu;
  a.fv = g->fv;
  a.geo = g->geo64;
  a.V = d.n_views;
  a.n_mu = d.n_mu;
  a.n_s = d.n_s;
  a.m = m;
  a.taper = taper;
  a.ds = (float)d.ds;
  a.W = W;
  cudaStream_t st = (cudaStream_t)stream;
  DC_CUDA(cudaFuncSetAttribute(k_crofton, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               200 * 1024));
  dim3 grid((d.n_s + CR_THREADS - 1) / CR_THREADS, d.n_mu, d.n_views);
  k_crofton<<<grid, CR_THREADS, smem, st>>>(a);
  DC_CHECK_LAUNCH("k_crofton");
  return DC_OK;
}
