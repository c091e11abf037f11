// dc_backproject.cu -- voxel-driven cone-beam backprojection A3d^T of the
// filtered projections (Ye et al., DRACO, Eq. 5 and the last layer of
// Eq. 12), optional ReLU (Sec. 2.3), and its transpose.
//
//   f(X) = sum_i bilinear(g^F_i, P_i X) / |X - a_i|^2
//
// Each thread owns a column of NZ voxels along z (register blocking); the
// projection of the column is affine in z before the perspective divide, so
// a voxel costs one reciprocal for the depth and one for the distance
// weight.  Coordinates are taken relative to the volume centre and to the
// principal point so that FP32 keeps ~1e-5 pixel accuracy.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "dc_async.cuh"
#include "dc_common.cuh"

namespace {

constexpr int BP_TX = 16, BP_TY = 16;
constexpr int BP_NZ = 16;      // voxels per thread along z
constexpr int BP_VCHUNK = 32;  // views staged in shared memory at a time

struct BPArgs {
  const void *gF;
  const float *scale;  // [B][V] for F16
  const dc::BPView *views;
  float *vol;
  unsigned flags;
  int V, H, W, nx, ny, nz, B;
  float dx, dy, dz;
};

template <typename T>
__device__ __forceinline__ float ld(const T *p);
template <>
__device__ __forceinline__ float ld<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p) {
  return __bfloat162float(__ldg(p));
}
template <>
__device__ __forceinline__ float ld<__half>(const __half *p) { return __half2float(__ldg(p)); }

// bilinear interpolation with zero outside the detector
template <typename T>
__device__ __forceinline__ float bilinear(const T *img, int H, int W, float u, float v) {
  u = fminf(fmaxf(u, -2.0f), (float)W + 1.0f);
  v = fminf(fmaxf(v, -2.0f), (float)H + 1.0f);
  float fu, fv;
  int j = dc::floor_frac(u, fu), r = dc::floor_frac(v, fv);
  bool j0 = (j >= 0 && j < W), j1 = (j + 1 >= 0 && j + 1 < W);
  bool r0 = (r >= 0 && r < H), r1 = (r + 1 >= 0 && r + 1 < H);
  const T *p = img + (ptrdiff_t)r * W + j;
  float g00 = (r0 && j0) ? ld(p) : 0.0f;
  float g01 = (r0 && j1) ? ld(p + 1) : 0.0f;
  float g10 = (r1 && j0) ? ld(p + W) : 0.0f;
  float g11 = (r1 && j1) ? ld(p + W + 1) : 0.0f;
  float a = fmaf(fu, g01 - g00, g00);
  float b = fmaf(fu, g11 - g10, g10);
  return fmaf(fv, b - a, a);
}

template <typename T, bool KAHAN>
__global__ void __launch_bounds__(BP_TX *BP_TY) k_bp3d(BPArgs a) {
  __shared__ dc::BPView sv[BP_VCHUNK];
  const int ix = blockIdx.x * BP_TX + threadIdx.x;
  const int iy = blockIdx.y * BP_TY + threadIdx.y;
  const int zblocks = (a.nz + BP_NZ - 1) / BP_NZ;
  const int b = blockIdx.z / zblocks;
  const int z0 = (blockIdx.z % zblocks) * BP_NZ;
  const int tid = threadIdx.y * BP_TX + threadIdx.x;
  const float xo = ((float)ix - 0.5f * (float)(a.nx - 1)) * a.dx;
  const float yo = ((float)iy - 0.5f * (float)(a.ny - 1)) * a.dy;
  const float zo = ((float)z0 - 0.5f * (float)(a.nz - 1)) * a.dz;
  const size_t np = (size_t)a.H * a.W;
  const T *gbase = (const T *)a.gF + (size_t)b * a.V * np;

  float acc[BP_NZ], cmp[BP_NZ];
#pragma unroll
  for (int k = 0; k < BP_NZ; ++k) acc[k] = cmp[k] = 0.0f;

  for (int i0 = 0; i0 < a.V; i0 += BP_VCHUNK) {
    int nvc = min(BP_VCHUNK, a.V - i0);
    __syncthreads();
    if (tid < nvc) sv[tid] = a.views[i0 + tid];
    __syncthreads();
    for (int ii = 0; ii < nvc; ++ii) {
      const dc::BPView w = sv[ii];
      const int i = i0 + ii;
      const T *img = gbase + (size_t)i * np;
      float sc = 1.0f;
      if (a.scale) sc = a.scale[(size_t)b * a.V + i];
      float U0 = fmaf(w.r0.x, xo, fmaf(w.r0.y, yo, fmaf(w.r0.z, zo, w.r0.w)));
      float V0 = fmaf(w.r1.x, xo, fmaf(w.r1.y, yo, fmaf(w.r1.z, zo, w.r1.w)));
      float W0 = fmaf(w.r2.x, xo, fmaf(w.r2.y, yo, fmaf(w.r2.z, zo, w.r2.w)));
      float dU = w.r0.z * a.dz, dV = w.r1.z * a.dz, dW = w.r2.z * a.dz;
      float ex = w.ca.x + xo, ey = w.ca.y + yo, ez0 = w.ca.z + zo;
      float rho2 = fmaf(ex, ex, ey * ey);
#pragma unroll
      for (int k = 0; k < BP_NZ; ++k) {
        float kf = (float)k;
        float dep = fmaf(kf, dW, W0);
        if (!(dep > 0.0f)) continue;
        float rw = __frcp_rn(dep);
        float u = fmaf(fmaf(kf, dU, U0), rw, w.pp.x);
        float v = fmaf(fmaf(kf, dV, V0), rw, w.pp.y);
        float val = bilinear<T>(img, a.H, a.W, u, v) * sc;
        float ez = fmaf(kf, a.dz, ez0);
        float wt = __frcp_rn(fmaf(ez, ez, rho2));
        float term = val * wt;
        if (KAHAN) {
          float y = term - cmp[k];
          float t = acc[k] + y;
          cmp[k] = (t - acc[k]) - y;
          acc[k] = t;
        } else {
          acc[k] += term;
        }
      }
    }
  }
  if (ix >= a.nx || iy >= a.ny) return;
  const size_t nvox = (size_t)a.nx * a.ny * a.nz;
#pragma unroll
  for (int k = 0; k < BP_NZ; ++k) {
    int iz = z0 + k;
    if (iz >= a.nz) break;
    size_t o = (size_t)b * nvox + ((size_t)iz * a.ny + iy) * a.nx + ix;
    float f = acc[k];
    if (a.flags & DC_ACCUM) f += a.vol[o];
    if ((a.flags & DC_RELU) && f < 0.0f) f = 0.0f;
    a.vol[o] = f;
  }
}

struct BPAdjArgs {
  const float *grad_vol;
  const float *relu_vol;
  const dc::BPView *views;
  float *grad_gF;
  int V, H, W, nx, ny, nz, B;
  float dx, dy, dz;
};

// transpose: every voxel scatters its weighted gradient onto the four taps
__global__ void __launch_bounds__(BP_TX *BP_TY) k_bp3d_adj(BPAdjArgs a) {
  __shared__ dc::BPView sv[BP_VCHUNK];
  const int ix = blockIdx.x * BP_TX + threadIdx.x;
  const int iy = blockIdx.y * BP_TY + threadIdx.y;
  const int zblocks = (a.nz + BP_NZ - 1) / BP_NZ;
  const int b = blockIdx.z / zblocks;
  const int z0 = (blockIdx.z % zblocks) * BP_NZ;
  const int tid = threadIdx.y * BP_TX + threadIdx.x;
  const float xo = ((float)ix - 0.5f * (float)(a.nx - 1)) * a.dx;
  const float yo = ((float)iy - 0.5f * (float)(a.ny - 1)) * a.dy;
  const float zo = ((float)z0 - 0.5f * (float)(a.nz - 1)) * a.dz;
  const size_t np = (size_t)a.H * a.W;
  const size_t nvox = (size_t)a.nx * a.ny * a.nz;
  const bool inside = (ix < a.nx && iy < a.ny);
  float gv[BP_NZ];
#pragma unroll
  for (int k = 0; k < BP_NZ; ++k) {
    int iz = z0 + k;
    gv[k] = 0.0f;
    if (inside && iz < a.nz) {
      size_t o = (size_t)b * nvox + ((size_t)iz * a.ny + iy) * a.nx + ix;
      float g = a.grad_vol[o];
      if (a.relu_vol && !(a.relu_vol[o] > 0.0f)) g = 0.0f;
      gv[k] = g;
    }
  }
  float *gbase = a.grad_gF + (size_t)b * a.V * np;
  for (int i0 = 0; i0 < a.V; i0 += BP_VCHUNK) {
    int nvc = min(BP_VCHUNK, a.V - i0);
    __syncthreads();
    if (tid < nvc) sv[tid] = a.views[i0 + tid];
    __syncthreads();
    if (!inside) continue;
    for (int ii = 0; ii < nvc; ++ii) {
      const dc::BPView w = sv[ii];
      float *img = gbase + (size_t)(i0 + ii) * np;
      float U0 = fmaf(w.r0.x, xo, fmaf(w.r0.y, yo, fmaf(w.r0.z, zo, w.r0.w)));
      float V0 = fmaf(w.r1.x, xo, fmaf(w.r1.y, yo, fmaf(w.r1.z, zo, w.r1.w)));
      float W0 = fmaf(w.r2.x, xo, fmaf(w.r2.y, yo, fmaf(w.r2.z, zo, w.r2.w)));
      float dU = w.r0.z * a.dz, dV = w.r1.z * a.dz, dW = w.r2.z * a.dz;
      float ex = w.ca.x + xo, ey = w.ca.y + yo, ez0 = w.ca.z + zo;
      float rho2 = fmaf(ex, ex, ey * ey);
#pragma unroll
      for (int k = 0; k < BP_NZ; ++k) {
        if (gv[k] == 0.0f) continue;
        float kf = (float)k;
        float dep = fmaf(kf, dW, W0);
        if (!(dep > 0.0f)) continue;
        float rw = __frcp_rn(dep);
        float u = fmaf(fmaf(kf, dU, U0), rw, w.pp.x);
        float v = fmaf(fmaf(kf, dV, V0), rw, w.pp.y);
        float ez = fmaf(kf, a.dz, ez0);
        float g = gv[k] * __frcp_rn(fmaf(ez, ez, rho2));
        u = fminf(fmaxf(u, -2.0f), (float)a.W + 1.0f);
        v = fminf(fmaxf(v, -2.0f), (float)a.H + 1.0f);
        float fu, fv;
        int j = dc::floor_frac(u, fu), r = dc::floor_frac(v, fv);
        bool j0 = (j >= 0 && j < a.W), j1 = (j + 1 >= 0 && j + 1 < a.W);
        bool r0 = (r >= 0 && r < a.H), r1 = (r + 1 >= 0 && r + 1 < a.H);
        float *p = img + (ptrdiff_t)r * a.W + j;
        if (r0 && j0) atomicAdd(p, g * (1.0f - fu) * (1.0f - fv));
        if (r0 && j1) atomicAdd(p + 1, g * fu * (1.0f - fv));
        if (r1 && j0) atomicAdd(p + a.W, g * (1.0f - fu) * fv);
        if (r1 && j1) atomicAdd(p + a.W + 1, g * fu * fv);
      }
    }
  }
}

int check_bp(const dc_geometry *g, int B, const char *who) {
  if (!g) return dc::fail(DC_ERR_ARG, std::string(who) + ": NULL geometry");
  if (B < 1) return dc::fail(DC_ERR_ARG, std::string(who) + ": batch must be >= 1");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != g->device)
    return dc::fail(DC_ERR_ARG, std::string(who) + ": geometry belongs to another device");
  return DC_OK;
}

}  // namespace

extern "C" {

int dc_backproject(const dc_geometry *g, int B, const void *gF, int dtype,
                   const float *gF_scale, float *vol, unsigned flags, void *stream) {
  int rc = check_bp(g, B, "dc_backproject");
  if (rc) return rc;
  if (!gF || !vol) return dc::fail(DC_ERR_ARG, "dc_backproject: NULL gF or vol");
  if (flags & ~(DC_ACCUM | DC_KAHAN | DC_RELU))
    return dc::fail(DC_ERR_ARG, "dc_backproject: unknown flag");
  if (dtype == DC_F16 && !gF_scale)
    return dc::fail(DC_ERR_ARG, "dc_backproject: DC_F16 needs gF_scale");
  const dc_geometry_desc &d = g->d;
  BPArgs a;
  a.gF = gF;
  a.scale = (dtype == DC_F16) ? gF_scale : nullptr;
  a.views = g->bpv;
  a.vol = vol;
  a.flags = flags;
  a.V = d.n_views;
  a.H = d.det_rows;
  a.W = d.det_cols;
  a.nx = d.vol_x;
  a.ny = d.vol_y;
  a.nz = d.vol_z;
  a.B = B;
  a.dx = (float)d.voxel[0];
  a.dy = (float)d.voxel[1];
  a.dz = (float)d.voxel[2];
  dim3 blk(BP_TX, BP_TY);
  dim3 grid((d.vol_x + BP_TX - 1) / BP_TX, (d.vol_y + BP_TY - 1) / BP_TY,
            ((d.vol_z + BP_NZ - 1) / BP_NZ) * B);
  cudaStream_t st = (cudaStream_t)stream;
  bool kahan = (flags & DC_KAHAN) != 0;
  dc::ProfScope ps(dc::KID_BP3D, st);
  switch (dtype) {
    case DC_F32:
      if (kahan) k_bp3d<float, true><<<grid, blk, 0, st>>>(a);
      else k_bp3d<float, false><<<grid, blk, 0, st>>>(a);
      break;
    case DC_BF16:
      if (kahan) k_bp3d<__nv_bfloat16, true><<<grid, blk, 0, st>>>(a);
      else k_bp3d<__nv_bfloat16, false><<<grid, blk, 0, st>>>(a);
      break;
    case DC_F16:
      if (kahan) k_bp3d<__half, true><<<grid, blk, 0, st>>>(a);
      else k_bp3d<__half, false><<<grid, blk, 0, st>>>(a);
      break;
    default:
      return dc::fail(DC_ERR_ARG, "dc_backproject: unknown dtype");
  }
  DC_CHECK_LAUNCH("k_bp3d");
  return DC_OK;
}

int dc_backproject_adjoint(const dc_geometry *g, int B, const float *grad_vol,
                           const float *relu_vol, float *grad_gF, void *stream) {
  int rc = check_bp(g, B, "dc_backproject_adjoint");
  if (rc) return rc;
  if (!grad_vol || !grad_gF)
    return dc::fail(DC_ERR_ARG, "dc_backproject_adjoint: NULL grad_vol or grad_gF");
  const dc_geometry_desc &d = g->d;
  cudaStream_t st = (cudaStream_t)stream;
  DC_CUDA(cudaMemsetAsync(grad_gF, 0,
                          sizeof(float) * (size_t)B * d.n_views * d.det_rows * d.det_cols, st));
  BPAdjArgs a;
  a.grad_vol = grad_vol;
  a.relu_vol = relu_vol;
  a.views = g->bpv;
  a.grad_gF = grad_gF;
  a.V = d.n_views;
  a.H = d.det_rows;
  a.W = d.det_cols;
  a.nx = d.vol_x;
  a.ny = d.vol_y;
  a.nz = d.vol_z;
  a.B = B;
  a.dx = (float)d.voxel[0];
  a.dy = (float)d.voxel[1];
  a.dz = (float)d.voxel[2];
  dim3 blk(BP_TX, BP_TY);
  dim3 grid((d.vol_x + BP_TX - 1) / BP_TX, (d.vol_y + BP_TY - 1) / BP_TY,
            ((d.vol_z + BP_NZ - 1) / BP_NZ) * B);
  dc::ProfScope ps(dc::KID_BP3D_ADJ, st);
  k_bp3d_adj<<<grid, blk, 0, st>>>(a);
  DC_CHECK_LAUNCH("k_bp3d_adj");
  return DC_OK;
}

}  // extern "C"
