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
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

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
  int z_begin, z_end;  // voxel planes [z_begin, z_end) of the staged kernels
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
// DC_F32X2: the value is the first half of the (g, right difference) pair
template <>
__device__ __forceinline__ float ld<float2>(const float2 *p) {
  return __ldg(reinterpret_cast<const float *>(p));
}

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


// ------------------------------------------------------------------------
// Shared-memory staged backprojection.  A CTA owns a 16 x 16 x 32 voxel box.
// For every view the box's eight corners are projected; the bounding box of
// the projections (plus a one-pixel margin) is the footprint of every voxel
// of the box on the detector.  A tiled TMA load copies that footprint
// (a 32x48 or 64x48 box, zero outside the detector) into shared memory
// through a three-stage mbarrier pipeline, and the voxels interpolate from
// shared memory without bounds checks.  Footprints are computed for 32 views
// at a time, one corner per thread.  Views whose footprint does not fit (or
// whose box reaches behind the source) fall back to bounds-checked global
// loads; views whose footprint misses the detector are skipped.
constexpr int TB_TX = 16, TB_TY = 16, TB_NZ = 32;
constexpr int TB_BWN = 32, TB_BWW = 64, TB_BH = 48;
constexpr int TB_NS = 3;
constexpr int TB_VCH = 32;
enum { FP_GLOBAL = 0, FP_NARROW = 1, FP_WIDE = 2, FP_SKIP = 3 };

// With DC_F32X2 storage g^F already holds the (g, right difference) pairs
// of the work tile, so the TMA box itself is the tile, read in place: boxes
// of 40 or 72 pairs give a row stride of 8 mod 16 pairs (the bank spread of
// the converted tile below), and every staged column is usable.
constexpr int TB_PBWN = 40, TB_PBWW = 72;
template <typename T>
struct TileShape {
  static constexpr bool PAIRS = false;
  static constexpr int BWN = TB_BWN, BWW = TB_BWW;
};
template <>
struct TileShape<float2> {
  static constexpr bool PAIRS = true;
  static constexpr int BWN = TB_PBWN, BWW = TB_PBWW;
};

template <typename T>
__device__ __forceinline__ float sld(const T *p);
template <>
__device__ __forceinline__ float sld<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float sld<__nv_bfloat16>(const __nv_bfloat16 *p) {
  return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ float sld<__half>(const __half *p) { return __half2float(*p); }

// Shared memory of k_bp3d_tma (dynamic): NS raw TMA stages, then two FP32
// work tiles of tap pairs (g[r][j], g[r][j+1] - g[r][j]) with a row stride
// of TB_S2 float2 (8 mod 16): adjacent rows put one column on different
// banks, a row's linear interpolation is one 64-bit load and one FMA.
// DC_F32X2 storage needs only the stages (the pairs come from g^F).
constexpr int TB_S2 = TB_BWW + 8;
template <typename T>
constexpr size_t bp_tma_smem() {
  return TileShape<T>::PAIRS
             ? (size_t)TB_NS * TB_BH * TB_PBWW * sizeof(T)
             : (size_t)TB_NS * TB_BH * TB_BWW * sizeof(T) +
                   2 * (size_t)TB_BH * TB_S2 * sizeof(float2);
}

// Tap addressing without integer conversions: x + kM rounded toward -inf is
// floor(x) + kM (unit spacing below 2^24), whose bit pattern is
// kFloorBits + floor(x); tile byte offsets fold kFloorBits in once per view.
constexpr float kM = 12582912.0f;  // 1.5 * 2^23
constexpr unsigned kFloorBits = 0x4B400000u;

__device__ __forceinline__ float2 ldpair(const char *sb, unsigned off) {
  return *reinterpret_cast<const float2 *>(sb + off);
}

// bilinear sample from the pair tile: the rows at byte offsets off and
// off + RS, each interpolated across columns by its (value, difference)
// pair, then across the two rows
template <unsigned RS>
__device__ __forceinline__ float tile_sample(const char *sb, unsigned off, float fu, float fv) {
  const float2 q0 = ldpair(sb, off), q1 = ldpair(sb, off + RS);
  const float x0 = fmaf(fu, q0.y, q0.x), x1 = fmaf(fu, q1.y, q1.x);
  return fmaf(fv, x1 - x0, x0);
}

// packed (two-lane) floor and fraction with the rounded-down offset: t holds
// floor(x) + kM (its bits are kFloorBits + floor(x)), f = x - floor(x) exactly
__device__ __forceinline__ void floor_frac2(float2 x, float2 &t, float2 &f) {
  t = __fadd2_rd(x, make_float2(kM, kM));
  f = __ffma2_rn(__fadd2_rn(t, make_float2(-kM, -kM)), make_float2(-1.0f, -1.0f), x);
}

// One CTA backprojects one box of 16 x 16 x NZ voxels (box indices bxi, byi
// and bzi = batch item * z-blocks + z-block) over every view.  `it` is the
// CTA's running view counter (mbarrier stage and parity), carried across
// boxes by the persistent kernel.  Returns false if a bounded wait gave up.
template <typename T, bool KAHAN, int NZ>
__device__ __forceinline__ bool bp_box(const BPArgs &a, float *vol, const CUtensorMap *tmn,
                                       const CUtensorMap *tmw, unsigned *err, int bxi, int byi,
                                       int bzi, unsigned char *dsm, uint64_t *full,
                                       dc::BPView *sv, int4 *vtab, unsigned &it) {
  constexpr bool PAIRS = TileShape<T>::PAIRS;
  constexpr int BWN = TileShape<T>::BWN, BWW = TileShape<T>::BWW;
  constexpr size_t STAGE_BYTES = (size_t)TB_BH * BWW * sizeof(T);
  float2 *wtile0 = (float2 *)(dsm + TB_NS * STAGE_BYTES);  // converted tiles (not PAIRS)
  const char *sb = reinterpret_cast<const char *>(dsm);

  const int tid = threadIdx.y * TB_TX + threadIdx.x;
  // each half-warp (the lanes of one 64-bit shared-memory wavefront) takes a
  // 4 x 4 patch of voxel columns: its taps span a few columns and at most two
  // rows of the pair tile, which the row stride maps to distinct banks
  static_assert(TB_TX == 16 && TB_TY == 16, "4 x 4 patches of a 16 x 16 box");
  const int hw = tid >> 4, l16 = tid & 15;
  const int ix = bxi * TB_TX + ((hw & 3) << 2) + (l16 & 3);
  const int iy = byi * TB_TY + ((hw >> 2) << 2) + (l16 >> 2);
  const int zblocks = (a.z_end - a.z_begin + NZ - 1) / NZ;
  const int b = bzi / zblocks;
  const int z0 = a.z_begin + (bzi % zblocks) * NZ;
  const float cx = 0.5f * (float)(a.nx - 1), cy = 0.5f * (float)(a.ny - 1),
              cz = 0.5f * (float)(a.nz - 1);
  const float xo = ((float)ix - cx) * a.dx;
  const float yo = ((float)iy - cy) * a.dy;
  const float zo = ((float)z0 - cz) * a.dz;
  // extremal voxel centres of this CTA's box (clipped to the volume)
  const float bx0 = ((float)(bxi * TB_TX) - cx) * a.dx;
  const float bx1 = ((float)min(bxi * TB_TX + TB_TX - 1, a.nx - 1) - cx) * a.dx;
  const float by0 = ((float)(byi * TB_TY) - cy) * a.dy;
  const float by1 = ((float)min(byi * TB_TY + TB_TY - 1, a.ny - 1) - cy) * a.dy;
  const float bz0 = zo;
  const float bz1 = ((float)min(z0 + NZ - 1, a.z_end - 1) - cz) * a.dz;
  const size_t np = (size_t)a.H * a.W;
  const T *gbase = (const T *)a.gF + (size_t)b * a.V * np;

  // The column's voxels in pairs: element h of acc2 holds voxels h and
  // h + NH, so that two voxels' positions, floors, weights and sums take one
  // packed FP32x2 operation each (sm_100+; each half rounded as the scalar
  // operation would round it).
  // With KAHAN each view chunk's terms are summed in plain FP32 into prt2,
  // and the chunk sums are added to acc2 with Kahan compensation (cmp2), so
  // the compensated sum runs over the V / TB_VCH chunk sums rather than
  // every view: the FP32 error is that of a TB_VCH-term sum, at 1/TB_VCH of
  // the per-view compensation cost.  Without KAHAN terms go to acc2.
  constexpr int NH = NZ / 2;
  float2 acc2[NH], cmp2[NH], prt2[NH];
#pragma unroll
  for (int h = 0; h < NH; ++h) acc2[h] = cmp2[h] = prt2[h] = make_float2(0.0f, 0.0f);
  // a pair of terms val * wt into voxels (h, h + NH); one term into voxel k
  auto add2 = [&](int h, float2 val, float2 wt) {
    if (KAHAN) prt2[h] = __ffma2_rn(val, wt, prt2[h]);
    else acc2[h] = __ffma2_rn(val, wt, acc2[h]);
  };
  auto add1 = [&](int k, float term) {
    float2 &c = KAHAN ? prt2[k < NH ? k : k - NH] : acc2[k < NH ? k : k - NH];
    if (k < NH) c.x += term;
    else c.y += term;
  };

  bool ok = true;
  for (int c0 = 0; c0 < a.V && ok; c0 += TB_VCH) {
    const int nvc = min(TB_VCH, a.V - c0);
    __syncthreads();
    {  // footprints of this chunk: thread = (view, corner)
      const int vi = tid >> 3, cr = tid & 7;
      float umin = 0.0f, umax = 0.0f, vmin = 0.0f, vmax = 0.0f;
      int good = 1;
      if (vi < nvc) {
        const dc::BPView w = a.views[c0 + vi];
        if (cr == 0) sv[vi] = w;
        float X = (cr & 1) ? bx1 : bx0, Y = (cr & 2) ? by1 : by0, Z = (cr & 4) ? bz1 : bz0;
        float U = fmaf(w.r0.x, X, fmaf(w.r0.y, Y, fmaf(w.r0.z, Z, w.r0.w)));
        float Vv = fmaf(w.r1.x, X, fmaf(w.r1.y, Y, fmaf(w.r1.z, Z, w.r1.w)));
        float Wd = fmaf(w.r2.x, X, fmaf(w.r2.y, Y, fmaf(w.r2.z, Z, w.r2.w)));
        good = (Wd > 1.0f);
        float u = good ? U / Wd + w.pp.x : 0.0f, v = good ? Vv / Wd + w.pp.y : 0.0f;
        umin = umax = u;
        vmin = vmax = v;
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, o));
        umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        good &= __shfl_xor_sync(0xffffffffu, good, o);
      }
      if (vi < nvc && cr == 0) {
        int4 t = make_int4(0, 0, FP_GLOBAL, BWW);
        if (good && fabsf(umin) < 1e6f && fabsf(umax) < 1e6f && fabsf(vmin) < 1e6f &&
            fabsf(vmax) < 1e6f) {
          constexpr int ALIGN = 16 / (int)sizeof(T);  // TMA x offset: 16-byte multiple
          int j0 = (int)floorf(umin) - 1, j1 = (int)floorf(umax) + 2;
          int r0 = (int)floorf(vmin) - 1, r1 = (int)floorf(vmax) + 2;
          int x0 = j0 & ~(ALIGN - 1);
          int ncol = j1 - x0 + 1, nrow = r1 - r0 + 1;
          if (j1 < 0 || x0 >= a.W || r1 < 0 || r0 >= a.H) {
            t = make_int4(x0, r0, FP_SKIP, BWW);
          } else if (nrow <= TB_BH && ncol <= BWN) {
            t = make_int4(x0, r0, FP_NARROW, BWN);
          } else if (nrow <= TB_BH && ncol <= BWW) {
            t = make_int4(x0, r0, FP_WIDE, BWW);
          }
        }
        vtab[vi] = t;
      }
    }
    __syncthreads();
    auto issue = [&](int vi, unsigned s) {
      const int4 t = vtab[vi];
      unsigned char *dst = dsm + s * STAGE_BYTES;
      dc::fence_proxy_async();
      if (t.z == FP_NARROW) {
        dc::mbar_arrive_expect_tx(&full[s], BWN * TB_BH * sizeof(T));
        dc::tma_load_3d(dst, tmn, t.x, t.y, b * a.V + c0 + vi, &full[s]);
      } else if (t.z == FP_WIDE) {
        dc::mbar_arrive_expect_tx(&full[s], BWW * TB_BH * sizeof(T));
        dc::tma_load_3d(dst, tmw, t.x, t.y, b * a.V + c0 + vi, &full[s]);
      } else {
        dc::mbar_arrive(&full[s]);
      }
    };
    if (tid == 0)
      for (int q = 0; q < TB_NS - 1 && q < nvc; ++q) issue(q, (it + q) % TB_NS);

    for (int vi = 0; vi < nvc; ++vi, ++it) {
      const unsigned s = it % TB_NS;
      const int4 t = vtab[vi];
      const int i = c0 + vi;
      float sc = 1.0f;
      if (a.scale) sc = a.scale[(size_t)b * a.V + i];
      bool w_ok = dc::mbar_wait_bounded(&full[s], (it / TB_NS) & 1, err);
      float2 *wt = wtile0 + (size_t)(it & 1) * TB_BH * TB_S2;
      // the pair tile (bytes from dsm) and its row stride: the converted tile,
      // or with PAIRS the TMA stage itself (row stride = box width)
      const unsigned wt_off = PAIRS ? s * (unsigned)STAGE_BYTES
                                    : (unsigned)((const unsigned char *)wt - dsm);
      const bool staged = (t.z == FP_NARROW || t.z == FP_WIDE);
      if (!PAIRS && w_ok && staged) {
        // raw box -> FP32 pair tile (times the FP16 scale)
        const T *raw = (const T *)(dsm + s * STAGE_BYTES);
        const int bw = t.w;
        if constexpr (sizeof(T) == 4) {
          // four pairs per thread and step: one 16-byte load (+ the next
          // element) and two 16-byte stores
          const int lg = (bw == TB_BWN) ? 3 : 4;  // log2 of the groups per row
          for (int e = tid; e < (TB_BH * bw) >> 2; e += TB_TX * TB_TY) {
            int r = e >> lg, j4 = (e - (r << lg)) << 2;
            const float *src = (const float *)raw + r * bw + j4;
            float4 v = *(const float4 *)src;
            float nx = (j4 + 4 < bw) ? src[4] : 0.0f;
            float4 *dst = (float4 *)(wt + r * TB_S2 + j4);
            dst[0] = make_float4(v.x, v.y - v.x, v.y, v.z - v.y);
            dst[1] = make_float4(v.z, v.w - v.z, v.w, nx - v.w);
          }
        } else if constexpr (sizeof(T) == 2) {
          // 16-bit storage: four values per 8-byte load, converted (and
          // scaled) to FP32 pairs with two 16-byte stores.  A BF16 value is
          // the upper half of the FP32 with the same bits, so its conversion
          // is a shift or a mask (exact), and BF16 storage has no scale.
          constexpr bool BF = std::is_same<T, __nv_bfloat16>::value;
          const int lg = (bw == TB_BWN) ? 3 : 4;
          for (int e = tid; e < (TB_BH * bw) >> 2; e += TB_TX * TB_TY) {
            int r = e >> lg, j4 = (e - (r << lg)) << 2;
            const T *src = raw + r * bw + j4;
            uint2 pk = *(const uint2 *)src;
            float v0, v1, v2, v3, nx;
            if (BF) {
              v0 = __uint_as_float(pk.x << 16);
              v1 = __uint_as_float(pk.x & 0xffff0000u);
              v2 = __uint_as_float(pk.y << 16);
              v3 = __uint_as_float(pk.y & 0xffff0000u);
              nx = (j4 + 4 < bw)
                       ? __uint_as_float((unsigned)*reinterpret_cast<const unsigned short *>(src + 4)
                                         << 16)
                       : 0.0f;
            } else {
              T h[4];
              memcpy(h, &pk, sizeof(pk));
              v0 = sld(&h[0]) * sc;
              v1 = sld(&h[1]) * sc;
              v2 = sld(&h[2]) * sc;
              v3 = sld(&h[3]) * sc;
              nx = (j4 + 4 < bw) ? sld(src + 4) * sc : 0.0f;
            }
            float4 *dst = (float4 *)(wt + r * TB_S2 + j4);
            dst[0] = make_float4(v0, v1 - v0, v1, v2 - v1);
            dst[1] = make_float4(v2, v3 - v2, v3, nx - v3);
          }
        }
      }
      if constexpr (PAIRS) {
        // the pair left of column 0 (fill zero from the copy) is (0, g[r][0]):
        // its difference is the first column's value, which the tile holds
        // whenever it reaches left of the detector (x0 < 0)
        if (w_ok && staged && t.x < 0 && tid < TB_BH) {
          float2 *row = reinterpret_cast<float2 *>(dsm + wt_off) + (size_t)tid * t.w;
          row[-1 - t.x].y = row[-t.x].x;
          dc::fence_proxy_async();  // before a later copy into this stage
        }
      }
      if (__syncthreads_or(!w_ok)) {
        ok = false;
        break;
      }
      if (tid == 0 && vi + TB_NS - 1 < nvc) issue(vi + TB_NS - 1, (it + TB_NS - 1) % TB_NS);
      const dc::BPView w = sv[vi];
      float U0 = fmaf(w.r0.x, xo, fmaf(w.r0.y, yo, fmaf(w.r0.z, zo, w.r0.w)));
      float V0 = fmaf(w.r1.x, xo, fmaf(w.r1.y, yo, fmaf(w.r1.z, zo, w.r1.w)));
      float W0 = fmaf(w.r2.x, xo, fmaf(w.r2.y, yo, fmaf(w.r2.z, zo, w.r2.w)));
      float dU = w.r0.z * a.dz, dV = w.r1.z * a.dz, dW = w.r2.z * a.dz;
      float ex = w.ca.x + xo, ey = w.ca.y + yo, ez0 = w.ca.z + zo;
      float rho2 = fmaf(ex, ex, ey * ey);
      // a staged view, with the tile's row stride RS (bytes) a constant: the
      // second row's taps are an immediate offset from the first's
      auto staged_view = [&](auto rs_const) {
        constexpr unsigned RS = decltype(rs_const)::value;
        // tile byte offset minus the floor's exponent bits of a row and a column
        const unsigned cbg = wt_off - kFloorBits * (RS + 8u);
        const float cul = w.pp.x - (float)t.x, cvl = w.pp.y - (float)t.y;
        const float umx = (float)t.w - 1.001f, vmx = (float)TB_BH - 1.001f;
        const float2 dz2 = make_float2(a.dz, a.dz), ez02 = make_float2(ez0, ez0);
        const float2 rho22 = make_float2(rho2, rho2);
        if (w.ca.w != 0.0f) {
          // circle view: u and the depth do not change along the column
          float rw = dc::rcp_approx(W0);
          float u = fminf(fmaxf(fmaf(U0, rw, cul), 0.0f), umx), fu;
          int j = dc::floor_frac(u, fu);
          // byte offset of column j, minus the floor's exponent bits per row
          const unsigned cbc = wt_off + (unsigned)j * 8u - kFloorBits * RS;
          float vb = fmaf(V0, rw, cvl), dv = dV * rw;
          const float2 vb2 = make_float2(vb, vb), dv2 = make_float2(dv, dv);
          // v is affine in k: the column stays inside the tile if both ends do
          float vlast = fmaf((float)(NZ - 1), dv, vb);
          const bool inside = fminf(vb, vlast) >= 0.01f && fmaxf(vb, vlast) <= vmx - 0.01f;
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            const float2 kf = make_float2((float)h, (float)(h + NH));
            float2 v = __ffma2_rn(kf, dv2, vb2);
            if (!inside) v = make_float2(fminf(fmaxf(v.x, 0.0f), vmx), fminf(fmaxf(v.y, 0.0f), vmx));
            float2 tv, fv;
            floor_frac2(v, tv, fv);
            const float2 val =
                make_float2(tile_sample<RS>(sb, __float_as_uint(tv.x) * RS + cbc, fu, fv.x),
                            tile_sample<RS>(sb, __float_as_uint(tv.y) * RS + cbc, fu, fv.y));
            const float2 ez = __ffma2_rn(kf, dz2, ez02);
            const float2 r2 = __ffma2_rn(ez, ez, rho22);
            add2(h, val, make_float2(dc::rcp_approx(r2.x), dc::rcp_approx(r2.y)));
          }
        } else {
          // (u, v) = (affine in k) / (affine depth > 0): monotonic in k, so
          // the column stays inside the tile if both end voxels do
          float kl = (float)(NZ - 1);
          float rwl = dc::rcp_approx(fmaf(kl, dW, W0)), rw0 = dc::rcp_approx(W0);
          float u0 = fmaf(U0, rw0, cul), ul = fmaf(fmaf(kl, dU, U0), rwl, cul);
          float v0 = fmaf(V0, rw0, cvl), vl = fmaf(fmaf(kl, dV, V0), rwl, cvl);
          const float m = 0.01f;  // margin for the rounding of the end points
          const bool inside = fminf(u0, ul) >= m && fmaxf(u0, ul) <= umx - m &&
                              fminf(v0, vl) >= m && fmaxf(v0, vl) <= vmx - m;
          const float2 dW2 = make_float2(dW, dW), W02 = make_float2(W0, W0);
          const float2 dU2 = make_float2(dU, dU), U02 = make_float2(U0, U0);
          const float2 dV2 = make_float2(dV, dV), V02 = make_float2(V0, V0);
          const float2 cul2 = make_float2(cul, cul), cvl2 = make_float2(cvl, cvl);
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            const float2 kf = make_float2((float)h, (float)(h + NH));
            const float2 dep = __ffma2_rn(kf, dW2, W02);
            const float2 rw = make_float2(dc::rcp_approx(dep.x), dc::rcp_approx(dep.y));
            float2 u = __ffma2_rn(__ffma2_rn(kf, dU2, U02), rw, cul2);
            float2 v = __ffma2_rn(__ffma2_rn(kf, dV2, V02), rw, cvl2);
            if (!inside) {
              u = make_float2(fminf(fmaxf(u.x, 0.0f), umx), fminf(fmaxf(u.y, 0.0f), umx));
              v = make_float2(fminf(fmaxf(v.x, 0.0f), vmx), fminf(fmaxf(v.y, 0.0f), vmx));
            }
            float2 tu, fu, tv, fv;
            floor_frac2(u, tu, fu);
            floor_frac2(v, tv, fv);
            const unsigned oa = __float_as_uint(tv.x) * RS + __float_as_uint(tu.x) * 8u + cbg;
            const unsigned ob = __float_as_uint(tv.y) * RS + __float_as_uint(tu.y) * 8u + cbg;
            const float2 val = make_float2(tile_sample<RS>(sb, oa, fu.x, fv.x),
                                           tile_sample<RS>(sb, ob, fu.y, fv.y));
            const float2 ez = __ffma2_rn(kf, dz2, ez02);
            const float2 r2 = __ffma2_rn(ez, ez, rho22);
            add2(h, val, make_float2(dc::rcp_approx(r2.x), dc::rcp_approx(r2.y)));
          }
        }
      };
      if (staged) {
        if constexpr (PAIRS) {
          if (t.w == BWN) staged_view(std::integral_constant<unsigned, BWN * 8u>());
          else staged_view(std::integral_constant<unsigned, BWW * 8u>());
        } else {
          staged_view(std::integral_constant<unsigned, TB_S2 * 8u>());
        }
      } else if (t.z == FP_GLOBAL) {
        const T *img = gbase + (size_t)i * np;
#pragma unroll
        for (int k = 0; k < NZ; ++k) {
          float kf = (float)k;
          float dep = fmaf(kf, dW, W0);
          if (!(dep > 0.0f)) continue;
          float rw = __frcp_rn(dep);
          float u = fmaf(fmaf(kf, dU, U0), rw, w.pp.x);
          float v = fmaf(fmaf(kf, dV, V0), rw, w.pp.y);
          float val = bilinear<T>(img, a.H, a.W, u, v) * sc;
          float ez = fmaf(kf, a.dz, ez0);
          add1(k, val * __frcp_rn(fmaf(ez, ez, rho2)));
        }
      }
    }
    if (KAHAN && ok) {
      auto kahan_step = [](float &acc, float &cmp, float &prt) {
        const float y = prt - cmp;
        const float tt = acc + y;
        cmp = (tt - acc) - y;
        acc = tt;
        prt = 0.0f;
      };
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        kahan_step(acc2[h].x, cmp2[h].x, prt2[h].x);
        kahan_step(acc2[h].y, cmp2[h].y, prt2[h].y);
      }
    }
  }
  if (!ok) return false;
  if (ix >= a.nx || iy >= a.ny) return true;
  const size_t nvox = (size_t)a.nx * a.ny * a.nz;
#pragma unroll
  for (int k = 0; k < NZ; ++k) {
    int iz = z0 + k;
    if (iz >= a.z_end) break;
    size_t o = (size_t)b * nvox + ((size_t)iz * a.ny + iy) * a.nx + ix;
    float f = (k < NH) ? acc2[k].x : acc2[k - NH].y;
    if (a.flags & DC_ACCUM) f += vol[o];
    if ((a.flags & DC_RELU) && f < 0.0f) f = 0.0f;
    vol[o] = f;
  }
  return true;
}

template <typename T, bool KAHAN, int NZ>
__global__ void __launch_bounds__(TB_TX *TB_TY, 2) k_bp3d_tma(BPArgs a, unsigned *err,
                                                             const __grid_constant__ CUtensorMap tmn,
                                                             const __grid_constant__ CUtensorMap tmw) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ uint64_t full[TB_NS];
  __shared__ dc::BPView sv[TB_VCH];
  __shared__ int4 vtab[TB_VCH];
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    for (int q = 0; q < TB_NS; ++q) dc::mbar_init(&full[q], 1);
    dc::fence_barrier_init();
  }
  __syncthreads();
  unsigned it = 0;
  if (!bp_box<T, KAHAN, NZ>(a, a.vol, &tmn, &tmw, err, blockIdx.x, blockIdx.y, blockIdx.z, dsm,
                            full, sv, vtab, it)) {
    for (int q = 0; q < TB_NS; ++q) dc::mbar_wait_bounded(&full[q], 0, nullptr);
  }
}

// Persistent backprojection of a batch of problems (orbits of uneven view
// counts, detectors and volumes): CTAs take (problem, box) items from a
// device counter until all are done.  Items are ordered by problem, largest
// view count first, so the long boxes start early.
constexpr int DC_MAX_BATCH = 32;
struct BatchProblem {
  BPArgs a;               // a.vol is unused: the output comes with the run
  const CUtensorMap *tmn; // global-memory tensor maps over the problem's g^F
  const CUtensorMap *tmw;
  int bx, by, bz;         // boxes per dimension (bz includes the batch)
  int nz;                 // voxels per thread along z (box depth) of this problem: 16 or 32
  long long first;        // first work item of this problem
};
struct BatchRun {
  float *vol[DC_MAX_BATCH];
};

template <typename T, bool KAHAN>
__global__ void __launch_bounds__(TB_TX *TB_TY, 2) k_bp3d_batched(const BatchProblem *probs,
                                                                 int nprob, long long total,
                                                                 unsigned long long *counter,
                                                                 unsigned *err, BatchRun run) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ uint64_t full[TB_NS];
  __shared__ dc::BPView sv[TB_VCH];
  __shared__ int4 vtab[TB_VCH];
  __shared__ long long item;
  const int tid = threadIdx.y * TB_TX + threadIdx.x;
  if (tid == 0) {
    for (int q = 0; q < TB_NS; ++q) dc::mbar_init(&full[q], 1);
    dc::fence_barrier_init();
  }
  unsigned it = 0;
  for (;;) {
    __syncthreads();
    if (tid == 0) item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long w = item;
    if (w >= total) break;
    int p = 0;
    while (p + 1 < nprob && probs[p + 1].first <= w) ++p;
    const BatchProblem &P = probs[p];
    long long lw = w - P.first;
    int bxi = (int)(lw % P.bx);
    long long rest = lw / P.bx;
    int byi = (int)(rest % P.by);
    int bzi = (int)(rest / P.by);
    // each problem has its own box depth (the autotuner's choice for its
    // detector-to-voxel scale); the CTA-uniform branch picks the instance
    const bool done = (P.nz == 16)
                          ? bp_box<T, KAHAN, 16>(P.a, run.vol[p], P.tmn, P.tmw, err, bxi, byi, bzi,
                                                 dsm, full, sv, vtab, it)
                          : bp_box<T, KAHAN, 32>(P.a, run.vol[p], P.tmn, P.tmw, err, bxi, byi, bzi,
                                                 dsm, full, sv, vtab, it);
    if (!done) {
      for (int q = 0; q < TB_NS; ++q) dc::mbar_wait_bounded(&full[q], 0, nullptr);
      return;
    }
  }
}

// ------------------------------------------------------------------------
// Transpose of the staged backprojection.  Same CTA boxes and footprints as
// the forward kernel; for every view the CTA's voxels scatter their weighted
// gradients into a shared-memory footprint tile (row stride 69: 5 mod 32, so
// the rows a warp's lanes reach fall on different banks for most view
// directions), which is then added to g^F's gradient with one global atomic
// per non-zero pixel.  Two tiles alternate: a view's tile is flushed while
// the next view scatters into the other, one barrier per view.
//
// The tile accumulates in 32-bit fixed point, because integer shared-memory
// atomics are native while floating-point ones are not.  The unit is chosen
// per (box, view) from a rigorous bound on any pixel sum: every voxel's four
// bilinear weights sum to one, so a pixel gets at most the box's total,
// nvox * max|g| / d_min^2, with d_min the source's distance to the box
// (centre distance minus half-diagonal); tighter and still rigorous is
// sum_box |g| / d_min^2, since every voxel's weights sum to one and each
// voxel's distance is at least d_min.  That bound maps to 2^30, so the sums
// cannot overflow; each contribution is rounded to the nearest unit.
constexpr int TA_S = 69;
static_assert(TA_S >= TB_BWW, "a tile row holds the widest footprint");
static_assert(TB_NZ == 32, "the adjoint rotates each lane's voxel order by its lane index");
static_assert(TB_BWW <= 64 && TB_BH <= 255, "the tile flush takes 32 columns per lane pass");

__global__ void __launch_bounds__(TB_TX *TB_TY, 2) k_bp3d_adj_tile(BPAdjArgs a) {
  __shared__ int tiles[2][TB_BH * TA_S];
  __shared__ dc::BPView sv[TB_VCH];
  __shared__ int4 vtab[TB_VCH];
  __shared__ float wsum[TB_TX * TB_TY / 32];
  __shared__ float wmax[TB_TX * TB_TY / 32];
  const int tid = threadIdx.y * TB_TX + threadIdx.x;
  const int ix = blockIdx.x * TB_TX + threadIdx.x;
  const int iy = blockIdx.y * TB_TY + threadIdx.y;
  const int zblocks = (a.nz + TB_NZ - 1) / TB_NZ;
  const int b = blockIdx.z / zblocks;
  const int z0 = (blockIdx.z % zblocks) * TB_NZ;
  const float cx = 0.5f * (float)(a.nx - 1), cy = 0.5f * (float)(a.ny - 1),
              cz = 0.5f * (float)(a.nz - 1);
  const float xo = ((float)ix - cx) * a.dx;
  const float yo = ((float)iy - cy) * a.dy;
  const float zo = ((float)z0 - cz) * a.dz;
  const float bx0 = ((float)(blockIdx.x * TB_TX) - cx) * a.dx;
  const float bx1 = ((float)min(blockIdx.x * TB_TX + TB_TX - 1, a.nx - 1) - cx) * a.dx;
  const float by0 = ((float)(blockIdx.y * TB_TY) - cy) * a.dy;
  const float by1 = ((float)min(blockIdx.y * TB_TY + TB_TY - 1, a.ny - 1) - cy) * a.dy;
  const float bz0 = zo;
  const float bz1 = ((float)min(z0 + TB_NZ - 1, a.nz - 1) - cz) * a.dz;
  // box centre and half-diagonal (for the distance bound)
  const float bcx = 0.5f * (bx0 + bx1), bcy = 0.5f * (by0 + by1), bcz = 0.5f * (bz0 + bz1);
  const float bhd = 0.5f * sqrtf((bx1 - bx0) * (bx1 - bx0) + (by1 - by0) * (by1 - by0) +
                                 (bz1 - bz0) * (bz1 - bz0)) + 0.5f * (a.dx + a.dy + a.dz);
  const size_t np = (size_t)a.H * a.W;
  const size_t nvox = (size_t)a.nx * a.ny * a.nz;
  const bool inside = (ix < a.nx && iy < a.ny);
  // Lane l takes its column's voxels in the rotated order kz = (k + l) mod
  // TB_NZ, so that at each step the lanes of a warp are at different depths
  // along z: lanes whose columns project to the same detector column (the
  // columns of a warp lined up with the view direction) then hit different
  // detector rows, and the row stride of the tile (TA_S) spreads those rows
  // over the banks.  The fixed-point sums are exact, so the order does not
  // change the result.  gv[k] holds voxel kz.
  const int rot = tid & 31;
  const float rotf = (float)rot;
  float gv[TB_NZ];
  float gs = 0.0f, gm = 0.0f;
#pragma unroll
  for (int k = 0; k < TB_NZ; ++k) {
    int iz = z0 + ((k + rot) & (TB_NZ - 1));
    gv[k] = 0.0f;
    if (inside && iz < a.nz) {
      size_t o = (size_t)b * nvox + ((size_t)iz * a.ny + iy) * a.nx + ix;
      float g = a.grad_vol[o];
      if (a.relu_vol && !(a.relu_vol[o] > 0.0f)) g = 0.0f;
      gv[k] = g;
      gs += fabsf(g);
      gm = fmaxf(gm, fabsf(g));
    }
  }
  const bool any = gs > 0.0f;
  for (int o = 16; o > 0; o >>= 1) {
    gs += __shfl_xor_sync(0xffffffffu, gs, o);
    gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
  }
  if ((tid & 31) == 0) {
    wsum[tid >> 5] = gs;
    wmax[tid >> 5] = gm;
  }
  for (int e = tid; e < 2 * TB_BH * TA_S; e += TB_TX * TB_TY) (&tiles[0][0])[e] = 0;
  __syncthreads();
  float gsum = 0.0f, gmax = 0.0f;
  for (int q = 0; q < TB_TX * TB_TY / 32; ++q) {
    gsum += wsum[q];
    gmax = fmaxf(gmax, wmax[q]);
  }
  gsum *= 1.0001f;  // headroom for the rounding of this sum
  if (!(gsum > 0.0f)) return;  // nothing to scatter from this box (CTA-uniform)
  // One contribution is at most gmax / d^2 <= gmax / dmin^2, i.e. at most
  // 2^30 gmax / gsum units.  When the box's gradient is spread over at least
  // 512 voxels' worth of its largest value, every contribution stays below
  // 2^21 units and is rounded to an integer by adding 1.5 * 2^23 (the sum
  // has unit spacing, and round-to-nearest-even is the same rounding as
  // __float2int_rn) instead of a conversion instruction.  CTA-uniform.
  const bool magic_round = gsum >= 512.0f * gmax;
  float *gbase = a.grad_gF + (size_t)b * a.V * np;

  // The pending tile: the last scattered view's, flushed while the next view
  // scatters into the other tile.  Its footprint rectangle (columns pt.w &
  // 255, rows pt.w >> 8) holds every tap of the view (one pixel of margin on
  // each side of the projected box), so flushing it clears the whole tile.
  int cur = 0;
  bool pending = false;
  int4 pt = make_int4(0, 0, 0, 0);
  float p_from_fix = 0.0f;
  float *p_img = nullptr;
  auto flush_pending = [&]() {
    int *T = tiles[cur ^ 1];
    const int nc = pt.w & 255, nr = pt.w >> 8;
    for (int c = tid & 31; c < nc; c += 32) {
      const int jj = pt.x + c;
      for (int r = tid >> 5; r < nr; r += (TB_TX * TB_TY) >> 5) {
        const int q = T[r * TA_S + c];
        if (q != 0) {
          T[r * TA_S + c] = 0;
          const int rr = pt.y + r;
          if (jj >= 0 && jj < a.W && rr >= 0 && rr < a.H)
            atomicAdd(p_img + (size_t)rr * a.W + jj, (float)q * p_from_fix);
        }
      }
    }
  };

  for (int c0 = 0; c0 < a.V; c0 += TB_VCH) {
    const int nvc = min(TB_VCH, a.V - c0);
    __syncthreads();
    {  // footprints: thread = (view, corner), as in the forward kernel
      const int vi = tid >> 3, cr = tid & 7;
      float umin = 0.0f, umax = 0.0f, vmin = 0.0f, vmax = 0.0f;
      int good = 1;
      if (vi < nvc) {
        const dc::BPView w = a.views[c0 + vi];
        if (cr == 0) sv[vi] = w;
        float X = (cr & 1) ? bx1 : bx0, Y = (cr & 2) ? by1 : by0, Z = (cr & 4) ? bz1 : bz0;
        float U = fmaf(w.r0.x, X, fmaf(w.r0.y, Y, fmaf(w.r0.z, Z, w.r0.w)));
        float Vv = fmaf(w.r1.x, X, fmaf(w.r1.y, Y, fmaf(w.r1.z, Z, w.r1.w)));
        float Wd = fmaf(w.r2.x, X, fmaf(w.r2.y, Y, fmaf(w.r2.z, Z, w.r2.w)));
        good = (Wd > 1.0f);
        float u = good ? U / Wd + w.pp.x : 0.0f, v = good ? Vv / Wd + w.pp.y : 0.0f;
        umin = umax = u;
        vmin = vmax = v;
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, o));
        umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        good &= __shfl_xor_sync(0xffffffffu, good, o);
      }
      if (vi < nvc && cr == 0) {
        int4 t = make_int4(0, 0, FP_GLOBAL, TB_BWW);
        if (good && fabsf(umin) < 1e6f && fabsf(umax) < 1e6f && fabsf(vmin) < 1e6f &&
            fabsf(vmax) < 1e6f) {
          int x0 = (int)floorf(umin) - 1, x1 = (int)floorf(umax) + 2;
          int r0 = (int)floorf(vmin) - 1, r1 = (int)floorf(vmax) + 2;
          if (x1 < 0 || x0 >= a.W || r1 < 0 || r0 >= a.H)
            t = make_int4(x0, r0, FP_SKIP, 0);
          else if (r1 - r0 + 1 <= TB_BH && x1 - x0 + 1 <= TB_BWW)
            t = make_int4(x0, r0, FP_WIDE, (x1 - x0 + 1) | ((r1 - r0 + 1) << 8));
        }
        vtab[vi] = t;
      }
    }
    __syncthreads();
    for (int vi = 0; vi < nvc; ++vi) {
      int4 t = vtab[vi];
      if (t.z == FP_SKIP) continue;
      const dc::BPView w = sv[vi];
      float *img = gbase + (size_t)(c0 + vi) * np;
      float U0 = fmaf(w.r0.x, xo, fmaf(w.r0.y, yo, fmaf(w.r0.z, zo, w.r0.w)));
      float V0 = fmaf(w.r1.x, xo, fmaf(w.r1.y, yo, fmaf(w.r1.z, zo, w.r1.w)));
      float W0 = fmaf(w.r2.x, xo, fmaf(w.r2.y, yo, fmaf(w.r2.z, zo, w.r2.w)));
      float dU = w.r0.z * a.dz, dV = w.r1.z * a.dz, dW = w.r2.z * a.dz;
      float ex = w.ca.x + xo, ey = w.ca.y + yo, ez0 = w.ca.z + zo;
      float rho2 = fmaf(ex, ex, ey * ey);
      // fixed-point unit of this (box, view); CTA-uniform
      float dcx = w.ca.x + bcx, dcy = w.ca.y + bcy, dcz = w.ca.z + bcz;
      float dmin = sqrtf(dcx * dcx + dcy * dcy + dcz * dcz) - bhd;
      if (t.z == FP_WIDE && !(dmin > 1.0f)) t.z = FP_GLOBAL;
      if (t.z == FP_WIDE) {
        const float bound = gsum / (dmin * dmin);             // >= any pixel sum
        const float to_fix = 1073741824.0f / bound;            // bound -> 2^30
        const float from_fix = bound * (1.0f / 1073741824.0f);
        const float cul = w.pp.x - (float)t.x, cvl = w.pp.y - (float)t.y;
        const float umx = (float)TB_BWW - 1.001f, vmx = (float)TB_BH - 1.001f;
        int *tile = tiles[cur];
        auto scatter = [&](auto to_int) {
#pragma unroll
          for (int k = 0; k < TB_NZ; ++k) {
            if (gv[k] == 0.0f) continue;
            float kf = rotf + (float)k;  // voxel (k + rot) mod TB_NZ
            kf = (kf >= (float)TB_NZ) ? kf - (float)TB_NZ : kf;
            float rw = dc::rcp_approx(fmaf(kf, dW, W0));
            float u = fminf(fmaxf(fmaf(fmaf(kf, dU, U0), rw, cul), 0.0f), umx);
            float v = fminf(fmaxf(fmaf(fmaf(kf, dV, V0), rw, cvl), 0.0f), vmx);
            float ez = fmaf(kf, a.dz, ez0);
            float gk = gv[k] * dc::rcp_approx(fmaf(ez, ez, rho2)) * to_fix;
            float fu, fv;
            int j = dc::floor_frac(u, fu), r = dc::floor_frac(v, fv);
            int *p = tile + r * TA_S + j;
            float g1 = gk * fv, g0 = gk - g1;
            float g01 = g0 * fu, g11 = g1 * fu;
            atomicAdd(p, to_int(g0 - g01));
            atomicAdd(p + 1, to_int(g01));
            atomicAdd(p + TA_S, to_int(g1 - g11));
            atomicAdd(p + TA_S + 1, to_int(g11));
          }
        };
        if (any) {
          if (magic_round)
            scatter([](float x) {
              return __float_as_int(__fadd_rn(x, 12582912.0f)) - 0x4B400000;  // |x| < 2^22
            });
          else
            scatter([](float x) { return __float2int_rn(x); });
        }
        // the previous view's tile (complete since the last barrier) to g^F's
        // gradient, cleared for the view after this one
        if (pending) flush_pending();
        __syncthreads();
        pending = true;
        pt = t;
        p_from_fix = from_fix;
        p_img = img;
        cur ^= 1;
      } else if (any) {
#pragma unroll
        for (int k = 0; k < TB_NZ; ++k) {
          if (gv[k] == 0.0f) continue;
          float kf = rotf + (float)k;  // voxel (k + rot) mod TB_NZ
          kf = (kf >= (float)TB_NZ) ? kf - (float)TB_NZ : kf;
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
  if (pending) flush_pending();  // its scatter ended at the last barrier
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// bytes per g^F pixel of a storage form
int pixel_bytes(int dtype) { return dtype == DC_F32 ? 4 : dtype == DC_F32X2 ? 8 : 2; }

// 3-D map over g^F viewed as [B*V][H][W] with a box of bw x TB_BH x 1 (a
// DC_F32X2 pair is one 8-byte element: the copy moves its bits)
bool make_map(CUtensorMap *m, const void *base, int dtype, int W, int H, long long nimg,
              int bw) {
  auto fn = encode_fn();
  if (!fn) return false;
  int es = pixel_bytes(dtype);
  CUtensorMapDataType t = (dtype == DC_F32)     ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                          : (dtype == DC_F32X2) ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                          : (dtype == DC_BF16)  ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)nimg};
  cuuint64_t strides[2] = {(cuuint64_t)W * es, (cuuint64_t)W * H * es};
  cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)TB_BH, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, t, 3, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <typename T, int NZ>
int launch_bp_tma_nz(const dc_geometry *g, BPArgs &a, bool kahan, cudaStream_t st,
                     const CUtensorMap &mn, const CUtensorMap &mw) {
  dim3 blk(TB_TX, TB_TY);
  dim3 grid((a.nx + TB_TX - 1) / TB_TX, (a.ny + TB_TY - 1) / TB_TY,
            ((a.z_end - a.z_begin + NZ - 1) / NZ) * a.B);
  const size_t sm = bp_tma_smem<T>();
  if (kahan) {
    DC_CUDA(cudaFuncSetAttribute(k_bp3d_tma<T, true, NZ>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_bp3d_tma<T, true, NZ><<<grid, blk, sm, st>>>(a, g->w_flags, mn, mw);
  } else {
    DC_CUDA(cudaFuncSetAttribute(k_bp3d_tma<T, false, NZ>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_bp3d_tma<T, false, NZ><<<grid, blk, sm, st>>>(a, g->w_flags, mn, mw);
  }
  return DC_OK;
}

bool tma_ok(const void *base, int W, int dtype) {
  int es = pixel_bytes(dtype);
  return ((size_t)W * es) % 16 == 0 && ((uintptr_t)base & 15) == 0 && encode_fn() != nullptr;
}

template <typename T>
int launch_bp_tma(const dc_geometry *g, BPArgs &a, int dtype, bool kahan, cudaStream_t st,
                  bool *used) {
  *used = false;
  if (!tma_ok(a.gF, a.W, dtype) || getenv("DC_BP_NO_TMA")) return DC_OK;
  CUtensorMap mn, mw;
  long long nimg = (long long)a.B * a.V;
  if (!make_map(&mn, a.gF, dtype, a.W, a.H, nimg, TileShape<T>::BWN) ||
      !make_map(&mw, a.gF, dtype, a.W, a.H, nimg, TileShape<T>::BWW))
    return DC_OK;
  int rc = (g->bp_nz == 16) ? launch_bp_tma_nz<T, 16>(g, a, kahan, st, mn, mw)
                            : launch_bp_tma_nz<T, 32>(g, a, kahan, st, mn, mw);
  if (rc) return rc;
  *used = true;
  return DC_OK;
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

BPArgs bp_args(const dc_geometry *g, int B, const void *gF, int dtype, const float *gF_scale,
               float *vol, unsigned flags) {
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
  a.z_begin = 0;
  a.z_end = d.vol_z;
  a.B = B;
  a.dx = (float)d.voxel[0];
  a.dy = (float)d.voxel[1];
  a.dz = (float)d.voxel[2];
  return a;
}

}  // namespace

namespace dc {

int backproject_check(const dc_geometry *g, int B, const void *gF, int dtype,
                      const float *gF_scale, const float *vol, unsigned flags, const char *who) {
  int rc = check_bp(g, B, who);
  if (rc) return rc;
  if (!gF || !vol) return fail(DC_ERR_ARG, std::string(who) + ": NULL gF or vol");
  if (flags & ~(DC_ACCUM | DC_KAHAN | DC_RELU))
    return fail(DC_ERR_ARG, std::string(who) + ": unknown flag");
  if (dtype != DC_F32 && dtype != DC_BF16 && dtype != DC_F16 && dtype != DC_F32X2)
    return fail(DC_ERR_ARG, std::string(who) + ": unknown dtype");
  if (dtype == DC_F16 && !gF_scale)
    return fail(DC_ERR_ARG, std::string(who) + ": DC_F16 needs gF_scale");
  return DC_OK;
}

int backproject_slab(const dc_geometry *g, int B, const void *gF, int dtype,
                     const float *gF_scale, float *vol, unsigned flags, int z_begin, int z_end,
                     cudaStream_t st, bool *used) {
  BPArgs a = bp_args(g, B, gF, dtype, gF_scale, vol, flags);
  a.z_begin = z_begin;
  a.z_end = z_end;
  const bool kahan = (flags & DC_KAHAN) != 0;
  ProfScope ps(KID_BP3D, st);
  int rc;
  switch (dtype) {
    case DC_F32: rc = launch_bp_tma<float>(g, a, dtype, kahan, st, used); break;
    case DC_F32X2: rc = launch_bp_tma<float2>(g, a, dtype, kahan, st, used); break;
    case DC_BF16: rc = launch_bp_tma<__nv_bfloat16>(g, a, dtype, kahan, st, used); break;
    default: rc = launch_bp_tma<__half>(g, a, dtype, kahan, st, used); break;
  }
  if (rc) return rc;
  if (*used) DC_CHECK_LAUNCH("k_bp3d_tma");
  return DC_OK;
}

}  // namespace dc

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
  a.z_begin = 0;
  a.z_end = d.vol_z;
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
  bool used = false;
  switch (dtype) {
    case DC_F32: rc = launch_bp_tma<float>(g, a, dtype, kahan, st, &used); break;
    case DC_F32X2: rc = launch_bp_tma<float2>(g, a, dtype, kahan, st, &used); break;
    case DC_BF16: rc = launch_bp_tma<__nv_bfloat16>(g, a, dtype, kahan, st, &used); break;
    case DC_F16: rc = launch_bp_tma<__half>(g, a, dtype, kahan, st, &used); break;
    default: return dc::fail(DC_ERR_ARG, "dc_backproject: unknown dtype");
  }
  if (rc) return rc;
  if (used) {
    DC_CHECK_LAUNCH("k_bp3d_tma");
    return DC_OK;
  }
  switch (dtype) {
    case DC_F32:
      if (kahan) k_bp3d<float, true><<<grid, blk, 0, st>>>(a);
      else k_bp3d<float, false><<<grid, blk, 0, st>>>(a);
      break;
    case DC_F32X2:
      if (kahan) k_bp3d<float2, true><<<grid, blk, 0, st>>>(a);
      else k_bp3d<float2, false><<<grid, blk, 0, st>>>(a);
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
  if (getenv("DC_BP_ADJ_GLOBAL")) {
    k_bp3d_adj<<<grid, blk, 0, st>>>(a);
  } else {
    dim3 gridt((d.vol_x + TB_TX - 1) / TB_TX, (d.vol_y + TB_TY - 1) / TB_TY,
               ((d.vol_z + TB_NZ - 1) / TB_NZ) * B);
    k_bp3d_adj_tile<<<gridt, blk, 0, st>>>(a);
  }
  DC_CHECK_LAUNCH("k_bp3d_adj");
  return DC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Batched reconstruction: the filter of every problem (its chunked launches,
// or with DC_PERSISTENT_FILTER one persistent kernel over the (problem,
// view) images of all problems), then one persistent backprojection over all
// problems' voxel boxes.  Everything a run needs is allocated by
// dc_batch_create, so dc_batch_run allocates nothing and can be captured in
// a CUDA graph.
struct dc_batch {
  int n;
  int dtype;
  unsigned flags;
  int nz;                         // 16 / 32 for every problem, 0: each geometry's own bp_nz
  int grid;
  long long total;
  int order[DC_MAX_BATCH];        // table position -> problem index
  dc_geometry *geoms[DC_MAX_BATCH];
  void *gF[DC_MAX_BATCH];         // owned filtered projections [V][H][W]
  float *scale[DC_MAX_BATCH];     // owned FP16 scales [V]
  BatchProblem *d_probs;
  CUtensorMap *d_maps;
  unsigned long long *d_counter;
  dc::BatchFilterPlan *fplan;     // persistent filter of every problem (NULL: per-problem calls)
};

namespace {

void free_batch(dc_batch *b) {
  if (!b) return;
  for (int i = 0; i < b->n; ++i) {
    cudaFree(b->gF[i]);
    cudaFree(b->scale[i]);
  }
  cudaFree(b->d_probs);
  cudaFree(b->d_maps);
  cudaFree(b->d_counter);
  dc::batch_filter_destroy(b->fplan);
  delete b;
}

int build_batch_tables(dc_batch *b) {
  std::vector<BatchProblem> probs(b->n);
  std::vector<CUtensorMap> maps(2 * b->n);
  long long first = 0;
  for (int t = 0; t < b->n; ++t) {
    int i = b->order[t];
    const dc_geometry *g = b->geoms[i];
    const dc_geometry_desc &d = g->d;
    BatchProblem &P = probs[t];
    memset(&P, 0, sizeof(P));
    P.a.gF = b->gF[i];
    P.a.scale = (b->dtype == DC_F16) ? b->scale[i] : nullptr;
    P.a.views = g->bpv;
    P.a.vol = nullptr;
    P.a.flags = b->flags & DC_RELU;
    P.a.V = d.n_views;
    P.a.H = d.det_rows;
    P.a.W = d.det_cols;
    P.a.nx = d.vol_x;
    P.a.ny = d.vol_y;
    P.a.nz = d.vol_z;
    P.a.z_begin = 0;
    P.a.z_end = d.vol_z;
    P.a.B = 1;
    P.a.dx = (float)d.voxel[0];
    P.a.dy = (float)d.voxel[1];
    P.a.dz = (float)d.voxel[2];
    const bool pairs = (b->dtype == DC_F32X2);
    if (!make_map(&maps[2 * t], b->gF[i], b->dtype, d.det_cols, d.det_rows, d.n_views,
                  pairs ? TB_PBWN : TB_BWN) ||
        !make_map(&maps[2 * t + 1], b->gF[i], b->dtype, d.det_cols, d.det_rows, d.n_views,
                  pairs ? TB_PBWW : TB_BWW))
      return dc::fail(DC_ERR_CUDA, "dc_batch: tensor map encoding failed");
    P.tmn = b->d_maps + 2 * t;
    P.tmw = b->d_maps + 2 * t + 1;
    P.bx = (d.vol_x + TB_TX - 1) / TB_TX;
    P.by = (d.vol_y + TB_TY - 1) / TB_TY;
    P.nz = b->nz ? b->nz : g->bp_nz;
    P.bz = (d.vol_z + P.nz - 1) / P.nz;
    P.first = first;
    first += (long long)P.bx * P.by * P.bz;
  }
  b->total = first;
  DC_CUDA(cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                     cudaMemcpyHostToDevice));
  DC_CUDA(cudaMemcpy(b->d_probs, probs.data(), sizeof(BatchProblem) * probs.size(),
                     cudaMemcpyHostToDevice));
  return DC_OK;
}

template <typename T, bool KAHAN>
int launch_batched(dc_batch *b, BatchRun &run, cudaStream_t st) {
  const size_t sm = bp_tma_smem<T>();
  DC_CUDA(cudaFuncSetAttribute(k_bp3d_batched<T, KAHAN>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_bp3d_batched<T, KAHAN><<<b->grid, dim3(TB_TX, TB_TY), sm, st>>>(
      b->d_probs, b->n, b->total, b->d_counter, b->geoms[0]->w_flags, run);
  return DC_OK;
}

template <typename T>
int launch_batched_t(dc_batch *b, BatchRun &run, cudaStream_t st) {
  return (b->flags & DC_KAHAN) ? launch_batched<T, true>(b, run, st)
                               : launch_batched<T, false>(b, run, st);
}

}  // namespace

extern "C" {

int dc_batch_create(int n, dc_geometry *const *geoms, int dtype, unsigned flags,
                    dc_batch **out) {
  if (!out || !geoms) return dc::fail(DC_ERR_ARG, "dc_batch_create: NULL argument");
  *out = nullptr;
  if (n < 1 || n > DC_MAX_BATCH)
    return dc::fail(DC_ERR_ARG, "dc_batch_create: 1 <= n <= " + std::to_string(DC_MAX_BATCH));
  if (dtype != DC_F32 && dtype != DC_BF16 && dtype != DC_F16 && dtype != DC_F32X2)
    return dc::fail(DC_ERR_ARG, "dc_batch_create: unknown dtype");
  if (flags & ~(DC_KAHAN | DC_RELU | DC_PERSISTENT_FILTER))
    return dc::fail(DC_ERR_ARG,
                    "dc_batch_create: flags may be DC_KAHAN | DC_RELU | DC_PERSISTENT_FILTER");
  if (!encode_fn()) return dc::fail(DC_ERR_UNSUPPORTED, "dc_batch_create: no TMA encoder");
  int dev = -1;
  cudaGetDevice(&dev);
  int es = pixel_bytes(dtype);
  for (int i = 0; i < n; ++i) {
    if (!geoms[i]) return dc::fail(DC_ERR_ARG, "dc_batch_create: NULL geometry");
    if (geoms[i]->device != dev)
      return dc::fail(DC_ERR_ARG, "dc_batch_create: geometry on another device");
    if (((size_t)geoms[i]->d.det_cols * es) % 16 != 0)
      return dc::fail(DC_ERR_UNSUPPORTED,
                      "dc_batch_create: detector rows must be a multiple of 16 bytes");
  }
  dc_batch *b = new dc_batch();
  memset((void *)b, 0, sizeof(dc_batch));
  b->n = n;
  b->dtype = dtype;
  b->flags = flags;
  b->nz = 0;  // each problem's box depth from its geometry (dc_geometry_set_tuning)
  for (int i = 0; i < n; ++i) b->geoms[i] = geoms[i];
  // largest view count first
  for (int i = 0; i < n; ++i) b->order[i] = i;
  std::sort(b->order, b->order + n, [&](int x, int y) {
    return geoms[x]->d.n_views > geoms[y]->d.n_views;
  });
  auto bail = [&](int code) {
    free_batch(b);
    return code;
  };
  for (int i = 0; i < n; ++i) {
    const dc_geometry_desc &d = geoms[i]->d;
    size_t bytes = (size_t)d.n_views * d.det_rows * d.det_cols * es;
    cudaError_t e = dc::dmalloc(&b->gF[i], bytes);
    if (e != cudaSuccess) return bail(dc::cuda_fail(e, "dc_batch_create: g^F"));
    if (dtype == DC_F16) {
      e = dc::dmalloc((void **)&b->scale[i], sizeof(float) * d.n_views);
      if (e != cudaSuccess) return bail(dc::cuda_fail(e, "dc_batch_create: scales"));
    }
  }
  cudaError_t e = dc::dmalloc((void **)&b->d_probs, sizeof(BatchProblem) * n);
  if (e == cudaSuccess) e = dc::dmalloc((void **)&b->d_maps, sizeof(CUtensorMap) * 2 * n);
  if (e == cudaSuccess) e = dc::dmalloc((void **)&b->d_counter, sizeof(unsigned long long));
  if (e != cudaSuccess) return bail(dc::cuda_fail(e, "dc_batch_create: tables"));
  int rc = build_batch_tables(b);
  if (rc) return bail(rc);
  // optionally one persistent launch filters every problem; problems whose
  // rows do not fit its shared memory keep the per-problem filter calls
  if (flags & DC_PERSISTENT_FILTER) {
    rc = dc::batch_filter_create(n, b->geoms, dtype, b->gF, b->scale, &b->fplan);
    if (rc == DC_ERR_UNSUPPORTED) {
      b->fplan = nullptr;
    } else if (rc) {
      return bail(rc);
    }
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->grid = std::max(1, sms) * 2;
  *out = b;
  return DC_OK;
}

int dc_batch_set_bp_nz(dc_batch *b, int nz) {
  if (!b || (nz != 0 && nz != 16 && nz != 32))
    return dc::fail(DC_ERR_ARG, "dc_batch_set_bp_nz: nz must be 16, 32 or 0 (per geometry)");
  b->nz = nz;
  return build_batch_tables(b);
}

int dc_batch_run(dc_batch *b, const float *const *g, const float *const *W, float *const *vol,
                 void *stream) {
  if (!b || !g || !vol) return dc::fail(DC_ERR_ARG, "dc_batch_run: NULL argument");
  for (int i = 0; i < b->n; ++i)
    if (!g[i] || !vol[i]) return dc::fail(DC_ERR_ARG, "dc_batch_run: NULL g or vol");
  cudaStream_t st = (cudaStream_t)stream;
  if (b->fplan) {
    int rc = dc::batch_filter_run(b->fplan, g, W, st);
    if (rc) return rc;
  } else {
    for (int i = 0; i < b->n; ++i) {
      int rc = dc_filter(b->geoms[i], 1, g[i], W ? W[i] : nullptr, b->gF[i], b->dtype,
                         b->scale[i], stream);
      if (rc) return rc;
    }
  }
  BatchRun run;
  memset(&run, 0, sizeof(run));
  for (int t = 0; t < b->n; ++t) run.vol[t] = vol[b->order[t]];
  DC_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), st));
  dc::ProfScope ps(dc::KID_BP3D, st);
  int rc = DC_OK;
  switch (b->dtype) {
    case DC_F32: rc = launch_batched_t<float>(b, run, st); break;
    case DC_F32X2: rc = launch_batched_t<float2>(b, run, st); break;
    case DC_BF16: rc = launch_batched_t<__nv_bfloat16>(b, run, st); break;
    default: rc = launch_batched_t<__half>(b, run, st); break;
  }
  if (rc) return rc;
  DC_CHECK_LAUNCH("k_bp3d_batched");
  return DC_OK;
}

void dc_batch_destroy(dc_batch *b) { free_batch(b); }

int dc_geometry_set_tuning(dc_geometry *g, int chunk_images, int bp_nz) {
  if (!g) return dc::fail(DC_ERR_ARG, "dc_geometry_set_tuning: NULL geometry");
  if (chunk_images < 0 || chunk_images > g->chunk_capacity)
    return dc::fail(DC_ERR_ARG, "dc_geometry_set_tuning: chunk_images must be in [1, " +
                                    std::to_string(g->chunk_capacity) + "] (0 keeps it)");
  if (bp_nz != 0 && bp_nz != 16 && bp_nz != 32)
    return dc::fail(DC_ERR_ARG, "dc_geometry_set_tuning: bp_nz must be 16 or 32 (0 keeps it)");
  if (chunk_images > 0) g->chunk_images = chunk_images;
  if (bp_nz > 0) g->bp_nz = bp_nz;
  return DC_OK;
}

int dc_geometry_get_tuning(const dc_geometry *g, int *chunk_images, int *chunk_capacity,
                           int *bp_nz) {
  if (!g) return dc::fail(DC_ERR_ARG, "dc_geometry_get_tuning: NULL geometry");
  if (chunk_images) *chunk_images = g->chunk_images;
  if (chunk_capacity) *chunk_capacity = g->chunk_capacity;
  if (bp_nz) *bp_nz = g->bp_nz;
  return DC_OK;
}

}  // extern "C"
