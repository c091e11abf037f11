// dc_microbench.cu -- interpolation peaks of this GPU for the benchmark: the
// bare inner steps of the three gather kernels, run on a resident shared-
// memory tile with nothing around them (no staging, no set-up, no epilogue):
//
//   kind 0  Joseph step (k_linesum): affine position, exact floor and
//           fraction, two taps of a [sample][33] band, linear interpolation,
//           accumulate; neighbouring lanes ~1.2 samples apart
//   kind 1  transposed-hat pair (k_bp2d): affine position, two taps of a row,
//           two saturated hat weights, accumulate; two pixels per thread in
//           packed FP32x2 operations
//   kind 2  bilinear sample (k_bp3d_tma): affine position in v with a fixed
//           column, exact floor and fraction, two (value, difference) pairs,
//           three interpolations, accumulate
//   kind 3  kind 2 times the voxel weight 1/|X - a|^2 (the circle-view update
//           of k_bp3d_tma: two more FMAs and a reciprocal)
//   kind 4  kind 3 from a tile of quads (both rows' value and difference of
//           a pixel in 16 bytes): one 16-byte load per sample, two samples
//           (voxels k and k + 16 of a column) per step in packed FP32x2
//
// Every thread runs `iters` rounds of 32 unrolled steps; the result goes to
// `sink` so that nothing is optimised away.  The measured steps per second
// are the practical peak of each kernel's core, against which bench.py
// reports the kernels' own rates.
#include <cstdint>

#include "dc_async.cuh"
#include "dc_common.cuh"

namespace {

constexpr int MB_THREADS = 512;
constexpr int MB_TILE = 16384;  // floats of the resident tile (64 KB)

__device__ __forceinline__ float ldf(const char *sb, unsigned off) {
  return *reinterpret_cast<const float *>(sb + off);
}
__device__ __forceinline__ float4 ldq(const char *sb, unsigned off) {
  return *reinterpret_cast<const float4 *>(sb + off);
}

__global__ void __launch_bounds__(MB_THREADS) k_microbench(int kind, int iters, float *sink) {
  extern __shared__ __align__(16) float tile[];
  for (int i = threadIdx.x; i < MB_TILE; i += MB_THREADS) tile[i] = (float)((i * 37) % 101) * 0.01f;
  __syncthreads();
  const char *sb = reinterpret_cast<const char *>(tile);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float M = 12582912.0f;
  float acc = 0.0f;
  if (kind == 0) {
    // [sample][33] band: 256 samples x 33 floats = 8448 floats
    const float dxi = 0.37f;
    for (int it = 0; it < iters; ++it) {
      const float fb = 0.25f + 0.001f * (float)(it & 7);
      const unsigned cb = (unsigned)((40 + (int)(1.2f * (float)lane) + warp) * 33 * 4) -
                          0x4B400000u * (unsigned)(33 * 4);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float x = fmaf((float)q, dxi, fb);
        const float t = __fadd_rd(x, M);
        const float f = x - (t - M);
        const unsigned off = __float_as_uint(t) * (unsigned)(33 * 4) + cb + 4u * q;
        const float g0 = ldf(sb, off), g1 = ldf(sb, off + 33 * 4);
        acc += fmaf(f, g1 - g0, g0);
      }
    }
  } else if (kind == 1) {
    // two pixels (columns lane, lane + 32) per thread in packed FP32x2, as in
    // k_bp2d; s-bin positions stay below 80 of the 520-float rows
    const float Bc = 0.83f, winv = 1.21f, w1c = 1.0f - 1.21f;
    const float2 M2 = make_float2(M, M), mM2 = make_float2(-M, -M), m12 = make_float2(-1.f, -1.f);
    float2 a2 = make_float2(0.0f, 0.0f);
    for (int it = 0; it < iters; ++it) {
      const float rt = 3.0f + 0.5f * (float)warp + 0.001f * (float)(it & 7);
      const unsigned cb = (unsigned)((it & 7) * 520 * 4) - 4u * 0x4B400000u;
      const float2 base = __ffma2_rn(make_float2((float)lane, (float)(lane + 32)),
                                     make_float2(Bc, Bc), make_float2(rt, rt));
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float2 x = __fadd2_rn(base, make_float2((float)q, (float)q));
        const float2 t = __fadd2_rd(x, M2);
        const float2 f = __ffma2_rn(__fadd2_rn(t, mM2), m12, x);
        const unsigned o0 = __float_as_uint(t.x) * 4u + cb, o1 = __float_as_uint(t.y) * 4u + cb;
        const float2 p0 = make_float2(ldf(sb, o0), ldf(sb, o1));
        const float2 p1 = make_float2(ldf(sb, o0 + 4), ldf(sb, o1 + 4));
        const float2 w0 = make_float2(__saturatef(fmaf(-f.x, winv, 1.0f)),
                                      __saturatef(fmaf(-f.y, winv, 1.0f)));
        const float2 w1 = make_float2(__saturatef(fmaf(f.x, winv, w1c)),
                                      __saturatef(fmaf(f.y, winv, w1c)));
        a2 = __ffma2_rn(w0, p0, __ffma2_rn(w1, p1, a2));
      }
    }
    acc = a2.x + a2.y;
  } else if (kind == 4) {
    // quad tile of 32 rows x 44 quads (row stride 704 bytes, 64 mod 128)
    const float fu = 0.3f + 0.01f * (float)lane;
    const float2 fu2 = make_float2(fu, fu);
    const float dv = 0.93f, dz = 0.375f;
    const float ez0 = -40.0f + 0.1f * (float)lane, rho2 = 5.0e5f + (float)warp;
    const float2 M2 = make_float2(M, M), mM2 = make_float2(-M, -M), m12 = make_float2(-1.f, -1.f);
    float2 a2 = make_float2(0.0f, 0.0f);
    for (int it = 0; it < iters; ++it) {
      const float vb = 1.0f + 0.25f * (float)(lane & 3) + 0.001f * (float)(it & 7);
      const unsigned cbc = (unsigned)((2 * warp + (lane >> 2) + 2) * 16) - 0x4B400000u * 704u;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float2 kf = make_float2((float)k, (float)(k + 16));
        const float2 v = __ffma2_rn(kf, make_float2(dv, dv), make_float2(vb, vb));
        const float2 t = __fadd2_rd(v, M2);
        const float2 f = __ffma2_rn(__fadd2_rn(t, mM2), m12, v);
        const float4 qa = ldq(sb, __float_as_uint(t.x) * 704u + cbc);
        const float4 qb = ldq(sb, __float_as_uint(t.y) * 704u + cbc);
        const float2 xa = __ffma2_rn(fu2, make_float2(qa.z, qa.w), make_float2(qa.x, qa.y));
        const float2 xb = __ffma2_rn(fu2, make_float2(qb.z, qb.w), make_float2(qb.x, qb.y));
        const float2 val = make_float2(fmaf(f.x, xa.y - xa.x, xa.x), fmaf(f.y, xb.y - xb.x, xb.x));
        const float2 ez = __ffma2_rn(kf, make_float2(dz, dz), make_float2(ez0, ez0));
        const float2 r2 = __ffma2_rn(ez, ez, make_float2(rho2, rho2));
        a2 = __ffma2_rn(val, make_float2(dc::rcp_approx(r2.x), dc::rcp_approx(r2.y)), a2);
      }
    }
    acc = a2.x + a2.y;
  } else {
    // pair tile of 40 rows x 72 float2 (row stride 576 bytes)
    const float fu = 0.3f + 0.01f * (float)lane;
    const float dv = 0.93f;
    const bool weighted = (kind == 3);
    const float ez0 = -40.0f + 0.1f * (float)lane, dz = 0.375f, rho2 = 5.0e5f + (float)warp;
    for (int it = 0; it < iters; ++it) {
      const float vb = 1.0f + 0.25f * (float)(lane & 3) + 0.001f * (float)(it & 7);
      const unsigned cbc = (unsigned)((4 * warp + (lane >> 2) + 2) * 8) - 0x4B400000u * 576u;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const float v = fmaf((float)k, dv, vb);
        const float tv = __fadd_rd(v, M), fv = v - (tv - M);
        const unsigned off = __float_as_uint(tv) * 576u + cbc;
        const float2 q0 = *reinterpret_cast<const float2 *>(sb + off);
        const float2 q1 = *reinterpret_cast<const float2 *>(sb + off + 576);
        const float x0 = fmaf(fu, q0.y, q0.x), x1 = fmaf(fu, q1.y, q1.x);
        const float val = fmaf(fv, x1 - x0, x0);
        if (weighted) {
          const float ez = fmaf((float)k, dz, ez0);
          acc = fmaf(val, dc::rcp_approx(fmaf(ez, ez, rho2)), acc);
        } else {
          acc += val;
        }
      }
    }
  }
  sink[blockIdx.x * MB_THREADS + threadIdx.x] = acc;
}

}  // namespace

extern "C" int dc_microbench(int kind, int n_blocks, int iters, float *sink, void *stream) {
  if (kind < 0 || kind > 4 || n_blocks < 1 || iters < 1 || !sink)
    return dc::fail(DC_ERR_ARG, "dc_microbench: kind 0..4, n_blocks >= 1, iters >= 1, sink");
  const size_t sm = sizeof(float) * MB_TILE;
  DC_CUDA(cudaFuncSetAttribute(k_microbench, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_microbench<<<n_blocks, MB_THREADS, sm, (cudaStream_t)stream>>>(kind, iters, sink);
  DC_CHECK_LAUNCH("k_microbench");
  return DC_OK;
}
