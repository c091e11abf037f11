// dc_common.cuh -- internal declarations shared by the CUDA sources of the
// Defrise-Clack library (handle layout, error plumbing, small device helpers).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/dracogb.h"

namespace dc {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
// counts kernel launches issued by this library (for benchmarks)
void count_launch(unsigned n = 1);
// allocation that honours the host-side allocation-failure hook
cudaError_t dmalloc(void **p, size_t bytes);

#define DC_CHECK_LAUNCH(what)                                   \
  do {                                                          \
    ::dc::count_launch();                                       \
    cudaError_t e_ = cudaGetLastError();                        \
    if (e_ != cudaSuccess) return ::dc::cuda_fail(e_, what);    \
  } while (0)

#define DC_CUDA(call)                                           \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return ::dc::cuda_fail(e_, #call);   \
  } while (0)

// --------------------------------------------------------------- profiling
// Kernel ids of the optional launch profiler (CUDA events around launches).
enum KernelId {
  KID_PREP = 0,
  KID_LINESUM,
  KID_BP2D,
  KID_TO_F16,
  KID_REDUCE_W,
  KID_SINO_IN,
  KID_BP3D,
  KID_BP3D_ADJ,
  KID_COUNT
};

// Records a start event on construction and an end event on destruction
// when profiling is enabled (dc_profile_enable); otherwise does nothing.
struct ProfScope {
  int slot;
  cudaStream_t st;
  ProfScope(int kid, cudaStream_t s);
  ~ProfScope();
};

// ---------------------------------------------------------------- tables
// FP32 per-view record used by the backprojector (5 x float4):
//  r0 = (f l_x) row, r1 = (f l_y) row, r2 = (-l_z) row of the principal-
//  point-free matrix applied to X - C (C = volume centre); q = that matrix
//  times (C - a); ca = C - a; cu, cv principal point.
struct BPView {
  float4 r0;   // m00 m01 m02 q0
  float4 r1;   // m10 m11 m12 q1
  float4 r2;   // m20 m21 m22 q2   (row 2 gives the depth)
  float4 ca;   // (C-a).x (C-a).y (C-a).z circle_flag
  float4 pp;   // cu cv 0 0
};

// FP32 per-view record used by the filter kernels.
struct FView {
  float D, cu, cv, ax;   // ax,ay,az = v.l_x, v.l_y, v.l_z (Eq. 10 weight)
  float ay, az, pad0, pad1;
};

// FP32 per-angle record: (cos, sin, joseph scale p/max(|c|,|s|), hat inverse
// half-width ds/(p*max(|c|,|s|)))
struct MuRec {
  float c, s, jscale, winv;
};

// A group of consecutive angles (all of one Joseph branch) handled by one
// CTA of the line-sum kernel.
struct MuGroup {
  int first;    // index into the ordered angle list
  int count;
  int branch;   // 0: step over detector rows (|cos| >= |sin|), 1: over columns
  int pad;
};

}  // namespace dc

// ---------------------------------------------------------------- handle
struct dc_geometry {
  dc_geometry_desc d;
  int device;
  // FP64 geometry (device) and a host copy
  double *geo64;             // [V][DC_VIEW_GEO_N]
  double *host_geo;          // [V][DC_VIEW_GEO_N]
  // FP32 tables (device)
  dc::BPView *bpv;           // [V]
  dc::FView *fv;             // [V]
  dc::MuRec *mu;             // [n_mu]
  int *mu_order;             // [n_mu] angle index in group order
  dc::MuGroup *groups;       // [n_groups]
  int n_groups;
  int n_groups_branch0;
  int mg;                    // max angles per group
  // work area
  int chunk_images;          // images (view x batch item) per chunk
  size_t img_stride;         // floats per padded image  (H * Wp)
  size_t imgT_stride;        // floats per padded transposed image (W * Hp)
  size_t sino_stride;        // floats per padded sinogram (n_mu * NSp)
  int Wp, Hp, NSp;           // padded row lengths (multiples of 4)
  float *w_img;              // [chunk][H][Wp]
  float *w_imgT;             // [chunk][W][Hp]
  float *w_sinoA;            // [chunk][n_mu][NSp]
  float *w_sinoB;            // [chunk][n_mu][NSp]
  unsigned *w_absmax;        // [chunk]
  unsigned *w_flags;         // [4] device-side error bits (bit 0: wait timeout)
};

namespace dc {

// host-side helpers defined in dc_filter.cu / dc_backproject.cu
int alloc_workspace(dc_geometry *g);
int build_mu_tables(dc_geometry *g);

}  // namespace dc
