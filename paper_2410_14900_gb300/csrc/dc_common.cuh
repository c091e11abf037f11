// dc_common.cuh -- internal declarations shared by the CUDA sources of the
// Defrise-Clack library (handle layout, error plumbing, small device helpers).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/dracogb.h"

// bits of a handle's device-side error word (w_flags[0])
#define DC_FLAG_TIMEOUT 1u        // a bounded wait gave up (the kernel skipped its output)
#define DC_FLAG_NONFINITE_W 2u    // a redundancy weight read by a filter kernel was NaN / inf

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
  KID_SMOOTH,
  KID_ADJ_S,
  KID_FILTER_BATCHED,
  KID_TO_PAIRS,
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

// FP32 per-angle record, from FP64 at set-up.  With (cs, sn) = (cos, sin)
// for the row-stepping Joseph branch and (sin, cos) for the column-stepping
// one, m = max(|cos|, |sin|) = |cs|:
//   jscale = p/m, winv = ds/(p m)             Joseph scale, hat half-width^-1
//   a = (ds/p)/cs, d = -sn/cs                 line-sum position per s-bin, per row
//   bc = cos p/ds, bs = sin p/ds              s-bin position per pixel column, row
// Pairs *_hi + *_lo are exact splits whose *_hi has 12 fractional bits, so
// products with small integers are exact in FP32.
struct MuRec {
  float c, s, jscale, winv;
  float a_hi, a_lo, d_hi, d_lo;
  float dxi, bc_hi, bc_lo, bs_hi;
  float bs_lo, pad0, pad1, pad2;
};

// FP32 per-(view, angle) record, from FP64 at set-up: the Joseph position of
// line s_0 at row 0, b = c_col + c_row sn/cs, and the s-bin position of pixel
// (0, 0), x = (n_s-1)/2 - (c_u cos + c_v sin) p/ds, each as an integer part
// and a fraction in [0, 1).
struct VMu {
  float b0i, b0f, xoi, xof;
};

// A group of consecutive angles (all of one Joseph branch) handled by one
// CTA of the line-sum kernel.
struct MuGroup {
  int first;    // index into the ordered angle list
  int count;
  int branch;   // 0: step over detector rows (|cos| >= |sin|), 1: over columns
  int pad;
};

// Line-sum CTAs hold at most DC_LS_MAX_MG angles and DC_LS_MAX_TASKS tasks
// (angle, chunk of 31 lines).  The group size fills the task table.
constexpr int DC_LS_MAX_MG = 16;
constexpr int DC_LS_MAX_TASKS = 256;
inline int linesum_group_size(int n_s) {
  int chunks = (n_s - 1 + 30) / 31;
  if (chunks < 1) chunks = 1;
  int mg = DC_LS_MAX_TASKS / chunks;
  return mg < 1 ? 1 : (mg > DC_LS_MAX_MG ? DC_LS_MAX_MG : mg);
}

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
  dc::VMu *vmu;              // [V][n_mu]
  int *mu_order;             // [n_mu] angle index in group order
  dc::MuGroup *groups;       // [n_groups]
  int n_groups;
  int n_groups_branch0;
  int mg;                    // max angles per group
  // work area
  int chunk_images;          // images (view x batch item) per chunk
  int chunk_capacity;        // images the work area was sized for
  int bp_nz;                 // voxels per thread along z in the backprojector (16, 32)
  size_t img_stride;         // floats per padded image  (H * Wp)
  size_t sino_stride;        // floats per padded sinogram (n_mu * NSp)
  int Wp, NSp;               // padded row lengths (multiples of 4)
  int ls_rb;                 // line-sum band height (32, 16 or 8 rows)
  float *w_img;              // [chunk][H][Wp]
  float *w_sinoA;            // [chunk][n_mu][NSp]
  float *w_sinoB;            // [chunk][n_mu][NSp]
  unsigned *w_absmax;        // [chunk]
  unsigned *w_flags;         // [4] device-side error bits (bit 0: wait timeout)
  // streams and events of dc_reconstruct_host (created by its first call)
  int aux_ready;
  cudaStream_t aux_copy, aux_compute;
  cudaEvent_t aux_ev[8];
};

namespace dc {

// host-side helpers defined in dc_filter.cu / dc_backproject.cu
int alloc_workspace(dc_geometry *g);
int build_mu_tables(dc_geometry *g);
// argument checks of the filter entry points (DC_OK or the error code)
int filter_check(const dc_geometry *g, int B, const float *gin, const void *gF, int dtype,
                 const float *gF_scale, const char *who);
// chunk sizes: bc batch items of cv views per chunk of the work area
void filter_chunk_plan(const dc_geometry *g, int B, int *bc, int *cv);
// the filter of one chunk: views [v0, v0 + nv) of items [b0, b0 + bc)
// (S: optional [B][V][n_mu][n_s] copy of Grangeat's function, or NULL)
int filter_chunk(const dc_geometry *g, const float *gin, const float *W, void *gF, int dtype,
                 float *gF_scale, int b0, int bc, int v0, int nv, cudaStream_t st,
                 float *S = nullptr);
// checks of dc_backproject's arguments
int backproject_check(const dc_geometry *g, int B, const void *gF, int dtype,
                      const float *gF_scale, const float *vol, unsigned flags, const char *who);
// backprojection of the z range [z_begin, z_end) of every batch item with the
// TMA kernel; *used = false (nothing launched) when that kernel cannot run
int backproject_slab(const dc_geometry *g, int B, const void *gF, int dtype,
                     const float *gF_scale, float *vol, unsigned flags, int z_begin, int z_end,
                     cudaStream_t st, bool *used);
// the batched persistent filter (dc_filter.cu): one launch filters every
// view of up to 32 problems into the given g^F buffers (and FP16 scales)
struct BatchFilterPlan;
int batch_filter_create(int n, dc_geometry *const *geoms, int dtype, void *const *gF,
                        float *const *scale, BatchFilterPlan **out);
int batch_filter_run(BatchFilterPlan *p, const float *const *g, const float *const *W,
                     cudaStream_t st);
void batch_filter_destroy(BatchFilterPlan *p);
// FP64 split of v into hi (12 fractional bits) + lo
inline __host__ __device__ float split_hi12(double v) {
  return (float)(rint(v * 4096.0) / 4096.0);
}

// The Joseph branch of angle m = mu_m / (pi / n_mu), decided exactly by
// integers: rows (|cos| > |sin|) when 4m < n_mu or 4m >= 3 n_mu.  Of the two
// 45-degree ties, mu = pi/4 steps over columns and mu = 3pi/4 over rows, so
// that each branch has n_mu / 2 angles when 4 divides n_mu (equal angle
// groups for the line sums); on a line of slope +-1 both branches sample the
// same points with the same weights, so the tie may go either way.
inline __host__ __device__ bool joseph_rows(int m, int n_mu) {
  return (4 * m < n_mu) || (4 * m >= 3 * n_mu);
}

// The per-angle record of angle m, from FP64 (host or device).
inline __host__ __device__ MuRec make_mu_rec(int m, int n_mu, double pitch, double ds) {
  double ang = m * 3.14159265358979323846 / n_mu, c = cos(ang), s = sin(ang);
  bool rows = joseph_rows(m, n_mu);
  double cs = rows ? c : s, sn = rows ? s : c;
  double mx = fabs(cs);
  MuRec r;
  r.c = (float)c;
  r.s = (float)s;
  r.jscale = (float)(pitch / mx);
  r.winv = (float)(ds / (pitch * mx));
  double A = (ds / pitch) / cs, dx = -sn / cs, bc = c * pitch / ds, bs = s * pitch / ds;
  r.a_hi = split_hi12(A);
  r.a_lo = (float)(A - (double)r.a_hi);
  r.d_hi = split_hi12(dx);
  r.d_lo = (float)(dx - (double)r.d_hi);
  r.dxi = (float)dx;
  r.bc_hi = split_hi12(bc);
  r.bc_lo = (float)(bc - (double)r.bc_hi);
  r.bs_hi = split_hi12(bs);
  r.bs_lo = (float)(bs - (double)r.bs_hi);
  r.pad0 = r.pad1 = r.pad2 = 0.0f;
  return r;
}

// the FP64 origins of one (view, angle): see VMu
inline __host__ __device__ VMu make_vmu(int m, int n_mu, int n_s, double pitch, double ds,
                                        double cu, double cv) {
  double ang = m * 3.14159265358979323846 / n_mu, c = cos(ang), s = sin(ang);
  bool rows = joseph_rows(m, n_mu);
  double cs = rows ? c : s, sn = rows ? s : c;
  double ccol = rows ? cu : cv, crow = rows ? cv : cu;
  double b0 = ccol + crow * sn / cs;
  double xo = 0.5 * (n_s - 1) - (cu * c + cv * s) * pitch / ds;
  VMu r;
  r.b0i = (float)floor(b0);
  r.b0f = (float)(b0 - floor(b0));
  r.xoi = (float)floor(xo);
  r.xof = (float)(xo - floor(xo));
  return r;
}

}  // namespace dc
