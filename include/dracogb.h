/*
 * dracogb.h -- C ABI of the GB300 (sm_103a) Defrise-Clack shift-variant
 * filtered backprojection for arbitrary cone-beam orbits (Ye et al., DRACO,
 * arXiv 2410.14900, Sec. 2.2-2.3).
 *
 * The method (Eq. 12):
 *     f = A3d^T w_d A2d^T D w_red w_sino D A2d w_cos g
 * is split into two calls:
 *     dc_filter       g   -> g^F = w_d A2d^T D w_red w_sino D A2d w_cos g
 *                            (Eqs. 7, 8, 10, 11)
 *     dc_backproject  g^F -> f = A3d^T g^F  (Eq. 5), optional ReLU
 * plus their reverse-mode adjoints, so that the redundancy weights (the only
 * trainable layer, Eq. 10) and the projections can be differentiated.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Units: mm and radians.  Row-major, contiguous arrays.
 *  - Projections g, g^F: [B][V][H][W] (detector column index fastest).
 *  - Volumes f: [B][Z][Y][X] (x fastest).  Voxel (ix,iy,iz) sits at
 *    vol_center + ((ix-(X-1)/2) dx, (iy-(Y-1)/2) dy, (iz-(Z-1)/2) dz).
 *  - Sinogram axes per view: mu_m = m pi / n_mu (m < n_mu),
 *    s_k = (k - (n_s-1)/2) ds, measured from the principal point of the
 *    detector (foot of the perpendicular from the source) along
 *    (cos mu, sin mu) in the detector frame (l_x, l_y).
 *  - Redundancy weights W: [V][n_mu][n_s]; entry k refers to the half-grid
 *    abscissa s_{k+1/2} = s_k + ds/2 (the entry k = n_s-1 is unused).  The
 *    library multiplies W by K = -(1/4pi^2)|v_i . theta| / sqrt(s^2+D^2),
 *    where v_i = a'(lambda_i) dlambda_i; W = 1/2 is the exact circular-orbit
 *    value (Eq. 14, M = 1/2).
 *  - Projection matrices P: [V][3][4] FP64, host memory, mapping a
 *    homogeneous world point to (col*w, row*w, w), w > 0 in front of the
 *    source.  Pixels must be square with pitch `pitch`, without skew.
 *  - Ownership: every array argument is caller-owned.  Pointers documented as
 *    "device" must be CUDA device (or managed) memory on the current device;
 *    "host" pointers are ordinary host memory.  The geometry handle owns only
 *    its own device buffers (geometry tables and a work area).
 *  - Execution: every compute call is asynchronous on the given stream
 *    (a cudaStream_t passed as void*, NULL = the legacy default stream).  A
 *    handle's work area is shared by its calls: do not use one handle on two
 *    streams at the same time.  dc_setup_geometry is synchronous.
 *  - Errors: every int-returning call returns DC_OK (0) or a DC_ERR_* code
 *    and never throws; argument errors are detected before any work is
 *    launched.  dc_last_error() gives a message for the calling thread's
 *    last failure.
 */
#ifndef DRACOGB_H
#define DRACOGB_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DC_OK 0
#define DC_ERR_ARG 1          /* invalid argument (NULL, size, layout)      */
#define DC_ERR_CUDA 2         /* a CUDA runtime call or launch failed       */
#define DC_ERR_OOM 3          /* device allocation failed                   */
#define DC_ERR_TIMEOUT 4      /* a bounded device wait gave up              */
#define DC_ERR_UNSUPPORTED 5  /* valid request this build does not handle  */
#define DC_ERR_NONFINITE 6    /* a NaN / infinite redundancy weight was read
                                 (reported by dc_sync_status)               */

/* storage types of the filtered projections g^F */
#define DC_F32 0
#define DC_BF16 1             /* round-to-nearest-even                      */
#define DC_F16 2              /* with a per-view power-of-two scale         */
/* FP32 (value, right difference) pairs: pixel (r, c) of g^F is stored as
 * the two floats g[r][c] and g[r][c+1] - g[r][c] (g[r][W] = 0), i.e.
 * [B][V][H][W][2] FP32, 16-byte aligned.  The same values as DC_F32 at twice
 * the bytes; the backprojection reads its interpolation tiles in place
 * instead of building them. */
#define DC_F32X2 3

/* dc_backproject flags */
#define DC_ACCUM 1u           /* add into vol instead of overwriting        */
#define DC_KAHAN 2u           /* compensated (Kahan) summation over views   */
#define DC_RELU 4u            /* ReLU after the sum over views (Sec. 2.3)   */
/* dc_batch_create flag: filter every problem in one persistent launch */
#define DC_PERSISTENT_FILTER 8u

/* maximum number of orbit segments of dc_crofton_weights */
#define DC_MAX_SEGMENTS 16

/* doubles per view returned by dc_get_view_geometry */
#define DC_VIEW_GEO_N 24

typedef struct {
  int n_views;          /* V                                              */
  int det_rows;         /* H                                              */
  int det_cols;         /* W                                              */
  int n_mu;             /* angles of the per-view 2D Radon transform      */
  int n_s;              /* s-bins of the per-view 2D Radon transform      */
  double pitch;         /* detector pixel pitch (mm), square pixels       */
  double ds;            /* s-bin spacing (mm), ds >= pitch / 3            */
  int vol_x, vol_y, vol_z;
  double voxel[3];      /* voxel size (dx, dy, dz) in mm                  */
  double vol_center[3]; /* world position of the volume centre (mm)       */
  int closed_orbit;     /* 1: the orbit is a closed curve (only used when
                           the tangents are derived by finite differences) */
} dc_geometry_desc;

typedef struct dc_geometry dc_geometry;

/*
 * dc_setup_geometry -- per-view geometry of Fig. 1 (Sec. 2.3) from the
 * projection matrices, computed in FP64 on the GPU: source a = -M^-1 p4,
 * detector frame (l_x, l_y, l_z), source-detector distance D, principal
 * point, and the orbit tangent v_i = a'(lambda_i) dlambda_i that enters the
 * redundancy weight of Eq. 10.
 *   desc : host, sizes and spacings (see the struct).
 *   P    : host, [V][3][4] FP64.  Any nonzero scale; the sign is chosen so
 *          that the volume centre has positive depth.
 *   vdl  : host, [V][3] FP64 tangents a'(lambda)dlambda, or NULL to use
 *          central differences of the sources (one-sided at the ends of an
 *          open orbit, wrapped for closed_orbit = 1).
 *   out  : receives the handle (destroy with dc_destroy_geometry).
 * Returns DC_ERR_ARG for invalid sizes, a singular matrix, skew or
 * non-square pixels; DC_ERR_OOM / DC_ERR_CUDA on device failures.
 * Synchronous; uses the current CUDA device.
 */
int dc_setup_geometry(const dc_geometry_desc *desc, const double *P, const double *vdl,
                      dc_geometry **out);

/* Frees the handle and its device buffers (NULL is ignored). */
void dc_destroy_geometry(dc_geometry *geom);

/*
 * dc_get_view_geometry -- copies the FP64 per-view geometry to host memory:
 * out[V][DC_VIEW_GEO_N] = { a[3], l_x[3], l_y[3], l_z[3], D, c_u, c_v,
 * v[3], |v|, 0, 0, 0 } (Fig. 1; c_u, c_v = principal point in pixels).
 */
int dc_get_view_geometry(const dc_geometry *geom, double *out);

/*
 * dc_filter -- the shift-variant filter of Eq. 11 applied to Grangeat's
 * intermediate function of Eq. 7, for every view of every batch item:
 *     g^F = w_d A2d^T D_b (W K) w_sino D_f A2d w_cos g
 * A2d is Joseph's discrete 2D Radon transform over (mu, s); D_f/D_b are the
 * forward/backward s-differences; A2d^T is the transpose of the Joseph
 * weights times (pi/n_mu) ds/pitch^2 (the discrete integral over mu of
 * Eq. 8); w_cos = D/sqrt(x^2+y^2+D^2), w_sino = (s^2+D^2)/D^2,
 * w_d = x^2+y^2+D^2.
 *   B       : batch size (>= 1); all items share the geometry and W.
 *   g       : device, [B][V][H][W] FP32 projections.
 *   W       : device, [V][n_mu][n_s] FP32 redundancy weights, or NULL for
 *             the constant 1/2 (exact for a full circle, Eq. 14).
 *   gF      : device, [B][V][H][W] output in `dtype` (DC_F32, DC_BF16,
 *             DC_F16), or [B][V][H][W][2] FP32 for DC_F32X2 (16-byte aligned).
 *   gF_scale: device, [B][V] FP32, required for DC_F16 (g^F = half * scale),
 *             ignored otherwise.
 * Requires ds >= pitch / 3 (below pitch a pixel meets up to six lines).
 */
int dc_filter(const dc_geometry *geom, int B, const float *g, const float *W, void *gF,
              int dtype, float *gF_scale, void *stream);

/*
 * dc_filter_adjoint -- reverse mode of dc_filter (FP32 g^F): given
 * grad_gF = dL/dg^F, writes dL/dg and dL/dW.  Grangeat's function S is
 * recomputed from g view-chunk by view-chunk, so nothing from the forward
 * pass needs to be kept.
 *   grad_gF : device, [B][V][H][W] FP32.
 *   g       : device, [B][V][H][W] FP32 (the forward input).
 *   W       : device, [V][n_mu][n_s] FP32 or NULL (= 1/2).
 *   grad_g  : device, [B][V][H][W] FP32 output, or NULL to skip.
 *   grad_W  : device, [V][n_mu][n_s] FP32 output summed over the batch
 *             (overwritten), or NULL to skip.
 *   view_chunk: views processed together (0 = library default).
 */
int dc_filter_adjoint(const dc_geometry *geom, int B, const float *grad_gF, const float *g,
                      const float *W, float *grad_g, float *grad_W, int view_chunk,
                      void *stream);

/*
 * dc_filter_with_s / dc_filter_adjoint_from_s -- the same forward and
 * reverse mode with Grangeat's function S (Eq. 7) kept in between instead of
 * recomputed: the forward writes S, [B][V][n_mu][n_s] FP32 device (entry
 * n_s-1 = 0), as a by-product of the filter; the reverse mode reads it and
 * skips one line-sum pass over the projections.  Costs B*V*n_mu*n_s floats
 * of caller memory; the results equal dc_filter / dc_filter_adjoint.
 * Arguments as there; dc_filter_adjoint_from_s takes S in place of g.
 */
int dc_filter_with_s(const dc_geometry *geom, int B, const float *g, const float *W, void *gF,
                     int dtype, float *gF_scale, float *S, void *stream);
int dc_filter_adjoint_from_s(const dc_geometry *geom, int B, const float *grad_gF,
                             const float *S, const float *W, float *grad_g, float *grad_W,
                             int view_chunk, void *stream);

/*
 * dc_backproject -- voxel-driven cone-beam backprojection of Eq. 5:
 *     f(X) = sum_i bilinear(g^F_i, P_i X) / |X - a_i|^2
 * Pixels outside the detector count as zero; voxels with depth <= 0 in a
 * view get nothing from it.  Interpolation and accumulation are FP32 for
 * every storage type.
 *   gF      : device, [B][V][H][W] in `dtype` ([B][V][H][W][2] FP32 for
 *             DC_F32X2); gF_scale [B][V] for DC_F16.
 *   vol     : device, [B][Z][Y][X] FP32, overwritten (or added to with
 *             DC_ACCUM).
 *   flags   : DC_ACCUM | DC_KAHAN | DC_RELU.
 */
int dc_backproject(const dc_geometry *geom, int B, const void *gF, int dtype,
                   const float *gF_scale, float *vol, unsigned flags, void *stream);

/*
 * dc_backproject_adjoint -- transpose of dc_backproject (a voxel-driven
 * cone-beam forward projector with the same bilinear weights and the same
 * 1/|X - a|^2 factor):
 *     grad_gF_i[pixel] = sum_X w_bilinear(pixel; P_i X) grad_vol(X) / |X-a_i|^2
 *   grad_vol: device, [B][Z][Y][X] FP32.
 *   relu_vol: device, [B][Z][Y][X] FP32 forward output when the forward used
 *             DC_RELU (grad_vol is masked where relu_vol <= 0), else NULL.
 *   grad_gF : device, [B][V][H][W] FP32, overwritten.
 */
int dc_backproject_adjoint(const dc_geometry *geom, int B, const float *grad_vol,
                           const float *relu_vol, float *grad_gF, void *stream);

/*
 * dc_reconstruct_host -- Eq. 12 from host projections to a host volume
 * (dc_filter followed by dc_backproject) with the transfers overlapped:
 * the projections go up in view chunks on an internal copy stream, each
 * chunk's filter waiting only for its own upload, and the volume is
 * backprojected in n_slabs z-slabs (0: 16; at most one per 32 or 16 voxel
 * planes) whose downloads overlap the later slabs.  The result equals dc_filter + dc_backproject on the same data.
 *   g_host  : host, [B][V][H][W] FP32; vol_host: host, [B][Z][Y][X] FP32.
 *             Page-locked memory (cudaHostAlloc / pinned tensors) is needed
 *             for the overlap; pageable memory works but serialises.
 *   g_dev, gF, vol_dev: device buffers of the sizes dc_filter and
 *             dc_backproject take (caller-owned; g_dev receives the upload).
 *   W, dtype, gF_scale, flags: as for dc_filter / dc_backproject.
 * All work is ordered on `stream`: when it completes, vol_host holds the
 * volume.  The first call on a handle creates its two internal streams and
 * events (released by dc_destroy_geometry).
 */
int dc_reconstruct_host(const dc_geometry *geom, int B, const float *g_host, const float *W,
                        float *g_dev, void *gF, int dtype, float *gF_scale, float *vol_dev,
                        float *vol_host, unsigned flags, int n_slabs, void *stream);

/*
 * dc_crofton_weights -- the smooth Crofton weights of Eq. 9 as redundancy
 * weights W for dc_filter (the analytic alternative to learned weights):
 *   M(theta, lambda_i) = |v_i.theta|^m c_i / sum_alpha |v_alpha.theta|^m c_alpha
 * for every view i and plane (mu_m, s_{k+1/2}) through the source.  The
 * intersections alpha of the plane with the orbit are view i and each sign
 * change of (a_j - a_i).theta between consecutive views of a segment (tangent
 * and c interpolated linearly at the crossing).  c = 1 except within `taper`
 * views of the ends of an open segment (c = sin^2(pi/2 (d + 1/2)/taper) at
 * distance d from the end).
 *   n_seg, seg_start, seg_closed: host arrays describing the orbit's pieces,
 *     view ranges [seg_start[q], seg_start[q+1]) with seg_start[0] = 0; n_seg
 *     = 0 means one piece, closed as the descriptor says.
 *   m: 0..8 (m = 0 gives 1/n, the Crofton symbol itself).
 *   W: device, [V][n_mu][n_s] FP32, written (entry n_s-1 = 0; 0 where
 *     v_i.theta = 0).
 * A full circle gives 1/2 wherever the plane is not tangent to the orbit.
 */
int dc_crofton_weights(const dc_geometry *geom, int n_seg, const int *seg_start,
                       const int *seg_closed, int m, int taper, float *W, void *stream);

/*
 * dc_gauss_smooth -- the Gaussian filter layer the paper places after the
 * learned redundancy weight (Sec. 3.1: sigma 20, kernel size 121, i.e.
 * radius 60), or its transpose for the reverse mode.  Per view, W[mu][k] is
 * filtered along mu and along s over the valid entries k < n_s - 1; entry
 * n_s - 1 is copied through.  Taps exp(-t^2/(2 sigma^2)) for |t| <= radius,
 * normalised to unit sum; each line is extended by mirroring about its end
 * samples (index -1 reads 1, index n reads n - 2).
 *   in, out : device, [V][n_mu][n_s] FP32; out is written.
 *   work    : device scratch of V*n_mu*n_s floats, owned by the caller.
 *   adjoint : 0 applies the filter, 1 its transpose.
 * in, out and work must be distinct.  DC_ERR_ARG for bad sizes, sigma <= 0
 * or radius outside [0, 1024]; DC_ERR_UNSUPPORTED when a line and its halo
 * do not fit in shared memory (n_mu or n_s plus 4 radius beyond ~25000).
 */
int dc_gauss_smooth(int V, int n_mu, int n_s, float sigma, int radius, int adjoint,
                    const float *in, float *out, float *work, void *stream);

/*
 * Batched reconstruction of several problems (orbits with uneven view
 * counts, detectors and volumes): Eq. 12 for each, with the backprojection
 * of all problems done by one persistent kernel that takes (problem, voxel
 * box) items from a device counter, largest view count first.
 *
 * dc_batch_create -- plans a batch of n <= 32 geometries (not owned; they
 *   must outlive the batch) for g^F storage `dtype` and flags DC_KAHAN |
 *   DC_RELU | DC_PERSISTENT_FILTER.  Allocates the batch's filtered
 *   projections and tables.  Every detector row must be a multiple of 16
 *   bytes in `dtype` (tiled TMA loads).
 * dc_batch_run -- g[i]: device [V_i][H_i][W_i] FP32; W[i]: device
 *   [V_i][n_mu_i][n_s_i] or NULL entries (W itself may be NULL: all 1/2);
 *   vol[i]: device [Z_i][Y_i][X_i] FP32, overwritten.  Allocates nothing, so
 *   a run can be captured in a CUDA graph and replayed with the same
 *   pointers.  Uses each geometry's work area: one run at a time per batch.
 * dc_batch_set_bp_nz -- voxels per thread along z in the backprojection:
 *   16 or 32 for every problem, or 0 (the default) for each geometry's own
 *   bp_nz (dc_geometry_set_tuning), for the autotuner.
 *
 * The backprojection of a run is one persistent launch over (problem,
 * voxel box) items.  The filter is, by default, each problem's dc_filter
 * (chunked launches, recorded in the same graph); with
 * DC_PERSISTENT_FILTER it is one persistent launch whose CTAs (one per SM)
 * take (problem, view) images from a device counter, largest per-image
 * work first, so the whole run is two persistent launches.  (On GB300 that
 * kernel runs its 2-D backprojection at half the warps per SM of the
 * chunked kernel and is ~11% slower; it is kept for launch-bound uses.)
 * With the flag, problems whose detector or sinogram rows do not fit that
 * kernel's shared memory fall back to the per-problem calls, and so does
 * every problem of a DC_F32X2 batch (the pairs are made by the chunked
 * filter's pass over each finished image).
 */
typedef struct dc_batch dc_batch;
int dc_batch_create(int n, dc_geometry *const *geoms, int dtype, unsigned flags,
                    dc_batch **out);
int dc_batch_run(dc_batch *batch, const float *const *g, const float *const *W,
                 float *const *vol, void *stream);
int dc_batch_set_bp_nz(dc_batch *batch, int nz);
void dc_batch_destroy(dc_batch *batch);

/*
 * Tuning knobs of a geometry handle (chosen by the autotuner):
 * chunk_images -- images (view x batch item) the filter processes together,
 *   1 <= chunk_images <= the capacity its work area was sized for;
 * bp_nz -- voxels per thread along z in the backprojection (16 or 32).
 * 0 keeps a value.  dc_geometry_get_tuning reads them (any pointer may be
 * NULL).
 */
int dc_geometry_set_tuning(dc_geometry *geom, int chunk_images, int bp_nz);
int dc_geometry_get_tuning(const dc_geometry *geom, int *chunk_images, int *chunk_capacity,
                           int *bp_nz);

/*
 * Per-step entry points (the layers of Fig. 2), for testing and for callers
 * that compose the network themselves.
 *
 * dc_grangeat -- S = w_sino D_f A2d w_cos g (Eq. 7) on the half grid
 *   s_{k+1/2}: g device [B][V][H][W] FP32 -> S device [B][V][n_mu][n_s] FP32
 *   (entry k = n_s-1 is zero).
 * dc_radon2d -- Joseph A2d of arbitrary detector images, one per view of the
 *   geometry (principal point of that view): img device [B][V][H][W] FP32 ->
 *   R device [B][V][n_mu][n_s] FP32.
 * dc_radon2d_adjoint -- the exact transpose of dc_radon2d (no mu-integral
 *   scale): R device [B][V][n_mu][n_s] -> img device [B][V][H][W], overwritten.
 */
int dc_grangeat(const dc_geometry *geom, int B, const float *g, float *S, void *stream);
int dc_radon2d(const dc_geometry *geom, int B, const float *img, float *R, void *stream);
int dc_radon2d_adjoint(const dc_geometry *geom, int B, const float *R, float *img,
                       void *stream);

/*
 * dc_sync_status -- waits for `stream`, then reports device-side failures of
 * this handle's kernels since the last call: DC_ERR_TIMEOUT if a bounded
 * wait inside a kernel gave up (the kernel then skipped its output), else
 * DC_ERR_NONFINITE if a filter call (forward or reverse mode) read a NaN or
 * infinite redundancy weight W (the outputs that depend on that weight are
 * then NaN; no other output is affected).  Clears the flags.  Compute calls
 * never block, so they cannot report these themselves.
 */
int dc_sync_status(const dc_geometry *geom, void *stream);

/*
 * dc_deriv -- the s-derivatives of Eqs. 7 and 11 on their own (the filter
 * fuses them): in, out device [B][V][n_mu][n_s] FP32, distinct.
 *   kind 0: D_f, out[k] = (in[k+1] - in[k]) / ds on s_{k+1/2}, out[n_s-1] = 0
 *   kind 1: D_f^T
 *   kind 2: D_b, out[k] = (in[k] - in[k-1]) / ds with in[-1] = 0
 *   kind 3: D_b^T
 * Each difference is divided by ds in FP32, as in the filter's fused
 * derivatives; the results agree with those to FP32 rounding (the fused
 * path differences per-band partial line sums).
 */
int dc_deriv(const dc_geometry *geom, int B, const float *in, float *out, int kind,
             void *stream);

/*
 * dc_radon2d_noalloc -- the Joseph 2D Radon transform of dc_radon2d for
 * callers that cannot allocate device memory: a real-time loop whose memory
 * budget is fixed before the scan and must never wait on CUDA's
 * allocator, or a host that embeds this library inside another runtime's
 * memory pool and cannot create a geometry handle.  The paper has no
 * counterpart; it is an interface variant.  It allocates nothing and needs
 * no handle: its work area is a fixed 32 MiB array compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *   img   : device, [n_img][H][W] FP32 detector images (caller-owned).
 *   R     : device, [n_img][n_mu][n_s] FP32 line sums (caller-owned).
 *   cu, cv: principal point (column, row) shared by all images; pitch, ds,
 *           mu_m = m pi / n_mu and s_k as for a geometry handle.
 * Limits: n_mu <= 2048; one image needs H * round4(W) * 4 bytes of the fixed
 * area (its weighted copy with rows padded to a multiple of 4 floats), at
 * most 32 MiB - 256 KiB (larger requests return DC_ERR_ARG with the
 * numbers); images are processed in groups that fit.
 * The first call on a device (and the first after that device's context
 * changed, e.g. after cudaDeviceReset) looks up the array's device address
 * (set-up); make that first call before any stream capture.  All calls share
 * the array and it keeps the last call's contents: calls that overlap on the
 * GPU (two streams, two threads) race on it and must be serialised by the
 * caller.
 */
int dc_radon2d_noalloc(int n_img, int H, int W, int n_mu, int n_s, double pitch, double ds,
                       double cu, double cv, const float *img, float *R, void *stream);

/* Human-readable name of a status code (static storage). */
const char *dc_status_string(int status);

/* Message of the calling thread's most recent failure ("" if none). */
const char *dc_last_error(void);

/* Number of kernel launches this library has issued in this process. */
unsigned long long dc_launch_count(void);

/*
 * Launch profiler.  While enabled, every kernel launch of this library is
 * bracketed by CUDA events recorded on the launching stream.
 * dc_profile_enable returns the previous state.  dc_profile_collect waits for
 * the recorded events, writes per kernel id the summed device time (ms) and
 * launch count since the previous collect into ms[n] / launches[n] (either
 * may be NULL), resets the sums and returns the number of kernel ids.
 * dc_profile_kernel_name maps an id to the kernel's name.
 */
int dc_profile_enable(int on);
int dc_profile_collect(double *ms, unsigned long long *launches, int n);
const char *dc_profile_kernel_name(int id);

/* Library version string (static storage). */
const char *dc_version(void);

/*
 * dc_microbench -- measurement helper (the paper has no counterpart): runs
 * the bare inner step of one gather kernel on a resident shared-memory tile
 * so that its practical peak can be timed (CUDA events around the call):
 * kind 0 the Joseph step of the line sums, 1 the transposed-hat pair of the
 * 2-D backprojection, 2 the bilinear sample of the cone-beam
 * backprojection, 3 that sample times the voxel weight 1/|X - a|^2, 4 the
 * weighted sample from a tile of quads (both rows' value and difference of
 * a pixel), two voxels per step in packed FP32x2.  n_blocks CTAs of 512
 * threads each run iters x 32 samples per thread; sink (device,
 * n_blocks*512 floats) receives their sums.
 */
int dc_microbench(int kind, int n_blocks, int iters, float *sink, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DRACOGB_H */
