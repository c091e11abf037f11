// dc_geometry.cu -- per-view geometry (paper Fig. 1) from 3x4 projection
// matrices, in FP64 on the GPU, and the FP32 tables the compute kernels use.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dc_common.cuh"

namespace {

constexpr int GN = DC_VIEW_GEO_N;  // a(3) lx(3) ly(3) lz(3) D cu cv v(3) |v| pad

__device__ inline double det3(const double m[3][3]) {
  return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
         m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
         m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

__device__ inline double ddot(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// One thread per view.  P = s [A | -A a] with A rows f l_x - c_u l_z,
// f l_y - c_v l_z, -l_z (f = D / pitch).  Writes the frame, D, principal
// point and the source; status[i] = 1 for a singular / skewed matrix.
__global__ void k_geometry_frames(int V, double pitch, double cx, double cy, double cz,
                                  const double *__restrict__ P, double *__restrict__ geo,
                                  double *__restrict__ Pn, int *__restrict__ status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  const double *Pi = P + 12 * i;
  double *g = geo + (size_t)GN * i;
  for (int t = 0; t < GN; ++t) g[t] = 0.0;
  status[i] = 1;
  double sc = sqrt(Pi[8] * Pi[8] + Pi[9] * Pi[9] + Pi[10] * Pi[10]);
  if (!(sc > 0.0)) return;
  double wc = Pi[8] * cx + Pi[9] * cy + Pi[10] * cz + Pi[11];
  if (wc < 0.0) sc = -sc;
  double n[12];
  for (int t = 0; t < 12; ++t) n[t] = Pi[t] / sc;
  double M[3][3] = {{n[0], n[1], n[2]}, {n[4], n[5], n[6]}, {n[8], n[9], n[10]}};
  double p4[3] = {n[3], n[7], n[11]};
  double det = det3(M);
  if (fabs(det) < 1e-300) return;
  double a[3];
  for (int c = 0; c < 3; ++c) {
    double Mc[3][3];
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) Mc[r][q] = (q == c) ? p4[r] : M[r][q];
    a[c] = -det3(Mc) / det;
  }
  double lz[3] = {-n[8], -n[9], -n[10]};
  double r1[3] = {n[0], n[1], n[2]}, r2[3] = {n[4], n[5], n[6]};
  double cu = -ddot(r1, lz), cv = -ddot(r2, lz);
  double fx[3], fy[3];
  for (int c = 0; c < 3; ++c) {
    fx[c] = r1[c] + cu * lz[c];
    fy[c] = r2[c] + cv * lz[c];
  }
  double nfx = sqrt(ddot(fx, fx)), nfy = sqrt(ddot(fy, fy));
  if (!(nfx > 0.0) || !(nfy > 0.0)) return;
  if (fabs(nfx - nfy) > 1e-9 * nfx) return;
  double lx[3], ly[3];
  for (int c = 0; c < 3; ++c) {
    lx[c] = fx[c] / nfx;
    ly[c] = fy[c] / nfy;
  }
  if (fabs(ddot(lx, ly)) > 1e-9) return;
  for (int c = 0; c < 3; ++c) {
    g[0 + c] = a[c];
    g[3 + c] = lx[c];
    g[6 + c] = ly[c];
    g[9 + c] = lz[c];
  }
  g[12] = nfx * pitch;
  g[13] = cu;
  g[14] = cv;
  for (int t = 0; t < 12; ++t) Pn[12 * i + t] = n[t];
  status[i] = 0;
}

// One thread per view: tangent v = a'(lambda) dlambda (given, or central
// differences of the sources), the plane-normal dot products v.l_x, v.l_y,
// v.l_z of the redundancy weight (Eq. 10), and the FP32 tables.
__global__ void k_geometry_tables(int V, int closed, double pitch, double cx, double cy,
                                  double cz, const double *__restrict__ vdl,
                                  double *__restrict__ geo, dc::BPView *__restrict__ bpv,
                                  dc::FView *__restrict__ fv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  double *g = geo + (size_t)GN * i;
  double v[3] = {0.0, 0.0, 0.0};
  if (vdl) {
    for (int c = 0; c < 3; ++c) v[c] = vdl[3 * i + c];
  } else if (V >= 2) {
    int ip = i + 1, im = i - 1;
    double half = 0.5;
    if (closed) {
      ip = (i + 1) % V;
      im = (i - 1 + V) % V;
    } else if (i == 0) {
      im = 0;
      half = 1.0;
    } else if (i == V - 1) {
      ip = V - 1;
      half = 1.0;
    }
    const double *ap = geo + (size_t)GN * ip, *am = geo + (size_t)GN * im;
    for (int c = 0; c < 3; ++c) v[c] = half * (ap[c] - am[c]);
  }
  for (int c = 0; c < 3; ++c) g[15 + c] = v[c];
  g[18] = sqrt(ddot(v, v));
  const double *a = g, *lx = g + 3, *ly = g + 6, *lz = g + 9;
  double D = g[12], f = D / pitch;
  double ca[3] = {cx - a[0], cy - a[1], cz - a[2]};
  double m0[3], m1[3], m2[3];
  for (int c = 0; c < 3; ++c) {
    m0[c] = f * lx[c];
    m1[c] = f * ly[c];
    m2[c] = -lz[c];
  }
  dc::BPView b;
  b.r0 = make_float4((float)m0[0], (float)m0[1], (float)m0[2], (float)ddot(m0, ca));
  b.r1 = make_float4((float)m1[0], (float)m1[1], (float)m1[2], (float)ddot(m1, ca));
  b.r2 = make_float4((float)m2[0], (float)m2[1], (float)m2[2], (float)ddot(m2, ca));
  // a view whose u and depth do not change along z (circle about the z axis)
  float circ = (b.r0.z == 0.0f && b.r2.z == 0.0f) ? 1.0f : 0.0f;
  b.ca = make_float4((float)ca[0], (float)ca[1], (float)ca[2], circ);
  b.pp = make_float4((float)g[13], (float)g[14], 0.0f, 0.0f);
  bpv[i] = b;
  dc::FView r;
  r.D = (float)D;
  r.cu = (float)g[13];
  r.cv = (float)g[14];
  r.ax = (float)ddot(v, lx);
  r.ay = (float)ddot(v, ly);
  r.az = (float)ddot(v, lz);
  r.pad0 = r.pad1 = 0.0f;
  fv[i] = r;
}

// One thread per (view, angle): FP64 origins of the line-sum and pixel
// gathers (the principal point enters here).
__global__ void k_geometry_angles(int V, int n_mu, int n_s, double pitch, double ds,
                                  const double *__restrict__ geo, dc::VMu *__restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= V * n_mu) return;
  int i = t / n_mu, m = t % n_mu;
  const double *g = geo + (size_t)GN * i;
  out[t] = dc::make_vmu(m, n_mu, n_s, pitch, ds, g[13], g[14]);
}

void free_geometry(dc_geometry *g) {
  if (!g) return;
  cudaFree(g->geo64);
  cudaFree(g->bpv);
  cudaFree(g->fv);
  cudaFree(g->mu);
  cudaFree(g->vmu);
  cudaFree(g->mu_order);
  cudaFree(g->groups);
  cudaFree(g->w_img);
  cudaFree(g->w_sinoA);
  cudaFree(g->w_sinoB);
  cudaFree(g->w_absmax);
  cudaFree(g->w_flags);
  if (g->aux_ready) {
    cudaStreamDestroy(g->aux_copy);
    cudaStreamDestroy(g->aux_compute);
    for (int i = 0; i < 8; ++i) cudaEventDestroy(g->aux_ev[i]);
  }
  free(g->host_geo);
  delete g;
}

}  // namespace

namespace dc {

// Angle tables: cos/sin in FP64 -> FP32, the Joseph branch decided exactly by
// an integer test (joseph_rows), and groups of angles of one branch for the
// line-sum kernel.
int build_mu_tables(dc_geometry *g) {
  const dc_geometry_desc &d = g->d;
  int n_mu = d.n_mu;
  std::vector<MuRec> mu(n_mu);
  std::vector<int> b0, b1;
  for (int m = 0; m < n_mu; ++m) {
    bool rows = joseph_rows(m, n_mu);
    mu[m] = make_mu_rec(m, n_mu, d.pitch, d.ds);
    (rows ? b0 : b1).push_back(m);
  }
  const int mg = linesum_group_size(d.n_s);
  g->mg = mg;
  std::vector<int> order;
  std::vector<MuGroup> groups;
  for (int br = 0; br < 2; ++br) {
    const std::vector<int> &lst = br ? b1 : b0;
    for (size_t t = 0; t < lst.size(); t += mg) {
      MuGroup G;
      G.first = (int)order.size();
      G.count = (int)std::min<size_t>(mg, lst.size() - t);
      G.branch = br;
      G.pad = 0;
      for (int q = 0; q < G.count; ++q) order.push_back(lst[t + q]);
      groups.push_back(G);
    }
    if (br == 0) g->n_groups_branch0 = (int)groups.size();
  }
  g->n_groups = (int)groups.size();
  DC_CUDA(dmalloc((void **)&g->mu, sizeof(MuRec) * n_mu));
  DC_CUDA(dmalloc((void **)&g->mu_order, sizeof(int) * n_mu));
  DC_CUDA(dmalloc((void **)&g->groups, sizeof(MuGroup) * groups.size()));
  DC_CUDA(cudaMemcpy(g->mu, mu.data(), sizeof(MuRec) * n_mu, cudaMemcpyHostToDevice));
  DC_CUDA(cudaMemcpy(g->mu_order, order.data(), sizeof(int) * n_mu, cudaMemcpyHostToDevice));
  DC_CUDA(cudaMemcpy(g->groups, groups.data(), sizeof(MuGroup) * groups.size(),
                     cudaMemcpyHostToDevice));
  size_t nvm = (size_t)d.n_views * n_mu;
  DC_CUDA(dmalloc((void **)&g->vmu, sizeof(VMu) * nvm));
  k_geometry_angles<<<(unsigned)((nvm + 127) / 128), 128>>>(d.n_views, n_mu, d.n_s, d.pitch,
                                                           d.ds, g->geo64, g->vmu);
  DC_CUDA(cudaGetLastError());
  DC_CUDA(cudaDeviceSynchronize());
  return DC_OK;
}

}  // namespace dc

extern "C" {

int dc_setup_geometry(const dc_geometry_desc *desc, const double *P, const double *vdl,
                      dc_geometry **out) {
  if (!desc || !P || !out) return dc::fail(DC_ERR_ARG, "dc_setup_geometry: NULL argument");
  *out = nullptr;
  const dc_geometry_desc &d = *desc;
  if (d.n_views < 1 || d.det_rows < 2 || d.det_cols < 2 || d.n_mu < 1 || d.n_s < 2 ||
      d.vol_x < 1 || d.vol_y < 1 || d.vol_z < 1)
    return dc::fail(DC_ERR_ARG, "dc_setup_geometry: sizes must be positive (H, W, n_s >= 2)");
  if (!(d.pitch > 0) || !(d.ds > 0) || !(d.voxel[0] > 0) || !(d.voxel[1] > 0) ||
      !(d.voxel[2] > 0))
    return dc::fail(DC_ERR_ARG, "dc_setup_geometry: spacings must be positive");
  if (d.det_rows > 2048 || d.det_cols > 2048 || d.n_s > 2048)
    return dc::fail(DC_ERR_UNSUPPORTED,
                    "dc_setup_geometry: detector rows/columns and n_s are limited to 2048");
  if ((long long)d.det_rows * d.det_cols > (1LL << 30) ||
      (long long)d.vol_x * d.vol_y * d.vol_z > (1LL << 34) || d.n_views > (1 << 20) ||
      (long long)d.n_mu * d.n_s > (1LL << 28))
    return dc::fail(DC_ERR_ARG, "dc_setup_geometry: sizes too large");
  for (int t = 0; t < 12 * d.n_views; ++t)
    if (!std::isfinite(P[t])) return dc::fail(DC_ERR_ARG, "dc_setup_geometry: non-finite P");
  if (vdl)
    for (int t = 0; t < 3 * d.n_views; ++t)
      if (!std::isfinite(vdl[t]))
        return dc::fail(DC_ERR_ARG, "dc_setup_geometry: non-finite tangent");

  dc_geometry *g = new dc_geometry();
  memset((void *)g, 0, sizeof(dc_geometry));
  g->d = d;
  cudaGetDevice(&g->device);
  int V = d.n_views;
  double *dP = nullptr, *dV = nullptr, *dPn = nullptr;
  int *dst = nullptr;
  int rc = DC_OK;
  auto cleanup = [&](int code) {
    cudaFree(dP);
    cudaFree(dV);
    cudaFree(dPn);
    cudaFree(dst);
    if (code != DC_OK) free_geometry(g);
    return code;
  };
#define SETUP_CUDA(call)                                         \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return cleanup(dc::cuda_fail(e_, #call)); \
  } while (0)
  SETUP_CUDA(dc::dmalloc((void **)&g->geo64, sizeof(double) * GN * V));
  SETUP_CUDA(dc::dmalloc((void **)&g->bpv, sizeof(dc::BPView) * V));
  SETUP_CUDA(dc::dmalloc((void **)&g->fv, sizeof(dc::FView) * V));
  SETUP_CUDA(dc::dmalloc((void **)&dP, sizeof(double) * 12 * V));
  SETUP_CUDA(dc::dmalloc((void **)&dPn, sizeof(double) * 12 * V));
  SETUP_CUDA(dc::dmalloc((void **)&dst, sizeof(int) * V));
  if (vdl) SETUP_CUDA(dc::dmalloc((void **)&dV, sizeof(double) * 3 * V));
  SETUP_CUDA(cudaMemcpy(dP, P, sizeof(double) * 12 * V, cudaMemcpyHostToDevice));
  if (vdl) SETUP_CUDA(cudaMemcpy(dV, vdl, sizeof(double) * 3 * V, cudaMemcpyHostToDevice));
  int tpb = 128, nb = (V + tpb - 1) / tpb;
  k_geometry_frames<<<nb, tpb>>>(V, d.pitch, d.vol_center[0], d.vol_center[1],
                                 d.vol_center[2], dP, g->geo64, dPn, dst);
  SETUP_CUDA(cudaGetLastError());
  std::vector<int> st(V);
  SETUP_CUDA(cudaMemcpy(st.data(), dst, sizeof(int) * V, cudaMemcpyDeviceToHost));
  for (int i = 0; i < V; ++i)
    if (st[i])
      return cleanup(dc::fail(DC_ERR_ARG, "dc_setup_geometry: projection matrix of view " +
                                              std::to_string(i) +
                                              " is singular, skewed or has non-square pixels"));
  k_geometry_tables<<<nb, tpb>>>(V, d.closed_orbit, d.pitch, d.vol_center[0], d.vol_center[1],
                                 d.vol_center[2], dV, g->geo64, g->bpv, g->fv);
  SETUP_CUDA(cudaGetLastError());
  g->host_geo = (double *)malloc(sizeof(double) * GN * V);
  if (!g->host_geo) return cleanup(dc::fail(DC_ERR_OOM, "dc_setup_geometry: host malloc"));
  SETUP_CUDA(cudaMemcpy(g->host_geo, g->geo64, sizeof(double) * GN * V,
                        cudaMemcpyDeviceToHost));
  for (int i = 0; i < V; ++i) {
    double D = g->host_geo[GN * i + 12];
    if (!(D > 0) || !std::isfinite(D))
      return cleanup(dc::fail(DC_ERR_ARG, "dc_setup_geometry: bad source-detector distance"));
  }
#undef SETUP_CUDA
  rc = dc::build_mu_tables(g);
  if (rc != DC_OK) return cleanup(rc);
  rc = dc::alloc_workspace(g);
  if (rc != DC_OK) return cleanup(rc);
  cleanup(DC_OK);
  *out = g;
  return DC_OK;
}

void dc_destroy_geometry(dc_geometry *geom) { free_geometry(geom); }

int dc_get_view_geometry(const dc_geometry *geom, double *out) {
  if (!geom || !out) return dc::fail(DC_ERR_ARG, "dc_get_view_geometry: NULL argument");
  memcpy(out, geom->host_geo, sizeof(double) * GN * geom->d.n_views);
  return DC_OK;
}

}  // extern "C"
