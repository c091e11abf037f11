// dc_host.cu -- the whole reconstruction of Eq. 12 from host buffers, with
// the host<->device copies overlapped with the kernels:
//   - the projections go up view chunk by view chunk on a copy stream, and
//     each chunk's filter waits only for its own copy;
//   - the volume is backprojected in z-slabs on two alternating streams (a
//     slab's last CTAs overlap the next slab's first), and each finished
//     slab goes down on the copy stream while later slabs compute.
// With page-locked host buffers only the first chunk's upload and the last
// slab's download stay outside the kernels' time.
#include <algorithm>
#include <mutex>
#include <string>

#include "dc_common.cuh"

namespace {

std::mutex g_aux_mu;

// the copy stream, the second compute stream and the events, once per handle
int ensure_aux(dc_geometry *g) {
  std::lock_guard<std::mutex> lk(g_aux_mu);
  if (g->aux_ready) return DC_OK;
  DC_CUDA(cudaStreamCreateWithFlags(&g->aux_copy, cudaStreamNonBlocking));
  DC_CUDA(cudaStreamCreateWithFlags(&g->aux_compute, cudaStreamNonBlocking));
  for (int i = 0; i < 8; ++i)
    DC_CUDA(cudaEventCreateWithFlags(&g->aux_ev[i], cudaEventDisableTiming));
  g->aux_ready = 1;
  return DC_OK;
}

}  // namespace

extern "C" int dc_reconstruct_host(const dc_geometry *geom, int B, const float *g_host,
                                   const float *W, float *g_dev, void *gF, int dtype,
                                   float *gF_scale, float *vol_dev, float *vol_host,
                                   unsigned flags, int n_slabs, void *stream) {
  int rc = dc::filter_check(geom, B, g_dev, gF, dtype, gF_scale, "dc_reconstruct_host");
  if (rc) return rc;
  rc = dc::backproject_check(geom, B, gF, dtype, gF_scale, vol_dev, flags, "dc_reconstruct_host");
  if (rc) return rc;
  if (!g_host || !vol_host) return dc::fail(DC_ERR_ARG, "dc_reconstruct_host: NULL host buffer");
  if (n_slabs < 0) return dc::fail(DC_ERR_ARG, "dc_reconstruct_host: negative n_slabs");
  dc_geometry *g = const_cast<dc_geometry *>(geom);  // only the stream/event cache changes
  if ((rc = ensure_aux(g))) return rc;
  const dc_geometry_desc &d = g->d;
  cudaStream_t st = (cudaStream_t)stream, cs = g->aux_copy, as = g->aux_compute;
  cudaEvent_t *ev = g->aux_ev;  // 0 start, 1 filtered, 2-3 uploads, 4-5 slabs, 6 done

  // nothing of this call may overwrite buffers earlier work on `stream` uses
  DC_CUDA(cudaEventRecord(ev[0], st));
  DC_CUDA(cudaStreamWaitEvent(cs, ev[0], 0));
  DC_CUDA(cudaStreamWaitEvent(as, ev[0], 0));

  // filter, chunk by chunk behind the uploads
  const size_t img = (size_t)d.det_rows * d.det_cols;
  int bcm, cvm, k = 0;
  dc::filter_chunk_plan(g, B, &bcm, &cvm);
  for (int b0 = 0; b0 < B; b0 += bcm) {
    const int bc = std::min(bcm, B - b0);
    for (int v0 = 0; v0 < d.n_views; v0 += cvm) {
      const int nv = std::min(cvm, d.n_views - v0);
      for (int b = b0; b < b0 + bc; ++b) {
        const size_t off = ((size_t)b * d.n_views + v0) * img;
        DC_CUDA(cudaMemcpyAsync(g_dev + off, g_host + off, sizeof(float) * nv * img,
                                cudaMemcpyHostToDevice, cs));
      }
      cudaEvent_t e = ev[2 + (k++ & 1)];
      DC_CUDA(cudaEventRecord(e, cs));
      DC_CUDA(cudaStreamWaitEvent(st, e, 0));
      if ((rc = dc::filter_chunk(g, g_dev, W, gF, dtype, gF_scale, b0, bc, v0, nv, st)))
        return rc;
    }
  }
  DC_CUDA(cudaEventRecord(ev[1], st));
  DC_CUDA(cudaStreamWaitEvent(as, ev[1], 0));

  // backprojection by z-slabs (multiples of the box depth), each slab down
  // as soon as it is complete
  const size_t nxy = (size_t)d.vol_x * d.vol_y, nvox = nxy * d.vol_z;
  const int zq = g->bp_nz;
  const int zblocks = (d.vol_z + zq - 1) / zq;
  const int ns = std::max(1, std::min(n_slabs == 0 ? 16 : n_slabs, zblocks));
  const int depth = ((zblocks + ns - 1) / ns) * zq;
  int s = 0;
  for (int z0 = 0; z0 < d.vol_z; z0 += depth, ++s) {
    const int z1 = std::min(d.vol_z, z0 + depth);
    cudaStream_t ss = (s & 1) ? as : st;
    bool used = false;
    if ((rc = dc::backproject_slab(g, B, gF, dtype, gF_scale, vol_dev, flags, z0, z1, ss, &used)))
      return rc;
    if (!used) {
      // the staged kernel cannot read this g^F layout: one plain launch
      if (s != 0) return dc::fail(DC_ERR_CUDA, "dc_reconstruct_host: backprojection path changed");
      if ((rc = dc_backproject(g, B, gF, dtype, gF_scale, vol_dev, flags, st))) return rc;
      DC_CUDA(cudaEventRecord(ev[4], st));
      DC_CUDA(cudaStreamWaitEvent(cs, ev[4], 0));
      DC_CUDA(cudaMemcpyAsync(vol_host, vol_dev, sizeof(float) * nvox * B,
                              cudaMemcpyDeviceToHost, cs));
      break;
    }
    cudaEvent_t e = ev[4 + (s & 1)];
    DC_CUDA(cudaEventRecord(e, ss));
    DC_CUDA(cudaStreamWaitEvent(cs, e, 0));
    for (int b = 0; b < B; ++b) {
      const size_t off = (size_t)b * nvox + (size_t)z0 * nxy;
      DC_CUDA(cudaMemcpyAsync(vol_host + off, vol_dev + off, sizeof(float) * (z1 - z0) * nxy,
                              cudaMemcpyDeviceToHost, cs));
    }
  }
  // the caller's stream ends after the last download (which waited for every slab)
  DC_CUDA(cudaEventRecord(ev[6], cs));
  DC_CUDA(cudaStreamWaitEvent(st, ev[6], 0));
  return DC_OK;
}
