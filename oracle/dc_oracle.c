/*
 * dc_oracle.c -- plain FP64 CPU oracle of the Defrise-Clack shift-variant
 * filtered backprojection as a layered network (Ye et al., DRACO, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: it exists so that the tests, the smoke check and the
 * CPU-baseline leg of the benchmark can compare the CUDA library against an
 * independent, slow, obviously correct implementation.  It shares no code,
 * header or table with the CUDA sources.
 *
 * Every step is written in the paper's order and notation:
 *
 *   S   = w_sino * D_f * A2d * w_cos * g              (Eq. 7; Eq. 6)
 *   g^F = w_d * A2d^T * D_b * w_red * S               (Eq. 11; Eq. 8)
 *   f   = A3d^T g^F, optionally followed by ReLU      (Eq. 5, Eq. 12)
 *
 * with w_cos = D / sqrt(x^2+y^2+D^2), w_sino = (s^2+D^2)/D^2, w_d = x^2+y^2+D^2
 * and w_red = W * K, K = -(1/4pi^2) |a'(lambda)dlambda . theta| / sqrt(s^2+D^2)
 * (Eq. 10; the trainable/Crofton part W is an input, dlambda is folded into
 * the tangent so that W = 1/2 is the exact circular-orbit value of Eq. 14).
 *
 * Discretisation (the paper defers it to its operator library; these are the
 * readings used throughout this project):
 *   - detector pixel (j, r) at x_j = (j - c_u) p, y_r = (r - c_v) p;
 *   - sinogram mu_m = m pi / N_mu, s_k = (k - (N_s-1)/2) ds;
 *   - A2d: Joseph's method (Joseph 1982).  Lines with |cos mu| >= |sin mu|
 *     (decided exactly as 4m <= N_mu or 4m >= 3 N_mu) step over detector rows
 *     and interpolate linearly between the two neighbouring columns, scaled
 *     by p/|cos mu|; the other lines step over columns symmetrically.  Samples
 *     outside the detector contribute zero.
 *   - D_f: forward difference onto the half grid s_{k+1/2};  S, W, K live on
 *     that grid; the entry k = N_s-1 is zero.  D_b: backward difference back
 *     onto s_k.  The two together form the compound 3-point stencil.
 *   - A2d^T: the literal transpose of the Joseph weights, times
 *     (pi/N_mu) * ds / p^2 so that it approximates the integral over mu of
 *     Eq. 8 (the Joseph weights of one pixel sum to p^2/ds over s on average).
 *   - A3d^T: voxel-driven; a voxel X projects through the 3x4 matrix of the
 *     view to (u, v) in pixel units, g^F is interpolated bilinearly (pixels
 *     outside the detector are zero) and weighted by 1/|X - a|^2 (Eq. 5).
 *     Voxels with depth <= 0 are skipped.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC dc_oracle.c -o libdc_oracle.so -lm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* per-view geometry record (doubles) */
#define GEO_N 32
#define G_P 0      /* 12: normalised projection matrix, row major 3x4   */
#define G_A 12     /* 3 : source position a                              */
#define G_LX 15    /* 3 : detector axis l_x                              */
#define G_LY 18    /* 3 : detector axis l_y                              */
#define G_LZ 21    /* 3 : unit vector from detector towards the source   */
#define G_D 24     /* source-detector distance D                         */
#define G_CU 25    /* principal point, column index                      */
#define G_CV 26    /* principal point, row index                         */
#define G_V 27     /* 3 : a'(lambda) dlambda                             */

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Geometry (Fig. 1: detector frame; source from the projection matrix)     */
/* ------------------------------------------------------------------------ */

static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/*
 * From P_i = s [A | -A a]: a = -M^{-1} p4 (Cramer's rule); the third row of
 * M is -l_z up to the scale s; the first two rows are f l_x - c_u l_z and
 * f l_y - c_v l_z with f = D/p.  The sign of s is chosen so that the volume
 * centre has positive depth.  Returns 0, or 1 for a singular / skewed /
 * non-square-pixel matrix.
 */
int orc_setup_geometry(int V, double pitch, const double *vol_center,
                       const double *P, const double *vdl, int closed,
                       double *geo) {
  for (int i = 0; i < V; ++i) {
    const double *Pi = P + 12 * i;
    double *g = geo + (size_t)GEO_N * i;
    memset(g, 0, sizeof(double) * GEO_N);
    double m3[3] = {Pi[8], Pi[9], Pi[10]};
    double sc = sqrt(dot3(m3, m3));
    if (!(sc > 0)) return 1;
    double wc = Pi[8] * vol_center[0] + Pi[9] * vol_center[1] +
                Pi[10] * vol_center[2] + Pi[11];
    if (wc < 0) sc = -sc;
    for (int t = 0; t < 12; ++t) g[G_P + t] = Pi[t] / sc;
    const double *n = g + G_P;
    /* a = -M^{-1} p4 */
    double M[3][3] = {{n[0], n[1], n[2]}, {n[4], n[5], n[6]}, {n[8], n[9], n[10]}};
    double p4[3] = {n[3], n[7], n[11]};
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                 M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                 M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (fabs(det) < 1e-300) return 1;
    for (int c = 0; c < 3; ++c) {
      double Mc[3][3];
      memcpy(Mc, M, sizeof(M));
      for (int r = 0; r < 3; ++r) Mc[r][c] = p4[r];
      double dc = Mc[0][0] * (Mc[1][1] * Mc[2][2] - Mc[1][2] * Mc[2][1]) -
                  Mc[0][1] * (Mc[1][0] * Mc[2][2] - Mc[1][2] * Mc[2][0]) +
                  Mc[0][2] * (Mc[1][0] * Mc[2][1] - Mc[1][1] * Mc[2][0]);
      g[G_A + c] = -dc / det;
    }
    for (int c = 0; c < 3; ++c) g[G_LZ + c] = -n[8 + c];
    double *lz = g + G_LZ;
    double r1[3] = {n[0], n[1], n[2]}, r2[3] = {n[4], n[5], n[6]};
    double cu = -dot3(r1, lz), cv = -dot3(r2, lz);
    double fx[3], fy[3];
    for (int c = 0; c < 3; ++c) {
      fx[c] = r1[c] + cu * lz[c];
      fy[c] = r2[c] + cv * lz[c];
    }
    double nfx = sqrt(dot3(fx, fx)), nfy = sqrt(dot3(fy, fy));
    if (!(nfx > 0) || !(nfy > 0)) return 1;
    if (fabs(nfx - nfy) > 1e-9 * nfx) return 1;
    for (int c = 0; c < 3; ++c) {
      g[G_LX + c] = fx[c] / nfx;
      g[G_LY + c] = fy[c] / nfy;
    }
    if (fabs(dot3(g + G_LX, g + G_LY)) > 1e-9) return 1;
    g[G_D] = nfx * pitch;
    g[G_CU] = cu;
    g[G_CV] = cv;
  }
  /* tangent a'(lambda) dlambda: given, or central differences of the sources */
  for (int i = 0; i < V; ++i) {
    double *g = geo + (size_t)GEO_N * i;
    if (vdl) {
      for (int c = 0; c < 3; ++c) g[G_V + c] = vdl[3 * i + c];
      continue;
    }
    if (V < 2) continue;
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
    const double *ap = geo + (size_t)GEO_N * ip + G_A;
    const double *am = geo + (size_t)GEO_N * im + G_A;
    for (int c = 0; c < 3; ++c) g[G_V + c] = half * (ap[c] - am[c]);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Pointwise weights (Eq. 7, Eq. 10, Eq. 11)                                */
/* ------------------------------------------------------------------------ */

/* w_cos(x, y) = D / sqrt(x^2 + y^2 + D^2)  (Eq. 6/7) */
void orc_cosine_weight(int H, int W, double p, const double *geo_i,
                       const double *g, double *out) {
  double D = geo_i[G_D], cu = geo_i[G_CU], cv = geo_i[G_CV];
  for (int r = 0; r < H; ++r)
    for (int j = 0; j < W; ++j) {
      double x = (j - cu) * p, y = (r - cv) * p;
      out[(size_t)r * W + j] = g[(size_t)r * W + j] * D / sqrt(x * x + y * y + D * D);
    }
}

/* w_d(x, y) = x^2 + y^2 + D^2  (Eq. 11) */
void orc_detector_weight(int H, int W, double p, const double *geo_i,
                         const double *h, double *out) {
  double D = geo_i[G_D], cu = geo_i[G_CU], cv = geo_i[G_CV];
  for (int r = 0; r < H; ++r)
    for (int j = 0; j < W; ++j) {
      double x = (j - cu) * p, y = (r - cv) * p;
      out[(size_t)r * W + j] = h[(size_t)r * W + j] * (x * x + y * y + D * D);
    }
}

static double s_of(int k, int n_s, double ds) { return (k - 0.5 * (n_s - 1)) * ds; }

/*
 * K(mu, s) = -(1/4pi^2) |v . theta| / sqrt(s^2 + D^2) on the half grid
 * s_{k+1/2} (Eq. 10 without the Crofton part), where theta is the unit normal
 * of the plane through the source containing the detector line
 * x cos mu + y sin mu = s:  theta = (D cos mu l_x + D sin mu l_y + s l_z) /
 * sqrt(D^2 + s^2).  out[m][k]; the entry k = N_s-1 is 0.
 */
void orc_redundancy_K(int n_mu, int n_s, double ds, const double *geo_i,
                      double *out) {
  double D = geo_i[G_D];
  const double *lx = geo_i + G_LX, *ly = geo_i + G_LY, *lz = geo_i + G_LZ;
  const double *v = geo_i + G_V;
  for (int m = 0; m < n_mu; ++m) {
    double mu = m * PI / n_mu, c = cos(mu), s = sin(mu);
    for (int k = 0; k < n_s; ++k) {
      if (k == n_s - 1) {
        out[(size_t)m * n_s + k] = 0.0;
        continue;
      }
      double sh = s_of(k, n_s, ds) + 0.5 * ds;
      double nrm = sqrt(D * D + sh * sh);
      double th[3];
      for (int t = 0; t < 3; ++t) th[t] = (D * c * lx[t] + D * s * ly[t] + sh * lz[t]) / nrm;
      out[(size_t)m * n_s + k] = -fabs(dot3(v, th)) / (4.0 * PI * PI * nrm);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* A2d: Joseph line sums, and its literal transpose                          */
/* ------------------------------------------------------------------------ */

static int cos_branch(int m, int n_mu) { return 4 * m <= n_mu || 4 * m >= 3 * n_mu; }

/* R[m][k] = sum over the line x cos mu + y sin mu = s_k of img (Joseph) */
void orc_radon(int H, int W, double p, double cu, double cv, int n_mu, int n_s,
               double ds, const double *img, double *R) {
  for (int m = 0; m < n_mu; ++m) {
    double mu = m * PI / n_mu, c = cos(mu), s = sin(mu);
    int vert = cos_branch(m, n_mu);
    for (int k = 0; k < n_s; ++k) {
      double sk = s_of(k, n_s, ds), acc = 0.0;
      if (vert) {
        for (int r = 0; r < H; ++r) {
          double y = (r - cv) * p;
          double xi = (sk - y * s) / (c * p) + cu;
          double j0 = floor(xi), t = xi - j0;
          long j = (long)j0;
          if (j >= 0 && j < W) acc += (1.0 - t) * img[(size_t)r * W + j];
          if (j + 1 >= 0 && j + 1 < W) acc += t * img[(size_t)r * W + j + 1];
        }
        acc *= p / fabs(c);
      } else {
        for (int j = 0; j < W; ++j) {
          double x = (j - cu) * p;
          double eta = (sk - x * c) / (s * p) + cv;
          double r0 = floor(eta), t = eta - r0;
          long r = (long)r0;
          if (r >= 0 && r < H) acc += (1.0 - t) * img[(size_t)r * W + j];
          if (r + 1 >= 0 && r + 1 < H) acc += t * img[(size_t)(r + 1) * W + j];
        }
        acc *= p / fabs(s);
      }
      R[(size_t)m * n_s + k] = acc;
    }
  }
}

/* img += J^T R : the same weights as orc_radon, scattered back */
void orc_radon_T(int H, int W, double p, double cu, double cv, int n_mu, int n_s,
                 double ds, const double *R, double *img) {
  for (int m = 0; m < n_mu; ++m) {
    double mu = m * PI / n_mu, c = cos(mu), s = sin(mu);
    int vert = cos_branch(m, n_mu);
    for (int k = 0; k < n_s; ++k) {
      double sk = s_of(k, n_s, ds);
      double val = R[(size_t)m * n_s + k];
      if (vert) {
        val *= p / fabs(c);
        for (int r = 0; r < H; ++r) {
          double y = (r - cv) * p;
          double xi = (sk - y * s) / (c * p) + cu;
          double j0 = floor(xi), t = xi - j0;
          long j = (long)j0;
          if (j >= 0 && j < W) img[(size_t)r * W + j] += (1.0 - t) * val;
          if (j + 1 >= 0 && j + 1 < W) img[(size_t)r * W + j + 1] += t * val;
        }
      } else {
        val *= p / fabs(s);
        for (int j = 0; j < W; ++j) {
          double x = (j - cu) * p;
          double eta = (sk - x * c) / (s * p) + cv;
          double r0 = floor(eta), t = eta - r0;
          long r = (long)r0;
          if (r >= 0 && r < H) img[(size_t)r * W + j] += (1.0 - t) * val;
          if (r + 1 >= 0 && r + 1 < H) img[(size_t)(r + 1) * W + j] += t * val;
        }
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* s-derivatives                                                              */
/* ------------------------------------------------------------------------ */

/* D_f: out[m][k] = (R[m][k+1] - R[m][k]) / ds on s_{k+1/2}; out[m][N_s-1] = 0 */
void orc_deriv_f(int n_mu, int n_s, double ds, const double *R, double *out) {
  for (int m = 0; m < n_mu; ++m)
    for (int k = 0; k < n_s; ++k)
      out[(size_t)m * n_s + k] =
          k < n_s - 1 ? (R[(size_t)m * n_s + k + 1] - R[(size_t)m * n_s + k]) / ds : 0.0;
}

/* D_f^T */
void orc_deriv_f_T(int n_mu, int n_s, double ds, const double *y, double *out) {
  for (int m = 0; m < n_mu; ++m)
    for (int k = 0; k < n_s; ++k) {
      double a = (k >= 1 && k - 1 < n_s - 1) ? y[(size_t)m * n_s + k - 1] : 0.0;
      double b = (k < n_s - 1) ? y[(size_t)m * n_s + k] : 0.0;
      out[(size_t)m * n_s + k] = (a - b) / ds;
    }
}

/* D_b: out[m][k] = (Q[m][k] - Q[m][k-1]) / ds with Q[m][-1] = 0 */
void orc_deriv_b(int n_mu, int n_s, double ds, const double *Q, double *out) {
  for (int m = 0; m < n_mu; ++m)
    for (int k = 0; k < n_s; ++k)
      out[(size_t)m * n_s + k] =
          (Q[(size_t)m * n_s + k] - (k > 0 ? Q[(size_t)m * n_s + k - 1] : 0.0)) / ds;
}

/* D_b^T */
void orc_deriv_b_T(int n_mu, int n_s, double ds, const double *y, double *out) {
  for (int m = 0; m < n_mu; ++m)
    for (int k = 0; k < n_s; ++k)
      out[(size_t)m * n_s + k] =
          (y[(size_t)m * n_s + k] - (k + 1 < n_s ? y[(size_t)m * n_s + k + 1] : 0.0)) / ds;
}

/* ------------------------------------------------------------------------ */
/* One view of the filter (Eqs. 7 and 11)                                    */
/* ------------------------------------------------------------------------ */

/* Grangeat's intermediate function S = w_sino D_f A2d w_cos g on s_{k+1/2} */
void orc_grangeat(int H, int W, double p, int n_mu, int n_s, double ds,
                  const double *geo_i, const double *g, double *S) {
  double D = geo_i[G_D];
  size_t np = (size_t)H * W, ns = (size_t)n_mu * n_s;
  double *gt = malloc(sizeof(double) * np), *R = malloc(sizeof(double) * ns);
  orc_cosine_weight(H, W, p, geo_i, g, gt);
  orc_radon(H, W, p, geo_i[G_CU], geo_i[G_CV], n_mu, n_s, ds, gt, R);
  orc_deriv_f(n_mu, n_s, ds, R, S);
  for (int m = 0; m < n_mu; ++m)
    for (int k = 0; k < n_s; ++k) {
      double sh = s_of(k, n_s, ds) + 0.5 * ds;
      S[(size_t)m * n_s + k] *= (sh * sh + D * D) / (D * D);
    }
  free(gt);
  free(R);
}

static double a2dT_scale(int n_mu, double ds, double p) { return (PI / n_mu) * ds / (p * p); }

/* g^F for one view; W_red [n_mu][n_s] (NULL -> 1/2) */
void orc_filter_view(int H, int W, double p, int n_mu, int n_s, double ds,
                     const double *geo_i, const double *g, const double *Wred,
                     double *gF) {
  size_t np = (size_t)H * W, ns = (size_t)n_mu * n_s;
  double *S = malloc(sizeof(double) * ns), *K = malloc(sizeof(double) * ns);
  double *Pm = malloc(sizeof(double) * ns), *h = calloc(np, sizeof(double));
  orc_grangeat(H, W, p, n_mu, n_s, ds, geo_i, g, S);
  orc_redundancy_K(n_mu, n_s, ds, geo_i, K);
  for (size_t t = 0; t < ns; ++t) S[t] *= (Wred ? Wred[t] : 0.5) * K[t]; /* Q */
  orc_deriv_b(n_mu, n_s, ds, S, Pm);
  double sc = a2dT_scale(n_mu, ds, p);
  for (size_t t = 0; t < ns; ++t) Pm[t] *= sc;
  orc_radon_T(H, W, p, geo_i[G_CU], geo_i[G_CV], n_mu, n_s, ds, Pm, h);
  orc_detector_weight(H, W, p, geo_i, h, gF);
  free(S);
  free(K);
  free(Pm);
  free(h);
}

/*
 * Reverse mode of orc_filter_view.  G = dL/dg^F.  Writes dL/dg (if grad_g)
 * and ADDS dL/dW_red into grad_W (if grad_W).
 */
void orc_filter_view_adjoint(int H, int W, double p, int n_mu, int n_s, double ds,
                             const double *geo_i, const double *g, const double *Wred,
                             const double *G, double *grad_g, double *grad_W) {
  size_t np = (size_t)H * W, ns = (size_t)n_mu * n_s;
  double *Hd = malloc(sizeof(double) * np), *Pg = malloc(sizeof(double) * ns);
  double *Qg = malloc(sizeof(double) * ns), *S = malloc(sizeof(double) * ns);
  double *K = malloc(sizeof(double) * ns), *y = malloc(sizeof(double) * ns);
  double *Rg = malloc(sizeof(double) * ns);
  double D = geo_i[G_D];
  orc_detector_weight(H, W, p, geo_i, G, Hd);                      /* w_d^T      */
  orc_radon(H, W, p, geo_i[G_CU], geo_i[G_CV], n_mu, n_s, ds, Hd, Pg); /* (A2d^T)^T */
  double sc = a2dT_scale(n_mu, ds, p);
  for (size_t t = 0; t < ns; ++t) Pg[t] *= sc;
  orc_deriv_b_T(n_mu, n_s, ds, Pg, Qg);                            /* D_b^T      */
  for (int m = 0; m < n_mu; ++m) Qg[(size_t)m * n_s + n_s - 1] = 0.0; /* Q[N_s-1] is fixed 0 */
  orc_grangeat(H, W, p, n_mu, n_s, ds, geo_i, g, S);               /* recompute  */
  orc_redundancy_K(n_mu, n_s, ds, geo_i, K);
  if (grad_W)
    for (size_t t = 0; t < ns; ++t) grad_W[t] += K[t] * S[t] * Qg[t];
  if (grad_g) {
    for (int m = 0; m < n_mu; ++m)
      for (int k = 0; k < n_s; ++k) {
        size_t t = (size_t)m * n_s + k;
        double sh = s_of(k, n_s, ds) + 0.5 * ds;
        double wsino = (sh * sh + D * D) / (D * D);
        y[t] = (Wred ? Wred[t] : 0.5) * K[t] * Qg[t] * wsino;        /* w_red^T, w_sino^T */
      }
    orc_deriv_f_T(n_mu, n_s, ds, y, Rg);                           /* D_f^T      */
    double *gt = calloc(np, sizeof(double));
    orc_radon_T(H, W, p, geo_i[G_CU], geo_i[G_CV], n_mu, n_s, ds, Rg, gt); /* A2d^T */
    orc_cosine_weight(H, W, p, geo_i, gt, grad_g);                 /* w_cos^T    */
    free(gt);
  }
  free(Hd);
  free(Pg);
  free(Qg);
  free(S);
  free(K);
  free(y);
  free(Rg);
}

/* All views of a batch.  g, gF: [B][nv][H][W] for the selected views `views`
 * (NULL -> 0..nv-1); W_red [V][n_mu][n_s] or NULL. */
void orc_filter(int B, int nv, const int *views, int H, int W, double p, int n_mu,
                int n_s, double ds, const double *geo, const double *g,
                const double *Wred, double *gF) {
  size_t np = (size_t)H * W, ns = (size_t)n_mu * n_s;
#pragma omp parallel for schedule(dynamic) collapse(2)
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < nv; ++i) {
      int v = views ? views[i] : i;
      size_t off = ((size_t)b * nv + i) * np;
      orc_filter_view(H, W, p, n_mu, n_s, ds, geo + (size_t)GEO_N * v, g + off,
                      Wred ? Wred + (size_t)v * ns : NULL, gF + off);
    }
}

/* Reverse mode for all views: grad_g [B][V][H][W] (nullable), grad_W
 * [V][n_mu][n_s] (nullable, summed over the batch, overwritten). */
void orc_filter_adjoint(int B, int V, int H, int W, double p, int n_mu, int n_s,
                        double ds, const double *geo, const double *g,
                        const double *Wred, const double *G, double *grad_g,
                        double *grad_W) {
  size_t np = (size_t)H * W, ns = (size_t)n_mu * n_s;
  if (grad_W) memset(grad_W, 0, sizeof(double) * ns * V);
#pragma omp parallel for schedule(dynamic)
  for (int v = 0; v < V; ++v)
    for (int b = 0; b < B; ++b) {
      size_t off = ((size_t)b * V + v) * np;
      orc_filter_view_adjoint(H, W, p, n_mu, n_s, ds, geo + (size_t)GEO_N * v, g + off,
                              Wred ? Wred + (size_t)v * ns : NULL, G + off,
                              grad_g ? grad_g + off : NULL,
                              grad_W ? grad_W + (size_t)v * ns : NULL);
    }
}

/* ------------------------------------------------------------------------ */
/* A3d^T: voxel-driven cone-beam backprojection (Eq. 5) and its transpose    */
/* ------------------------------------------------------------------------ */

static void voxel_pos(int ix, int iy, int iz, int nx, int ny, int nz,
                      const double *vox, const double *ctr, double *X) {
  X[0] = ctr[0] + (ix - 0.5 * (nx - 1)) * vox[0];
  X[1] = ctr[1] + (iy - 0.5 * (ny - 1)) * vox[1];
  X[2] = ctr[2] + (iz - 0.5 * (nz - 1)) * vox[2];
}

/* Bilinear taps of detector position (u, v): up to 4 (index, weight) pairs */
static int bilinear_taps(int H, int W, double u, double v, long *idx, double *wt) {
  double j0 = floor(u), r0 = floor(v);
  double fu = u - j0, fv = v - r0;
  long j = (long)j0, r = (long)r0;
  int n = 0;
  for (int dr = 0; dr < 2; ++dr)
    for (int dj = 0; dj < 2; ++dj) {
      long jj = j + dj, rr = r + dr;
      if (jj < 0 || jj >= W || rr < 0 || rr >= H) continue;
      idx[n] = rr * W + jj;
      wt[n] = (dj ? fu : 1.0 - fu) * (dr ? fv : 1.0 - fv);
      ++n;
    }
  return n;
}

/* Projection of X in view i: returns depth w, writes (u, v) and 1/|X-a|^2 */
static double project(const double *geo_i, const double *X, double *u, double *v,
                      double *inv_d2) {
  const double *n = geo_i + G_P, *a = geo_i + G_A;
  double U = n[0] * X[0] + n[1] * X[1] + n[2] * X[2] + n[3];
  double Vv = n[4] * X[0] + n[5] * X[1] + n[6] * X[2] + n[7];
  double w = n[8] * X[0] + n[9] * X[1] + n[10] * X[2] + n[11];
  if (w > 0) {
    *u = U / w;
    *v = Vv / w;
  }
  double d[3] = {X[0] - a[0], X[1] - a[1], X[2] - a[2]};
  *inv_d2 = 1.0 / dot3(d, d);
  return w;
}

static double bp_voxel(int V, int H, int W, const double *geo, const double *gF,
                       const double *X) {
  double acc = 0.0;
  size_t np = (size_t)H * W;
  for (int i = 0; i < V; ++i) {
    double u, v, w2;
    if (project(geo + (size_t)GEO_N * i, X, &u, &v, &w2) <= 0) continue;
    long idx[4];
    double wt[4];
    int n = bilinear_taps(H, W, u, v, idx, wt);
    double val = 0.0;
    for (int t = 0; t < n; ++t) val += wt[t] * gF[(size_t)i * np + idx[t]];
    acc += val * w2;
  }
  return acc;
}

/* vol [B][nz][ny][nx] (=, or += when accum); relu after the sum */
void orc_backproject(int B, int V, int H, int W, int nx, int ny, int nz,
                     const double *vox, const double *ctr, const double *geo,
                     const double *gF, int accum, int relu, double *vol) {
  size_t np = (size_t)H * W, nvox = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(dynamic) collapse(2)
  for (int b = 0; b < B; ++b)
    for (int iz = 0; iz < nz; ++iz)
      for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix) {
          double X[3];
          voxel_pos(ix, iy, iz, nx, ny, nz, vox, ctr, X);
          size_t o = (size_t)b * nvox + ((size_t)iz * ny + iy) * nx + ix;
          double f = bp_voxel(V, H, W, geo, gF + (size_t)b * V * np, X);
          if (accum) f += vol[o];
          if (relu && f < 0) f = 0;
          vol[o] = f;
        }
}

/* The same sum at selected flat voxel indices (z*ny + y)*nx + x of item b */
void orc_backproject_points(int V, int H, int W, int nx, int ny, int nz,
                            const double *vox, const double *ctr, const double *geo,
                            const double *gF, int npts, const long *flat, int relu,
                            double *out) {
#pragma omp parallel for schedule(dynamic)
  for (int t = 0; t < npts; ++t) {
    long f = flat[t];
    int ix = (int)(f % nx), iy = (int)((f / nx) % ny), iz = (int)(f / ((long)nx * ny));
    double X[3];
    voxel_pos(ix, iy, iz, nx, ny, nz, vox, ctr, X);
    double r = bp_voxel(V, H, W, geo, gF, X);
    out[t] = (relu && r < 0) ? 0.0 : r;
  }
}

/* grad_gF [B][V][H][W] = (A3d^T)^T grad_vol (overwritten) */
void orc_backproject_adjoint(int B, int V, int H, int W, int nx, int ny, int nz,
                             const double *vox, const double *ctr, const double *geo,
                             const double *grad_vol, double *grad_gF) {
  size_t np = (size_t)H * W, nvox = (size_t)nx * ny * nz;
  memset(grad_gF, 0, sizeof(double) * np * V * B);
#pragma omp parallel for schedule(dynamic) collapse(2)
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < V; ++i) {
      double *out = grad_gF + ((size_t)b * V + i) * np;
      const double *gi = geo + (size_t)GEO_N * i;
      for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
          for (int ix = 0; ix < nx; ++ix) {
            double X[3], u, v, w2;
            voxel_pos(ix, iy, iz, nx, ny, nz, vox, ctr, X);
            if (project(gi, X, &u, &v, &w2) <= 0) continue;
            double gv = grad_vol[(size_t)b * nvox + ((size_t)iz * ny + iy) * nx + ix];
            long idx[4];
            double wt[4];
            int n = bilinear_taps(H, W, u, v, idx, wt);
            for (int t = 0; t < n; ++t) out[idx[t]] += wt[t] * w2 * gv;
          }
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Smooth Crofton weight of Eq. 9                                            */
/* ------------------------------------------------------------------------ */

/*
 * M(theta, lambda_i) = |v_i.theta|^m c_i / sum_alpha |v_alpha.theta|^m c_alpha
 * for every view i and plane (mu, s_{k+1/2}) through a_i.  The sum runs over
 * the intersections of that plane with the orbit: view i itself, and every
 * sign change of f_j = (a_j - a_i).theta between consecutive views j, j+1 of
 * a segment (wrapping for a closed segment; pairs that contain i are skipped
 * because the crossing at i is counted by the first term).  At a crossing
 * t = f_j / (f_j - f_{j+1}) interpolates the tangent v and the taper c.
 * c is 1 except within `taper` views of the ends of an open segment, where
 * c = sin^2(pi/2 (d + 1/2) / taper) at distance d from the end.  Segments:
 * view ranges [seg_start[q], seg_start[q+1]) (the last ends at V) with
 * seg_closed[q].  out[V][n_mu][n_s]; entry n_s-1 is 0; M = 0 where
 * |v_i.theta| = 0.
 */
static double crofton_taper(int j, int lo, int hi, int closed, int taper) {
  if (closed || taper <= 0) return 1.0;
  int d = j - lo < hi - 1 - j ? j - lo : hi - 1 - j;
  if (d >= taper) return 1.0;
  double x = sin(0.5 * PI * (d + 0.5) / taper);
  return x * x;
}

void orc_crofton_weights(int V, int n_mu, int n_s, double ds, const double *geo,
                         int n_seg, const int *seg_start, const int *seg_closed, int m,
                         int taper, double *out) {
  double *cj = malloc(sizeof(double) * V);
  int *segof = malloc(sizeof(int) * V);
  for (int q = 0; q < n_seg; ++q) {
    int lo = seg_start[q], hi = q + 1 < n_seg ? seg_start[q + 1] : V;
    for (int j = lo; j < hi; ++j) {
      cj[j] = crofton_taper(j, lo, hi, seg_closed[q], taper);
      segof[j] = q;
    }
  }
#pragma omp parallel for schedule(dynamic) collapse(2)
  for (int i = 0; i < V; ++i)
    for (int mm = 0; mm < n_mu; ++mm) {
      const double *gi = geo + (size_t)GEO_N * i;
      double D = gi[G_D];
      const double *lx = gi + G_LX, *ly = gi + G_LY, *lz = gi + G_LZ, *ai = gi + G_A;
      double mu = mm * PI / n_mu, cm = cos(mu), sm = sin(mu);
      for (int k = 0; k < n_s; ++k) {
        double *o = out + ((size_t)i * n_mu + mm) * n_s + k;
        if (k == n_s - 1) {
          *o = 0.0;
          continue;
        }
        double sh = s_of(k, n_s, ds) + 0.5 * ds;
        double nrm = sqrt(D * D + sh * sh), th[3];
        for (int t = 0; t < 3; ++t) th[t] = (D * cm * lx[t] + D * sm * ly[t] + sh * lz[t]) / nrm;
        double own = pow(fabs(dot3(gi + G_V, th)), m) * cj[i];
        if (!(own > 0.0)) {
          *o = 0.0;
          continue;
        }
        double sum = own;
        for (int q = 0; q < n_seg; ++q) {
          int lo = seg_start[q], hi = q + 1 < n_seg ? seg_start[q + 1] : V;
          int npair = seg_closed[q] ? hi - lo : hi - lo - 1;
          for (int e = 0; e < npair; ++e) {
            int j0 = lo + e, j1 = (j0 + 1 < hi) ? j0 + 1 : lo;
            if (j0 == i || j1 == i) continue;
            const double *a0 = geo + (size_t)GEO_N * j0 + G_A, *a1 = geo + (size_t)GEO_N * j1 + G_A;
            double f0 = (a0[0] - ai[0]) * th[0] + (a0[1] - ai[1]) * th[1] + (a0[2] - ai[2]) * th[2];
            double f1 = (a1[0] - ai[0]) * th[0] + (a1[1] - ai[1]) * th[1] + (a1[2] - ai[2]) * th[2];
            if ((f0 < 0.0) == (f1 < 0.0)) continue;
            double t = f0 / (f0 - f1), va[3];
            const double *v0 = geo + (size_t)GEO_N * j0 + G_V, *v1 = geo + (size_t)GEO_N * j1 + G_V;
            for (int c = 0; c < 3; ++c) va[c] = (1.0 - t) * v0[c] + t * v1[c];
            double ca = (1.0 - t) * cj[j0] + t * cj[j1];
            sum += pow(fabs(dot3(va, th)), m) * ca;
          }
        }
        *o = own / sum;
      }
    }
  (void)segof;
  free(cj);
  free(segof);
}

/* ------------------------------------------------------------------------ */
/* Gaussian smoothing of the learned redundancy weight (Sec. 3.1)            */
/* ------------------------------------------------------------------------ */

/*
 * The paper smooths the learned weight with a Gaussian filter layer (sigma
 * 20, kernel size 121) without stating the axes or the boundary.  Reading
 * used here: per view, a separable filter along mu and along s over the
 * valid half-grid entries k < n_s - 1 (the unused entry n_s - 1 passes
 * through); taps exp(-t^2 / (2 sigma^2)) for |t| <= radius, normalised to
 * unit sum; mirror extension at both ends of a line (index -1 reads index 1,
 * index n reads n - 2, repeated for lines shorter than the radius).
 */
static int mirror_index(int p, int n) {
  if (n == 1) return 0;
  int T = 2 * (n - 1);
  p %= T;
  if (p < 0) p += T;
  return p < n ? p : T - p;
}

static void gauss_taps(double sigma, int radius, double *w) {
  double sum = 0.0;
  for (int t = -radius; t <= radius; ++t) {
    w[t + radius] = exp(-0.5 * (double)t * t / (sigma * sigma));
    sum += w[t + radius];
  }
  for (int t = 0; t <= 2 * radius; ++t) w[t] /= sum;
}

/* y = G x along one line of n elements spaced `stride` apart */
static void smooth_line(const double *x, double *y, int n, size_t stride, const double *w,
                        int radius) {
  for (int i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int t = -radius; t <= radius; ++t) acc += w[t + radius] * x[mirror_index(i + t, n) * stride];
    y[i * stride] = acc;
  }
}

/* x = G^T y along one line: the literal transpose (scatter) of smooth_line */
static void smooth_line_T(const double *y, double *x, int n, size_t stride, const double *w,
                          int radius) {
  for (int i = 0; i < n; ++i) x[i * stride] = 0.0;
  for (int i = 0; i < n; ++i)
    for (int t = -radius; t <= radius; ++t) x[mirror_index(i + t, n) * stride] += w[t + radius] * y[i * stride];
}

/* adjoint = 0: out = G_s G_mu in;  adjoint = 1: out = G_mu^T G_s^T in.
 * in, out: [V][n_mu][n_s] (may not alias). */
void orc_gauss_smooth(int V, int n_mu, int n_s, double sigma, int radius, int adjoint,
                      const double *in, double *out) {
  double *w = malloc(sizeof(double) * (2 * radius + 1));
  gauss_taps(sigma, radius, w);
  size_t nv = (size_t)n_mu * n_s;
  double *tmp = malloc(sizeof(double) * nv * V);
  memcpy(out, in, sizeof(double) * nv * V);
  memcpy(tmp, in, sizeof(double) * nv * V);
  int ns1 = n_s - 1;
#pragma omp parallel for schedule(static)
  for (int v = 0; v < V; ++v) {
    const double *x = in + v * nv;
    double *t = tmp + v * nv, *y = out + v * nv;
    if (!adjoint) {
      for (int k = 0; k < ns1; ++k) smooth_line(x + k, t + k, n_mu, (size_t)n_s, w, radius);
      for (int m = 0; m < n_mu; ++m) smooth_line(t + (size_t)m * n_s, y + (size_t)m * n_s, ns1, 1, w, radius);
    } else {
      for (int m = 0; m < n_mu; ++m) smooth_line_T(x + (size_t)m * n_s, t + (size_t)m * n_s, ns1, 1, w, radius);
      for (int k = 0; k < ns1; ++k) smooth_line_T(t + k, y + k, n_mu, (size_t)n_s, w, radius);
    }
  }
  free(tmp);
  free(w);
}
